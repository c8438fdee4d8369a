// te_sell.cu -- sliced-ELLPACK (SELL-C-sigma) form of H and the SpMV that uses it.
//
// On GB300 the FP64 pipe executes 2 lanes per SM per cycle (1.26 TFLOP/s for
// the whole GPU), while a complex128 multiply-add costs 4 DFMA per stored entry
// of 20 bytes.  The product y = H x is therefore bound by FP64 issue, not by
// HBM, and the layout is chosen to waste no FP64 lane: one lane per row, 32
// rows per slice (a warp), every row of a slice padded to the slice's widest
// row, and rows sorted by length inside windows of kSigma rows so that padding
// is rare.  No lane idles inside the loop and no shuffle reduction is needed.
//
// The sort is a symmetric permutation of the basis: new index i holds old row
// perm[i], columns are renumbered through iperm, and the solver works on
// permuted vectors (copied in and out once per solve).  Entries of slice s
// are stored lane-interleaved: entry k of lane l sits at off[s] + 32 k + l, so
// each warp load is 32 consecutive values.  Padding entries hold 0 and point at
// the lane's own row.
//
// Each complex multiply-add costs three DFMA instead of four: for an entry
// h = a + ib and a vector element x + iy,
//     Re(h x) = a (x + y) - (a + b) y,   Im(h x) = a (x + y) + (b - a) x
// (Gauss's three-multiplication complex product; normwise stable, Higham, SIAM
// J. Matrix Anal. Appl. 13 (1992) 681).  The matrix keeps a and the pair
// (b - a, a + b) per entry, and the product reads the sums s = x + y of the
// vector from a companion array that the kernels writing Lanczos vectors fill.
// The three sums are accumulated separately over the row and combined at its
// end.  The gathers this adds go to the load/store path, which this kernel
// leaves mostly idle.
#include <algorithm>
#include <vector>

#include "te_internal.cuh"

namespace {

constexpr int kSigma = 1024;     // rows per sorting window (multiple of 32)
constexpr int kChunk = 4;        // slices per work item of the SpMV

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    return warp_sum(r);
}

// ---------------------------------------------------------------- conversion

// One block per window: rank of each row = rows that are longer, or equally
// long with a smaller index (a stable descending sort by length).
__global__ void __launch_bounds__(kSigma) k_sell_rank(const int32_t* __restrict__ rowptr, int64_t d,
                                                      int32_t* __restrict__ perm,
                                                      int32_t* __restrict__ iperm) {
    __shared__ int32_t len[kSigma];
    const int64_t base = (int64_t)blockIdx.x * kSigma;
    const int n = (int)((d - base) < kSigma ? (d - base) : kSigma);
    const int t = threadIdx.x;
    if (t < n) len[t] = rowptr[base + t + 1] - rowptr[base + t];
    __syncthreads();
    if (t >= n) return;
    const int mine = len[t];
    int rank = 0;
    for (int q = 0; q < n; ++q) {
        const int l = len[q];
        rank += (l > mine) || (l == mine && q < t);
    }
    perm[base + rank] = (int32_t)(base + t);
    iperm[base + t] = (int32_t)(base + rank);
}

// Entries of slice s: 32 x (length of its first, longest row).
__global__ void k_sell_width(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ perm,
                             int64_t d, int64_t nslices, int32_t* __restrict__ cnt) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nslices) return;
    const int64_t r = perm[s * 32];
    cnt[s] = 32 * (rowptr[r + 1] - rowptr[r]);
}

__global__ void k_sell_fill(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const double2* __restrict__ val, const int32_t* __restrict__ perm,
                            const int32_t* __restrict__ iperm, const int32_t* __restrict__ off,
                            int64_t d, int64_t nslices, int32_t* __restrict__ scol,
                            double* __restrict__ sa, double2* __restrict__ spq) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nslices * 32) return;
    const int64_t s = i >> 5;
    const int lane = (int)(i & 31);
    const int64_t o = off[s];
    const int w = (off[s + 1] - off[s]) >> 5;
    int b = 0, len = 0;
    if (i < d) {
        const int64_t old = perm[i];
        b = rowptr[old];
        len = rowptr[old + 1] - b;
    }
    const int32_t self = (int32_t)(i < d ? i : 0);
    for (int k = 0; k < w; ++k) {
        const int64_t p = o + 32ll * k + lane;
        if (k < len) {
            const double2 v = val[b + k];
            scol[p] = iperm[col[b + k]];
            sa[p] = v.x;                                   // a
            spq[p] = make_double2(v.y - v.x, v.x + v.y);   // (b - a, a + b)
        } else {
            scol[p] = self;
            sa[p] = 0.0;
            spq[p] = make_double2(0.0, 0.0);
        }
    }
}

// ---------------------------------------------------------------- SpMV

// mode 0: Lanczos step j (y = sign scale[j] H u_j - beta[j-1] scale[j-1] u_{j-1},
// partial Re<u_j, y>, matvec count); mode 1: y = H x and Re<x, y>.  xs[i] must
// hold Re x_i + Im x_i.
//
// Work is handed out in chunks of kChunk slices through an atomic counter, so
// SMs that run slower (far-die L2 traffic, other streams) simply take fewer
// chunks.  Each chunk stores its own partial of Re<x, y>; the last block adds
// the chunk partials in chunk order, so the result does not depend on which
// warp took which chunk.
__global__ void __launch_bounds__(TE_BLOCK, 5) k_spmv_sell(
    const int32_t* __restrict__ off, const int32_t* __restrict__ col,
    const double* __restrict__ va, const double2* __restrict__ vpq,
    const double2* __restrict__ x, const double* __restrict__ xs,
    const double2* __restrict__ xprev, double2* __restrict__ y, int64_t d, int64_t nslices,
    DevState* st, int j, int mode, double* partials) {
    __shared__ double sh[32];
    __shared__ bool am_last;
    double cx = 1.0, bp = 0.0;
    if (mode == 0) {
        if (st->status != 0 || st->done != 0 || st->stop) return;
        cx = st->sign * st->scale[j];
        if (j > 0) bp = st->beta[j - 1] * st->scale[j - 1];
    }
    const int lane = threadIdx.x & 31;
    const int64_t nchunks = (nslices + kChunk - 1) / kChunk;
    unsigned int* next = &st->counter[6];
    for (;;) {
        unsigned int c = 0;
        if (lane == 0) c = atomicAdd(next, 1u);
        c = __shfl_sync(0xffffffffu, c, 0);
        if ((int64_t)c >= nchunks) break;
        const int64_t s1 = ((int64_t)c + 1) * kChunk < nslices ? ((int64_t)c + 1) * kChunk : nslices;
        double acc = 0.0;
        for (int64_t s = (int64_t)c * kChunk; s < s1; ++s) {
            const int32_t o = __ldg(off + s);
            const int w = (__ldg(off + s + 1) - o) >> 5;
            const double* ap = va + o + lane;
            const double2* qp = vpq + o + lane;
            const int32_t* cp = col + o + lane;
            // k1 = sum a s, k2 = sum (b - a) x, k3 = sum (a + b) y
            double k1 = 0.0, k2 = 0.0, k3 = 0.0;
            int k = 0;
            for (; k + 2 <= w; k += 2) {
                const double a0 = __ldcs(ap + 32 * k), a1 = __ldcs(ap + 32 * (k + 1));
                const double2 q0 = __ldcs(qp + 32 * k), q1 = __ldcs(qp + 32 * (k + 1));
                const int c0 = __ldcs(cp + 32 * k), c1 = __ldcs(cp + 32 * (k + 1));
                const double2 x0 = __ldg(x + c0), x1 = __ldg(x + c1);
                const double z0 = __ldg(xs + c0), z1 = __ldg(xs + c1);
                k1 = fma(a0, z0, k1);
                k2 = fma(q0.x, x0.x, k2);
                k3 = fma(q0.y, x0.y, k3);
                k1 = fma(a1, z1, k1);
                k2 = fma(q1.x, x1.x, k2);
                k3 = fma(q1.y, x1.y, k3);
            }
            if (k < w) {
                const double a0 = __ldcs(ap + 32 * k);
                const double2 q0 = __ldcs(qp + 32 * k);
                const int c0 = __ldcs(cp + 32 * k);
                const double2 x0 = __ldg(x + c0);
                const double z0 = __ldg(xs + c0);
                k1 = fma(a0, z0, k1);
                k2 = fma(q0.x, x0.x, k2);
                k3 = fma(q0.y, x0.y, k3);
            }
            const int64_t row = s * 32 + lane;
            if (row < d) {
                double2 out = make_double2(cx * (k1 - k3), cx * (k1 + k2));
                if (bp != 0.0) {
                    const double2 p = __ldcs(xprev + row);
                    out.x = fma(-bp, p.x, out.x);
                    out.y = fma(-bp, p.y, out.y);
                }
                y[row] = out;
                const double2 xr = __ldg(x + row);
                acc = fma(xr.x, out.x, acc);
                acc = fma(xr.y, out.y, acc);
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) {
            partials[c] = acc;
            __threadfence();
        }
    }
    __syncthreads();
    unsigned int* ctr = &st->counter[1];
    if (threadIdx.x == 0) {
        __threadfence();
        am_last = (atomicAdd(ctr, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < nchunks; i += blockDim.x) v += __ldcg(partials + i);
    const double tot = block_sum(v, sh);
    if (threadIdx.x == 0) {
        if (mode == 0) {
            const double a = st->scale[j] * tot;
            st->alpha[j] = a;
            st->as_cur = a * st->scale[j];
            st->matvecs += 1;
        } else {
            st->spmv_dot = tot;
        }
        *ctr = 0;
        *next = 0;
    }
}

// dst[i] = src[map[i]]  (map = perm: old -> new order; map = iperm: back);
// with dsum, also dsum[i] = Re dst[i] + Im dst[i] for the product's 3M form.
__global__ void k_gather(const double2* __restrict__ src, const int32_t* __restrict__ map,
                         int64_t d, double2* __restrict__ dst, double* __restrict__ dsum) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = src[map[i]];
        dst[i] = v;
        if (dsum) dsum[i] = v.x + v.y;
    }
}

}  // namespace

te_status build_sell(te_ctx* ctx, te_matrix* H) {
    cudaStream_t s = ctx->stream;
    const int64_t d = H->d;
    const int64_t nslices = (d + 31) / 32;
    const int64_t windows = (d + kSigma - 1) / kSigma;
    TE_CUDA_TRY(ctx, cudaMalloc(&H->perm, sizeof(int32_t) * (size_t)nslices * 32));
    TE_CUDA_TRY(ctx, cudaMalloc(&H->iperm, sizeof(int32_t) * (size_t)d));
    TE_CUDA_TRY(ctx, cudaMalloc(&H->sell_off, sizeof(int32_t) * (size_t)(nslices + 1)));
    // rows past d (in the last slice) map to row 0's length: give perm a valid entry there
    TE_CUDA_TRY(ctx, cudaMemsetAsync(H->perm, 0, sizeof(int32_t) * (size_t)nslices * 32, s));
    k_sell_rank<<<(int)windows, kSigma, 0, s>>>(H->rowptr, d, H->perm, H->iperm);
    TE_CUDA_TRY(ctx, cudaGetLastError());
    int32_t* cnt = nullptr;
    TE_CUDA_TRY(ctx, cudaMalloc(&cnt, sizeof(int32_t) * (size_t)nslices));
    k_sell_width<<<(int)((nslices + TE_BLOCK - 1) / TE_BLOCK), TE_BLOCK, 0, s>>>(H->rowptr, H->perm,
                                                                                d, nslices, cnt);
    cudaError_t e = cudaGetLastError();
    int64_t total = 0;
    te_status st = TE_OK;
    if (e == cudaSuccess) st = scan_counts(ctx, cnt, nslices, H->sell_off, &total, s);
    cudaFree(cnt);
    if (e != cudaSuccess) return cuda_error(ctx, e, "k_sell_width");
    if (st) return st;
    H->nslices = nslices;
    H->sell_nnz = total;
    TE_CUDA_TRY(ctx, cudaMalloc(&H->sell_col, sizeof(int32_t) * (size_t)std::max<int64_t>(total, 1)));
    TE_CUDA_TRY(ctx, cudaMalloc(&H->sell_a, sizeof(double) * (size_t)std::max<int64_t>(total, 1)));
    TE_CUDA_TRY(ctx, cudaMalloc(&H->sell_pq, sizeof(double2) * (size_t)std::max<int64_t>(total, 1)));
    k_sell_fill<<<(int)((nslices * 32 + TE_BLOCK - 1) / TE_BLOCK), TE_BLOCK, 0, s>>>(
        H->rowptr, H->col, H->val, H->perm, H->iperm, H->sell_off, d, nslices, H->sell_col,
        H->sell_a, H->sell_pq);
    TE_CUDA_TRY(ctx, cudaGetLastError());
    H->sell_grid = sell_grid(nslices, ctx->num_sms);
    TE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    return TE_OK;
}

int sell_grid(int64_t nslices, int num_sms) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv_sell, TE_BLOCK, 0);
    if (nb < 1) nb = 1;
    const int64_t need = (nslices + (TE_BLOCK / 32) - 1) / (TE_BLOCK / 32);
    const int64_t full = (int64_t)nb * num_sms;
    return (int)std::max<int64_t>(1, std::min(need, full));
}

// partials must hold sell_partials(H) doubles (one per chunk of slices); xs holds
// Re x + Im x.
cudaError_t launch_spmv_sell(const te_matrix* H, const double2* x, const double* xs,
                             const double2* xprev, double2* y, DevState* st, int j, int mode,
                             double* partials, cudaStream_t s) {
    k_spmv_sell<<<H->sell_grid, TE_BLOCK, 0, s>>>(H->sell_off, H->sell_col, H->sell_a, H->sell_pq,
                                                 x, xs, xprev, y, H->d, H->nslices, st, j, mode,
                                                 partials);
    return cudaGetLastError();
}

cudaError_t launch_gather(const double2* src, const int32_t* map, int64_t d, double2* dst,
                          double* dsum, int num_sms, cudaStream_t s) {
    const int64_t want = (d + TE_BLOCK - 1) / TE_BLOCK;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms * 8));
    k_gather<<<grid, TE_BLOCK, 0, s>>>(src, map, d, dst, dsum);
    return cudaGetLastError();
}

int64_t sell_partials(const te_matrix* H) { return (H->nslices + kChunk - 1) / kChunk; }
