// te_block.cu -- batched solves: many initial vectors evolved under one H.
//
// Algorithm 1 of arXiv 2205.15346 is a per-vector method: each of the B vectors
// builds its own Krylov space, takes its own steps and finishes after its own
// number of restarts.  What B solves under one H share is the operator, so the
// batch runs the restarts in lock step and turns the B products H u_j into one
// block product Y = H X with X, Y stored row-major as d x B (row r holds element
// r of every vector, so a gathered row of X is one contiguous 16 B-per-vector
// stretch).  Every other step stays per vector: each vector keeps its own
// DevState, its own alpha / beta / scale, its own breakdown test and its own
// step search (the step kernel runs one CTA per vector), and a vector that has
// reached t simply stops being updated while the others go on.
//
// On GB300 the products are bound by FP64 issue (2 DFMA lanes per SM per cycle),
// not by HBM, so the block product spends fewer FP64 instructions per complex
// multiply-add instead of saving bytes: with H_rc = a + ib and x_c = x + iy,
//     Re(H_rc x_c) = a (x + y) - (a + b) y,   Im(H_rc x_c) = a (x + y) + (b - a) x,
// three real products per entry (Gauss's three-multiplication complex product;
// Higham, SIAM J. Matrix Anal. Appl. 13 (1992) 681, shows it is normwise stable).
// The matrix side (a, b - a, a + b) is stored once per entry and the vector side
// s = x + y once per vector element (written by whichever kernel writes the
// Lanczos vector), so every entry of every vector costs three DFMA instead of
// four.  Each of the three sums is accumulated separately over the row and
// combined once at its end.
//
// Kernels of one Lanczos step (all deterministic: per-chunk or per-block
// partials are summed in a fixed order by a second kernel with one CTA per
// vector):
//   KB1  k_spmm_block   Y = cx_b H X - bp_b X_prev (per vector b), partials of Re<u_b, y_b>
//   KB1r k_alpha_block  alpha_b, as_cur_b
//   KB2  k_orth_block   W = Y - as_b U, s = Re W + Im W, partials of ||w_b||^2
//   KB2r k_decide_block beta_b, breakdown test, scale_b[j+1]
// per restart: K3 (k_step, grid = B), KB4 k_recombine_block (+ KB4r), state copy.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>

#include "te_internal.cuh"

namespace {

// threads of the one-CTA-per-vector / per-problem reductions (they add up to tens of
// thousands of partials each)
constexpr int kReduceThreads = 1024;

constexpr int kRowsPerWarp = 8;                          // rows of one warp in a chunk
constexpr int kChunkRows = kRowsPerWarp * (TE_BLOCK / 32);   // rows of one chunk (one CTA task)

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

__device__ __forceinline__ bool vec_halted(const DevState* s) {
    return s->status != 0 || s->done != 0 || s->stop != 0;
}

// Sum of partials[0..n) by one CTA in a fixed order (valid in every thread).
__device__ __forceinline__ double sum_partials(const double* p, int64_t n, double* sh) {
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v += __ldcg(p + i);
    return block_sum(v, sh);
}

// ---------------------------------------------------------------- 3M form of H

__global__ void k_make_3m(const double2* __restrict__ val, int64_t nnz, double* __restrict__ m3) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = val[k];
        m3[k] = v.x;                 // a
        m3[nnz + k] = v.y - v.x;     // b - a
        m3[2 * nnz + k] = v.x + v.y; // a + b
    }
}

// ---------------------------------------------------------------- packing

// V0[r, b] = v_in[b][r] for b < nvec, 0 for the padding vectors; s = Re + Im.
__global__ void k_pack(const double2* __restrict__ src, int64_t d, int nvec, int B,
                       double2* __restrict__ X, double* __restrict__ S) {
    const int64_t n = d * B;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / B;
        const int b = (int)(e - r * B);
        const double2 v = b < nvec ? src[(int64_t)b * d + r] : make_double2(0.0, 0.0);
        X[e] = v;
        S[e] = v.x + v.y;
    }
}

// v_out[b][r] = V0[r, b] for b < nvec.
__global__ void k_unpack(const double2* __restrict__ X, int64_t d, int nvec, int B,
                         double2* __restrict__ dst) {
    const int64_t n = d * nvec;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / d;
        const int64_t r = e - b * d;
        dst[e] = X[r * B + b];
    }
}

// ---------------------------------------------------------------- KB0 / KB2 / KB4 block partials

// Threads of a CTA with equal (threadIdx.x mod B) hold the same vector; their
// values are added in thread order and written to partials[b * G + blockIdx.x].
__device__ __forceinline__ void per_vector_partials(double acc, int B, double* sh,
                                                    double* partials, int G) {
    sh[threadIdx.x] = acc;
    __syncthreads();
    if ((int)threadIdx.x < B) {
        double s = 0.0;
        for (int t = threadIdx.x; t < (int)blockDim.x; t += B) s += sh[t];
        partials[(size_t)threadIdx.x * G + blockIdx.x] = s;
    }
}

// KB0: ||v_b||^2 partials of the packed initial block.
__global__ void __launch_bounds__(TE_BLOCK) k_norm_block(const double2* __restrict__ X, int64_t d,
                                                         int B, double* partials) {
    __shared__ double sh[TE_BLOCK];
    const int64_t n = d * B;
    double acc = 0.0;
    bool finite = true;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = X[e];
        finite &= isfinite(v.x) && isfinite(v.y);
        acc = fma(v.x, v.x, acc);
        acc = fma(v.y, v.y, acc);
    }
    if (!finite) acc = __longlong_as_double(0x7ff8000000000000LL);
    per_vector_partials(acc, B, sh, partials, gridDim.x);
}

// KB0r / KB4r: beta0_b = ||w_b|| opens the next Krylov space (one CTA per vector).
// init: validation of v_in (Sec. 2.1 assumes ||v(0)|| = 1); otherwise only the
// vectors whose step kernel took a step in this restart are updated.
__global__ void __launch_bounds__(kReduceThreads) k_beta0_block(DevState* st_base, const double* partials,
                                                          int G, int init) {
    __shared__ double sh[32];
    DevState* st = st_base + blockIdx.x;
    if (init ? (st->done != 0) : (st->active == 0 || st->status != 0)) return;
    const double tot = sum_partials(partials + (size_t)blockIdx.x * G, G, sh);
    if (threadIdx.x == 0) {
        const double nrm = sqrt(tot);
        st->beta0 = nrm;
        st->scale[0] = 1.0 / nrm;
        st->stop = 0;
        st->m_eff = st->m;
        st->breakdown = 0;
        st->active = 0;
        if (!isfinite(nrm)) st->status = TE_ERR_NONFINITE;
        else if (init && fabs(nrm - 1.0) > 1e-10) st->status = TE_ERR_NOT_NORMALIZED;
    }
}

// ---------------------------------------------------------------- KB1

// One CTA task is a chunk of kChunkRows consecutive rows (warp w takes rows
// w * kRowsPerWarp .. + kRowsPerWarp - 1 of it), handed out through an atomic
// counter; lane l of a warp owns vectors l, l + 32, ... (VPL of them).  The
// chunk's partials of Re<u_b, y_b> are written to partials[b * nchunks + chunk],
// so the sum does not depend on which CTA took which chunk.
template <int VPL>
__global__ void __launch_bounds__(TE_BLOCK, 3) k_spmm_block(
    const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const double* __restrict__ m3, int64_t nnz, const double2* __restrict__ X,
    const double* __restrict__ S, const double2* __restrict__ Xprev, double2* __restrict__ Y,
    int64_t d, int B, DevState* st_base, int j, double* partials, int64_t nchunks,
    unsigned int* ctr) {
    __shared__ double red[2][TE_BLOCK / 32][64];
    __shared__ int64_t sh_chunk;
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double cx[VPL], bp[VPL];
    bool on[VPL];
#pragma unroll
    for (int q = 0; q < VPL; ++q) {
        const int b = lane + 32 * q;
        on[q] = b < B;
        cx[q] = 0.0;
        bp[q] = 0.0;
        if (on[q]) {
            const DevState* s = st_base + b;
            if (!vec_halted(s)) {
                cx[q] = s->sign * s->scale[j];
                if (j > 0) bp[q] = s->beta[j - 1] * s->scale[j - 1];
            }
        }
    }
    const double* ma = m3;
    const double* mba = m3 + nnz;
    const double* mab = m3 + 2 * nnz;
    for (int it = 0;; it ^= 1) {
        if (threadIdx.x == 0) sh_chunk = (int64_t)atomicAdd(&ctr[0], 1u);
        __syncthreads();
        const int64_t c = sh_chunk;
        if (c >= nchunks) break;
        double al[VPL];
#pragma unroll
        for (int q = 0; q < VPL; ++q) al[q] = 0.0;
        const int64_t r0 = c * kChunkRows + (int64_t)wid * kRowsPerWarp;
        for (int i = 0; i < kRowsPerWarp; ++i) {
            const int64_t r = r0 + i;
            if (r >= d) break;
            const int e0 = __ldg(rowptr + r), e1 = __ldg(rowptr + r + 1);
            double k1[VPL], k2[VPL], k3[VPL];
#pragma unroll
            for (int q = 0; q < VPL; ++q) k1[q] = k2[q] = k3[q] = 0.0;
            int k = e0;
            for (; k + 1 < e1; k += 2) {
                const int c0 = __ldg(col + k), c1 = __ldg(col + k + 1);
                const double a0 = __ldg(ma + k), a1 = __ldg(ma + k + 1);
                const double p0 = __ldg(mba + k), p1 = __ldg(mba + k + 1);
                const double s0 = __ldg(mab + k), s1 = __ldg(mab + k + 1);
                double2 x0[VPL], x1[VPL];
                double z0[VPL], z1[VPL];
#pragma unroll
                for (int q = 0; q < VPL; ++q) {
                    if (on[q]) {
                        x0[q] = __ldg(X + (int64_t)c0 * B + lane + 32 * q);
                        z0[q] = __ldg(S + (int64_t)c0 * B + lane + 32 * q);
                        x1[q] = __ldg(X + (int64_t)c1 * B + lane + 32 * q);
                        z1[q] = __ldg(S + (int64_t)c1 * B + lane + 32 * q);
                    } else {
                        x0[q] = x1[q] = make_double2(0.0, 0.0);
                        z0[q] = z1[q] = 0.0;
                    }
                }
#pragma unroll
                for (int q = 0; q < VPL; ++q) {
                    k1[q] = fma(a0, z0[q], k1[q]);
                    k2[q] = fma(p0, x0[q].x, k2[q]);
                    k3[q] = fma(s0, x0[q].y, k3[q]);
                    k1[q] = fma(a1, z1[q], k1[q]);
                    k2[q] = fma(p1, x1[q].x, k2[q]);
                    k3[q] = fma(s1, x1[q].y, k3[q]);
                }
            }
            if (k < e1) {
                const int c0 = __ldg(col + k);
                const double a0 = __ldg(ma + k), p0 = __ldg(mba + k), s0 = __ldg(mab + k);
#pragma unroll
                for (int q = 0; q < VPL; ++q) {
                    if (on[q]) {
                        const double2 x0 = __ldg(X + (int64_t)c0 * B + lane + 32 * q);
                        const double z0 = __ldg(S + (int64_t)c0 * B + lane + 32 * q);
                        k1[q] = fma(a0, z0, k1[q]);
                        k2[q] = fma(p0, x0.x, k2[q]);
                        k3[q] = fma(s0, x0.y, k3[q]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < VPL; ++q) {
                if (!on[q]) continue;
                const int64_t e = r * B + lane + 32 * q;
                const double re = k1[q] - k3[q];
                const double im = k1[q] + k2[q];
                double2 out = make_double2(cx[q] * re, cx[q] * im);
                if (bp[q] != 0.0) {
                    const double2 p = __ldcs(Xprev + e);
                    out.x = fma(-bp[q], p.x, out.x);
                    out.y = fma(-bp[q], p.y, out.y);
                }
                Y[e] = out;
                const double2 xr = __ldg(X + e);
                al[q] = fma(xr.x, out.x, al[q]);
                al[q] = fma(xr.y, out.y, al[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < VPL; ++q) red[it][wid][lane + 32 * q] = al[q];
        __syncthreads();
        if ((int)threadIdx.x < B) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < TE_BLOCK / 32; ++w) s += red[it][w][threadIdx.x];
            partials[(size_t)threadIdx.x * nchunks + c] = s;
        }
    }
    // the last CTA to leave resets the chunk counter for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        am_last = (atomicAdd(&ctr[1], 1u) == gridDim.x - 1);
        if (am_last) {
            ctr[0] = 0;
            ctr[1] = 0;
        }
    }
}

// KB1r: alpha_b = scale_b[j]^2 Re<u_b, y_b> (one CTA per vector).
__global__ void __launch_bounds__(kReduceThreads) k_alpha_block(DevState* st_base, const double* partials,
                                                          int64_t nchunks, int j) {
    __shared__ double sh[32];
    DevState* st = st_base + blockIdx.x;
    if (vec_halted(st)) return;
    const double tot = sum_partials(partials + (size_t)blockIdx.x * nchunks, nchunks, sh);
    if (threadIdx.x == 0) {
        const double a = st->scale[j] * tot;
        st->alpha[j] = a;
        st->as_cur = a * st->scale[j];
        st->matvecs += 1;
    }
}

// ---------------------------------------------------------------- KB2

// w = y - as_b u in place (write), s = Re w + Im w, ||w_b||^2 partials.  The
// grid stride is a multiple of B, so every thread stays on one vector.
__global__ void __launch_bounds__(TE_BLOCK) k_orth_block(double2* __restrict__ W,
                                                         const double2* __restrict__ U,
                                                         double* __restrict__ S, int64_t d, int B,
                                                         const DevState* st_base, int write,
                                                         double* partials) {
    __shared__ double sh[TE_BLOCK];
    const int64_t n = d * B;
    const int b = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) % B);
    const DevState* s = st_base + b;
    const double as = vec_halted(s) ? 0.0 : s->as_cur;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double acc = 0.0;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; e + 3 * stride < n; e += 4 * stride) {
        double2 y[4], u[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            y[q] = W[e + q * stride];
            u[q] = __ldcs(U + e + q * stride);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            y[q].x = fma(-as, u[q].x, y[q].x);
            y[q].y = fma(-as, u[q].y, y[q].y);
            if (write) {
                W[e + q * stride] = y[q];
                S[e + q * stride] = y[q].x + y[q].y;
            }
            acc = fma(y[q].x, y[q].x, acc);
            acc = fma(y[q].y, y[q].y, acc);
        }
    }
    for (; e < n; e += stride) {
        double2 y = W[e];
        const double2 u = __ldcs(U + e);
        y.x = fma(-as, u.x, y.x);
        y.y = fma(-as, u.y, y.y);
        if (write) {
            W[e] = y;
            S[e] = y.x + y.y;
        }
        acc = fma(y.x, y.x, acc);
        acc = fma(y.y, y.y, acc);
    }
    per_vector_partials(acc, B, sh, partials, gridDim.x);
}

// KB2r: h_{j+1,j} = ||w~_b||, the breakdown test of Algorithm 1 step 1 and
// scale_b[j+1] (one CTA per vector).
__global__ void __launch_bounds__(kReduceThreads) k_decide_block(DevState* st_base, const double* partials,
                                                           int G, int j) {
    __shared__ double sh[32];
    DevState* st = st_base + blockIdx.x;
    if (vec_halted(st)) return;
    const double nrm = sqrt(sum_partials(partials + (size_t)blockIdx.x * G, G, sh));
    if (threadIdx.x == 0) {
        st->beta[j] = nrm;
        if (!(nrm >= st->tol_rate)) {        // also catches NaN
            if (!isfinite(nrm)) st->status = TE_ERR_NONFINITE;
            st->stop = 1;
            st->m_eff = j + 1;
            st->breakdown = 1;
        } else if (j + 1 < st->m) {
            st->scale[j + 1] = 1.0 / nrm;
        } else {
            st->m_eff = st->m;
        }
    }
}

// ---------------------------------------------------------------- KB4

// w_b = sum_{k < m_eff_b} coef_b[k] u_{b,k} into block 0 for the vectors whose
// step kernel took a step (Algorithm 1 step 3), s = Re w + Im w, ||w_b||^2
// partials.  Coefficients of all vectors sit in shared memory (B x m double2).
__global__ void __launch_bounds__(TE_BLOCK) k_recombine_block(double2* __restrict__ V,
                                                              double* __restrict__ S, int64_t d,
                                                              int B, int m, const DevState* st_base,
                                                              double* partials) {
    extern __shared__ double2 cf[];                      // [B][m]
    __shared__ double sh[TE_BLOCK];
    for (int i = threadIdx.x; i < B * m; i += blockDim.x) {
        const int b = i / m, k = i - b * m;
        cf[i] = st_base[b].coef[k];
    }
    __syncthreads();
    const int64_t n = d * B;
    const int64_t blk = d * B;                            // elements per Krylov block
    const int b = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) % B);
    const DevState* s = st_base + b;
    const bool act = s->active != 0 && s->status == 0;
    const int nk = act ? s->last_m_eff : 0;
    const double2* c = cf + (size_t)b * m;
    double acc = 0.0;
    if (act) {
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
             e += (int64_t)gridDim.x * blockDim.x) {
            double re = 0.0, im = 0.0;
            int k = 0;
            for (; k + 4 <= nk; k += 4) {
                double2 a[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) a[q] = __ldcs(V + (size_t)(k + q) * blk + e);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    re = fma(c[k + q].x, a[q].x, re);
                    re = fma(-c[k + q].y, a[q].y, re);
                    im = fma(c[k + q].x, a[q].y, im);
                    im = fma(c[k + q].y, a[q].x, im);
                }
            }
            for (; k < nk; ++k) {
                const double2 a = __ldcs(V + (size_t)k * blk + e);
                re = fma(c[k].x, a.x, re);
                re = fma(-c[k].y, a.y, re);
                im = fma(c[k].x, a.y, im);
                im = fma(c[k].y, a.x, im);
            }
            V[e] = make_double2(re, im);
            S[e] = re + im;
            acc = fma(re, re, acc);
            acc = fma(im, im, acc);
        }
    }
    per_vector_partials(acc, B, sh, partials, gridDim.x);
}

template <int VPL>
int spmm_occ() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmm_block<VPL>, TE_BLOCK, 0);
    return nb > 0 ? nb : 1;
}

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

// ------------------------------------------------------------------ engine

struct BlockPlan {
    te_ctx* ctx = nullptr;           // owner (device memory through its allocator)
    uint64_t matrix_id = 0;
    int m = 0, B = 0, profile = 0;
    int64_t d = 0;
    int64_t nchunks = 0;
    int grid_spmm = 0, grid_stream = 0;
    double2* V = nullptr;           // (m + 1) blocks of d x B
    double* S = nullptr;            // d x B: Re + Im of the current Lanczos block
    double* partials = nullptr;
    DevState* st = nullptr;         // B states
    DevState* st_host = nullptr;    // pinned copy written at the end of each restart
    DevState* st_init = nullptr;    // pinned
    unsigned int* ctr = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> ev;
    bool in_use = false;
};

namespace {

std::mutex g_block_mu;
std::vector<std::pair<te_ctx*, BlockPlan*>> g_block_plans;

void free_block_plan(BlockPlan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
    for (void* q : {(void*)p->V, (void*)p->S, (void*)p->partials, (void*)p->st, (void*)p->ctr})
        if (q) dev_free(p->ctx, q);
    if (p->st_host) cudaFreeHost(p->st_host);
    if (p->st_init) cudaFreeHost(p->st_init);
    delete p;
}

cudaError_t launch_spmm(const te_matrix* H, const BlockPlan* p, int j, cudaStream_t s) {
    const double2* X = p->V + (size_t)j * p->d * p->B;
    const double2* Xp = j > 0 ? p->V + (size_t)(j - 1) * p->d * p->B : nullptr;
    double2* Y = p->V + (size_t)(j + 1) * p->d * p->B;
    if (p->B > 32)
        k_spmm_block<2><<<p->grid_spmm, TE_BLOCK, 0, s>>>(H->rowptr, H->col, H->m3, H->nnz, X, p->S,
                                                          Xp, Y, p->d, p->B, p->st, j, p->partials,
                                                          p->nchunks, p->ctr);
    else
        k_spmm_block<1><<<p->grid_spmm, TE_BLOCK, 0, s>>>(H->rowptr, H->col, H->m3, H->nnz, X, p->S,
                                                          Xp, Y, p->d, p->B, p->st, j, p->partials,
                                                          p->nchunks, p->ctr);
    return cudaGetLastError();
}

te_status capture_block_restart(te_ctx* ctx, const te_matrix* H, BlockPlan* p, cudaStream_t s) {
    const int64_t blk = p->d * p->B;
    const int m = p->m, B = p->B;
    TE_CUDA_TRY(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < m && e == cudaSuccess; ++j) {
        const bool timed = p->profile && j == m / 2;     // one product per round is timed
        if (timed) e = cudaEventRecordWithFlags(p->ev[0], s, cudaEventRecordExternal);
        if (e == cudaSuccess) e = launch_spmm(H, p, j, s);
        if (timed && e == cudaSuccess)
            e = cudaEventRecordWithFlags(p->ev[1], s, cudaEventRecordExternal);
        if (e != cudaSuccess) break;
        k_alpha_block<<<B, kReduceThreads, 0, s>>>(p->st, p->partials, p->nchunks, j);
        k_orth_block<<<p->grid_stream, TE_BLOCK, 0, s>>>(p->V + (size_t)(j + 1) * blk,
                                                         p->V + (size_t)j * blk, p->S, p->d, B,
                                                         p->st, j + 1 < m, p->partials);
        k_decide_block<<<B, kReduceThreads, 0, s>>>(p->st, p->partials, p->grid_stream, j);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_step_batch(p->st, B, m, s);
    if (e == cudaSuccess) {
        k_recombine_block<<<p->grid_stream, TE_BLOCK, sizeof(double2) * B * m, s>>>(
            p->V, p->S, p->d, B, m, p->st, p->partials);
        k_beta0_block<<<B, kReduceThreads, 0, s>>>(p->st, p->partials, p->grid_stream, 0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->st_host, p->st, sizeof(DevState) * B, cudaMemcpyDeviceToHost, s);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_error(ctx, e, "capturing the batched restart graph");
    }
    if (e2 != cudaSuccess) return cuda_error(ctx, e2, "cudaStreamEndCapture");
    cudaError_t e3 = cudaGraphInstantiate(&p->exec, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return cuda_error(ctx, e3, "cudaGraphInstantiate (batched restart)");
    return TE_OK;
}

te_status ensure_3m(te_ctx* ctx, const te_matrix* Hc, cudaStream_t s) {
    te_matrix* H = const_cast<te_matrix*>(Hc);   // library-owned; the 3M copy is a cache
    std::lock_guard<std::mutex> lk(g_block_mu);
    if (H->m3) return TE_OK;
    double* m3 = nullptr;
    TE_CUDA_TRY(ctx, dev_alloc(ctx, &m3, sizeof(double) * 3 * (size_t)std::max<int64_t>(H->nnz, 1)));
    const int64_t want = (H->nnz + TE_BLOCK - 1) / TE_BLOCK;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)ctx->num_sms * 8));
    k_make_3m<<<grid, TE_BLOCK, 0, s>>>(H->val, H->nnz, m3);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        dev_free(ctx, m3);
        return cuda_error(ctx, e, "building the 3M form of H");
    }
    H->m3 = m3;
    return TE_OK;
}

te_status create_block_plan(te_ctx* ctx, const te_matrix* H, int m, int B, int profile,
                            cudaStream_t s, BlockPlan** out) {
    BlockPlan* p = new BlockPlan();
    p->ctx = ctx;
    p->matrix_id = H->id;
    p->m = m;
    p->B = B;
    p->profile = profile;
    p->d = H->d;
    p->nchunks = (H->d + kChunkRows - 1) / kChunkRows;
    const int occ = B > 32 ? spmm_occ<2>() : spmm_occ<1>();
    p->grid_spmm = (int)std::max<int64_t>(1, std::min<int64_t>(p->nchunks, (int64_t)occ * ctx->num_sms));
    const int64_t want = (H->d * B + TE_BLOCK - 1) / TE_BLOCK;
    p->grid_stream = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)ctx->num_sms * 8);
    const size_t blk = (size_t)H->d * B;
    const size_t npart = (size_t)B * std::max<int64_t>(p->nchunks, p->grid_stream);
    cudaError_t e = dev_alloc(ctx, &p->V, sizeof(double2) * (size_t)(m + 1) * blk);
    if (e == cudaSuccess) e = dev_alloc(ctx, &p->S, sizeof(double) * blk);
    if (e == cudaSuccess) e = dev_alloc(ctx, &p->partials, sizeof(double) * npart);
    if (e == cudaSuccess) e = dev_alloc(ctx, &p->st, sizeof(DevState) * B);
    if (e == cudaSuccess) e = dev_alloc(ctx, &p->ctr, sizeof(unsigned int) * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&p->st_host, sizeof(DevState) * B);
    if (e == cudaSuccess) e = cudaMallocHost(&p->st_init, sizeof(DevState) * B);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_block_plan(p);
        return set_error(ctx, e == cudaErrorMemoryAllocation ? TE_ERR_OOM : TE_ERR_CUDA,
                         std::string("allocating the batched workspace: ") + cudaGetErrorString(e));
    }
    if (cudaMemsetAsync(p->ctr, 0, sizeof(unsigned int) * 4, s) != cudaSuccess ||
        cudaMemsetAsync(p->st, 0, sizeof(DevState) * B, s) != cudaSuccess) {
        cudaGetLastError();
        free_block_plan(p);
        return set_error(ctx, TE_ERR_CUDA, "preparing the batched workspace");
    }
    if (profile) {
        p->ev.resize(2);
        for (auto& ev : p->ev) cudaEventCreate(&ev);
    }
    te_status st = capture_block_restart(ctx, H, p, s);
    if (st) {
        free_block_plan(p);
        return st;
    }
    *out = p;
    return TE_OK;
}

te_status acquire_block_plan(te_ctx* ctx, const te_matrix* H, int m, int B, int profile,
                             cudaStream_t s, BlockPlan** out) {
    {
        std::lock_guard<std::mutex> lk(g_block_mu);
        for (auto& cp : g_block_plans) {
            BlockPlan* p = cp.second;
            if (cp.first == ctx && !p->in_use && p->matrix_id == H->id && p->m == m && p->B == B &&
                p->profile == profile) {
                p->in_use = true;
                *out = p;
                return TE_OK;
            }
        }
    }
    BlockPlan* p = nullptr;
    te_status st = create_block_plan(ctx, H, m, B, profile, s, &p);
    if (st == TE_ERR_OOM) {
        // drop this context's idle batched plans and try once more
        std::vector<BlockPlan*> idle;
        {
            std::lock_guard<std::mutex> lk(g_block_mu);
            auto it = std::partition(g_block_plans.begin(), g_block_plans.end(),
                                     [&](const std::pair<te_ctx*, BlockPlan*>& q) {
                                         return q.first != ctx || q.second->in_use;
                                     });
            for (auto q = it; q != g_block_plans.end(); ++q) idle.push_back(q->second);
            g_block_plans.erase(it, g_block_plans.end());
        }
        cudaStreamSynchronize(s);
        for (BlockPlan* q : idle) free_block_plan(q);
        st = create_block_plan(ctx, H, m, B, profile, s, &p);
    }
    if (st) return st;
    p->in_use = true;
    std::lock_guard<std::mutex> lk(g_block_mu);
    g_block_plans.emplace_back(ctx, p);
    *out = p;
    return TE_OK;
}

}  // namespace

// Drop the batched plans of a context (all of them) or of one matrix.
void block_plans_release(te_ctx* ctx, uint64_t matrix_id) {
    std::vector<BlockPlan*> drop;
    {
        std::lock_guard<std::mutex> lk(g_block_mu);
        auto it = std::partition(g_block_plans.begin(), g_block_plans.end(),
                                 [&](const std::pair<te_ctx*, BlockPlan*>& q) {
                                     return !(q.first == ctx && (matrix_id == 0 ||
                                                                 q.second->matrix_id == matrix_id));
                                 });
        for (auto q = it; q != g_block_plans.end(); ++q) drop.push_back(q->second);
        g_block_plans.erase(it, g_block_plans.end());
    }
    for (BlockPlan* p : drop) free_block_plan(p);
}

// The dynamic shared memory of the recombination (B x m coefficients) can pass
// the default 48 KB; its limit is set once for the largest B and m.
cudaError_t block_prepare() {
    return cudaFuncSetAttribute(k_recombine_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(double2) * TE_BATCH_MAX * TE_M_MAX));
}

// One group of nvec <= TE_BATCH_MAX vectors through a batched plan.  v_in /
// v_out hold nvec vectors of length d one after the other (device pointers if
// dev, else host; host data is staged through the plan's last Krylov block,
// which is free outside a restart).
te_status run_block_solve(te_ctx* ctx, const te_matrix* H, int nvec, const double* v_in, double t,
                          double tol, int m, const te_options& o, double* v_out, bool dev,
                          te_stats* stats, int32_t* status, cudaStream_t s) {
    const double t0 = now_ms();
    int B = 1;
    while (B < nvec) B <<= 1;
    const int profile = (o.flags & TE_OPT_PROFILE) ? 1 : 0;
    te_status rs = ensure_3m(ctx, H, s);
    if (rs) return rs;
    BlockPlan* p = nullptr;
    rs = acquire_block_plan(ctx, H, m, B, profile, s, &p);
    if (rs) return rs;
    const int64_t d = H->d;
    DevState* ini = p->st_init;
    memset(ini, 0, sizeof(DevState) * B);
    for (int b = 0; b < B; ++b) {
        DevState& x = ini[b];
        x.T = fabs(t);
        x.tol_rate = (t != 0.0) ? tol / fabs(t) : tol;
        x.sign = (t >= 0.0) ? 1.0 : -1.0;
        x.t_step0 = o.t_step0;
        x.shrink = o.shrink;
        x.quad_rel_tol = o.quad_rel_tol;
        x.min_step = o.min_step_rel * fabs(t);
        x.m = m;
        x.n_substeps = o.n_substeps;
        x.quad = o.quad;
        x.gauss_n = o.gauss_n;
        x.quad_max_levels = o.quad_max_levels;
        x.max_substeps = o.max_substeps;
        x.smallexp = o.small_exp;
        x.first = 1;
        x.m_eff = m;
        x.min_err_step = INFINITY;
        x.done = (b >= nvec) ? 1 : 0;                  // padding vectors never run
    }
    gauss_legendre_table(o.gauss_n, ini[0].gx, ini[0].gw);
    double2* stage = p->V + (size_t)m * (size_t)d * B;
    for (int b = 1; b < B; ++b) {
        memcpy(ini[b].gx, ini[0].gx, sizeof(ini[0].gx));
        memcpy(ini[b].gw, ini[0].gw, sizeof(ini[0].gw));
    }
    auto fail = [&](cudaError_t e, const char* what) {
        std::lock_guard<std::mutex> lk(g_block_mu);
        p->in_use = false;
        return cuda_error(ctx, e, what);
    };
    cudaError_t e = cudaMemcpyAsync(p->st, ini, sizeof(DevState) * B, cudaMemcpyHostToDevice, s);
    const int64_t want = (d * B + TE_BLOCK - 1) / TE_BLOCK;
    const int gpk = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)ctx->num_sms * 8));
    const double2* src = (const double2*)v_in;
    if (e == cudaSuccess && !dev) {
        e = cudaMemcpyAsync(stage, v_in, sizeof(double2) * (size_t)nvec * d, cudaMemcpyHostToDevice, s);
        src = stage;
    }
    if (e == cudaSuccess) {
        k_pack<<<gpk, TE_BLOCK, 0, s>>>(src, d, nvec, B, p->V, p->S);
        k_norm_block<<<p->grid_stream, TE_BLOCK, 0, s>>>(p->V, d, B, p->partials);
        k_beta0_block<<<B, kReduceThreads, 0, s>>>(p->st, p->partials, p->grid_stream, 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->st_host, p->st, sizeof(DevState) * B, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(e, "starting the batched solve");
    const DevState* h = p->st_host;
    double spmv_ms = 0.0;
    int64_t spmv_launches = 0;
    auto running = [&]() {
        for (int b = 0; b < nvec; ++b)
            if (h[b].status == 0 && h[b].done == 0) return true;
        return false;
    };
    while (t != 0.0 && running()) {
        e = cudaGraphLaunch(p->exec, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(e, "batched restart");
        if (profile) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p->ev[0], p->ev[1]) == cudaSuccess) {
                spmv_ms += ms;
                spmv_launches += 1;
            } else {
                cudaGetLastError();
            }
        }
    }
    k_unpack<<<gpk, TE_BLOCK, 0, s>>>(p->V, d, nvec, B, dev ? (double2*)v_out : stage);
    e = cudaGetLastError();
    if (e == cudaSuccess && !dev)
        e = cudaMemcpyAsync(v_out, stage, sizeof(double2) * (size_t)nvec * d, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(e, "unpacking the batched result");
    const double per_restart = (double)d * H->norm1 * 2.220446049250313e-16;
    te_status worst = TE_OK;
    for (int b = 0; b < nvec; ++b) {
        const DevState& x = h[b];
        const te_status sb = x.status;
        if (status) status[b] = sb;
        if (sb != TE_OK && worst == TE_OK) worst = sb;
        if (!stats) continue;
        te_stats S;
        memset(&S, 0, sizeof(S));
        S.norm_in = b < nvec ? x.beta0 : 0.0;
        S.m_used = m;
        S.restarts = x.restarts;
        S.matvecs = x.matvecs;
        S.breakdowns = x.breakdowns;
        S.quad_warnings = x.quad_warnings;
        S.quad_integrals = x.quad_integrals;
        S.quad_nodes = x.quad_nodes;
        S.eig_mcycles = 1e-6 * (double)x.eig_cycles;
        S.search_mcycles = 1e-6 * (double)x.search_cycles;
        S.err_bound = x.err_acc;
        S.roundoff_est = per_restart * (double)x.restarts;
        if (x.restarts > 0 && per_restart > x.min_err_step) S.flags |= TE_WARN_ROUNDOFF;
        if (x.breakdowns) S.flags |= TE_FLAG_BREAKDOWN;
        if (x.quad_warnings) S.flags |= TE_WARN_QUAD;
        S.t_reached = (t == 0.0) ? 0.0 : (t >= 0.0 ? 1.0 : -1.0) * x.t_now;
        S.spmv_ms = spmv_ms;
        S.spmv_launches = spmv_launches;
        stats[b] = S;
    }
    // the initial norm check reports the first bad vector of the group
    if (worst == TE_ERR_NOT_NORMALIZED)
        set_error(ctx, worst, "a vector of v_in is not normalised (| ||v|| - 1 | > 1e-10)");
    else if (worst == TE_ERR_NONFINITE)
        set_error(ctx, worst, "non-finite values in a batched solve");
    else if (worst == TE_ERR_STEP_UNDERFLOW)
        set_error(ctx, worst, "step size underflow in a batched solve");
    else if (worst == TE_ERR_UNSUPPORTED)
        set_error(ctx, worst, kSeriesRangeMsg);
    else if (worst != TE_OK)
        set_error(ctx, worst, "batched solve failed on the device");
    const double el = now_ms() - t0;
    if (stats)
        for (int b = 0; b < nvec; ++b) stats[b].solve_ms = el;
    {
        std::lock_guard<std::mutex> lk(g_block_mu);
        p->in_use = false;
    }
    return worst;
}
