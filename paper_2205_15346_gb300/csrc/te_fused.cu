// te_fused.cu -- the m Lanczos steps of one restart as one cooperative kernel,
// for small matrices.
//
// Each step of eq. arnoldi (Sec. 2.1) needs two grid-wide sums: alpha_j after
// the product and ||w~_j|| after the orthogonalisation.  As separate launches
// (K1, K2 in te_sell.cu / te_lanczos.cu) a step costs two kernel boundaries
// plus the last-block reductions, about 20 us whatever the size; below ~10^5
// rows that latency, not the FP64 pipe, sets the time of a solve.  Here every
// block stays resident for the whole loop (a cooperative launch guarantees
// it) and the two sums become grid barriers: each block publishes one partial,
// waits at the barrier, and then adds all partials itself in a fixed order, so
// every block holds the same alpha_j and beta_j without another round trip.
//
// Work split: warp g owns slices g, g + W, g + 2W, g + 3W of the sliced copy
// (W = warps in the grid, at most TE_FUSED_SLICES_PER_WARP slices per warp),
// one lane per row, in the same length-sorted basis and with the same row
// products as K1.  A lane keeps its rows of u_{j-1}, u_j and y in registers
// across the whole loop, so the orthogonalisation reads nothing from memory and
// the product gathers only the other rows of u_j (and of u_j's Re + Im) through
// L2, where the writes of other blocks are visible after the barrier.
//
// Each step computes exactly what K1 and K2 compute (the same scales, the same
// breakdown rule and the same stored vectors and sums Re + Im); only the order
// in which the grid-wide sums are added differs.
//
// The barrier never waits without bound: a block that sees no release within
// about a second, or finds the abort word set, sets the abort word and the
// solve's status (TE_ERR_TIMEOUT) and returns, and so does every other block
// at its next wait.  The words are cleared (a memset node) before each launch.
// te_fused_barrier_check runs the same barrier with one block absent, so that a
// test can see a wait that cannot complete end with that status.
#include "te_internal.cuh"
#include "te_slices.cuh"

using te_slices::FullSlices;
using te_slices::IndexedSlices;
using te_slices::RealIndexedSlices;

namespace {

constexpr int kSlices = TE_FUSED_SLICES_PER_WARP;
constexpr unsigned long long kWaitNs = 1000000000ull;   // give up after 1 s at one barrier
constexpr long long kWaitPolls = 1ll << 26;             // and after this many polls

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

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int ld_relaxed(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int* p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v)
                 : "memory");
    return old;
}

__device__ __forceinline__ void st_release(unsigned int* p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier over all blocks of the launch.  bar[0]: arrivals, bar[1]:
// generation (barriers completed), bar[2]: abort.  `gen` (thread 0 only) is the
// number of barriers this block has passed.  The arrival is a release (after
// the block barrier, it publishes the writes of every thread of the block) and
// the last arrival also an acquire; the waiters acquire the generation the last
// one releases.  Returns false in the whole block when it gave up; the caller
// then leaves the loop.
__device__ bool grid_barrier(unsigned int* bar, unsigned int& gen, int* ok_sh) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int target = gen + 1;
        int ok = 1;
        if (atom_add_acq_rel(bar, 1u) == gridDim.x - 1) {
            bar[0] = 0;                               // nobody arrives before the release
            st_release(bar + 1, target);
        } else {
            const unsigned long long t0 = global_ns();
            for (long long poll = 0;; ++poll) {
                const unsigned int g = ld_acquire(bar + 1);
                const unsigned int abort = ld_relaxed(bar + 2);
                if (g == target) break;
                if (abort != 0 || poll >= kWaitPolls || global_ns() - t0 > kWaitNs) {
                    ok = 0;
                    break;
                }
                __nanosleep(16);
            }
        }
        if (!ok) atomicExch(bar + 2, 1u);
        gen = target;
        *ok_sh = ok;
    }
    __syncthreads();
    return *ok_sh != 0;
}

// Sum of part[0..n) in a fixed order (the same in every block), broadcast to
// the block.
__device__ __forceinline__ double sum_partials(const double* part, int n, double* slot) {
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int i = threadIdx.x; i < n; i += 32) v += __ldcg(part + i);
        v = warp_sum(v);
        if (threadIdx.x == 0) *slot = v;
    }
    __syncthreads();
    return *slot;
}

// V: (m + 1) columns of length d (column 0 = u_0 on entry); S: Re + Im of each
// column; part: 2 x gridDim.x doubles; bar: 3 words, zero on entry.
template <class Slices>
__global__ void __launch_bounds__(256) k_lanczos_fused(Slices M, double2* __restrict__ V,
                                                       double* __restrict__ S, int64_t d,
                                                       int64_t nslices, DevState* st, int m,
                                                       double* part, unsigned int* bar) {
    __shared__ double sh[32];
    __shared__ double slot;
    __shared__ int ok_sh;
    // written by earlier kernels only: every block reads the same values
    if (st->status != 0 || st->done != 0 || st->stop) return;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    // test aid (TE_OPT_TEST_FUSED_TIMEOUT): the last block leaves before the first
    // barrier, so that the others' bounded wait runs out
    const bool hold = st->test_hold != 0 && blockIdx.x == gridDim.x - 1;
    const double sign = st->sign, tol_rate = st->tol_rate;
    double scale_j = st->scale[0];
    double bp = 0.0;                                  // beta[j-1] * scale[j-1]
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int G = gridDim.x;
    unsigned int gen = 0;
    double2 ucur[kSlices], uprev[kSlices], w[kSlices];
#pragma unroll
    for (int q = 0; q < kSlices; ++q) {
        const int64_t row = (warp + q * nwarps) * 32 + lane;
        ucur[q] = (row < d) ? V[row] : make_double2(0.0, 0.0);
        uprev[q] = make_double2(0.0, 0.0);
    }
    bool ok = true;
    for (int j = 0; j < m; ++j) {
        // K1: y = (sign scale_j) H u_j - bp u_{j-1}; partial of Re <u_j, y>
        const double cx = sign * scale_j;
        const double2* x = V + (size_t)j * d;
        const double* xs = S + (size_t)j * d;
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < kSlices; ++q) {
            const int64_t s = warp + q * nwarps;
            w[q] = make_double2(0.0, 0.0);
            if (s < nslices) {                        // warp-uniform
                const int64_t row = s * 32 + lane;
                const bool real_row = row < d;
                const double2 hx = M.template row<true>(s, lane, x, xs, real_row ? row : -1, ucur[q]);
                if (real_row) {
                    double2 out = make_double2(cx * hx.x, cx * hx.y);
                    if (bp != 0.0) {
                        out.x = fma(-bp, uprev[q].x, out.x);
                        out.y = fma(-bp, uprev[q].y, out.y);
                    }
                    w[q] = out;
                    acc = fma(ucur[q].x, out.x, acc);
                    acc = fma(ucur[q].y, out.y, acc);
                }
            }
        }
        double b = block_sum(acc, sh);
        if (threadIdx.x == 0) part[blockIdx.x] = b;
        if (hold) return;
        if (!grid_barrier(bar, gen, &ok_sh)) {
            ok = false;
            break;
        }
        const double a = scale_j * sum_partials(part, G, &slot);
        const double as = a * scale_j;
        if (lead) {
            st->alpha[j] = a;
            st->as_cur = as;
            st->matvecs += 1;
        }
        // K2: w~ = y - alpha_j scale_j u_j (stored with its Re + Im while a next
        // vector is needed); partial of ||w~||^2
        const bool write = j + 1 < m;
        double2* y = V + (size_t)(j + 1) * d;
        double* sy = S + (size_t)(j + 1) * d;
        double acc2 = 0.0;
#pragma unroll
        for (int q = 0; q < kSlices; ++q) {
            const int64_t row = (warp + q * nwarps) * 32 + lane;
            if (row < d) {
                double2 v = w[q];
                v.x = fma(-as, ucur[q].x, v.x);
                v.y = fma(-as, ucur[q].y, v.y);
                if (write) {
                    y[row] = v;
                    sy[row] = v.x + v.y;
                }
                acc2 = fma(v.x, v.x, acc2);
                acc2 = fma(v.y, v.y, acc2);
                w[q] = v;
            }
        }
        b = block_sum(acc2, sh);
        if (threadIdx.x == 0) part[G + blockIdx.x] = b;
        if (!grid_barrier(bar, gen, &ok_sh)) {
            ok = false;
            break;
        }
        // the breakdown rule of K2, taken by every block on the same numbers
        const double nrm = sqrt(sum_partials(part + G, G, &slot));
        if (lead) st->beta[j] = nrm;
        if (!(nrm >= tol_rate)) {                     // also catches NaN
            if (lead) {
                if (!isfinite(nrm)) st->status = TE_ERR_NONFINITE;
                st->stop = 1;
                st->m_eff = j + 1;
                st->breakdown = 1;
            }
            break;
        }
        if (j + 1 < m) {
            const double sc = 1.0 / nrm;
            if (lead) st->scale[j + 1] = sc;
            bp = nrm * scale_j;
            scale_j = sc;
#pragma unroll
            for (int q = 0; q < kSlices; ++q) {
                uprev[q] = ucur[q];
                ucur[q] = w[q];
            }
        } else if (lead) {
            st->m_eff = m;
        }
    }
    if (!ok && threadIdx.x == 0) atomicCAS(&st->status, 0, (int)TE_ERR_TIMEOUT);
}

// One grid barrier; block `absent` leaves without arriving.  passed counts the
// blocks that got through.
__global__ void k_barrier_check(unsigned int* bar, int absent, int* passed) {
    __shared__ int ok_sh;
    if ((int)blockIdx.x == absent) return;
    unsigned int gen = 0;
    const bool ok = grid_barrier(bar, gen, &ok_sh);
    if (threadIdx.x == 0 && ok) atomicAdd(passed, 1);
}

template <class Slices>
cudaError_t launch_fused(const Slices& M, double2* V, double* S, int64_t d, int64_t nslices,
                         DevState* st, int m, double* part, unsigned int* bar, int grid,
                         int threads, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_lanczos_fused<Slices>, M, V, S, d, nslices, st, m, part, bar);
}

}  // namespace

bool fused_shape(const te_matrix* H, int num_sms, int* grid, int* threads) {
    if (!H->sell_col || num_sms < 1) return false;
    const int64_t ns = H->nslices;
    if (ns < 1 || ns > (int64_t)num_sms * 8 * kSlices) return false;
    // spread the rows over as many SMs as possible, one block per SM
    const int64_t wpb = std::min<int64_t>(8, std::max<int64_t>(1, (ns + num_sms - 1) / num_sms));
    int64_t g = (ns + wpb - 1) / wpb;
    if (g > num_sms) g = num_sms;
    *grid = (int)g;
    *threads = (int)(32 * wpb);
    return true;
}

cudaError_t launch_lanczos_fused(const te_matrix* H, double2* V, double* S, DevState* st, int m,
                                 double* part, unsigned int* bar, int grid, int threads,
                                 cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bar, 0, 3 * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    if (H->sell_idx && H->dict_real) {
        const RealIndexedSlices M{H->sell_off, H->sell_col, H->sell_idx, H->dict_a, H->sell_diag};
        return launch_fused(M, V, S, H->d, H->nslices, st, m, part, bar, grid, threads, s);
    }
    if (H->sell_idx) {
        const IndexedSlices M{H->sell_off, H->sell_col, H->sell_idx, H->dict_a, H->dict_pq,
                              H->sell_diag};
        return launch_fused(M, V, S, H->d, H->nslices, st, m, part, bar, grid, threads, s);
    }
    const FullSlices M{H->sell_off, H->sell_col, H->sell_a, H->sell_pq};
    return launch_fused(M, V, S, H->d, H->nslices, st, m, part, bar, grid, threads, s);
}

extern "C" te_status te_fused_barrier_check(te_ctx* ctx, int32_t absent_block, int32_t* passed,
                                            double* ms) {
    if (!ctx || !passed) return TE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaGetLastError();
    if (!ctx->coop) return set_error(ctx, TE_ERR_UNSUPPORTED, "device without cooperative launches");
    const int grid = ctx->num_sms;
    if (absent_block >= grid) return set_error(ctx, TE_ERR_INVALID_ARG, "absent_block >= number of SMs");
    cudaStream_t s = ctx->stream;
    TE_CUDA_TRY(ctx, cudaEventRecord(ctx->user_ev, ctx->user_stream));
    TE_CUDA_TRY(ctx, cudaStreamWaitEvent(s, ctx->user_ev, 0));
    unsigned int* bar = nullptr;
    TE_CUDA_TRY(ctx, dev_alloc(ctx, &bar, 4 * sizeof(unsigned int)));
    int* cnt = reinterpret_cast<int*>(bar + 3);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3(32);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, k_barrier_check, bar, (int)absent_block, cnt);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, cnt, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(ctx, bar);
    if (e != cudaSuccess) return cuda_error(ctx, e, "te_fused_barrier_check");
    *passed = h;
    if (ms) *ms = t;
    const int expect = absent_block >= 0 ? grid - 1 : grid;
    if (h != expect) return set_error(ctx, TE_ERR_TIMEOUT, "a grid barrier gave up waiting");
    return TE_OK;
}
