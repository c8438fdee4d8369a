// te_multi.cu -- many independent solves (each its own H, v, t) advanced together.
//
// Algorithm 1 of arXiv 2205.15346 runs per problem; what a group of small and
// large problems gains from running together is that every Lanczos step of all
// of them is one launch instead of one per problem, so the small problems stop
// paying a launch latency per step and fill the GPU beside the large ones.  The
// problems keep separate Krylov spaces, states, steps and restart counts: the
// restarts run in lock step (one CUDA graph per round), each problem's state is
// updated only while it runs, and a finished problem drops out of the work.
//
// Layout: the Krylov blocks of all problems are concatenated (problem p at
// element offset elem0_p of every block), each problem in the length-sorted
// basis of its own sliced copy.  Work items:
//   * SpMV tasks (tpt_p slices of problem p), numbered problem after problem and
//     handed out by an atomic counter;
//   * element chunks (kChunkElems consecutive elements of one problem) for the
//     streaming kernels, assigned to CTAs by a fixed grid stride.
// Every reduction keeps one partial per task or chunk, and one CTA per problem
// adds the partials of its problem in order, so results do not depend on which
// warp or CTA did which item.
//
// Kernels of one Lanczos step: KM1 k_spmv_multi, KM1r k_alpha_multi, KM2
// k_orth_multi, KM2r k_decide_multi.  Per round: K3 (k_step, one CTA per
// problem), KM4 k_recombine_multi, KM4r k_beta0_multi, state copy.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>

#include "te_internal.cuh"
#include "te_slices.cuh"

using te_slices::FullSlices;
using te_slices::IndexedSlices;
using te_slices::RealIndexedSlices;

struct MProb {
    const int32_t* off;
    const int32_t* col;
    const uint16_t* vidx;      // value-indexed form (null: full-value form)
    const double* ta;
    const double2* tpq;
    const double* diag;
    const double* va;          // full-value form
    const double2* vpq;
    int64_t d;
    int64_t nslices;
    int64_t elem0;             // element offset in every concatenated block
    int32_t tpt;               // slices per SpMV task
    int32_t real;              // value-indexed form with a real table (2-DFMA product)
};

namespace {

// threads of the one-CTA-per-vector / per-problem reductions (they add up to tens of
// thousands of partials each)
constexpr int kReduceThreads = 1024;

constexpr int kChunkElems = 2048;   // elements per chunk of the streaming kernels

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

__device__ __forceinline__ double sum_range(const double* p, int64_t n, double* sh) {
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v += __ldcg(p + i);
    return block_sum(v, sh);
}

// Problem of item c: the last p with start[p] <= c (start has n + 1 entries).
__device__ __forceinline__ int owner(const int64_t* start, int n, int64_t c) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The initial normalisation (init mode of KM0 / beta0) is for problems that have
// not started: a problem that already took a restart (a request carried over
// into a new group by the serving loop) keeps its vector and scale.
__device__ __forceinline__ bool fresh_skip(const DevState* s) {
    return s->done != 0 || s->restarts != 0;
}

// A problem takes part in Lanczos step j while it runs and j is inside its
// Krylov dimension (m_p = min(m, d_p)).
__device__ __forceinline__ bool step_idle(const DevState* s, int j) {
    return s->status != 0 || s->done != 0 || s->stop != 0 || j >= s->m;
}

// ---------------------------------------------------------------- KM1

template <class Slices>
__device__ __forceinline__ double run_task(const Slices& M, int64_t s0, int64_t s1, int lane,
                                           int64_t d, const double2* __restrict__ x,
                                           const double* __restrict__ xs,
                                           const double2* __restrict__ xprev,
                                           double2* __restrict__ y, double cx, double bp) {
    double acc = 0.0;
#pragma unroll 1
    for (int64_t s = s0; s < s1; ++s) {
        const int64_t row = s * 32 + lane;
        const bool real_row = row < d;
        const double2 xr = real_row ? __ldg(x + row) : make_double2(0.0, 0.0);
        const double2 hx = M.row(s, lane, x, xs, real_row ? row : -1, xr);
        if (real_row) {
            double2 out = make_double2(cx * hx.x, cx * hx.y);
            if (bp != 0.0) {
                const double2 p = __ldcs(xprev + row);
                out.x = fma(-bp, p.x, out.x);
                out.y = fma(-bp, p.y, out.y);
            }
            y[row] = out;
            acc = fma(xr.x, out.x, acc);
            acc = fma(xr.y, out.y, acc);
        }
    }
    return acc;
}

// Lanczos step j of every running problem: y_p = s_p H_p u_p - b_p u_{p,j-1},
// one partial of Re<u_p, y_p> per task.
__global__ void __launch_bounds__(TE_BLOCK, 4) k_spmv_multi(
    const MProb* __restrict__ probs, const int64_t* __restrict__ task_start, int n,
    const double2* __restrict__ X, const double* __restrict__ S, const double2* __restrict__ Xp,
    double2* __restrict__ Y, DevState* st, int j, double* partials, unsigned int* ctr) {
    __shared__ int64_t ts[TE_MULTI_MAX + 1];
    __shared__ bool am_last;
    for (int i = threadIdx.x; i <= n; i += blockDim.x) ts[i] = task_start[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t total = ts[n];
    for (;;) {
        unsigned int c = 0;
        if (lane == 0) c = atomicAdd(&ctr[0], 1u);
        c = __shfl_sync(0xffffffffu, c, 0);
        if ((int64_t)c >= total) break;
        const int p = owner(ts, n, c);
        const DevState* sp = st + p;
        if (step_idle(sp, j)) continue;
        const double cx = sp->sign * sp->scale[j];
        const double bp = j > 0 ? sp->beta[j - 1] * sp->scale[j - 1] : 0.0;
        const MProb P = probs[p];
        const int64_t s0 = ((int64_t)c - ts[p]) * P.tpt;
        const int64_t s1 = s0 + P.tpt < P.nslices ? s0 + P.tpt : P.nslices;
        const double2* x = X + P.elem0;
        const double* xs = S + P.elem0;
        const double2* xprev = Xp ? Xp + P.elem0 : nullptr;
        double2* y = Y + P.elem0;
        double acc;
        if (P.vidx && P.real) {
            const RealIndexedSlices M{P.off, P.col, P.vidx, P.ta, P.diag};
            acc = run_task(M, s0, s1, lane, P.d, x, xs, xprev, y, cx, bp);
        } else if (P.vidx) {
            const IndexedSlices M{P.off, P.col, P.vidx, P.ta, P.tpq, P.diag};
            acc = run_task(M, s0, s1, lane, P.d, x, xs, xprev, y, cx, bp);
        } else {
            const FullSlices M{P.off, P.col, P.va, P.vpq};
            acc = run_task(M, s0, s1, lane, P.d, x, xs, xprev, y, cx, bp);
        }
        acc = warp_sum(acc);
        if (lane == 0) partials[c] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        am_last = (atomicAdd(&ctr[1], 1u) == gridDim.x - 1);
        if (am_last) {
            ctr[0] = 0;
            ctr[1] = 0;
        }
    }
}

// KM1r: alpha_p = scale_p[j]^2 Re<u_p, y_p> (one CTA per problem).
__global__ void __launch_bounds__(kReduceThreads) k_alpha_multi(DevState* st, const int64_t* task_start,
                                                          const double* partials, int j) {
    __shared__ double sh[32];
    DevState* sp = st + blockIdx.x;
    if (step_idle(sp, j)) return;
    const int64_t t0 = task_start[blockIdx.x];
    const double tot = sum_range(partials + t0, task_start[blockIdx.x + 1] - t0, sh);
    if (threadIdx.x == 0) {
        const double a = sp->scale[j] * tot;
        sp->alpha[j] = a;
        sp->as_cur = a * sp->scale[j];
        sp->matvecs += 1;
    }
}

// ---------------------------------------------------------------- KM2 / KM2r

// w = y - as_p u (in place, when the vector is needed), s = Re w + Im w,
// ||w||^2 partial per chunk.
__global__ void __launch_bounds__(TE_BLOCK) k_orth_multi(
    const MProb* __restrict__ probs, const int64_t* __restrict__ chunk_start, int n,
    double2* __restrict__ W, const double2* __restrict__ U, double* __restrict__ S,
    const DevState* st, int j, double* partials) {
    __shared__ int64_t cs[TE_MULTI_MAX + 1];
    __shared__ double sh[32];
    for (int i = threadIdx.x; i <= n; i += blockDim.x) cs[i] = chunk_start[i];
    __syncthreads();
    const int64_t total = cs[n];
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        const int p = owner(cs, n, g);
        const DevState* sp = st + p;
        if (step_idle(sp, j)) continue;                  // uniform over the CTA
        const double as = sp->as_cur;
        const bool write = j + 1 < sp->m;
        const int64_t e0 = probs[p].elem0, d = probs[p].d;
        const int64_t b = e0 + (g - cs[p]) * kChunkElems;
        const int64_t e = b + kChunkElems < e0 + d ? b + kChunkElems : e0 + d;
        double acc = 0.0;
        for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
            double2 y = W[i];
            const double2 u = __ldcs(U + i);
            y.x = fma(-as, u.x, y.x);
            y.y = fma(-as, u.y, y.y);
            if (write) {
                W[i] = y;
                S[i] = y.x + y.y;
            }
            acc = fma(y.x, y.x, acc);
            acc = fma(y.y, y.y, acc);
        }
        const double tot = block_sum(acc, sh);
        if (threadIdx.x == 0) partials[g] = tot;
    }
}

// KM2r: h_{j+1,j} of problem p, its breakdown test (Algorithm 1 step 1) and
// scale_p[j+1].
__global__ void __launch_bounds__(kReduceThreads) k_decide_multi(DevState* st, const int64_t* chunk_start,
                                                           const double* partials, int j) {
    __shared__ double sh[32];
    DevState* sp = st + blockIdx.x;
    if (step_idle(sp, j)) return;
    const int64_t c0 = chunk_start[blockIdx.x];
    const double nrm = sqrt(sum_range(partials + c0, chunk_start[blockIdx.x + 1] - c0, sh));
    if (threadIdx.x == 0) {
        sp->beta[j] = nrm;
        if (!(nrm >= sp->tol_rate)) {        // also catches NaN
            if (!isfinite(nrm)) sp->status = TE_ERR_NONFINITE;
            sp->stop = 1;
            sp->m_eff = j + 1;
            sp->breakdown = 1;
        } else if (j + 1 < sp->m) {
            sp->scale[j + 1] = 1.0 / nrm;
        } else {
            sp->m_eff = sp->m;
        }
    }
}

// ---------------------------------------------------------------- KM0 / KM4 / beta0

// init: ||v||^2 (and a non-finite marker) per chunk of the initial block, s = Re + Im.
// Otherwise w_p = sum_{k < m_eff} coef_p[k] u_{p,k} into block 0 for the problems
// whose step kernel took a step (Algorithm 1 step 3), s, ||w||^2 per chunk.
__global__ void __launch_bounds__(TE_BLOCK) k_recombine_multi(
    const MProb* __restrict__ probs, const int64_t* __restrict__ chunk_start, int n,
    double2* __restrict__ V, double* __restrict__ S, int64_t blk, const DevState* st, int init,
    double* partials) {
    __shared__ int64_t cs[TE_MULTI_MAX + 1];
    __shared__ double sh[32];
    __shared__ double2 c[TE_M_MAX];
    for (int i = threadIdx.x; i <= n; i += blockDim.x) cs[i] = chunk_start[i];
    __syncthreads();
    const int64_t total = cs[n];
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        const int p = owner(cs, n, g);
        const DevState* sp = st + p;
        if (init ? fresh_skip(sp) : (sp->active == 0 || sp->status != 0)) continue;
        const int nk = init ? 0 : sp->last_m_eff;
        __syncthreads();                                // c[] of the previous chunk is consumed
        for (int k = threadIdx.x; k < nk; k += blockDim.x) c[k] = sp->coef[k];
        __syncthreads();
        const int64_t e0 = probs[p].elem0, d = probs[p].d;
        const int64_t b = e0 + (g - cs[p]) * kChunkElems;
        const int64_t e = b + kChunkElems < e0 + d ? b + kChunkElems : e0 + d;
        double acc = 0.0;
        bool finite = true;
        for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
            double re, im;
            if (init) {
                const double2 v = V[i];
                re = v.x;
                im = v.y;
                finite &= isfinite(re) && isfinite(im);
            } else {
                re = 0.0;
                im = 0.0;
                for (int k = 0; k < nk; ++k) {
                    const double2 a = __ldcs(V + (size_t)k * blk + i);
                    re = fma(c[k].x, a.x, re);
                    re = fma(-c[k].y, a.y, re);
                    im = fma(c[k].x, a.y, im);
                    im = fma(c[k].y, a.x, im);
                }
                V[i] = make_double2(re, im);
            }
            S[i] = re + im;
            acc = fma(re, re, acc);
            acc = fma(im, im, acc);
        }
        if (!finite) acc = __longlong_as_double(0x7ff8000000000000LL);
        const double tot = block_sum(acc, sh);
        if (threadIdx.x == 0) partials[g] = tot;
    }
}

// beta0_p = ||w_p|| opens problem p's next Krylov space (init: validation of
// v_in, Sec. 2.1 assumes ||v(0)|| = 1).
__global__ void __launch_bounds__(kReduceThreads) k_beta0_multi(DevState* st, const int64_t* chunk_start,
                                                          const double* partials, int init) {
    __shared__ double sh[32];
    DevState* sp = st + blockIdx.x;
    if (init ? fresh_skip(sp) : (sp->active == 0 || sp->status != 0)) return;
    const int64_t c0 = chunk_start[blockIdx.x];
    const double nrm = sqrt(sum_range(partials + c0, chunk_start[blockIdx.x + 1] - c0, sh));
    if (threadIdx.x == 0) {
        sp->beta0 = nrm;
        sp->scale[0] = 1.0 / nrm;
        sp->stop = 0;
        sp->m_eff = sp->m;
        sp->breakdown = 0;
        sp->active = 0;
        if (!isfinite(nrm)) sp->status = TE_ERR_NONFINITE;
        else if (init && fabs(nrm - 1.0) > 1e-10) sp->status = TE_ERR_NOT_NORMALIZED;
        if (init && sp->T == 0.0) sp->done = 1;       // t = 0: validated, nothing to evolve
    }
}

// The state of a problem before its first restart (constants of the solve).
void initial_state(DevState* x, double t, double tol, int m, const te_options& o) {
    memset(x, 0, sizeof(DevState));
    double gx[TE_GAUSS_MAX], gw[TE_GAUSS_MAX];
    gauss_legendre_table(o.gauss_n, gx, gw);
    x->T = fabs(t);
    x->tol_rate = (t != 0.0) ? tol / fabs(t) : tol;      // eq. errorRate
    x->sign = (t >= 0.0) ? 1.0 : -1.0;
    x->t_step0 = o.t_step0;
    x->shrink = o.shrink;
    x->quad_rel_tol = o.quad_rel_tol;
    x->min_step = o.min_step_rel * fabs(t);
    x->m = m;
    x->n_substeps = o.n_substeps;
    x->quad = o.quad;
    x->gauss_n = o.gauss_n;
    x->quad_max_levels = o.quad_max_levels;
    x->max_substeps = o.max_substeps;
    x->smallexp = o.small_exp;
    x->first = 1;
    x->m_eff = m;
    x->min_err_step = INFINITY;
    memcpy(x->gx, gx, sizeof(gx));
    memcpy(x->gw, gw, sizeof(gw));
}

// te_stats of a finished problem from its device state.
te_stats stats_from_state(const DevState& x, const te_matrix* H, double t) {
    const double per_restart = (double)H->d * H->norm1 * 2.220446049250313e-16;
    te_stats S;
    memset(&S, 0, sizeof(S));
    S.norm_in = x.beta0;
    S.m_used = x.m;
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
    return S;
}

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

// ------------------------------------------------------------------ engine

struct MultiPlan {
    te_ctx* ctx = nullptr;
    std::vector<uint64_t> ids;      // matrix of each problem
    int m = 0, n = 0, profile = 0;
    int64_t dsum = 0;
    int64_t ntasks = 0, nchunks = 0;
    int grid_spmv = 0, grid_stream = 0;
    std::vector<int64_t> elem0;     // host copy of the element offsets
    double2* V = nullptr;           // (m + 1) concatenated blocks of dsum elements
    double* S = nullptr;
    double* partials = nullptr;
    DevState* st = nullptr;
    DevState* st_host = nullptr;
    DevState* st_init = nullptr;
    MProb* probs = nullptr;
    int64_t* task_start = nullptr;
    int64_t* chunk_start = nullptr;
    unsigned int* ctr = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> ev;
    bool in_use = false;
};

namespace {

std::mutex g_multi_mu;
std::vector<MultiPlan*> g_multi_plans;

void free_multi_plan(MultiPlan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
    for (void* q : {(void*)p->V, (void*)p->S, (void*)p->partials, (void*)p->st, (void*)p->probs,
                    (void*)p->task_start, (void*)p->chunk_start, (void*)p->ctr})
        if (q) dev_free(p->ctx, q);
    if (p->st_host) cudaFreeHost(p->st_host);
    if (p->st_init) cudaFreeHost(p->st_init);
    delete p;
}

te_status capture_multi_round(te_ctx* ctx, MultiPlan* p, cudaStream_t s) {
    const int64_t blk = p->dsum;
    const int m = p->m, n = p->n;
    TE_CUDA_TRY(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < m && e == cudaSuccess; ++j) {
        const double2* X = p->V + (size_t)j * blk;
        const double2* Xp = j > 0 ? p->V + (size_t)(j - 1) * blk : nullptr;
        double2* Y = p->V + (size_t)(j + 1) * blk;
        const bool timed = p->profile && j == m / 2;     // one product per round is timed
        if (timed) e = cudaEventRecordWithFlags(p->ev[0], s, cudaEventRecordExternal);
        if (e != cudaSuccess) break;
        k_spmv_multi<<<p->grid_spmv, TE_BLOCK, 0, s>>>(p->probs, p->task_start, n, X, p->S, Xp, Y,
                                                      p->st, j, p->partials, p->ctr);
        if (timed) e = cudaEventRecordWithFlags(p->ev[1], s, cudaEventRecordExternal);
        if (e != cudaSuccess) break;
        k_alpha_multi<<<n, kReduceThreads, 0, s>>>(p->st, p->task_start, p->partials, j);
        k_orth_multi<<<p->grid_stream, TE_BLOCK, 0, s>>>(p->probs, p->chunk_start, n, Y, X, p->S,
                                                         p->st, j, p->partials);
        k_decide_multi<<<n, kReduceThreads, 0, s>>>(p->st, p->chunk_start, p->partials, j);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_step_batch(p->st, n, m, s);
    if (e == cudaSuccess) {
        k_recombine_multi<<<p->grid_stream, TE_BLOCK, 0, s>>>(p->probs, p->chunk_start, n, p->V,
                                                              p->S, blk, p->st, 0, p->partials);
        k_beta0_multi<<<n, kReduceThreads, 0, s>>>(p->st, p->chunk_start, p->partials, 0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->st_host, p->st, sizeof(DevState) * n, cudaMemcpyDeviceToHost, s);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_error(ctx, e, "capturing the grouped restart graph");
    }
    if (e2 != cudaSuccess) return cuda_error(ctx, e2, "cudaStreamEndCapture");
    cudaError_t e3 = cudaGraphInstantiate(&p->exec, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return cuda_error(ctx, e3, "cudaGraphInstantiate (grouped restart)");
    return TE_OK;
}

te_status create_multi_plan(te_ctx* ctx, int n, const te_matrix* const* H, int m, int profile,
                            cudaStream_t s, MultiPlan** out) {
    MultiPlan* p = new MultiPlan();
    p->ctx = ctx;
    p->m = m;
    p->n = n;
    p->profile = profile;
    std::vector<MProb> hp(n);
    std::vector<int64_t> ts(n + 1, 0), cs(n + 1, 0);
    int64_t off = 0;
    for (int i = 0; i < n; ++i) {
        const te_matrix* A = H[i];
        p->ids.push_back(A->id);
        MProb& q = hp[i];
        memset(&q, 0, sizeof(q));
        q.off = A->sell_off;
        q.col = A->sell_col;
        q.vidx = A->sell_idx;
        q.ta = A->dict_a;
        q.tpq = A->dict_pq;
        q.diag = A->sell_diag;
        q.va = A->sell_a;
        q.vpq = A->sell_pq;
        q.d = A->d;
        q.nslices = A->nslices;
        q.tpt = A->sell_tpt;
        q.real = A->dict_real ? 1 : 0;
        q.elem0 = off;
        p->elem0.push_back(off);
        // keep every problem's segment 16-byte aligned and a whole number of slices
        off += (A->d + 31) / 32 * 32;
        ts[i + 1] = ts[i] + (A->nslices + A->sell_tpt - 1) / A->sell_tpt;
        cs[i + 1] = cs[i] + (A->d + kChunkElems - 1) / kChunkElems;
    }
    p->dsum = off;
    p->ntasks = ts[n];
    p->nchunks = cs[n];
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv_multi, TE_BLOCK, 0);
    p->grid_spmv = (int)std::max<int64_t>(1, std::min<int64_t>((p->ntasks + 7) / 8,
                                                                (int64_t)std::max(occ, 1) * ctx->num_sms));
    p->grid_stream = (int)std::max<int64_t>(1, std::min<int64_t>(p->nchunks, (int64_t)ctx->num_sms * 8));
    const size_t npart = (size_t)std::max(p->ntasks, p->nchunks);
    cudaError_t e = dev_alloc(ctx, &p->V, sizeof(double2) * (size_t)(m + 1) * (size_t)p->dsum);
    if (e == cudaSuccess) e = dev_alloc(ctx, &p->S, sizeof(double) * (size_t)p->dsum);
    if (e == cudaSuccess) e = dev_alloc(ctx, &p->partials, sizeof(double) * npart);
    if (e == cudaSuccess) e = dev_alloc(ctx, &p->st, sizeof(DevState) * n);
    if (e == cudaSuccess) e = dev_alloc(ctx, &p->probs, sizeof(MProb) * n);
    if (e == cudaSuccess) e = dev_alloc(ctx, &p->task_start, sizeof(int64_t) * (n + 1));
    if (e == cudaSuccess) e = dev_alloc(ctx, &p->chunk_start, sizeof(int64_t) * (n + 1));
    if (e == cudaSuccess) e = dev_alloc(ctx, &p->ctr, sizeof(unsigned int) * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&p->st_host, sizeof(DevState) * n);
    if (e == cudaSuccess) e = cudaMallocHost(&p->st_init, sizeof(DevState) * n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->probs, hp.data(), sizeof(MProb) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->task_start, ts.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->chunk_start, cs.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->ctr, 0, sizeof(unsigned int) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->st, 0, sizeof(DevState) * n, s);
    // the gaps between segments are never written: keep them at zero
    if (e == cudaSuccess) e = cudaMemsetAsync(p->S, 0, sizeof(double) * (size_t)p->dsum, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_multi_plan(p);
        return set_error(ctx, e == cudaErrorMemoryAllocation ? TE_ERR_OOM : TE_ERR_CUDA,
                         std::string("allocating the grouped workspace: ") + cudaGetErrorString(e));
    }
    if (profile) {
        p->ev.resize(2);
        for (auto& ev : p->ev) cudaEventCreate(&ev);
    }
    te_status st = capture_multi_round(ctx, p, s);
    if (st) {
        free_multi_plan(p);
        return st;
    }
    *out = p;
    return TE_OK;
}

te_status acquire_multi_plan(te_ctx* ctx, int n, const te_matrix* const* H, int m, int profile,
                             cudaStream_t s, MultiPlan** out) {
    {
        std::lock_guard<std::mutex> lk(g_multi_mu);
        for (MultiPlan* p : g_multi_plans) {
            if (p->ctx != ctx || p->in_use || p->n != n || p->m != m || p->profile != profile) continue;
            bool same = true;
            for (int i = 0; i < n && same; ++i) same = p->ids[i] == H[i]->id;
            if (!same) continue;
            p->in_use = true;
            *out = p;
            return TE_OK;
        }
    }
    MultiPlan* p = nullptr;
    te_status st = create_multi_plan(ctx, n, H, m, profile, s, &p);
    if (st == TE_ERR_OOM) {
        std::vector<MultiPlan*> idle;
        {
            std::lock_guard<std::mutex> lk(g_multi_mu);
            auto it = std::partition(g_multi_plans.begin(), g_multi_plans.end(),
                                     [&](MultiPlan* q) { return q->ctx != ctx || q->in_use; });
            idle.assign(it, g_multi_plans.end());
            g_multi_plans.erase(it, g_multi_plans.end());
        }
        cudaStreamSynchronize(s);
        for (MultiPlan* q : idle) free_multi_plan(q);
        st = create_multi_plan(ctx, n, H, m, profile, s, &p);
    }
    if (st) return st;
    p->in_use = true;
    std::lock_guard<std::mutex> lk(g_multi_mu);
    g_multi_plans.push_back(p);
    *out = p;
    return TE_OK;
}

}  // namespace

// A grouped solve that uses the matrix is running.
bool multi_plans_in_use(te_ctx* ctx, uint64_t matrix_id) {
    std::lock_guard<std::mutex> lk(g_multi_mu);
    for (MultiPlan* q : g_multi_plans)
        if (q->ctx == ctx && q->in_use &&
            std::find(q->ids.begin(), q->ids.end(), matrix_id) != q->ids.end())
            return true;
    return false;
}

// Drop the grouped plans of a context (matrix_id 0) or those that use one matrix.
void multi_plans_release(te_ctx* ctx, uint64_t matrix_id) {
    std::vector<MultiPlan*> drop;
    {
        std::lock_guard<std::mutex> lk(g_multi_mu);
        auto it = std::partition(g_multi_plans.begin(), g_multi_plans.end(), [&](MultiPlan* q) {
            if (q->ctx != ctx) return true;
            if (matrix_id == 0) return false;
            return std::find(q->ids.begin(), q->ids.end(), matrix_id) == q->ids.end();
        });
        drop.assign(it, g_multi_plans.end());
        g_multi_plans.erase(it, g_multi_plans.end());
    }
    for (MultiPlan* p : drop) free_multi_plan(p);
}

// One group of n <= TE_MULTI_MAX problems.
te_status run_multi_solve(te_ctx* ctx, int n, const te_matrix* const* H, const double* const* v_in,
                          const double* t, double tol, int m, const te_options& o,
                          double* const* v_out, bool dev, te_stats* stats, int32_t* status,
                          cudaStream_t s) {
    const double t0 = now_ms();
    const int profile = (o.flags & TE_OPT_PROFILE) ? 1 : 0;
    MultiPlan* p = nullptr;
    te_status rs = acquire_multi_plan(ctx, n, H, m, profile, s, &p);
    if (rs) return rs;
    auto release = [&]() {
        std::lock_guard<std::mutex> lk(g_multi_mu);
        p->in_use = false;
    };
    auto fail = [&](cudaError_t e, const char* what) {
        release();
        return cuda_error(ctx, e, what);
    };
    DevState* ini = p->st_init;
    for (int i = 0; i < n; ++i)
        initial_state(&ini[i], t[i], tol, (int)std::min<int64_t>(m, H[i]->d), o);
    const int64_t blk = p->dsum;
    double2* stage = p->V + (size_t)m * (size_t)blk;   // the last block is free outside a round
    cudaError_t e = cudaMemcpyAsync(p->st, ini, sizeof(DevState) * n, cudaMemcpyHostToDevice, s);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const int64_t d = H[i]->d;
        double2* seg = p->V + p->elem0[i];
        const double2* src = (const double2*)v_in[i];
        if (!dev) {
            e = cudaMemcpyAsync(stage + p->elem0[i], v_in[i], sizeof(double2) * d,
                                cudaMemcpyHostToDevice, s);
            src = stage + p->elem0[i];
        }
        if (e == cudaSuccess)
            e = launch_gather(src, H[i]->perm, d, seg, p->S + p->elem0[i], ctx->num_sms, s);
    }
    if (e == cudaSuccess) {
        k_recombine_multi<<<p->grid_stream, TE_BLOCK, 0, s>>>(p->probs, p->chunk_start, n, p->V,
                                                              p->S, blk, p->st, 1, p->partials);
        k_beta0_multi<<<n, kReduceThreads, 0, s>>>(p->st, p->chunk_start, p->partials, 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->st_host, p->st, sizeof(DevState) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(e, "starting the grouped solve");
    const DevState* h = p->st_host;
    double spmv_ms = 0.0;
    int64_t spmv_launches = 0, rounds = 0;
    auto running = [&]() {
        for (int i = 0; i < n; ++i)
            if (h[i].status == 0 && h[i].done == 0 && t[i] != 0.0) return true;
        return false;
    };
    while (running()) {
        e = cudaGraphLaunch(p->exec, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(e, "grouped restart round");
        ++rounds;
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
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const int64_t d = H[i]->d;
        const double2* seg = p->V + p->elem0[i];
        if (dev) {
            e = launch_gather(seg, H[i]->iperm, d, (double2*)v_out[i], nullptr, ctx->num_sms, s);
        } else {
            e = launch_gather(seg, H[i]->iperm, d, stage + p->elem0[i], nullptr, ctx->num_sms, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(v_out[i], stage + p->elem0[i], sizeof(double2) * d,
                                    cudaMemcpyDeviceToHost, s);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(e, "returning the grouped results");
    te_status worst = TE_OK;
    const double el = now_ms() - t0;
    for (int i = 0; i < n; ++i) {
        const DevState& x = h[i];
        const te_status si = x.status;
        if (status) status[i] = si;
        if (si != TE_OK && worst == TE_OK) worst = si;
        if (!stats) continue;
        te_stats S = stats_from_state(x, H[i], t[i]);
        S.spmv_ms = spmv_ms;
        S.spmv_launches = spmv_launches;
        S.solve_ms = el;
        stats[i] = S;
    }
    if (worst == TE_ERR_NOT_NORMALIZED)
        set_error(ctx, worst, "an input vector is not normalised (| ||v|| - 1 | > 1e-10)");
    else if (worst == TE_ERR_NONFINITE)
        set_error(ctx, worst, "non-finite values in a grouped solve");
    else if (worst == TE_ERR_STEP_UNDERFLOW)
        set_error(ctx, worst, "step size underflow in a grouped solve");
    else if (worst == TE_ERR_UNSUPPORTED)
        set_error(ctx, worst, kSeriesRangeMsg);
    else if (worst != TE_OK)
        set_error(ctx, worst, "grouped solve failed on the device");
    release();
    (void)rounds;
    return worst;
}

// ------------------------------------------------------------------ continuous batching
//
// The serving loop behind te_submit.  Algorithm 1's restart boundary (a state is
// fully described by the vector w and a few scalars once step 3 has formed w) is
// the checkpoint at which requests join and leave: every running request takes
// part in each round (one restart of all of them through the grouped kernels of
// this file, one captured graph per composition), a queued request is admitted
// at the next round boundary as soon as a slot of the Krylov arena is free, and
// a finished request leaves at the end of its round.  The arena holds the
// (m_max + 1) Krylov columns of every slot at a fixed column stride, so a
// request keeps its place while others come and go; admission by HBM footprint
// is admission by free arena space.

namespace {

struct ServeSlot {
    te_request* r = nullptr;
    int64_t elem0 = 0, seg = 0;     // arena segment
    int idx = -1;                   // position in the captured composition (-1: new)
    double t_admit = 0.0;
};

struct ServeEngine {
    te_ctx* ctx = nullptr;
    cudaStream_t s = nullptr;
    int depth = 0;                  // Krylov dimension of the arena
    int64_t cap = 0;                // elements per Krylov column
    size_t npart = 0;
    size_t bytes = 0;
    double2* V = nullptr;
    double* S = nullptr;
    double* partials = nullptr;
    DevState* st = nullptr;
    DevState* st_host = nullptr;
    DevState* st_init = nullptr;
    MProb* probs = nullptr;
    int64_t* task_start = nullptr;
    int64_t* chunk_start = nullptr;
    unsigned int* ctr = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<ServeSlot> slots;   // running requests, in composition order
    std::vector<std::pair<int64_t, int64_t>> holes;   // free arena segments (offset, length)
    bool dirty = true;              // composition changed since the last capture

    int cls = 0;                    // 0: small batch, 1: medium batch

    te_status init(te_ctx* c, int m_max, int64_t capacity, int cls_) {
        ctx = c;
        cls = cls_;
        depth = m_max;
        cap = capacity / 32 * 32;
        npart = (size_t)(cap / 32 + 2 * TE_MULTI_MAX + 1);
        int lo = 0, hi = 0;              // small batch: the highest priority; medium: the lowest
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        const int prio = cls == 0 ? hi : lo;
        cudaError_t e = cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio);
        if (e == cudaSuccess) e = dev_alloc(ctx, &V, sizeof(double2) * (size_t)(depth + 1) * (size_t)cap);
        if (e == cudaSuccess) e = dev_alloc(ctx, &S, sizeof(double) * (size_t)cap);
        if (e == cudaSuccess) e = dev_alloc(ctx, &partials, sizeof(double) * npart);
        if (e == cudaSuccess) e = dev_alloc(ctx, &st, sizeof(DevState) * TE_MULTI_MAX);
        if (e == cudaSuccess) e = dev_alloc(ctx, &probs, sizeof(MProb) * TE_MULTI_MAX);
        if (e == cudaSuccess) e = dev_alloc(ctx, &task_start, sizeof(int64_t) * (TE_MULTI_MAX + 1));
        if (e == cudaSuccess) e = dev_alloc(ctx, &chunk_start, sizeof(int64_t) * (TE_MULTI_MAX + 1));
        if (e == cudaSuccess) e = dev_alloc(ctx, &ctr, sizeof(unsigned int) * 4);
        if (e == cudaSuccess) e = cudaMallocHost(&st_host, sizeof(DevState) * TE_MULTI_MAX);
        if (e == cudaSuccess) e = cudaMallocHost(&st_init, sizeof(DevState) * TE_MULTI_MAX);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctr, 0, sizeof(unsigned int) * 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(S, 0, sizeof(double) * (size_t)cap, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(ctx, e == cudaErrorMemoryAllocation ? TE_ERR_OOM : TE_ERR_CUDA,
                             std::string("allocating the serving arena: ") + cudaGetErrorString(e));
        }
        bytes = sizeof(double2) * (size_t)(depth + 1) * (size_t)cap + sizeof(double) * ((size_t)cap + npart);
        holes.push_back({0, cap});
        return TE_OK;
    }

    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        for (void* q : {(void*)V, (void*)S, (void*)partials, (void*)st, (void*)probs,
                        (void*)task_start, (void*)chunk_start, (void*)ctr})
            if (q) dev_free(ctx, q);
        if (st_host) cudaFreeHost(st_host);
        if (st_init) cudaFreeHost(st_init);
        if (s) cudaStreamDestroy(s);
        V = nullptr;
        S = nullptr;
        st_host = st_init = nullptr;
        s = nullptr;
    }

    // first-fit arena segment of `len` elements (-1: none)
    int64_t take(int64_t len) {
        for (size_t i = 0; i < holes.size(); ++i) {
            if (holes[i].second < len) continue;
            const int64_t off = holes[i].first;
            holes[i].first += len;
            holes[i].second -= len;
            if (holes[i].second == 0) holes.erase(holes.begin() + (long)i);
            return off;
        }
        return -1;
    }

    void give(int64_t off, int64_t len) {
        holes.push_back({off, len});
        std::sort(holes.begin(), holes.end());
        std::vector<std::pair<int64_t, int64_t>> merged;
        for (auto& h : holes) {
            if (!merged.empty() && merged.back().first + merged.back().second == h.first)
                merged.back().second += h.second;
            else
                merged.push_back(h);
        }
        holes.swap(merged);
    }
};

// Tables, states and graph of the current composition; new slots are started
// (vector gathered into the arena in the matrix's sorted basis, normalisation
// checked).  Carried slots keep their arena columns and continue from their
// state of the last round.
te_status serve_compose(ServeEngine& E) {
    te_ctx* ctx = E.ctx;
    const int n = (int)E.slots.size();
    std::vector<MProb> hp(n);
    std::vector<int64_t> ts(n + 1, 0), cs(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        const te_matrix* A = E.slots[i].r->H;
        MProb& q = hp[i];
        memset(&q, 0, sizeof(q));
        q.off = A->sell_off;
        q.col = A->sell_col;
        q.vidx = A->sell_idx;
        q.ta = A->dict_a;
        q.tpq = A->dict_pq;
        q.diag = A->sell_diag;
        q.va = A->sell_a;
        q.vpq = A->sell_pq;
        q.d = A->d;
        q.nslices = A->nslices;
        q.tpt = A->sell_tpt;
        q.real = A->dict_real ? 1 : 0;
        q.elem0 = E.slots[i].elem0;
        ts[i + 1] = ts[i] + (A->nslices + A->sell_tpt - 1) / A->sell_tpt;
        cs[i + 1] = cs[i] + (A->d + kChunkElems - 1) / kChunkElems;
        const ServeSlot& sl = E.slots[i];
        if (sl.idx >= 0) {
            E.st_init[i] = E.st_host[sl.idx];
        } else {
            const te_request* r = sl.r;
            initial_state(&E.st_init[i], r->t, r->tol, r->m, r->opt);
        }
    }
    cudaStream_t s = E.s;
    cudaError_t e = cudaMemcpyAsync(E.probs, hp.data(), sizeof(MProb) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(E.task_start, ts.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(E.chunk_start, cs.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(E.st, E.st_init, sizeof(DevState) * n, cudaMemcpyHostToDevice, s);
    bool fresh = false;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        ServeSlot& sl = E.slots[i];
        if (sl.idx >= 0) continue;
        fresh = true;
        e = launch_gather((const double2*)sl.r->v_in_dev, sl.r->H->perm, sl.r->H->d, E.V + sl.elem0,
                          E.S + sl.elem0, ctx->num_sms, s);
    }
    int grid_stream = (int)std::max<int64_t>(1, std::min<int64_t>(cs[n], (int64_t)ctx->num_sms * 8));
    if (e == cudaSuccess && fresh) {
        k_recombine_multi<<<grid_stream, TE_BLOCK, 0, s>>>(E.probs, E.chunk_start, n, E.V, E.S, E.cap,
                                                           E.st, 1, E.partials);
        k_beta0_multi<<<n, kReduceThreads, 0, s>>>(E.st, E.chunk_start, E.partials, 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(E.st_host, E.st, sizeof(DevState) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(ctx, e, "starting a serving round");
    for (int i = 0; i < n; ++i) E.slots[i].idx = i;
    // the round graph of this composition
    if (E.exec) cudaGraphExecDestroy(E.exec);
    E.exec = nullptr;
    MultiPlan mp;
    mp.ctx = ctx;
    mp.m = E.depth;
    mp.n = n;
    mp.dsum = E.cap;
    mp.ntasks = ts[n];
    mp.nchunks = cs[n];
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv_multi, TE_BLOCK, 0);
    // the medium batch's grouped SpMV (its blocks stay resident for the whole
    // product) leaves one block slot per SM to the small batch
    if (E.cls == 1 && occ >= 2) occ -= 1;
    mp.grid_spmv = (int)std::max<int64_t>(1, std::min<int64_t>((mp.ntasks + 7) / 8,
                                                                (int64_t)std::max(occ, 1) * ctx->num_sms));
    mp.grid_stream = grid_stream;
    mp.V = E.V;
    mp.S = E.S;
    mp.partials = E.partials;
    mp.st = E.st;
    mp.st_host = E.st_host;
    mp.probs = E.probs;
    mp.task_start = E.task_start;
    mp.chunk_start = E.chunk_start;
    mp.ctr = E.ctr;
    te_status cst = capture_multi_round(ctx, &mp, s);
    E.exec = mp.exec;
    mp.exec = nullptr;
    E.dirty = false;
    return cst;
}

// Publish a request's outcome (the vector is already in r->v_out_dev when ok).
void serve_publish(te_request* r, te_status res, const te_stats& S, const std::string& msg) {
    {
        std::lock_guard<std::mutex> lk(r->ctx->qmu);
        r->ctx->pending -= 1;
    }
    {
        // notified under the lock: r is not touched after it is released (its owner
        // may free it then)
        std::lock_guard<std::mutex> lk(r->mu);
        r->stats = S;
        r->result = res;
        r->err = msg;
        r->state.store(2);
        r->cv.notify_all();
    }
}

// Finished or failed slot i: its result leaves the arena (back to the caller's
// basis) and the slot is released.
void serve_finish(ServeEngine& E, size_t i, te_status res, const std::string& msg) {
    ServeSlot sl = E.slots[i];
    te_request* r = sl.r;
    te_stats S;
    memset(&S, 0, sizeof(S));
    if (sl.idx >= 0) S = stats_from_state(E.st_host[sl.idx], r->H, r->t);
    if (res == TE_OK || res == TE_ERR_STEP_UNDERFLOW) {
        cudaError_t e = launch_gather(E.V + sl.elem0, r->H->iperm, r->H->d, (double2*)r->v_out_dev,
                                      nullptr, E.ctx->num_sms, E.s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(E.s);
        if (e != cudaSuccess) {
            res = TE_ERR_CUDA;
            cudaGetLastError();
        }
    }
    S.solve_ms = now_ms() - sl.t_admit;
    E.slots.erase(E.slots.begin() + (long)i);
    E.give(sl.elem0, sl.seg);
    E.dirty = true;
    serve_publish(r, res, S, msg);
}

const char* device_status_msg(te_status s) {
    switch (s) {
        case TE_ERR_NOT_NORMALIZED: return "the request vector is not normalised (| ||v|| - 1 | > 1e-10)";
        case TE_ERR_NONFINITE: return "non-finite values in the request";
        case TE_ERR_STEP_UNDERFLOW: return "step size underflow: no step meets the error rate";
        case TE_ERR_UNSUPPORTED: return kSeriesRangeMsg;
        default: return "the request failed on the device";
    }
}

}  // namespace

// The small batch's arena holds a quarter of the medium one's columns.
int64_t serve_class_capacity(const te_ctx* ctx, int cls) {
    return cls == 0 ? std::max<int64_t>(32, ctx->serve_cap / 4 / 32 * 32) : ctx->serve_cap;
}

int serve_class(const te_ctx* ctx, const te_request* r) {
    const bool batchable = ctx->serve_mode == TE_SERVE_BATCH && r->opt.reorth == TE_REORTH_NONE &&
                           r->opt.spmv_lanes == 0 && !(r->opt.flags & TE_OPT_PROFILE) &&
                           r->m <= ctx->serve_m && r->H->sell_off != nullptr;
    if (!batchable) return -1;
    if (ctx->serve_large_nnz > 0 && r->H->nnz >= ctx->serve_large_nnz) return -1;
    const int64_t seg = (r->H->d + 31) / 32 * 32;
    if (r->H->nnz < ctx->serve_small_nnz && seg <= serve_class_capacity(ctx, 0)) return 0;
    return seg <= serve_class_capacity(ctx, 1) ? 1 : -1;
}

// A serving loop (one thread per context and class, started by the first request of its
// class).  The small batch's stream has the highest priority (its kernels are short), the
// large lane's the next and the medium batch's the lowest, so the short rounds of small
// requests are not held up behind long rounds.
void serve_loop(te_ctx* ctx, int cls) {
    cudaSetDevice(ctx->device);
    ServeEngine E;
    te_status init_st = TE_OK;
    bool ready = false;
    for (;;) {
        std::vector<te_request*> cancelled;
        {
            std::unique_lock<std::mutex> lk(ctx->qmu);
            ctx->qcv.wait(lk, [&] { return ctx->stopping || !ctx->bqueue[cls].empty() || !E.slots.empty(); });
            if (ctx->stopping) {
                for (te_request* r : ctx->bqueue[cls]) {
                    r->state.store(1);
                    cancelled.push_back(r);
                }
                ctx->bqueue[cls].clear();
            } else {
                if (!ready && init_st == TE_OK) {
                    lk.unlock();
                    init_st = E.init(ctx, ctx->serve_m, serve_class_capacity(ctx, cls), cls);
                    lk.lock();
                    if (init_st == TE_OK) {
                        ready = true;
                        ctx->in_use += (int64_t)E.bytes;
                    }
                }
                if (!ready) {                           // no arena: every queued request fails
                    for (te_request* r : ctx->bqueue[cls]) {
                        r->state.store(1);
                        cancelled.push_back(r);
                    }
                    ctx->bqueue[cls].clear();
                }
                // admission in arrival order while slots and arena space last
                while (ready && !ctx->bqueue[cls].empty() && (int)E.slots.size() < TE_MULTI_MAX) {
                    te_request* r = ctx->bqueue[cls].front();
                    if (r->cancel.load()) {
                        ctx->bqueue[cls].pop_front();
                        r->state.store(1);
                        cancelled.push_back(r);
                        continue;
                    }
                    const int64_t seg = (r->H->d + 31) / 32 * 32;
                    const int64_t off = E.take(seg);
                    if (off < 0) break;
                    ctx->bqueue[cls].pop_front();
                    r->state.store(1);
                    ServeSlot sl;
                    sl.r = r;
                    sl.elem0 = off;
                    sl.seg = seg;
                    sl.t_admit = now_ms();
                    E.slots.push_back(sl);
                    E.dirty = true;
                }
            }
        }
        for (te_request* r : cancelled) {
            te_stats S;
            memset(&S, 0, sizeof(S));
            if (!ready && init_st != TE_OK && !ctx->stopping)
                serve_publish(r, init_st, S, "the serving arena could not be allocated");
            else
                serve_publish(r, TE_ERR_CANCELLED, S, "request cancelled");
        }
        if (ctx->stopping) {
            while (!E.slots.empty()) serve_finish(E, 0, TE_ERR_CANCELLED, "request cancelled");
            break;
        }
        for (size_t i = 0; i < E.slots.size();) {
            if (E.slots[i].r->cancel.load()) serve_finish(E, i, TE_ERR_CANCELLED, "request cancelled");
            else ++i;
        }
        if (E.slots.empty()) continue;
        if (E.dirty) {
            const te_status cs = serve_compose(E);
            if (cs != TE_OK) {
                std::string msg;
                {
                    std::lock_guard<std::mutex> lk(ctx->mu);
                    msg = ctx->err;
                }
                while (!E.slots.empty()) {
                    E.slots[0].idx = -1;
                    serve_finish(E, 0, cs, msg);
                }
                continue;
            }
            // requests that failed their start (normalisation, t = 0 done)
            for (size_t i = 0; i < E.slots.size();) {
                const DevState& x = E.st_host[E.slots[i].idx];
                if (x.status != 0) serve_finish(E, i, x.status, device_status_msg(x.status));
                else if (x.done) serve_finish(E, i, TE_OK, std::string());
                else ++i;
            }
            if (E.dirty) continue;                      // recompose before the round
        }
        cudaError_t e = cudaGraphLaunch(E.exec, E.s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(E.s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            const std::string msg = std::string("serving round: ") + cudaGetErrorString(e);
            while (!E.slots.empty()) serve_finish(E, 0, TE_ERR_CUDA, msg);
            continue;
        }
        for (size_t i = 0; i < E.slots.size();) {
            const DevState& x = E.st_host[E.slots[i].idx];
            if (x.status != 0) serve_finish(E, i, x.status, device_status_msg(x.status));
            else if (x.done) serve_finish(E, i, TE_OK, std::string());
            else ++i;
        }
        ctx->qcv.notify_all();
    }
    if (ready) {
        std::lock_guard<std::mutex> lk(ctx->qmu);
        ctx->in_use -= (int64_t)E.bytes;
    }
    E.release();
}
