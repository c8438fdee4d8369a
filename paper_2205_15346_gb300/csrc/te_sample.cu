// te_sample.cu -- states at intermediate times and diagonal observables.
//
// Sec. 2.4 of arXiv 2205.15346 remarks that Algorithm 1 extends to sampling the
// state at any time t_s inside a step: in step 3 the restart's H_m and V_m give
//     v(t_s) = beta0 V_m exp(-i H_m (t_s - t_now)) e_1,   t_now <= t_s <= t_now + t_step.
// A sampled solve puts two kernels into the restart graph, after the step kernel
// (which records the step's window) and before the recombination overwrites the
// first Krylov column:
//   KS1 k_sample_omega    one CTA per sample inside the window: omega_s by the
//                         Chebyshev / Jacobi-Anger series of te_smallexp.cuh, then the
//                         coefficients beta0 scale[k] omega_s[k];
//   KS2 k_sample_combine  w_s = sum_k c_{s,k} u_k for up to kGroup samples per pass
//                         over the Krylov basis, into the sample buffer.
// A sample time s belongs to the first restart whose window reaches it
// (|s| <= t_now + t_step; every remaining sample in the restart that reaches t),
// which is the oracle's rule.  After the solve KO k_observables reduces the
// diagonal observables <w_s| O_l |w_s> = sum_i O_l[i] |w_s[i]|^2 (e.g. the mode
// occupations whose time dependence Sec. 5 plots), one partial per (sample,
// observable, CTA) added in CTA order.
#include <math.h>

#include "te_internal.cuh"
#include "te_smallexp.cuh"

namespace {

constexpr int kGroup = 8;            // samples recombined per pass over V

// First index k in [lo, n) with ts[k] > x (ts non-decreasing).
__device__ __forceinline__ int upper_bound(const double* ts, int lo, int n, double x) {
    int hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ts[mid] <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Samples covered by the step the step kernel just took: [lo, hi).
__device__ __forceinline__ void window(const DevState* st, const double* ts, int ns, int* lo, int* hi) {
    *lo = st->samp_next;
    *hi = st->win_last ? ns : upper_bound(ts, *lo, ns, st->win_t1);
}

// ---------------------------------------------------------------- KS1

__global__ void __launch_bounds__(TE_STEP_THREADS) k_sample_omega(DevState* st, const double* ts,
                                                                  int ns, int mcap,
                                                                  double2* coef, double* bound) {
    extern __shared__ double2 smem[];
    __shared__ double sh_S, red[64];
    if (!st->active || st->status != 0) return;
    int lo, hi;
    window(st, ts, ns, &lo, &hi);
    if (blockIdx.x == 0) {
        // the bound at a sample is the bound accumulated through this step
        for (int k = lo + (int)threadIdx.x; k < hi; k += blockDim.x) bound[k] = st->err_acc;
        if (threadIdx.x == 0) {
            st->samp_lo = lo;
            st->samp_hi = hi;
        }
    }
    if (lo + (int)blockIdx.x >= hi) return;
    const int n = st->last_m_eff;
    const int tid = threadIdx.x, nt = blockDim.x;
    double2* om = reinterpret_cast<double2*>(smem);      // first: 16-byte aligned for any mcap
    double* al = reinterpret_cast<double*>(om + mcap);
    double* be = al + mcap;
    double* v3 = be + mcap;
    double* jk = v3 + 3 * mcap;
    for (int i = tid; i < n; i += nt) {
        al[i] = st->alpha[i];
        be[i] = (i + 1 < n) ? st->beta[i] : 0.0;
    }
    __syncthreads();
    // Gershgorin interval [b - a, b + a] of H_m, as in the step kernel
    double l = INFINITY, h = -INFINITY;
    for (int i = tid; i < n; i += nt) {
        const double rad = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i + 1 < n ? fabs(be[i]) : 0.0);
        l = fmin(l, al[i] - rad);
        h = fmax(h, al[i] + rad);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l = fmin(l, __shfl_xor_sync(0xffffffffu, l, o));
        h = fmax(h, __shfl_xor_sync(0xffffffffu, h, o));
    }
    if ((tid & 31) == 0) {
        red[tid >> 5] = l;
        red[32 + (tid >> 5)] = h;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < nt / 32; ++w) {
            red[0] = fmin(red[0], red[w]);
            red[32] = fmax(red[32], red[32 + w]);
        }
    }
    __syncthreads();
    const double b = 0.5 * (red[32] + red[0]);
    double a = 0.5 * (red[32] - red[0]);
    if (!(a > 0.0)) a = 1.0;
    const double inv_a = 1.0 / a;
    const double beta0 = st->beta0;
    for (int s = lo + blockIdx.x; s < hi; s += gridDim.x) {
        const double tau = fmax(ts[s] - st->win_t0, 0.0);
        __syncthreads();
        if (!cheb_exp_e1(al, be, n, a, b, inv_a, tau, jk, v3, mcap, &sh_S, om)) {
            if (threadIdx.x == 0) {
                st->status = TE_ERR_UNSUPPORTED;   // sample beyond the series' pieces
                st->done = 1;
            }
            return;
        }
        __syncthreads();
        for (int r = tid; r < n; r += nt) {
            const double sc = beta0 * st->scale[r];
            coef[(size_t)s * mcap + r] = make_double2(sc * om[r].x, sc * om[r].y);
        }
    }
}

// ---------------------------------------------------------------- KS2

// With S (Re + Im of every Krylov column, the sliced path) each product takes the
// three-multiplication form of the recombination kernel, summed in the same order,
// so the sample at the end of a step equals the state that step returns bit for bit.
__global__ void __launch_bounds__(TE_BLOCK) k_sample_combine(const double2* __restrict__ V,
                                                             const double* __restrict__ S,
                                                             int64_t d, DevState* st,
                                                             const double2* __restrict__ coef,
                                                             int mcap, double2* __restrict__ out) {
    __shared__ double ca[kGroup][TE_M_MAX], cp[kGroup][TE_M_MAX], cq[kGroup][TE_M_MAX];
    if (!st->active || st->status != 0) return;
    const int lo = st->samp_lo, hi = st->samp_hi;
    const int n = st->last_m_eff;
    for (int g0 = lo; g0 < hi; g0 += kGroup) {
        const int ng = hi - g0 < kGroup ? hi - g0 : kGroup;
        __syncthreads();
        for (int i = threadIdx.x; i < ng * n; i += blockDim.x) {
            const int q = i / n, k = i - q * n;
            const double2 c = coef[(size_t)(g0 + q) * mcap + k];
            if (S) {
                ca[q][k] = c.x;            // a
                cp[q][k] = c.y - c.x;      // b - a
                cq[q][k] = c.x + c.y;      // a + b
            } else {
                ca[q][k] = c.x;
                cp[q][k] = c.y;
            }
        }
        __syncthreads();
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < d;
             e += (int64_t)gridDim.x * blockDim.x) {
            double re[kGroup], im[kGroup];
#pragma unroll
            for (int q = 0; q < kGroup; ++q) re[q] = im[q] = 0.0;
            if (S) {
                double k3[kGroup];
#pragma unroll
                for (int q = 0; q < kGroup; ++q) k3[q] = 0.0;
                // re carries sum a (x + y), im sum (b - a) x, k3 sum (a + b) y
                for (int k = 0; k < n; ++k) {
                    const double2 u = __ldg(V + (size_t)k * d + e);
                    const double z = __ldg(S + (size_t)k * d + e);
#pragma unroll
                    for (int q = 0; q < kGroup; ++q) {
                        if (q < ng) {
                            re[q] = fma(ca[q][k], z, re[q]);
                            im[q] = fma(cp[q][k], u.x, im[q]);
                            k3[q] = fma(cq[q][k], u.y, k3[q]);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < kGroup; ++q) {
                    const double k1 = re[q];
                    re[q] = k1 - k3[q];
                    im[q] = k1 + im[q];
                }
            } else {
                for (int k = 0; k < n; ++k) {
                    const double2 u = __ldg(V + (size_t)k * d + e);
#pragma unroll
                    for (int q = 0; q < kGroup; ++q) {
                        if (q < ng) {
                            re[q] = fma(ca[q][k], u.x, re[q]);
                            re[q] = fma(-cp[q][k], u.y, re[q]);
                            im[q] = fma(ca[q][k], u.y, im[q]);
                            im[q] = fma(cp[q][k], u.x, im[q]);
                        }
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < kGroup; ++q)
                if (q < ng) out[(size_t)(g0 + q) * d + e] = make_double2(re[q], im[q]);
        }
    }
}

// The sampler's cursor moves past the window once both kernels are done with it.
__global__ void k_sample_advance(DevState* st) {
    if (threadIdx.x == 0 && st->active && st->status == 0) st->samp_next = st->samp_hi;
}

// ---------------------------------------------------------------- KO

// partials[(s nobs + l) gridDim.x + blockIdx.x] = sum over this CTA's elements of
// O_l[i] |w_s[i]|^2 (blockIdx.y = s; observables in groups of 8).
__global__ void __launch_bounds__(TE_BLOCK) k_observables(const double2* __restrict__ W, int64_t d,
                                                          const double* __restrict__ O, int nobs,
                                                          double* __restrict__ partials) {
    __shared__ double sh[TE_BLOCK / 32][8];
    const int s = blockIdx.y;
    const double2* w = W + (size_t)s * d;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int l0 = 0; l0 < nobs; l0 += 8) {
        double acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = 0.0;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d;
             i += (int64_t)gridDim.x * blockDim.x) {
            const double2 x = w[i];
            const double p = fma(x.x, x.x, x.y * x.y);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (l0 + q < nobs) acc[q] = fma(__ldg(O + (size_t)(l0 + q) * d + i), p, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            double v = acc[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            acc[q] = v;
        }
        __syncthreads();
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < 8; ++q) sh[wid][q] = acc[q];
        __syncthreads();
        if (threadIdx.x < 8 && l0 + (int)threadIdx.x < nobs) {
            double v = 0.0;
            for (int w2 = 0; w2 < TE_BLOCK / 32; ++w2) v += sh[w2][threadIdx.x];
            partials[((size_t)s * nobs + l0 + threadIdx.x) * gridDim.x + blockIdx.x] = v;
        }
    }
}

__global__ void k_gather_real(const double* __restrict__ src, const int32_t* __restrict__ map,
                              int64_t d, double* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[map[i]];
}

__global__ void k_observables_sum(const double* __restrict__ partials, int npairs, int G,
                                  double* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npairs) return;
    double v = 0.0;
    for (int b = 0; b < G; ++b) v += partials[(size_t)k * G + b];
    out[k] = v;
}

}  // namespace

int sample_omega_smem(int mcap) {
    return (int)(sizeof(double) * ((size_t)5 * mcap + kKcap) + sizeof(double2) * (size_t)mcap);
}

cudaError_t sample_prepare() {
    return cudaFuncSetAttribute(k_sample_omega, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                sample_omega_smem(TE_M_MAX));
}

cudaError_t launch_sample_kernels(DevState* st, const double* ts, int ns, int mcap, double2* coef,
                                  double* bound, const double2* V, const double* S, int64_t d,
                                  double2* out, int grid_stream, cudaStream_t s) {
    const int g1 = ns < 32 ? (ns > 0 ? ns : 1) : 32;
    k_sample_omega<<<g1, TE_STEP_THREADS, sample_omega_smem(mcap), s>>>(st, ts, ns, mcap, coef,
                                                                      bound);
    k_sample_combine<<<grid_stream, TE_BLOCK, 0, s>>>(V, S, d, st, coef, mcap, out);
    k_sample_advance<<<1, 32, 0, s>>>(st);
    return cudaGetLastError();
}

cudaError_t launch_observables(const double2* W, int64_t d, int ns, const double* O, int nobs,
                               double* partials, int G, double* out, cudaStream_t s) {
    dim3 grid(G, ns);
    k_observables<<<grid, TE_BLOCK, 0, s>>>(W, d, O, nobs, partials);
    const int npairs = ns * nobs;
    k_observables_sum<<<(npairs + 255) / 256, 256, 0, s>>>(partials, npairs, G, out);
    return cudaGetLastError();
}

cudaError_t launch_gather_real(const double* src, const int32_t* map, int64_t d, double* dst,
                               int num_sms, cudaStream_t s) {
    const int64_t want = (d + TE_BLOCK - 1) / TE_BLOCK;
    const int grid = (int)(want < (int64_t)num_sms * 8 ? (want > 0 ? want : 1) : (int64_t)num_sms * 8);
    k_gather_real<<<grid, TE_BLOCK, 0, s>>>(src, map, d, dst);
    return cudaGetLastError();
}
