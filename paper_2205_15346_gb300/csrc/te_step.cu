// te_step.cu -- K3: step 2 of Algorithm 1 (arXiv 2205.15346) in one thread block.
//
// Per restart, with H_m the real symmetric tridiagonal Lanczos matrix
// (alpha on the diagonal, beta off it) and h = h_{m+1,m}:
//  1. diagonalise H_m = Q diag(lam) Q^T once (Sec. 2.4, first remark), by the
//     implicit QL iteration with shifts (Golub and Van Loan, "Matrix
//     Computations", Sec. 8.3): one thread runs the scalar sweep and records its
//     Givens rotations, then every thread applies them to its own row of Q;
//  2. error integrand f(tau) = h |e_m^T exp(-i H_m tau) e_1|
//                            = h |sum_k Q[m,k] Q[1,k] e^{-i lam_k tau}|   (eq. errorIntegral);
//  3. E(a, b) = int_a^b f by adaptive tanh-sinh (Takahasi and Mori 1974): step
//     2^-k on |u| <= 3.15, relative stop |I_k - I_{k-1}| <= quad_rel_tol |I_k| from
//     level 3, warning after quad_max_levels (Sec. 4); or the non-adaptive
//     Gauss-Legendre option;
//  4. step size: largest admissible step by the search of Algorithm 1 step 2
//     (first restart: start at t_step0 and double; later: shrink the previous
//     step; then halve while E(0, tau) > tol_rate tau; then grow by substeps of
//     tau / n_substeps while the accumulated integral stays within tol_rate times
//     the new end), every candidate clipped to the remaining time; after a lucky
//     breakdown the whole remaining time is taken with the bound h * t_rem;
//  5. omega = exp(-i H_m tau) e_1 = Q diag(e^{-i lam tau}) Q^T e_1
//     (eq. krylovApproximation) and the recombination coefficients
//     coef[k] = beta0 scale[k] omega_k for K4.
// All threads run the same control flow: every decision is taken from values
// reduced over the block and broadcast through shared memory.
#include <float.h>

#include "te_internal.cuh"

namespace {

constexpr double kUMax = 3.15;
constexpr int kMinLevel = 3;
constexpr double kHalfPi = 1.5707963267948966;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum broadcast to every thread (fixed reduction order).
__device__ double block_sum_all(double v, double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double r = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
        r = warp_sum(r);
        if (lane == 0) red[32] = r;
    }
    __syncthreads();
    return red[32];
}

struct Integrand {
    const double* lam;
    const double* q;
    int n;
    double h;
};

__device__ __forceinline__ double f_at(const Integrand& F, double tau) {
    double re = 0.0, im = 0.0;
    for (int k = 0; k < F.n; ++k) {
        double s, c;
        sincos(F.lam[k] * tau, &s, &c);
        re = fma(F.q[k], c, re);
        im = fma(-F.q[k], s, im);
    }
    return F.h * sqrt(re * re + im * im);
}

struct Quad {
    int method;
    double rel_tol;
    int max_levels;
    int gauss_n;
    const double* gx;
    const double* gw;
};

// E(a, b); every thread gets the same value.  *warn counts non-converged calls
// (incremented by thread 0 only).
__device__ double integrate(const Integrand& F, const Quad& Qd, double a, double b, double* red,
                            int* warn, long long* nodes) {
    if (a == b) return 0.0;
    const double c = 0.5 * (a + b), r = 0.5 * (b - a);
    const int tid = threadIdx.x, nt = blockDim.x;
    if (Qd.method == TE_QUAD_GAUSS) {
        double loc = 0.0;
        for (int i = tid; i < Qd.gauss_n; i += nt) loc += Qd.gw[i] * f_at(F, c + r * Qd.gx[i]);
        if (tid == 0) *nodes += Qd.gauss_n;
        return r * block_sum_all(loc, red);
    }
    auto node = [&](double u, double& x, double& w) {
        const double s = kHalfPi * sinh(u);
        const double ch = cosh(s);
        x = c + r * tanh(s);
        w = r * kHalfPi * cosh(u) / (ch * ch);
    };
    double loc = 0.0;
    const int j0 = (int)floor(kUMax);
    for (int i = tid; i < 2 * j0 + 1; i += nt) {
        double x, w;
        node((double)(i - j0), x, w);
        loc += w * f_at(F, x);
    }
    double total = block_sum_all(loc, red);
    if (tid == 0) *nodes += 2 * j0 + 1;
    double step = 1.0;
    for (int level = 1; level <= Qd.max_levels; ++level) {
        step *= 0.5;
        const int kmax = (int)floor((kUMax / step - 1.0) * 0.5);
        const int count = 2 * (kmax + 1);
        loc = 0.0;
        for (int i = tid; i < count; i += nt) {
            const int k = i - (kmax + 1);
            double x, w;
            node((2.0 * k + 1.0) * step, x, w);
            loc += w * f_at(F, x);
        }
        const double s = block_sum_all(loc, red);
        if (tid == 0) *nodes += count;
        const double nt_total = 0.5 * total + step * s;
        if (level >= kMinLevel && fabs(nt_total - total) <= Qd.rel_tol * fabs(nt_total))
            return nt_total;
        total = nt_total;
    }
    if (tid == 0) *warn += 1;
    return total;
}

__global__ void __launch_bounds__(TE_STEP_THREADS) k_step(DevState* st, int mcap) {
    extern __shared__ double smem[];
    __shared__ double red[33];
    __shared__ int sh_mm, sh_nrot, sh_fail, sh_warn;
    __shared__ long long sh_nodes;
    if (st->status != 0 || st->done != 0) return;
    const long long clk0 = clock64();
    const int n = st->m_eff;
    const int tid = threadIdx.x, nt = blockDim.x;
    double2* ph = reinterpret_cast<double2*>(smem);   // 16-byte aligned first
    double* Zt = reinterpret_cast<double*>(ph + mcap);  // Zt[k*n + r] = Q[r][k]
    double* dd = Zt + (size_t)mcap * mcap;              // eigenvalues
    double* ee = dd + mcap;
    double* q = ee + mcap;
    double* z0 = q + mcap;
    double* rc = z0 + mcap;
    double* rs = rc + mcap;
    int* ri = reinterpret_cast<int*>(rs + mcap);

    for (int i = tid; i < n * n; i += nt) Zt[i] = ((i / n) == (i % n)) ? 1.0 : 0.0;
    for (int i = tid; i < n; i += nt) {
        dd[i] = st->alpha[i];
        ee[i] = (i + 1 < n) ? st->beta[i] : 0.0;
    }
    if (tid == 0) {
        sh_fail = 0;
        sh_warn = 0;
        sh_nodes = 0;
    }
    __syncthreads();

    // ---- 1. implicit QL with shifts
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        for (;;) {
            if (tid == 0) {
                int mm = l;
                while (mm < n - 1) {
                    const double tst = fabs(dd[mm]) + fabs(dd[mm + 1]);
                    if (fabs(ee[mm]) <= DBL_EPSILON * tst) break;
                    ++mm;
                }
                sh_mm = mm;
                sh_nrot = 0;
                if (mm != l) {
                    if (++iter > 64) {
                        sh_fail = 1;
                    } else {
                        double g = (dd[l + 1] - dd[l]) / (2.0 * ee[l]);
                        double r = hypot(g, 1.0);
                        g = dd[mm] - dd[l] + ee[l] / (g + copysign(r, g));
                        double s = 1.0, c = 1.0, p = 0.0;
                        int nrot = 0;
                        bool early = false;
                        for (int i = mm - 1; i >= l; --i) {
                            const double f = s * ee[i];
                            const double bb = c * ee[i];
                            r = hypot(f, g);
                            ee[i + 1] = r;
                            if (r == 0.0) {
                                dd[i + 1] -= p;
                                ee[mm] = 0.0;
                                early = true;
                                break;
                            }
                            s = f / r;
                            c = g / r;
                            g = dd[i + 1] - p;
                            r = (dd[i] - g) * s + 2.0 * c * bb;
                            p = s * r;
                            dd[i + 1] = g + p;
                            g = c * r - bb;
                            rc[nrot] = c;
                            rs[nrot] = s;
                            ri[nrot] = i;
                            ++nrot;
                        }
                        if (!early) {
                            dd[l] -= p;
                            ee[l] = g;
                            ee[mm] = 0.0;
                        }
                        sh_nrot = nrot;
                    }
                }
            }
            __syncthreads();
            const bool converged = (sh_mm == l) || (sh_fail != 0);
            const int nrot = sh_nrot;
            __syncthreads();                  // thread 0 may overwrite sh_* only after this
            if (converged) break;
            for (int r = tid; r < n; r += nt) {
                for (int qd = 0; qd < nrot; ++qd) {
                    const int i = ri[qd];
                    const double c = rc[qd], s = rs[qd];
                    const double zi = Zt[i * n + r], zi1 = Zt[(i + 1) * n + r];
                    Zt[(i + 1) * n + r] = s * zi + c * zi1;
                    Zt[i * n + r] = c * zi - s * zi1;
                }
            }
            __syncthreads();
        }
        if (sh_fail) break;
    }
    if (sh_fail) {
        if (tid == 0) {
            st->status = TE_ERR_INTERNAL;
            st->done = 1;
        }
        return;
    }
    for (int k = tid; k < n; k += nt) {
        z0[k] = Zt[k * n + 0];
        q[k] = Zt[k * n + (n - 1)] * Zt[k * n + 0];
    }
    __syncthreads();

    const long long clk1 = clock64();
    int n_integrals = 0;
    // ---- 2-4. step size from the error integral
    const double h = st->beta[n - 1];
    const double T = st->T, t_now = st->t_now;
    const double t_rem = T - t_now;
    const double tol_rate = st->tol_rate;
    Integrand F{dd, q, n, h};
    Quad Qd{st->quad, st->quad_rel_tol, st->quad_max_levels, st->gauss_n, st->gx, st->gw};
    double tau = 0.0, err = 0.0;
    bool underflow = false;
    const bool brk = st->breakdown != 0;
    if (brk) {
        tau = t_rem;
        err = h * t_rem;
    } else {
        if (st->first) {
            tau = fmin(st->t_step0, t_rem);
            err = (++n_integrals, integrate(F, Qd, 0.0, tau, red, &sh_warn, &sh_nodes));
            if (err <= tol_rate * tau) {
                while (2.0 * tau <= t_rem) {
                    const double e2 = (++n_integrals, integrate(F, Qd, 0.0, 2.0 * tau, red, &sh_warn, &sh_nodes));
                    if (!(e2 <= tol_rate * (2.0 * tau))) break;
                    tau = 2.0 * tau;
                    err = e2;
                }
            }
        } else {
            tau = fmin(st->shrink * st->prev_step, t_rem);
            err = (++n_integrals, integrate(F, Qd, 0.0, tau, red, &sh_warn, &sh_nodes));
        }
        while (!(err <= tol_rate * tau)) {
            tau = 0.5 * tau;
            if (tau < st->min_step) {
                underflow = true;
                break;
            }
            err = (++n_integrals, integrate(F, Qd, 0.0, tau, red, &sh_warn, &sh_nodes));
        }
        if (!underflow) {
            const double s = tau / st->n_substeps;
            const double base = tau;
            int nsub = 0;
            while (nsub < st->max_substeps && tau < t_rem) {
                const double end = fmin(base + (nsub + 1) * s, t_rem);
                const double delta = (++n_integrals, integrate(F, Qd, tau, end, red, &sh_warn, &sh_nodes));
                if (!(err + delta <= tol_rate * end)) break;
                err += delta;
                tau = end;
                ++nsub;
            }
        }
    }
    __syncthreads();
    if (underflow) {
        if (tid == 0) {
            st->status = TE_ERR_STEP_UNDERFLOW;
            st->done = 1;
            st->quad_warnings += sh_warn;
        }
        return;
    }

    // ---- 5. omega = Q diag(e^{-i lam tau}) Q^T e_1, recombination coefficients
    for (int k = tid; k < n; k += nt) {
        double s, c;
        sincos(dd[k] * tau, &s, &c);
        ph[k] = make_double2(c * z0[k], -s * z0[k]);
    }
    __syncthreads();
    const double beta0 = st->beta0;
    for (int r = tid; r < n; r += nt) {
        double re = 0.0, im = 0.0;
        for (int k = 0; k < n; ++k) {
            const double z = Zt[k * n + r];
            re = fma(z, ph[k].x, re);
            im = fma(z, ph[k].y, im);
        }
        const double sc = beta0 * st->scale[r];
        st->coef[r] = make_double2(sc * re, sc * im);
    }
    if (tid == 0) {
        st->quad_integrals += n_integrals;
        st->quad_nodes += sh_nodes;
        st->eig_cycles += clk1 - clk0;
        st->search_cycles += clock64() - clk1;
        st->t_now = (tau == t_rem) ? T : t_now + tau;
        st->err_acc += err;
        st->prev_step = tau;
        st->first = 0;
        st->restarts += 1;
        st->breakdowns += brk ? 1 : 0;
        st->quad_warnings += sh_warn;
        st->last_m_eff = n;
        st->last_step = tau;
        st->last_err = err;
        st->done = (st->t_now >= T) ? 1 : 0;
    }
}

}  // namespace

int step_smem_bytes(int m) {
    return (int)(sizeof(double) * ((size_t)m * m + 6 * (size_t)m) + sizeof(double2) * m +
                 sizeof(int) * m);
}

// The limit is a property of the function, shared by every plan and thread, so
// it is set once to the size needed by the largest Krylov dimension.
cudaError_t step_prepare() {
    return cudaFuncSetAttribute(k_step, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                step_smem_bytes(TE_M_MAX));
}

cudaError_t launch_step(DevState* st, int m, cudaStream_t s) {
    k_step<<<1, TE_STEP_THREADS, step_smem_bytes(m), s>>>(st, m);
    return cudaGetLastError();
}
