// te_step.cu -- K3: step 2 of Algorithm 1 (arXiv 2205.15346) in one thread block.
//
// Per restart, with H_m = T the real symmetric tridiagonal Lanczos matrix
// (alpha on the diagonal, beta off it) and h = h_{m+1,m}, K3
//  a. evaluates the error integrand f(tau) = h |e_m^T exp(-i T tau) e_1| (eq. errorIntegral),
//  b. integrates it, E(a, b) = int_a^b f, by adaptive tanh-sinh (Takahasi and Mori 1974):
//     step 2^-k on |u| <= 3.15, stop when |I_k - I_{k-1}| <= quad_rel_tol |I_k| from
//     level 3 on, warning after quad_max_levels (Sec. 4); or by the non-adaptive
//     Gauss-Legendre option,
//  c. searches the largest admissible step (Algorithm 1 step 2 and the Sec. 2.4
//     remarks: first restart from t_step0 with doubling; later restarts from the
//     shrunk previous step; halve while E(0, tau) > tol_rate tau; grow by
//     substeps of tau / n_substeps while the accumulated integral stays within
//     tol_rate times the new end; candidates clipped to the remaining time;
//     after a lucky breakdown the whole remaining time with the bound h t_rem),
//  d. forms omega = exp(-i T tau) e_1 (eq. krylovApproximation) and the
//     recombination coefficients coef[k] = beta0 scale[k] omega_k for K4.
//
// exp(-i T tau) e_1 is evaluated in one of two ways:
//  * diagonalisation (the paper's choice, Sec. 2.4): T = Q diag(lam) Q^T by the
//    implicit QL iteration with shifts (Golub and Van Loan, "Matrix Computations",
//    Sec. 8.3); one thread runs the scalar sweep, all threads apply its Givens
//    rotations to their rows of Q; then f = h |sum_k Q[m,k] Q[1,k] e^{-i lam_k tau}|.
//  * Chebyshev expansion (default): with [b - a, b + a] a Gershgorin interval
//    of T and T~ = (T - b) / a, the Jacobi-Anger expansion gives
//      exp(-i T tau) = e^{-i b tau} sum_k c_k (-i)^k J_k(a tau) T_k(T~),  c_0 = 1, c_k = 2,
//    with Bessel functions J_k and Chebyshev polynomials T_k.  The integrand
//    only needs the scalars g_k = e_m^T T_k(T~) e_1 (zero for k < m - 1), built
//    by the three-term Chebyshev recurrence; each node then costs one backward
//    Bessel recurrence (Miller's algorithm, normalised by J_0 + 2 sum J_2k = 1),
//    with no sin/cos and no serial eigensolver.  GB300 issues FP64 at 2 lanes
//    per SM per cycle, so the long serial FP64 chain of QL dominates a restart;
//    the Chebyshev route is lane-parallel over quadrature nodes.
// All threads run the same control flow: every decision is taken from values
// reduced over the block and broadcast through shared memory.
#include <float.h>

#include "te_internal.cuh"
#include "te_smallexp.cuh"

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

// Block minimum and maximum broadcast to every thread.
__device__ void block_minmax_all(double lo, double hi, double* red, double* out_lo, double* out_hi) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    __syncthreads();
    if (lane == 0) {
        red[wid] = lo;
        red[16 + wid] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double l = red[0], h = red[16];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            l = fmin(l, red[w]);
            h = fmax(h, red[16 + w]);
        }
        red[32] = l;
        red[31] = h;
    }
    __syncthreads();
    *out_lo = red[32];
    *out_hi = red[31];
    __syncthreads();
}


struct Small {                       // what the integrand needs, in shared memory
    int method;                      // TE_SMALLEXP_*
    int n;
    double h;
    // diagonalisation
    const double* lam;
    const double* q;                 // Q[m,k] Q[1,k]
    // Chebyshev
    double a, b, inv_a;
    const double* g;                 // g_k = e_m^T T_k(T~) e_1, valid for k <= K
    int K, M;                        // terms kept and start of the backward recurrence
};

// f(tau) by the eigen-decomposition
__device__ __forceinline__ double f_eig(const Small& F, double tau) {
    double re = 0.0, im = 0.0;
    for (int k = 0; k < F.n; ++k) {
        double s, c;
        sincos(F.lam[k] * tau, &s, &c);
        re = fma(F.q[k], c, re);
        im = fma(-F.q[k], s, im);
    }
    return F.h * hypot(re, im);
}

// f(tau) by the Chebyshev expansion: |sum_k c_k (-i)^k J_k(a tau) g_k| with
// J_k from Miller's backward recurrence J_{k-1} = (2k / z) J_k - J_{k+1},
// started at M = K(z) + kMillerExtra with J_{M+1} = 0 (K(z) terms for this
// node's own argument z, at most the integral's F.K) and normalised by
// J_0 + 2 sum J_{2k} = 1.  Every FP64 instruction of a warp occupies the FP64
// pipe for ~64 cycles on GB300, so the loop is written for few of them: the
// weights c_k = 2 (k > 0) and the factor 2 of the normalisation are applied
// once at the end, the (-i)^k pattern is unrolled by four, and (for z >= 1,
// where one step grows J by at most 2M/z <= 2M) the overflow guard runs once per
// four steps.  Nodes with z < 1 take the same recurrence with a guard per step.
__device__ __forceinline__ double f_cheb(const Small& F, double tau) {
    const double z = F.a * tau;
    const int first = F.n - 1;       // g_k = 0 below this index
    if (!(z > 1e-300)) return first == 0 ? F.h * fabs(F.g[0]) : 0.0;
    const int Kn = min(bessel_terms(z), F.K);
    const int M = Kn + kMillerExtra;
    const double inv = 2.0 / z;
    double t = inv * M;              // 2k / z for the current k
    double jp = 0.0, jc = 1e-300;    // J_{k+1}, J_k (unnormalised)
    double S2 = 0.0, re = 0.0, im = 0.0, j0 = 0.0;
    const double* g = F.g;
    // |J_k| > kBig tested on the bit pattern (ordered like the magnitude), on the
    // integer pipe instead of the FP64 pipe
    const unsigned long long kBigBits = (unsigned long long)__double_as_longlong(kBig);
    // one step at index k: accumulate, then move to k - 1
#define TE_ACC(k, q)                                                       \
    if ((k) >= first && (k) <= Kn) {                                        \
        if ((q) == 0) re = fma(g[k], jc, re);                               \
        else if ((q) == 1) im = fma(-g[k], jc, im);                         \
        else if ((q) == 2) re = fma(-g[k], jc, re);                         \
        else im = fma(g[k], jc, im);                                        \
    }                                                                       \
    if (((q) & 1) == 0) S2 += jc;
#define TE_REC()                                                           \
    {                                                                       \
        const double jn = fma(t, jc, -jp);                                  \
        jp = jc;                                                            \
        jc = jn;                                                            \
        t -= inv;                                                           \
    }
#define TE_GUARD()                                                         \
    if (((unsigned long long)__double_as_longlong(jc) & 0x7fffffffffffffffull) > kBigBits) { \
        jc *= kSmall;                                                       \
        jp *= kSmall;                                                       \
        S2 *= kSmall;                                                       \
        re *= kSmall;                                                       \
        im *= kSmall;                                                       \
    }
    int k = M;
    if (z < 1.0) {
        for (; k >= 0; --k) {
            const int q = k & 3;
            TE_ACC(k, q)
            if (k == 0) break;
            TE_REC()
            TE_GUARD()
        }
        j0 = jc;
    } else {
        for (; (k & 3) != 3; --k) {             // down to the next k = 3 (mod 4)
            const int q = k & 3;
            TE_ACC(k, q)
            TE_REC()
        }
        TE_GUARD()
        for (; k >= 3; k -= 4) {
            // 2k/z from the index once per group: the running t -= inv drifts by one
            // rounding per step, which would shift the phase of J_k at large z
            t = inv * (double)k;
            TE_ACC(k, 3)
            TE_REC()
            TE_ACC(k - 1, 2)
            TE_REC()
            TE_ACC(k - 2, 1)
            TE_REC()
            TE_ACC(k - 3, 0)
            if (k == 3) break;                  // J_0 reached
            TE_REC()
            TE_GUARD()
        }
        j0 = jc;
    }
#undef TE_ACC
#undef TE_REC
#undef TE_GUARD
    // sum_k c_k (...) = 2 sum_k (...) - [k = 0 term];  J_0 + 2 sum J_2k = 2 S2 - J_0
    re = 2.0 * re - (first == 0 ? g[0] * j0 : 0.0);
    im = 2.0 * im;
    const double S = 2.0 * S2 - j0;
    // hypot: the unnormalised sums can be near 1e-215, where re * re underflows
    return F.h * hypot(re, im) / fabs(S);
}

__device__ __forceinline__ double f_at(const Small& F, double tau) {
    return F.method == TE_SMALLEXP_EIG ? f_eig(F, tau) : f_cheb(F, tau);
}

// Unit tanh-sinh nodes of levels 0..kTabLevels-1 on [-1, 1] (x = tanh(pi/2 sinh u),
// w = pi/2 cosh u / cosh^2(pi/2 sinh u)), in the order the levels visit them.
constexpr int kTabLevels = 6;
constexpr int kTabNodes = 201;       // 7 + 6 + 12 + 26 + 50 + 100
__constant__ int kTabOff[kTabLevels + 1] = {0, 7, 13, 25, 51, 101, 201};

struct Quad {
    int method;
    double rel_tol;
    int max_levels;
    int gauss_n;
    const double* gx;
    const double* gw;
    const double* tx;                // unit nodes and weights of the first levels
    const double* tw;
    double* vals;                    // kTabNodes scratch doubles
};

// The u of node i of level `level` (same order as the level loops below).
__device__ __forceinline__ double ts_u(int level, int i) {
    if (level == 0) return (double)(i - (int)floor(kUMax));
    const double step = ldexp(1.0, -level);
    const int kmax = (int)floor((kUMax / step - 1.0) * 0.5);
    return (2.0 * (i - (kmax + 1)) + 1.0) * step;
}

// Fill the unit node table (one thread per node).
__device__ void ts_table(double* tx, double* tw) {
    for (int i = threadIdx.x; i < kTabNodes; i += blockDim.x) {
        int level = 0;
        while (i >= kTabOff[level + 1]) ++level;
        const double u = ts_u(level, i - kTabOff[level]);
        const double sv = kHalfPi * sinh(u);
        const double ch = cosh(sv);
        tx[i] = tanh(sv);
        tw[i] = kHalfPi * cosh(u) / (ch * ch);
    }
}

// Chebyshev vectors v_k = T_k(T~) e_1 (three buffers rotated in shared memory),
// extended until g is valid up to index K.  Each v_k with k < nkeep is also kept
// at keep + k * mcap, for the evaluation of omega at the chosen step.
struct ChebState {
    double* v[3];
    int cur;                         // v[cur] = v_kdone, v[(cur + 2) % 3] = v_{kdone-1}
    int kdone;
    double* keep;
    int nkeep, mcap;
};

static_assert(TE_M_MAX <= TE_STEP_THREADS, "the step kernel keeps one Krylov row per thread");

__device__ void cheb_extend(ChebState& cs, double* g, int K, int n, const double* alpha,
                            const double* beta, double a_inv, double b) {
    // one row per thread (n <= TE_M_MAX <= blockDim.x): the row's coefficients stay
    // in registers, (alpha_i - b) is formed once, and the owner of row n - 1 writes
    // g_k itself, so a step needs one block barrier.  Three rotating buffers make
    // that barrier enough: step k reads v_k (neighbouring rows) and v_{k-1} (own
    // row) and writes v_{k+1} over v_{k-2}, which no thread still reads.
    const int i = threadIdx.x;
    const bool own = i < n;
    const double ab = own ? alpha[i] - b : 0.0;
    const double bl = (own && i > 0) ? beta[i - 1] : 0.0;
    const double br = (own && i + 1 < n) ? beta[i] : 0.0;
    while (cs.kdone < K) {
        const double* vc = cs.v[cs.cur];
        const double* vp = cs.v[(cs.cur + 2) % 3];
        double* vn = cs.v[(cs.cur + 1) % 3];
        if (own) {
            double tv = ab * vc[i];
            if (i > 0) tv = fma(bl, vc[i - 1], tv);
            if (i + 1 < n) tv = fma(br, vc[i + 1], tv);
            tv *= a_inv;
            tv = (cs.kdone == 0) ? tv : 2.0 * tv - vp[i];
            vn[i] = tv;
            if (cs.kdone + 1 < cs.nkeep) cs.keep[(size_t)(cs.kdone + 1) * cs.mcap + i] = tv;
            if (i == n - 1) g[cs.kdone + 1] = tv;
        }
        cs.cur = (cs.cur + 1) % 3;
        cs.kdone += 1;
        __syncthreads();
    }
}

// E(a, b); every thread gets the same value.  *warn counts non-converged calls and
// *nodes the integrand evaluations (both updated by thread 0 only).
__device__ double integrate(const Small& F, const Quad& Qd, double a, double b, double* red,
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
    // Levels 0..kMinLevel are always needed: their nodes are evaluated in one
    // parallel round (each level's dependent chains used to run one after another),
    // then the trapezoid estimates are refined level by level as before.
    const int n0 = kTabOff[kMinLevel + 1];
    for (int i = tid; i < n0; i += nt) Qd.vals[i] = r * Qd.tw[i] * f_at(F, c + r * Qd.tx[i]);
    __syncthreads();
    if (tid <= kMinLevel) {                              // per-level sums in node order
        double sum = 0.0;
        for (int i = kTabOff[tid]; i < kTabOff[tid + 1]; ++i) sum += Qd.vals[i];
        red[tid] = sum;
    }
    __syncthreads();
    double lsum[kMinLevel + 1];
    for (int l = 0; l <= kMinLevel; ++l) lsum[l] = red[l];
    __syncthreads();
    if (tid == 0) *nodes += n0;
    double total = lsum[0];
    double step = 1.0;
    for (int level = 1; level <= Qd.max_levels; ++level) {
        step *= 0.5;
        double s;
        if (level <= kMinLevel) {
            s = lsum[level];
        } else {
            const int kmax = (int)floor((kUMax / step - 1.0) * 0.5);
            const int count = 2 * (kmax + 1);
            double loc = 0.0;
            if (level < kTabLevels) {
                const int o = kTabOff[level];
                for (int i = tid; i < count; i += nt) loc += r * Qd.tw[o + i] * f_at(F, c + r * Qd.tx[o + i]);
            } else {
                for (int i = tid; i < count; i += nt) {
                    const int k = i - (kmax + 1);
                    double x, w;
                    node((2.0 * k + 1.0) * step, x, w);
                    loc += w * f_at(F, x);
                }
            }
            s = block_sum_all(loc, red);
            if (tid == 0) *nodes += count;
        }
        const double nt_total = 0.5 * total + step * s;
        if (level >= kMinLevel && fabs(nt_total - total) <= Qd.rel_tol * fabs(nt_total))
            return nt_total;
        total = nt_total;
    }
    if (tid == 0) *warn += 1;
    return total;
}

// The Chebyshev vectors the step search computes are kept for omega while they
// fit in this much shared memory (about 150 vectors at m = 40; a longer series
// runs its recurrence again); the step kernel then still fits twice per SM.
constexpr int kKeepBytes = 48 * 1024;
__host__ __device__ constexpr int keep_vectors(int mcap) { return kKeepBytes / (8 * mcap); }

// Shared-memory carve-up (16-byte aligned blocks first).
struct Layout {
    double2* ph;     // mcap
    double2* om;     // mcap
    double* Zt;      // mcap * mcap (diagonalisation only)
    double* dd;      // mcap: eigenvalues / working diagonal
    double* ee;      // mcap
    double* q;       // mcap
    double* z0;      // mcap
    double* rc;      // mcap
    double* rs;      // mcap
    double* al;      // mcap: alpha
    double* be;      // mcap: beta
    double* v3;      // 3 * mcap: Chebyshev vectors
    double* g;       // kKcap: g_k
    double* jk;      // kKcap: J_k for omega
    double* vk;      // keep_vectors(mcap) * mcap: T_k(T~) e_1 kept for omega
    double* tx;      // kTabNodes: unit tanh-sinh nodes
    double* tw;      // kTabNodes: their weights
    double* tv;      // kTabNodes: weighted integrand values of one round
    int* ri;         // mcap
};

__device__ Layout carve(double* smem, int mcap, int method) {
    Layout L;
    L.ph = reinterpret_cast<double2*>(smem);
    L.om = L.ph + mcap;
    double* p = reinterpret_cast<double*>(L.om + mcap);
    if (method == TE_SMALLEXP_EIG) {
        L.Zt = p;
        p += (size_t)mcap * mcap;
    } else {
        L.Zt = nullptr;
    }
    L.dd = p; p += mcap;
    L.ee = p; p += mcap;
    L.q = p; p += mcap;
    L.z0 = p; p += mcap;
    L.rc = p; p += mcap;
    L.rs = p; p += mcap;
    L.al = p; p += mcap;
    L.be = p; p += mcap;
    L.tx = p; p += kTabNodes;
    L.tw = p; p += kTabNodes;
    L.tv = p; p += kTabNodes;
    if (method == TE_SMALLEXP_EIG) {
        L.v3 = L.g = L.jk = L.vk = nullptr;
    } else {
        L.v3 = p; p += 3 * (size_t)mcap;
        L.g = p; p += kKcap;
        L.jk = p; p += kKcap;
        L.vk = p; p += (size_t)keep_vectors(mcap) * mcap;
    }
    L.ri = reinterpret_cast<int*>(p);
    return L;
}

// Implicit QL with shifts on (dd, ee); eigenvectors accumulated into Zt
// (Zt[k * n + r] = Q[r][k]).  Returns false if an eigenvalue needed more than 64
// iterations.
__device__ bool ql_eigen(const Layout& L, int n, int* sh_mm, int* sh_nrot, int* sh_fail) {
    const int tid = threadIdx.x, nt = blockDim.x;
    double* Zt = L.Zt;
    double* dd = L.dd;
    double* ee = L.ee;
    for (int i = tid; i < n * n; i += nt) Zt[i] = ((i / n) == (i % n)) ? 1.0 : 0.0;
    __syncthreads();
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
                *sh_mm = mm;
                *sh_nrot = 0;
                if (mm != l) {
                    if (++iter > 64) {
                        *sh_fail = 1;
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
                            L.rc[nrot] = c;
                            L.rs[nrot] = s;
                            L.ri[nrot] = i;
                            ++nrot;
                        }
                        if (!early) {
                            dd[l] -= p;
                            ee[l] = g;
                            ee[mm] = 0.0;
                        }
                        *sh_nrot = nrot;
                    }
                }
            }
            __syncthreads();
            const bool converged = (*sh_mm == l) || (*sh_fail != 0);
            const int nrot = *sh_nrot;
            __syncthreads();                  // thread 0 may overwrite sh_* only after this
            if (converged) break;
            for (int r = tid; r < n; r += nt) {
                for (int qd = 0; qd < nrot; ++qd) {
                    const int i = L.ri[qd];
                    const double c = L.rc[qd], s = L.rs[qd];
                    const double zi = Zt[i * n + r], zi1 = Zt[(i + 1) * n + r];
                    Zt[(i + 1) * n + r] = s * zi + c * zi1;
                    Zt[i * n + r] = c * zi - s * zi1;
                }
            }
            __syncthreads();
        }
        if (*sh_fail) break;
    }
    return *sh_fail == 0;
}

// One CTA per solve: CTA b works on st_base[b] (a batch of independent solves
// sharing H launches one CTA per vector).
// omega = exp(-i H_m tau) e_1 by the Chebyshev series (every thread of the block).
// A one-piece series whose vectors fit the kept ones extends them as far as it
// needs (a lucky breakdown evaluates none during the search) and sums them.
__device__ bool omega_cheb(const Layout& L, ChebState& cs, int n, const Small& F, double tau,
                           int mcap, double* sh_S) {
    const double z = F.a * tau;
    if (n > 1 && z <= kZPiece) {
        const int K = min(bessel_terms(fmin(z, (double)kKcap)), kKcap - kMillerExtra - 1);
        if (K < cs.nkeep && cs.kdone < K) cheb_extend(cs, L.g, K, n, L.al, L.be, F.inv_a, F.b);
    }
    return cheb_exp_e1(L.al, L.be, n, F.a, F.b, F.inv_a, tau, L.jk, L.v3, mcap, sh_S, L.om, L.vk,
                       min(cs.kdone + 1, cs.nkeep));
}

__global__ void __launch_bounds__(TE_STEP_THREADS, 1) k_step(DevState* st_base, int mcap) {
    DevState* st = st_base + blockIdx.x;
    extern __shared__ double smem[];
    __shared__ double red[33];
    __shared__ int sh_mm, sh_nrot, sh_fail, sh_warn;
    __shared__ long long sh_nodes;
    __shared__ double sh_S;
    if (st->status != 0 || st->done != 0) return;
    const long long clk0 = clock64();
    const int n = st->m_eff;
    const int method = st->smallexp;
    const int tid = threadIdx.x, nt = blockDim.x;
    const Layout L = carve(smem, mcap, method);
    for (int i = tid; i < n; i += nt) {
        L.al[i] = st->alpha[i];
        L.be[i] = (i + 1 < n) ? st->beta[i] : 0.0;
        L.dd[i] = L.al[i];
        L.ee[i] = L.be[i];
    }
    if (tid == 0) {
        sh_fail = 0;
        sh_warn = 0;
        sh_nodes = 0;
    }
    __syncthreads();

    const double h = st->beta[n - 1];
    Small F;
    F.method = method;
    F.n = n;
    F.h = h;
    F.lam = L.dd;
    F.q = L.q;
    F.g = L.g;
    F.K = 0;
    F.M = 0;
    ChebState cs{};
    if (method == TE_SMALLEXP_EIG) {
        // ---- diagonalisation of H_m
        if (!ql_eigen(L, n, &sh_mm, &sh_nrot, &sh_fail)) {
            if (tid == 0) {
                st->status = TE_ERR_INTERNAL;
                st->done = 1;
            }
            return;
        }
        for (int k = tid; k < n; k += nt) {
            L.z0[k] = L.Zt[k * n + 0];
            L.q[k] = L.Zt[k * n + (n - 1)] * L.Zt[k * n + 0];
        }
        F.a = F.b = F.inv_a = 0.0;
    } else {
        // ---- Gershgorin interval [b - a, b + a] and the Chebyshev recurrence start
        double lo = INFINITY, hi = -INFINITY;
        for (int i = tid; i < n; i += nt) {
            const double rad = (i > 0 ? fabs(L.be[i - 1]) : 0.0) + (i + 1 < n ? fabs(L.be[i]) : 0.0);
            lo = fmin(lo, L.al[i] - rad);
            hi = fmax(hi, L.al[i] + rad);
        }
        block_minmax_all(lo, hi, red, &lo, &hi);
        F.b = 0.5 * (hi + lo);
        F.a = 0.5 * (hi - lo);
        if (!(F.a > 0.0)) F.a = 1.0;          // n = 1: any positive a gives the same series
        F.inv_a = 1.0 / F.a;
        cs.v[0] = L.v3;
        cs.v[1] = L.v3 + mcap;
        cs.v[2] = L.v3 + 2 * mcap;
        cs.cur = 0;
        cs.kdone = 0;
        cs.keep = L.vk;
        cs.nkeep = keep_vectors(mcap);
        cs.mcap = mcap;
        for (int i = tid; i < n; i += nt) {
            cs.v[0][i] = (i == 0) ? 1.0 : 0.0;
            cs.v[2][i] = 0.0;
            L.vk[i] = cs.v[0][i];
        }
        if (tid == 0) L.g[0] = (n == 1) ? 1.0 : 0.0;
        __syncthreads();
    }
    const long long clk1 = clock64();

    // ---- step size from the error integral
    const double T = st->T, t_now = st->t_now;
    const double t_rem = T - t_now;
    const double tol_rate = st->tol_rate;
    Quad Qd{st->quad, st->quad_rel_tol, st->quad_max_levels, st->gauss_n, st->gx, st->gw,
            L.tx, L.tw, L.tv};
    if (Qd.method != TE_QUAD_GAUSS) {
        ts_table(L.tx, L.tw);
        __syncthreads();
    }
    int n_integrals = 0;
    // E over [lo_t, hi_t]; for the Chebyshev route first make sure g covers the
    // largest argument a * hi_t (an integral that would need more than kKcap terms
    // is reported as infinite, i.e. the step is rejected: a conservative outcome).
    auto E = [&](double lo_t, double hi_t) -> double {
        ++n_integrals;
        if (method != TE_SMALLEXP_EIG) {
            const double zmax = F.a * hi_t;
            if (!(zmax < (double)(kKcap - kMillerExtra - 200))) return INFINITY;
            const int K = bessel_terms(zmax);
            if (K + kMillerExtra >= kKcap) return INFINITY;
            cheb_extend(cs, L.g, K, n, L.al, L.be, F.inv_a, F.b);
            F.K = K;
            F.M = K + kMillerExtra;
        }
        return integrate(F, Qd, lo_t, hi_t, red, &sh_warn, &sh_nodes);
    };
    double tau = 0.0, err = 0.0;
    bool underflow = false;
    const bool brk = st->breakdown != 0;
    if (brk) {
        tau = t_rem;
        err = h * t_rem;
    } else {
        if (st->first) {
            tau = fmin(st->t_step0, t_rem);
            err = E(0.0, tau);
            if (err <= tol_rate * tau) {
                while (2.0 * tau <= t_rem) {
                    const double e2 = E(0.0, 2.0 * tau);
                    if (!(e2 <= tol_rate * (2.0 * tau))) break;
                    tau = 2.0 * tau;
                    err = e2;
                }
            }
        } else {
            tau = fmin(st->shrink * st->prev_step, t_rem);
            err = E(0.0, tau);
        }
        while (!(err <= tol_rate * tau)) {
            tau = 0.5 * tau;
            if (tau < st->min_step) {
                underflow = true;
                break;
            }
            err = E(0.0, tau);
        }
        if (!underflow) {
            const double s = tau / st->n_substeps;
            const double base = tau;
            int nsub = 0;
            while (nsub < st->max_substeps && tau < t_rem) {
                const double end = fmin(base + (nsub + 1) * s, t_rem);
                const double delta = E(tau, end);
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

    // ---- omega = exp(-i H_m tau) e_1
    const double beta0 = st->beta0;
    if (method == TE_SMALLEXP_EIG) {
        for (int k = tid; k < n; k += nt) {
            double s, c;
            sincos(L.dd[k] * tau, &s, &c);
            L.ph[k] = make_double2(c * L.z0[k], -s * L.z0[k]);
        }
        __syncthreads();
        for (int r = tid; r < n; r += nt) {
            double re = 0.0, im = 0.0;
            for (int k = 0; k < n; ++k) {
                const double z = L.Zt[k * n + r];
                re = fma(z, L.ph[k].x, re);
                im = fma(z, L.ph[k].y, im);
            }
            L.om[r] = make_double2(re, im);
        }
    } else if (!omega_cheb(L, cs, n, F, tau, mcap, &sh_S)) {
        // a step longer than the series' pieces reach (only a lucky breakdown takes one)
        if (tid == 0) {
            st->status = TE_ERR_UNSUPPORTED;
            st->done = 1;
            st->quad_warnings += sh_warn;
        }
        return;
    }
    __syncthreads();
    for (int r = tid; r < n; r += nt) {
        const double sc = beta0 * st->scale[r];
        st->coef[r] = make_double2(sc * L.om[r].x, sc * L.om[r].y);
    }
    if (tid == 0) {
        st->quad_integrals += n_integrals;
        st->quad_nodes += sh_nodes;
        st->eig_cycles += clk1 - clk0;
        st->search_cycles += clock64() - clk1;
        st->t_now = (tau == t_rem) ? T : t_now + tau;
        st->win_t0 = t_now;                     // window of this step, for intermediate samples
        st->win_t1 = t_now + tau;
        st->win_last = (tau == t_rem) ? 1 : 0;
        st->err_acc += err;
        st->prev_step = tau;
        st->first = 0;
        st->restarts += 1;
        st->breakdowns += brk ? 1 : 0;
        st->quad_warnings += sh_warn;
        st->last_m_eff = n;
        st->last_step = tau;
        st->last_err = err;
        st->min_err_step = fmin(st->min_err_step, err);
        st->done = (st->t_now >= T) ? 1 : 0;
        st->active = 1;                         // a step was taken: K4 recombines this solve
    }
}

}  // namespace

int step_smem_bytes(int m) {
    const size_t eig = sizeof(double2) * 2 * m +
                       sizeof(double) * ((size_t)m * m + 8 * (size_t)m + 3 * kTabNodes) +
                       sizeof(int) * m;
    const size_t cheb = sizeof(double2) * 2 * m +
                        sizeof(double) * (11 * (size_t)m + 2 * kKcap + 3 * kTabNodes +
                                          (size_t)keep_vectors(m) * m) +
                        sizeof(int) * m;
    return (int)(eig > cheb ? eig : cheb);
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

cudaError_t launch_step_batch(DevState* st, int nvec, int m, cudaStream_t s) {
    k_step<<<nvec, TE_STEP_THREADS, step_smem_bytes(m), s>>>(st, m);
    return cudaGetLastError();
}
