// te_smallexp.cuh -- exp(-i T tau) e_1 for a real symmetric tridiagonal T by the
// Jacobi-Anger / Chebyshev series, shared by the step kernel (te_step.cu) and
// the intermediate-time sampler (te_sample.cu).
//
// With [b - a, b + a] an interval containing the spectrum of T and
// T~ = (T - b) / a,
//   exp(-i T tau) = e^{-i b tau} sum_k c_k (-i)^k J_k(a tau) T_k(T~),  c_0 = 1, c_k = 2,
// with Bessel functions J_k (Miller's backward recurrence, normalised by
// J_0 + 2 sum J_2k = 1) and Chebyshev polynomials T_k applied to e_1 by their
// three-term recurrence.
#pragma once

#include "te_internal.cuh"

constexpr int kKcap = 3072;          // largest Chebyshev / Bessel index
constexpr int kMillerExtra = 20;     // backward recurrence starts this far above the last term
constexpr double kBig = 1e250, kSmall = 1e-250;

// Number of Bessel terms kept at argument z: J_k(z) is below 1e-30 past it.
__device__ __forceinline__ int bessel_terms(double z) {
    return (int)ceil(z + 10.0 * cbrt(z) + 30.0);
}

// Largest argument z = a tau the series takes in one piece (K(2048) = 2205 terms,
// well inside kKcap), and the most pieces one call may take.  A longer tau is
// split into p equal pieces, exp(-i T tau) = (exp(-i T tau / p))^p, each piece
// applied to the previous piece's complex result: exact on the Krylov space, so
// a lucky breakdown (which takes the whole remaining time in one step, Sec. 2.4)
// may evaluate any tau without truncating the series.  Beyond kMaxPieces pieces
// (z > 2048 x 512) the call reports failure instead of truncating.
constexpr double kZPiece = 2048.0;
constexpr int kMaxPieces = 512;

// One application of the truncated series to a real vector x (x = e_1 when
// u == nullptr, else x_i = Re u_i (part 0) or Im u_i (part 1)):
//   (accr + i acci) = sum_{k<=K} c_k (-i)^k J_k T_k(T~) x,   row tid of the result.
// jk[0..K] holds J_k unnormalised; invS is the normalisation.  n <= blockDim.x.
__device__ __forceinline__ void cheb_pass(const double* al, const double* be, int n, double b,
                                          double inv_a, int K, const double* jk, double invS,
                                          double* v3, int mcap, const double2* u, int part,
                                          double* accr_out, double* acci_out) {
    const int tid = threadIdx.x, nt = blockDim.x;
    double* v0 = v3;
    double* v1 = v3 + mcap;
    double* v2 = v3 + 2 * mcap;
    double accr = 0.0, acci = 0.0;
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
        v0[i] = (u == nullptr) ? ((i == 0) ? 1.0 : 0.0) : (part == 0 ? u[i].x : u[i].y);
        v2[i] = 0.0;
    }
    __syncthreads();
    double* vc = v0;
    double* vp = v2;
    double* vn = v1;
    for (int k = 0; k <= K; ++k) {
        const double c = (k == 0 ? 1.0 : 2.0) * jk[k] * invS;
        if (tid < n) {
            const double x = vc[tid];
            switch (k & 3) {
                case 0: accr = fma(c, x, accr); break;
                case 1: acci = fma(-c, x, acci); break;
                case 2: accr = fma(-c, x, accr); break;
                default: acci = fma(c, x, acci); break;
            }
        }
        if (k == K) break;
        for (int i = tid; i < n; i += nt) {
            double tv = (al[i] - b) * vc[i];
            if (i > 0) tv = fma(be[i - 1], vc[i - 1], tv);
            if (i + 1 < n) tv = fma(be[i], vc[i + 1], tv);
            tv *= inv_a;
            vn[i] = (k == 0) ? tv : 2.0 * tv - vp[i];
        }
        __syncthreads();
        double* tmp = vp;
        vp = vc;
        vc = vn;
        vn = tmp;
    }
    *accr_out = accr;
    *acci_out = acci;
}

// Miller's coefficients 2k/z go through a table of this many entries, filled by
// all threads of the block, so the serial recurrence issues one FP64 instruction
// per step (two on even k) instead of also forming 2k/z and testing |J_k|.
constexpr int kMillerChunk = 256;

// om[0..n) = exp(-i T tau) e_1.  T: diagonal al, off-diagonal be (be[n-1] unused),
// n <= blockDim.x.  Called by every thread of the block with the same arguments;
// jk: kKcap shared doubles, v3: 3 mcap shared doubles, sh_S: one shared double.
// vk (optional): the vectors T_k(T~) e_1 for k < nvk, vk + k * mcap, as the
// recurrence of cheb_pass computes them (the step kernel keeps those of its step
// search); a one-piece series with K < nvk then sums them directly instead of
// running the recurrence again, with the same sums in the same order, so the
// result is bitwise the one cheb_pass gives.  n = 1 takes the closed form
// e^{-i al_0 tau}.  Returns false (every thread, om untouched) when a tau would
// need more than kMaxPieces pieces.
__device__ __forceinline__ bool cheb_exp_e1(const double* al, const double* be, int n, double a,
                                            double b, double inv_a, double tau, double* jk,
                                            double* v3, int mcap, double* sh_S, double2* om,
                                            const double* vk = nullptr, int nvk = 0) {
    __shared__ double tk[kMillerChunk];
    const int tid = threadIdx.x, nt = blockDim.x;
    if (n == 1) {
        if (tid == 0) {
            double s, c;
            sincos(al[0] * tau, &s, &c);
            om[0] = make_double2(c, -s);
        }
        return true;
    }
    int p = 1;
    if (a * tau > kZPiece) {
        const double pf = ceil(a * tau / kZPiece);
        if (!(pf <= (double)kMaxPieces)) return false;
        p = (int)pf;
    }
    const double tp = (p == 1) ? tau : tau / p;          // one piece
    const double z = a * tp;
    const int K = min(bessel_terms(fmin(z, (double)kKcap)), kKcap - kMillerExtra - 1);
    const int M = K + kMillerExtra;
    // J_0..J_K(z) by Miller's backward recurrence, normalised by J_0 + 2 sum J_2k,
    // on thread 0.  The coefficient 2k/z is formed from k (a table of
    // kMillerChunk values at a time, filled by the block): decrementing it by 2/z
    // instead accumulates one rounding per step, which shifts the phase of the
    // oscillating J_k (k < z) by ~1e-11 at z = 2000.  The overflow test
    // |J_k| > kBig compares the bit patterns (ordered like the magnitudes for
    // non-negative doubles), on the integer pipe.
    double* J = jk;
    __syncthreads();
    if (!(z > 1e-300)) {
        if (tid == 0) {
            J[0] = 1.0;
            for (int k = 1; k <= K; ++k) J[k] = 0.0;
            (*sh_S) = 1.0;
        }
    } else {
        const double inv = 2.0 / z;
        const unsigned long long big = (unsigned long long)__double_as_longlong(kBig);
        double jp = 0.0, jc = 1e-300, S = 0.0;              // thread 0's recurrence state
        for (int top = M; top >= 0; top -= kMillerChunk) {
            const int lo = max(top - (kMillerChunk - 1), 0);
            for (int k = lo + tid; k <= top; k += nt) tk[k - lo] = inv * (double)k;
            __syncthreads();
            if (tid == 0) {
                for (int k = top; k >= lo; --k) {
                    if (k <= K) J[k] = jc;
                    if ((k & 1) == 0) S += (k == 0) ? jc : 2.0 * jc;
                    if (k == 0) break;
                    const double jn = fma(tk[k - lo], jc, -jp);
                    jp = jc;
                    jc = jn;
                    if (((unsigned long long)__double_as_longlong(jc) & 0x7fffffffffffffffull) > big) {
                        jc *= kSmall;
                        jp *= kSmall;
                        S *= kSmall;
                        for (int q = k; q <= K; ++q) J[q] *= kSmall;
                    }
                }
                if (lo == 0) (*sh_S) = S;
            }
            __syncthreads();
        }
    }
    __syncthreads();
    const double invS = 1.0 / (*sh_S);
    double sb, cb;
    sincos(b * tp, &sb, &cb);                 // e^{-i b tp}
    // first piece from e_1
    double accr = 0.0, acci = 0.0;
    if (p == 1 && vk != nullptr && K < nvk) {
        // the vectors T_k(T~) e_1 are stored: sum c_k (-i)^k J_k v_k row by row
        // (cheb_pass's coefficients and order), J_k replaced by c_k in place
        for (int k = tid; k <= K; k += nt) jk[k] = (k == 0 ? 1.0 : 2.0) * jk[k] * invS;
        __syncthreads();
        if (tid < n) {
            for (int k = 0; k <= K; ++k) {
                const double c = jk[k];
                const double x = vk[(size_t)k * mcap + tid];
                switch (k & 3) {
                    case 0: accr = fma(c, x, accr); break;
                    case 1: acci = fma(-c, x, acci); break;
                    case 2: accr = fma(-c, x, accr); break;
                    default: acci = fma(c, x, acci); break;
                }
            }
        }
    } else {
        cheb_pass(al, be, n, b, inv_a, K, jk, invS, v3, mcap, nullptr, 0, &accr, &acci);
    }
    // the phase e^{-i b tp} applied with explicit FMAs: a free-standing
    // x * y + u * v leaves the compiler the choice of product to fuse, which can
    // differ between the kernels that evaluate this series
    double2 r = make_double2(fma(cb, accr, sb * acci), fma(cb, acci, -(sb * accr)));
    // later pieces from the previous result u = x + i y:
    //   S(u) = S(x) + i S(y), S the real-coefficient series applied to a real vector
    for (int q = 1; q < p; ++q) {
        __syncthreads();
        if (tid < n) om[tid] = r;
        double xr, xi, yr, yi;
        cheb_pass(al, be, n, b, inv_a, K, jk, invS, v3, mcap, om, 0, &xr, &xi);
        cheb_pass(al, be, n, b, inv_a, K, jk, invS, v3, mcap, om, 1, &yr, &yi);
        const double sr = xr - yi, si = xi + yr;
        r = make_double2(fma(cb, sr, sb * si), fma(cb, si, -(sb * sr)));
    }
    __syncthreads();
    if (tid < n) om[tid] = r;
    return true;
}
