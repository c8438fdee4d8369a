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

// om[0..n) = exp(-i T tau) e_1.  T: diagonal al, off-diagonal be (be[n-1] unused),
// n <= blockDim.x.  Called by every thread of the block with the same arguments;
// jk: kKcap shared doubles, v3: 3 mcap shared doubles, sh_S: one shared double.
__device__ __forceinline__ void cheb_exp_e1(const double* al, const double* be, int n, double a,
                                            double b, double inv_a, double tau, double* jk,
                                            double* v3, int mcap, double* sh_S, double2* om) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const double z = a * tau;
    const int K = min(bessel_terms(fmin(z, (double)kKcap)), kKcap - kMillerExtra - 1);
    const int M = K + kMillerExtra;
    if (tid == 0) {
        // J_0..J_K(z) by Miller's backward recurrence, normalised by J_0 + 2 sum J_2k
        double* J = jk;
        if (!(z > 1e-300)) {
            J[0] = 1.0;
            for (int k = 1; k <= K; ++k) J[k] = 0.0;
            (*sh_S) = 1.0;
        } else {
            const double inv = 2.0 / z;
            double t = inv * M, jp = 0.0, jc = 1e-300, S = 0.0;
            for (int k = M; k >= 0; --k) {
                if (k <= K) J[k] = jc;
                if ((k & 1) == 0) S += (k == 0) ? jc : 2.0 * jc;
                if (k == 0) break;
                const double jn = fma(t, jc, -jp);
                jp = jc;
                jc = jn;
                t -= inv;
                if (fabs(jc) > kBig) {
                    jc *= kSmall;
                    jp *= kSmall;
                    S *= kSmall;
                    for (int q = k; q <= K; ++q) J[q] *= kSmall;
                }
            }
            (*sh_S) = S;
        }
    }
    __syncthreads();
    const double invS = 1.0 / (*sh_S);
    // sum_k c_k (-i)^k J_k T_k(T~) e_1, recomputing the Chebyshev vectors
    double* v0 = v3;
    double* v1 = v3 + mcap;
    double* v2 = v3 + 2 * mcap;
    double accr = 0.0, acci = 0.0;
    for (int i = tid; i < n; i += nt) {
        v0[i] = (i == 0) ? 1.0 : 0.0;
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
    double sb, cb;
    sincos(b * tau, &sb, &cb);                // e^{-i b tau}
    if (tid < n) om[tid] = make_double2(cb * accr + sb * acci, cb * acci - sb * accr);
}
