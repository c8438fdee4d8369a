// te_slices.cuh -- row products of the two sliced-ELLPACK forms of H, shared by
// the single-solve SpMV (te_sell.cu) and the grouped SpMV of many independent
// problems (te_multi.cu).  See te_sell.cu for the storage and the
// three-multiplication product.
#pragma once

#include "te_internal.cuh"

namespace te_slices {

// Loads of the vector being multiplied.  kL2 = false: through the read-only
// path (the vector does not change during the launch).  kL2 = true: from L2,
// for a kernel that reads vectors other blocks wrote earlier in the same launch
// (the fused Lanczos loop), where a line held in another SM's L1 could be stale.
template <bool kL2, class T>
__device__ __forceinline__ T ldx(const T* p) {
    if constexpr (kL2) return __ldcg(p);
    else return __ldg(p);
}

// Loads of the stored matrix: streamed once per product (evict-first) in the
// large-matrix kernels; kept cacheable in the fused loop, which re-reads the
// whole (small) matrix at every Lanczos step.
template <bool kL2, class T>
__device__ __forceinline__ T ldm(const T* p) {
    if constexpr (kL2) return __ldg(p);
    else return __ldcs(p);
}

// Asynchronous copies global -> shared (cp.async, sm_80 and later): the gathered
// vector elements of a later trip are in flight without holding registers.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Shared staging of one warp for the asynchronous row products: kStages trips of
// kTrip entries, each lane its own slots (x at sx[(stage * kTrip + u) * 32 + lane],
// x + y at ss[...]).  Bytes per warp: kStages * kTrip * 32 * 24.
template <int kTrip, int kStages>
struct Staging {
    static constexpr int kBytesPerWarp = kStages * kTrip * 32 * 24;
    double2* sx;
    double* ss;
    __device__ __forceinline__ Staging(unsigned char* warp_base)
        : sx(reinterpret_cast<double2*>(warp_base)),
          ss(reinterpret_cast<double*>(warp_base + kStages * kTrip * 32 * 16)) {}
};

// Slice products of the two stored forms.  row() returns, for the lane's row of
// slice s, the sums k1 = sum a (x + y), k2 = sum (b - a) x, k3 = sum (a + b) y
// over its stored entries, combined as (k1 - k3, k1 + k2), plus the diagonal
// term d_r x_r of the value-indexed form.
struct FullSlices {
    const int32_t* __restrict__ off;
    const int32_t* __restrict__ col;
    const double* __restrict__ va;
    const double2* __restrict__ vpq;
    template <bool kL2 = false>
    __device__ __forceinline__ double2 row(int64_t s, int lane, const double2* __restrict__ x,
                                           const double* __restrict__ xs, int64_t r,
                                           double2 xr) const {
        const int32_t o = __ldg(off + s);
        const int w = (__ldg(off + s + 1) - o) >> 5;
        const double* ap = va + o + lane;
        const double2* qp = vpq + o + lane;
        const int32_t* cp = col + o + lane;
        double k1 = 0.0, k2 = 0.0, k3 = 0.0;
        // four entries per trip, as in the value-indexed form below
        int k = 0;
#pragma unroll 1
        for (; k + 4 <= w; k += 4) {
            int c[4];
            double a[4], z[4];
            double2 q[4], xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                c[u] = ldm<kL2>(cp + 32 * (k + u));
                a[u] = ldm<kL2>(ap + 32 * (k + u));
                q[u] = ldm<kL2>(qp + 32 * (k + u));
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                xv[u] = ldx<kL2>(x + c[u]);
                z[u] = ldx<kL2>(xs + c[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                k1 = fma(a[u], z[u], k1);
                k2 = fma(q[u].x, xv[u].x, k2);
                k3 = fma(q[u].y, xv[u].y, k3);
            }
        }
#pragma unroll 1
        for (; k < w; ++k) {
            const double a0 = ldm<kL2>(ap + 32 * k);
            const double2 q0 = ldm<kL2>(qp + 32 * k);
            const int c0 = ldm<kL2>(cp + 32 * k);
            const double2 x0 = ldx<kL2>(x + c0);
            const double z0 = ldx<kL2>(xs + c0);
            k1 = fma(a0, z0, k1);
            k2 = fma(q0.x, x0.x, k2);
            k3 = fma(q0.y, x0.y, k3);
        }
        return make_double2(k1 - k3, k1 + k2);
    }
};

struct IndexedSlices {
    const int32_t* __restrict__ off;
    const int32_t* __restrict__ col;
    const uint16_t* __restrict__ vidx;
    const double* __restrict__ ta;
    const double2* __restrict__ tpq;
    const double* __restrict__ diag;
    template <bool kL2 = false>
    __device__ __forceinline__ double2 row(int64_t s, int lane, const double2* __restrict__ x,
                                           const double* __restrict__ xs, int64_t r,
                                           double2 xr) const {
        const int32_t o = __ldg(off + s);
        const int w = (__ldg(off + s + 1) - o) >> 5;
        const uint16_t* ip = vidx + o + lane;
        const int32_t* cp = col + o + lane;
        double k1 = 0.0, k2 = 0.0, k3 = 0.0;
        // four entries per trip: sixteen gathers in flight per lane before the FMAs
        int k = 0;
#pragma unroll 1
        for (; k + 4 <= w; k += 4) {
            int c[4], q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                c[u] = ldm<kL2>(cp + 32 * (k + u));
                q[u] = ldm<kL2>(ip + 32 * (k + u));
            }
            double a[4], z[4];
            double2 p[4], xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = __ldg(ta + q[u]);
                p[u] = __ldg(tpq + q[u]);
                xv[u] = ldx<kL2>(x + c[u]);
                z[u] = ldx<kL2>(xs + c[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                k1 = fma(a[u], z[u], k1);
                k2 = fma(p[u].x, xv[u].x, k2);
                k3 = fma(p[u].y, xv[u].y, k3);
            }
        }
#pragma unroll 1
        for (; k < w; ++k) {
            const int qq = ldm<kL2>(ip + 32 * k);
            const int cc = ldm<kL2>(cp + 32 * k);
            const double a0 = __ldg(ta + qq);
            const double2 p0 = __ldg(tpq + qq);
            const double2 x0 = ldx<kL2>(x + cc);
            const double z0 = ldx<kL2>(xs + cc);
            k1 = fma(a0, z0, k1);
            k2 = fma(p0.x, x0.x, k2);
            k3 = fma(p0.y, x0.y, k3);
        }
        const double dg = r >= 0 ? ldm<kL2>(diag + r) : 0.0;
        return make_double2(fma(dg, xr.x, k1 - k3), fma(dg, xr.y, k1 + k2));
    }

    // The same row product (same sums, same order) with the gathers of x and x + y
    // software-pipelined: the column and table indices are loaded two trips ahead into
    // registers, the gathers of the next trip go to the warp's shared staging by
    // cp.async while the FMAs of this trip run, so a warp never waits for its own
    // gathers.  Three stages: a stage is refilled one full trip after it was read.
    // The lane's rows of two slices at once (rows r0 of s0 and r1 of s1): over the
    // entries both rows have, each trip gathers two entries of each, so twice as many
    // independent loads and FMA chains are in flight per lane; the longer row then
    // finishes alone.  Each row's sums take its entries in storage order, as row()
    // does, so the results are bitwise row()'s.
    __device__ __forceinline__ void row_pair(int64_t s0, int64_t s1, int lane,
                                             const double2* __restrict__ x,
                                             const double* __restrict__ xs, int64_t r0, int64_t r1,
                                             double2 xr0, double2 xr1, double2* h0,
                                             double2* h1) const {
        const int32_t o0 = __ldg(off + s0), o1 = __ldg(off + s1);
        const int w0 = (__ldg(off + s0 + 1) - o0) >> 5;
        const int w1 = (__ldg(off + s1 + 1) - o1) >> 5;
        const uint16_t* ip0 = vidx + o0 + lane;
        const uint16_t* ip1 = vidx + o1 + lane;
        const int32_t* cp0 = col + o0 + lane;
        const int32_t* cp1 = col + o1 + lane;
        double a1 = 0.0, a2 = 0.0, a3 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0;
        const int wc = w0 < w1 ? w0 : w1;
        int k = 0;
#pragma unroll 1
        for (; k + 2 <= wc; k += 2) {
            int c[4], q[4];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                c[u] = __ldcs(cp0 + 32 * (k + u));
                q[u] = __ldcs(ip0 + 32 * (k + u));
                c[2 + u] = __ldcs(cp1 + 32 * (k + u));
                q[2 + u] = __ldcs(ip1 + 32 * (k + u));
            }
            double a[4], z[4];
            double2 p[4], xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = __ldg(ta + q[u]);
                p[u] = __ldg(tpq + q[u]);
                xv[u] = __ldg(x + c[u]);
                z[u] = __ldg(xs + c[u]);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                a1 = fma(a[u], z[u], a1);
                a2 = fma(p[u].x, xv[u].x, a2);
                a3 = fma(p[u].y, xv[u].y, a3);
                b1 = fma(a[2 + u], z[2 + u], b1);
                b2 = fma(p[2 + u].x, xv[2 + u].x, b2);
                b3 = fma(p[2 + u].y, xv[2 + u].y, b3);
            }
        }
        // the rest of each row alone, in storage order
        auto rest = [&](const int32_t* cp, const uint16_t* ip, int w, double& k1, double& k2,
                        double& k3) {
#pragma unroll 1
            for (int kk = k; kk < w; ++kk) {
                const int qq = __ldcs(ip + 32 * kk);
                const int cc = __ldcs(cp + 32 * kk);
                const double a0 = __ldg(ta + qq);
                const double2 p0 = __ldg(tpq + qq);
                const double2 x0 = __ldg(x + cc);
                const double z0 = __ldg(xs + cc);
                k1 = fma(a0, z0, k1);
                k2 = fma(p0.x, x0.x, k2);
                k3 = fma(p0.y, x0.y, k3);
            }
        };
        rest(cp0, ip0, w0, a1, a2, a3);
        rest(cp1, ip1, w1, b1, b2, b3);
        const double d0 = r0 >= 0 ? __ldcs(diag + r0) : 0.0;
        const double d1 = r1 >= 0 ? __ldcs(diag + r1) : 0.0;
        *h0 = make_double2(fma(d0, xr0.x, a1 - a3), fma(d0, xr0.y, a1 + a2));
        *h1 = make_double2(fma(d1, xr1.x, b1 - b3), fma(d1, xr1.y, b1 + b2));
    }

    template <int kTrip>
    __device__ __forceinline__ double2 row_async(int64_t s, int lane, const double2* __restrict__ x,
                                                 const double* __restrict__ xs, int64_t r,
                                                 double2 xr, Staging<kTrip, 3> st) const {
        const int32_t o = __ldg(off + s);
        const int w = (__ldg(off + s + 1) - o) >> 5;
        const uint16_t* ip = vidx + o + lane;
        const int32_t* cp = col + o + lane;
        double k1 = 0.0, k2 = 0.0, k3 = 0.0;
        const int nt = w / kTrip;                        // full trips
        int qc[kTrip], q1[kTrip], c1[kTrip];
        if (nt > 0) {
#pragma unroll
            for (int u = 0; u < kTrip; ++u) {            // trip 0: indices, then its gathers
                const int c0 = __ldcs(cp + 32 * u);
                qc[u] = __ldcs(ip + 32 * u);
                cp_async16(st.sx + u * 32 + lane, x + c0);
                cp_async8(st.ss + u * 32 + lane, xs + c0);
            }
            cp_async_commit();
            if (nt > 1) {
#pragma unroll
                for (int u = 0; u < kTrip; ++u) {        // trip 1: indices only
                    c1[u] = __ldcs(cp + 32 * (kTrip + u));
                    q1[u] = __ldcs(ip + 32 * (kTrip + u));
                }
            }
        }
#pragma unroll 1
        for (int t = 0; t < nt; ++t) {
            int q2[kTrip], c2[kTrip];
            if (t + 2 < nt) {                            // indices of trip t + 2
#pragma unroll
                for (int u = 0; u < kTrip; ++u) {
                    c2[u] = __ldcs(cp + 32 * ((t + 2) * kTrip + u));
                    q2[u] = __ldcs(ip + 32 * ((t + 2) * kTrip + u));
                }
            }
            if (t + 1 < nt) {                            // gathers of trip t + 1
                const int sg = (t + 1) % 3;
#pragma unroll
                for (int u = 0; u < kTrip; ++u) {
                    cp_async16(st.sx + (sg * kTrip + u) * 32 + lane, x + c1[u]);
                    cp_async8(st.ss + (sg * kTrip + u) * 32 + lane, xs + c1[u]);
                }
            }
            cp_async_commit();
            cp_async_wait<1>();                          // trip t has landed
            const int sc = t % 3;
#pragma unroll
            for (int u = 0; u < kTrip; ++u) {
                const double a = __ldg(ta + qc[u]);
                const double2 p = __ldg(tpq + qc[u]);
                const double2 xv = st.sx[(sc * kTrip + u) * 32 + lane];
                const double z = st.ss[(sc * kTrip + u) * 32 + lane];
                k1 = fma(a, z, k1);
                k2 = fma(p.x, xv.x, k2);
                k3 = fma(p.y, xv.y, k3);
            }
#pragma unroll
            for (int u = 0; u < kTrip; ++u) {
                qc[u] = q1[u];
                q1[u] = q2[u];
                c1[u] = c2[u];
            }
        }
        cp_async_wait<0>();
#pragma unroll 1
        for (int k = nt * kTrip; k < w; ++k) {
            const int qq = __ldcs(ip + 32 * k);
            const int cc = __ldcs(cp + 32 * k);
            const double a0 = __ldg(ta + qq);
            const double2 p0 = __ldg(tpq + qq);
            const double2 x0 = __ldg(x + cc);
            const double z0 = __ldg(xs + cc);
            k1 = fma(a0, z0, k1);
            k2 = fma(p0.x, x0.x, k2);
            k3 = fma(p0.y, x0.y, k3);
        }
        const double dg = r >= 0 ? __ldcs(diag + r) : 0.0;
        return make_double2(fma(dg, xr.x, k1 - k3), fma(dg, xr.y, k1 + k2));
    }
};

// Value-indexed form of a matrix whose off-diagonal values are all real (b = 0,
// e.g. the transverse-field Ising chain): Re(h x) = a x and Im(h x) = a y, two
// DFMA per entry instead of three, and no gather of x + y.  The table is the
// same a column of the complex form.
struct RealIndexedSlices {
    const int32_t* __restrict__ off;
    const int32_t* __restrict__ col;
    const uint16_t* __restrict__ vidx;
    const double* __restrict__ ta;
    const double* __restrict__ diag;
    template <bool kL2 = false>
    __device__ __forceinline__ double2 row(int64_t s, int lane, const double2* __restrict__ x,
                                           const double* __restrict__ /*xs*/, int64_t r,
                                           double2 xr) const {
        const int32_t o = __ldg(off + s);
        const int w = (__ldg(off + s + 1) - o) >> 5;
        const uint16_t* ip = vidx + o + lane;
        const int32_t* cp = col + o + lane;
        double k1 = 0.0, k2 = 0.0;
        int k = 0;
#pragma unroll 1
        for (; k + 4 <= w; k += 4) {
            int c[4], q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                c[u] = ldm<kL2>(cp + 32 * (k + u));
                q[u] = ldm<kL2>(ip + 32 * (k + u));
            }
            double a[4];
            double2 xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = __ldg(ta + q[u]);
                xv[u] = ldx<kL2>(x + c[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                k1 = fma(a[u], xv[u].x, k1);
                k2 = fma(a[u], xv[u].y, k2);
            }
        }
#pragma unroll 1
        for (; k < w; ++k) {
            const int qq = ldm<kL2>(ip + 32 * k);
            const int cc = ldm<kL2>(cp + 32 * k);
            const double a0 = __ldg(ta + qq);
            const double2 x0 = ldx<kL2>(x + cc);
            k1 = fma(a0, x0.x, k1);
            k2 = fma(a0, x0.y, k2);
        }
        const double dg = r >= 0 ? ldm<kL2>(diag + r) : 0.0;
        return make_double2(fma(dg, xr.x, k1), fma(dg, xr.y, k2));
    }
};

}  // namespace te_slices
