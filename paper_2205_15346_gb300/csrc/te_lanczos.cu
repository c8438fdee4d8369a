// te_lanczos.cu -- bandwidth-bound kernels of the Lanczos cycle (sm_103a).
//
// Sec. 2.1 of arXiv 2205.15346 (eq. arnoldi) builds v_{j+1} from
//     w_j = H v_j - h_{j-1,j} v_{j-1},  h_{j,j} = <v_j, w_j>,
//     w~_j = w_j - h_{j,j} v_j,          h_{j+1,j} = ||w~_j||,  v_{j+1} = w~_j / h_{j+1,j}.
// Here the basis is stored unnormalised: column j of V holds u_j with
// v_j = scale[j] * u_j, so the division by h_{j+1,j} is folded into the next
// product instead of costing a pass over the vector.  Each Lanczos step is two
// kernels:
//   K1: y = (sign * scale[j]) H u_j - (beta[j-1] scale[j-1]) u_{j-1}, written to
//       column j+1, with the per-block partials of Re <u_j, y> (alpha_j);
//   K2: w~ = y - alpha_j scale[j] u_j in place, with ||w~||^2 partials; its last
//       block takes the square root, tests for breakdown and sets scale[j+1].
// Reductions are deterministic: each block writes one partial, the last block
// to arrive (atomic counter) adds all partials in a fixed order.
#include "te_internal.cuh"

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; the result is valid in every thread.  sh >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = (lane < nw) ? sh[lane] : 0.0;
    r = warp_sum(r);
    return r;
}

// Thread 0 publishes the block's partial; returns true in every thread of the
// block that arrives last.  That block then reads all partials.
__device__ __forceinline__ bool publish_partial(double v, double* partials, int slot,
                                                unsigned int* counter) {
    __shared__ bool am_last;
    if (threadIdx.x == 0) {
        partials[slot] = v;
        __threadfence();
        unsigned int prev = atomicAdd(counter, 1u);
        am_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    return am_last;
}

// Fixed-order sum of partials[0..n) by one block (reads through L2).
__device__ __forceinline__ double gather_partials(const double* partials, int n, int stride,
                                                  double* sh) {
    __threadfence();
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += __ldcg(partials + (size_t)i * stride);
    return block_sum(v, sh);
}

__device__ __forceinline__ bool halted(const DevState* st) {
    return st->status != 0 || st->done != 0;
}

// ---------------------------------------------------------------- K0

__global__ void __launch_bounds__(TE_BLOCK) k_init_norm(const double2* __restrict__ v,
                                                        double* __restrict__ S, int64_t d,
                                                        DevState* st, double* partials) {
    __shared__ double sh[32];
    double acc = 0.0;
    bool finite = true;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d;
         i += (int64_t)gridDim.x * blockDim.x) {
        double2 a = v[i];
        finite &= isfinite(a.x) && isfinite(a.y);
        acc += a.x * a.x + a.y * a.y;
        if (S) S[i] = a.x + a.y;
    }
    if (!finite) acc = __longlong_as_double(0x7ff8000000000000LL);   // NaN marks it
    double s = block_sum(acc, sh);
    if (publish_partial(s, partials, blockIdx.x, &st->counter[0])) {
        double tot = gather_partials(partials, gridDim.x, 1, sh);
        if (threadIdx.x == 0) {
            double nrm = sqrt(tot);
            st->beta0 = nrm;
            st->scale[0] = 1.0 / nrm;
            st->stop = 0;
            st->m_eff = st->m;
            st->breakdown = 0;
            if (!isfinite(nrm)) {
                st->status = TE_ERR_NONFINITE;
            } else if (fabs(nrm - 1.0) > 1e-10) {
                st->status = TE_ERR_NOT_NORMALIZED;
            }
            st->counter[0] = 0;
        }
    }
}

// ---------------------------------------------------------------- K1

// G lanes per CSR row; a warp covers 32 / G consecutive rows per iteration, so
// the value/column loads of a warp are one contiguous stretch of the CSR arrays.
// mode 0: Lanczos step j (coefficients from st); mode 1: plain y = H x.
template <int G>
__global__ void __launch_bounds__(TE_BLOCK) k_spmv_lanczos(
    const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const double2* __restrict__ val, const double2* __restrict__ x,
    const double2* __restrict__ xprev, double2* __restrict__ y, int64_t d, DevState* st, int j,
    int mode, double* partials) {
    __shared__ double sh[32];
    double cx = 1.0, bp = 0.0;
    if (mode == 0) {
        if (halted(st) || st->stop) return;
        cx = st->sign * st->scale[j];
        if (j > 0) bp = st->beta[j - 1] * st->scale[j - 1];
    }
    const int lane = threadIdx.x & 31;
    const int sub = lane & (G - 1);
    constexpr int RPW = 32 / G;                       // rows per warp iteration
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double acc = 0.0;
    for (int64_t base = warp * RPW; base < d; base += nwarps * RPW) {
        const int64_t row = base + lane / G;
        double re = 0.0, im = 0.0;
        if (row < d) {
            const int b = __ldg(rowptr + row), e = __ldg(rowptr + row + 1);
            int k = b + sub;
            // two entries per lane per trip keep more loads in flight
            for (; k + G < e; k += 2 * G) {
                const double2 a0 = __ldcs(val + k);
                const double2 a1 = __ldcs(val + k + G);
                const int c0 = __ldcs(col + k);
                const int c1 = __ldcs(col + k + G);
                const double2 x0 = __ldg(x + c0);
                const double2 x1 = __ldg(x + c1);
                re = fma(a0.x, x0.x, re);
                re = fma(-a0.y, x0.y, re);
                im = fma(a0.x, x0.y, im);
                im = fma(a0.y, x0.x, im);
                re = fma(a1.x, x1.x, re);
                re = fma(-a1.y, x1.y, re);
                im = fma(a1.x, x1.y, im);
                im = fma(a1.y, x1.x, im);
            }
            if (k < e) {
                const double2 a0 = __ldcs(val + k);
                const double2 x0 = __ldg(x + __ldcs(col + k));
                re = fma(a0.x, x0.x, re);
                re = fma(-a0.y, x0.y, re);
                im = fma(a0.x, x0.y, im);
                im = fma(a0.y, x0.x, im);
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o, G);
            im += __shfl_xor_sync(0xffffffffu, im, o, G);
        }
        if (sub == 0 && row < d) {
            double2 out;
            out.x = cx * re;
            out.y = cx * im;
            if (bp != 0.0) {
                const double2 p = __ldcs(xprev + row);
                out.x -= bp * p.x;
                out.y -= bp * p.y;
            }
            y[row] = out;
            const double2 xr = __ldg(x + row);
            acc += xr.x * out.x + xr.y * out.y;       // Re(conj(x_r) y_r)
        }
    }
    const double s = block_sum(acc, sh);
    unsigned int* ctr = &st->counter[1];
    if (publish_partial(s, partials, blockIdx.x, ctr)) {
        const double tot = gather_partials(partials, gridDim.x, 1, sh);
        if (threadIdx.x == 0) {
            if (mode == 0) {
                const double a = st->scale[j] * tot;  // alpha_j = Re <v_j, w_j>
                st->alpha[j] = a;
                st->as_cur = a * st->scale[j];
                st->matvecs += 1;
            } else {
                st->spmv_dot = tot;
            }
            *ctr = 0;
        }
    }
}

// ---------------------------------------------------------------- K2

// Breakdown decision after ||w~_j|| is known (Algorithm 1 step 1; the test is
// h_{j+1,j} < tol_rate, the inner loop then ends with m_eff = j + 1).
__device__ __forceinline__ void lanczos_decide(DevState* st, int j, double nrm) {
    st->beta[j] = nrm;
    if (!(nrm >= st->tol_rate)) {            // also catches NaN
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

__global__ void __launch_bounds__(TE_BLOCK) k_orth_norm(double2* __restrict__ w,
                                                        double* __restrict__ S,
                                                        const double2* __restrict__ u, int64_t d,
                                                        DevState* st, int j, int write,
                                                        int decide, double* partials) {
    __shared__ double sh[32];
    if (halted(st) || st->stop) return;
    const double as = st->as_cur;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // four independent elements per trip keep enough loads in flight
    for (; i + 3 * stride < d; i += 4 * stride) {
        double2 yv[4], uv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            yv[q] = w[i + q * stride];
            uv[q] = __ldg(u + i + q * stride);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            yv[q].x = fma(-as, uv[q].x, yv[q].x);
            yv[q].y = fma(-as, uv[q].y, yv[q].y);
            if (write) {
                w[i + q * stride] = yv[q];
                if (S) S[i + q * stride] = yv[q].x + yv[q].y;
            }
            acc = fma(yv[q].x, yv[q].x, acc);
            acc = fma(yv[q].y, yv[q].y, acc);
        }
    }
    for (; i < d; i += stride) {
        double2 y0 = w[i];
        const double2 u0 = __ldg(u + i);
        y0.x = fma(-as, u0.x, y0.x);
        y0.y = fma(-as, u0.y, y0.y);
        if (write) {
            w[i] = y0;
            if (S) S[i] = y0.x + y0.y;
        }
        acc = fma(y0.x, y0.x, acc);
        acc = fma(y0.y, y0.y, acc);
    }
    if (!decide) return;
    const double s = block_sum(acc, sh);
    if (publish_partial(s, partials, blockIdx.x, &st->counter[2])) {
        const double tot = gather_partials(partials, gridDim.x, 1, sh);
        if (threadIdx.x == 0) {
            lanczos_decide(st, j, sqrt(tot));
            st->counter[2] = 0;
        }
    }
}

// ---------------------------------------------------------------- KR (option)

// c_k = <u_k, w> for k = 0..j (one pass over the j+1 stored vectors); the last
// block turns them into rcoef[k] = scale[k]^2 c_k so that the projection of w on
// v_k is rcoef[k] u_k.
__global__ void __launch_bounds__(TE_BLOCK) k_reorth_dots(const double2* __restrict__ V,
                                                          const double2* __restrict__ w,
                                                          int64_t d, DevState* st, int j,
                                                          double* partials) {
    __shared__ double sh[32];
    if (halted(st) || st->stop) return;
    const int nk = j + 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int k = 0; k < nk; ++k) {
        const double2* u = V + (size_t)k * d;
        double re = 0.0, im = 0.0;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += stride) {
            const double2 a = __ldg(u + i);
            const double2 b = w[i];
            re += a.x * b.x + a.y * b.y;       // conj(a) b
            im += a.x * b.y - a.y * b.x;
        }
        const double sre = block_sum(re, sh);
        const double sim = block_sum(im, sh);
        if (threadIdx.x == 0) {
            partials[((size_t)blockIdx.x * TE_M_MAX + k) * 2 + 0] = sre;
            partials[((size_t)blockIdx.x * TE_M_MAX + k) * 2 + 1] = sim;
        }
    }
    __shared__ bool am_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        am_last = (atomicAdd(&st->counter[3], 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    for (int k = 0; k < nk; ++k) {
        const double re = gather_partials(partials + 2 * k, gridDim.x, 2 * TE_M_MAX, sh);
        const double im = gather_partials(partials + 2 * k + 1, gridDim.x, 2 * TE_M_MAX, sh);
        if (threadIdx.x == 0) {
            const double s2 = st->scale[k] * st->scale[k];
            st->rcoef[k] = make_double2(s2 * re, s2 * im);
        }
    }
    if (threadIdx.x == 0) st->counter[3] = 0;
}

// w -= sum_k rcoef[k] u_k; with decide, also ||w|| and the breakdown test.
__global__ void __launch_bounds__(TE_BLOCK) k_reorth_update(const double2* __restrict__ V,
                                                            double2* __restrict__ w,
                                                            double* __restrict__ S, int64_t d,
                                                            DevState* st, int j, int decide,
                                                            double* partials) {
    __shared__ double sh[32];
    __shared__ double2 c[TE_M_MAX];
    if (halted(st) || st->stop) return;
    const int nk = j + 1;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) c[k] = st->rcoef[k];
    __syncthreads();
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d;
         i += (int64_t)gridDim.x * blockDim.x) {
        double2 r = w[i];
        for (int k = 0; k < nk; ++k) {
            const double2 a = __ldg(V + (size_t)k * d + i);
            r.x -= c[k].x * a.x - c[k].y * a.y;
            r.y -= c[k].x * a.y + c[k].y * a.x;
        }
        w[i] = r;
        if (S) S[i] = r.x + r.y;
        acc += r.x * r.x + r.y * r.y;
    }
    if (!decide) return;
    const double s = block_sum(acc, sh);
    if (publish_partial(s, partials, blockIdx.x, &st->counter[4])) {
        const double tot = gather_partials(partials, gridDim.x, 1, sh);
        if (threadIdx.x == 0) {
            lanczos_decide(st, j, sqrt(tot));
            st->counter[4] = 0;
        }
    }
}

// ---------------------------------------------------------------- K4

// w = sum_{k < m_eff} coef[k] u_k into column 0, then ||w|| for the next restart
// (Algorithm 1 step 3; v_1 of the next Krylov space is w / ||w||).
// With S (the sliced path: Re + Im of every column, S[k d + i]) the sum uses the
// three-multiplication product of the SpMV: for c_k = a + ib and u = x + iy,
// Re(c u) = a (x + y) - (a + b) y and Im(c u) = a (x + y) + (b - a) x, three DFMA
// per element and column instead of four.
__global__ void __launch_bounds__(TE_BLOCK) k_recombine(double2* __restrict__ V,
                                                        double* __restrict__ S, int64_t d,
                                                        DevState* st, double* partials) {
    __shared__ double sh[32];
    __shared__ double2 c[TE_M_MAX];
    __shared__ double ca[TE_M_MAX], cp[TE_M_MAX], cq[TE_M_MAX];
    if (st->status != 0) return;
    const int nk = st->last_m_eff;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        const double2 ck = st->coef[k];
        c[k] = ck;
        ca[k] = ck.x;                // a
        cp[k] = ck.y - ck.x;         // b - a
        cq[k] = ck.x + ck.y;         // a + b
    }
    __syncthreads();
    double acc = 0.0;
    if (S) {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d;
             i += (int64_t)gridDim.x * blockDim.x) {
            double k1 = 0.0, k2 = 0.0, k3 = 0.0;
            int k = 0;
            for (; k + 4 <= nk; k += 4) {
                double2 a[4];
                double z[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    a[q] = __ldcs(V + (size_t)(k + q) * d + i);
                    z[q] = __ldcs(S + (size_t)(k + q) * d + i);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    k1 = fma(ca[k + q], z[q], k1);
                    k2 = fma(cp[k + q], a[q].x, k2);
                    k3 = fma(cq[k + q], a[q].y, k3);
                }
            }
            for (; k < nk; ++k) {
                const double2 a = __ldcs(V + (size_t)k * d + i);
                const double z = __ldcs(S + (size_t)k * d + i);
                k1 = fma(ca[k], z, k1);
                k2 = fma(cp[k], a.x, k2);
                k3 = fma(cq[k], a.y, k3);
            }
            const double re = k1 - k3, im = k1 + k2;
            V[i] = make_double2(re, im);
            S[i] = re + im;
            acc = fma(re, re, acc);
            acc = fma(im, im, acc);
        }
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d && !S;
         i += (int64_t)gridDim.x * blockDim.x) {
        double re = 0.0, im = 0.0;
        int k = 0;
        for (; k + 4 <= nk; k += 4) {
            double2 a[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) a[q] = __ldcs(V + (size_t)(k + q) * d + i);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                re = fma(c[k + q].x, a[q].x, re);
                re = fma(-c[k + q].y, a[q].y, re);
                im = fma(c[k + q].x, a[q].y, im);
                im = fma(c[k + q].y, a[q].x, im);
            }
        }
        for (; k < nk; ++k) {
            const double2 a = __ldcs(V + (size_t)k * d + i);
            re = fma(c[k].x, a.x, re);
            re = fma(-c[k].y, a.y, re);
            im = fma(c[k].x, a.y, im);
            im = fma(c[k].y, a.x, im);
        }
        V[i] = make_double2(re, im);
        acc += re * re + im * im;
    }
    const double s = block_sum(acc, sh);
    if (publish_partial(s, partials, blockIdx.x, &st->counter[5])) {
        const double tot = gather_partials(partials, gridDim.x, 1, sh);
        if (threadIdx.x == 0) {
            const double nrm = sqrt(tot);
            st->beta0 = nrm;
            st->scale[0] = 1.0 / nrm;
            st->stop = 0;
            st->m_eff = st->m;
            st->breakdown = 0;
            if (!isfinite(nrm)) st->status = TE_ERR_NONFINITE;
            st->counter[5] = 0;
        }
    }
}

template <int G>
int spmv_occ() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv_lanczos<G>, TE_BLOCK, 0);
    return nb > 0 ? nb : 1;
}

}  // namespace

int spmv_lanes_for(double avg) {
    if (avg <= 3.0) return 2;
    if (avg <= 20.0) return 4;
    if (avg <= 40.0) return 8;
    if (avg <= 72.0) return 16;
    return 32;
}

int occupancy_grid_spmv(int lanes, int num_sms) {
    int nb = 1;
    switch (lanes) {
        case 1: nb = spmv_occ<1>(); break;
        case 2: nb = spmv_occ<2>(); break;
        case 4: nb = spmv_occ<4>(); break;
        case 8: nb = spmv_occ<8>(); break;
        case 16: nb = spmv_occ<16>(); break;
        default: nb = spmv_occ<32>(); break;
    }
    return nb * num_sms;
}

int spmv_grid(int lanes, int64_t d, int num_sms) {
    const int64_t rows_per_block = (TE_BLOCK / 32) * (32 / lanes);
    const int64_t need = (d + rows_per_block - 1) / rows_per_block;
    const int64_t full = occupancy_grid_spmv(lanes, num_sms);
    return (int)(need < full ? (need > 0 ? need : 1) : full);
}

cudaError_t launch_init_norm(const double2* v, double* S, int64_t d, DevState* st,
                             double* partials, int grid, cudaStream_t s) {
    k_init_norm<<<grid, TE_BLOCK, 0, s>>>(v, S, d, st, partials);
    return cudaGetLastError();
}

cudaError_t launch_spmv_lanczos(const te_matrix* H, int lanes, const double2* x,
                                const double2* xprev, double2* y, DevState* st, int j, int mode,
                                double* partials, int grid, cudaStream_t s) {
#define TE_K1(G)                                                                             \
    k_spmv_lanczos<G><<<grid, TE_BLOCK, 0, s>>>(H->rowptr, H->col, H->val, x, xprev, y, H->d, \
                                                st, j, mode, partials)
    switch (lanes) {
        case 1: TE_K1(1); break;
        case 2: TE_K1(2); break;
        case 4: TE_K1(4); break;
        case 8: TE_K1(8); break;
        case 16: TE_K1(16); break;
        default: TE_K1(32); break;
    }
#undef TE_K1
    return cudaGetLastError();
}

cudaError_t launch_orth_norm(double2* w, double* S, const double2* u, int64_t d, DevState* st,
                             int j, int write, int decide, double* partials, int grid,
                             cudaStream_t s) {
    k_orth_norm<<<grid, TE_BLOCK, 0, s>>>(w, S, u, d, st, j, write, decide, partials);
    return cudaGetLastError();
}

cudaError_t launch_reorth_dots(const double2* V, const double2* w, int64_t d, DevState* st,
                               int j, double* partials, int grid, cudaStream_t s) {
    k_reorth_dots<<<grid, TE_BLOCK, 0, s>>>(V, w, d, st, j, partials);
    return cudaGetLastError();
}

cudaError_t launch_reorth_update(const double2* V, double2* w, double* S, int64_t d, DevState* st,
                                 int j, int decide, double* partials, int grid, cudaStream_t s) {
    k_reorth_update<<<grid, TE_BLOCK, 0, s>>>(V, w, S, d, st, j, decide, partials);
    return cudaGetLastError();
}

cudaError_t launch_recombine(double2* V, double* S, int64_t d, DevState* st, double* partials,
                             int grid, cudaStream_t s) {
    k_recombine<<<grid, TE_BLOCK, 0, s>>>(V, S, d, st, partials);
    return cudaGetLastError();
}
