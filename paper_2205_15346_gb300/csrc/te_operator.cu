// te_operator.cu -- createMatrix (Sec. 3 of arXiv 2205.15346) on the device.
//
// The operator is a sum of terms c_t * (product of creation / annihilation
// operators), the basis all occupation tuples (n_1..n_L) with sum N and
// n_l <= cap_l (Sec. 3, eq. totalOccupationNumber; the fixed maximal occupations
// of Sec. 4), in descending lexicographic order.  The paper inverts the index
// map ind with a hash table; here ind and its inverse are the combinatorial
// rank / unrank of that order (cnt[p][r] = tuples of modes p..L-1 holding r
// particles), exact and without memory per state.
//
// One warp builds one row j: lane 0 unranks j, the lanes apply the terms in
// parallel (a_l |n> = sqrt(n_l) |n - 1_l>, a_l^dag |n> = sqrt(n_l + 1) |n + 1_l>,
// rightmost operator first; a result outside the space is dropped) and append
// (column, term) keys with values conj(c_t) sqrt(prod) -- row j holds
// <j|H|i> = conj(<i|H|j>) for a Hermitian operator -- to a buffer in shared
// memory; the warp sorts the buffer (bitonic) and lane 0 adds the contributions
// to each column in term order.  The diagonal entry is always stored.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "te_internal.cuh"

namespace {

constexpr int kMaxModes = 32;
constexpr int kMaxN = 64;
constexpr int kMaxFactors = 8;
constexpr int kMaxTerms = 4096;
constexpr int kRowBuf = 256;            // entries per row before merging (one warp's buffer)
constexpr int kWarps = 4;               // warps per CTA

struct OpTables {
    int L, N;
    int cap[kMaxModes];
    unsigned long long cnt[kMaxModes + 1][kMaxN + 1];
};

void op_tables(const te_operator_desc* o, OpTables* T) {
    memset(T, 0, sizeof(*T));
    T->L = o->n_modes;
    T->N = o->n_particles;
    for (int l = 0; l < T->L; ++l)
        T->cap[l] = o->max_occ ? std::min(std::max(o->max_occ[l], 0), T->N) : T->N;
    T->cnt[T->L][0] = 1;
    for (int p = T->L - 1; p >= 0; --p)
        for (int r = 0; r <= T->N; ++r) {
            unsigned long long s = 0;
            for (int a = 0; a <= std::min(r, T->cap[p]); ++a) s += T->cnt[p + 1][r - a];
            T->cnt[p][r] = s;
        }
}

__host__ __device__ void op_unrank(const OpTables& T, long long r, int* occ) {
    int rem = T.N;
    for (int p = 0; p < T.L; ++p) {
        int a = rem < T.cap[p] ? rem : T.cap[p];
        for (; a > 0; --a) {
            const unsigned long long c = T.cnt[p + 1][rem - a];
            if ((unsigned long long)r < c) break;
            r -= (long long)c;
        }
        occ[p] = a;
        rem -= a;
    }
}

__host__ __device__ long long op_rank(const OpTables& T, const int* occ) {
    long long idx = 0;
    int rem = T.N;
    for (int p = 0; p < T.L; ++p) {
        const int top = rem < T.cap[p] ? rem : T.cap[p];
        for (int a = top; a > occ[p]; --a) idx += (long long)T.cnt[p + 1][rem - a];
        rem -= occ[p];
    }
    return idx;
}

// flags[0]: a row produced more than kRowBuf entries.
__global__ void __launch_bounds__(32 * kWarps) k_op_rows(
    const OpTables* __restrict__ Tg, int nterms, const int32_t* __restrict__ toff,
    const int32_t* __restrict__ fmode, const int32_t* __restrict__ fdag,
    const double2* __restrict__ coef, int64_t d, int fill, int32_t* __restrict__ cnt,
    const int32_t* __restrict__ rowptr, int32_t* __restrict__ col, double2* __restrict__ val,
    int* flags) {
    __shared__ long long key[kWarps][kRowBuf];
    __shared__ double2 v[kWarps][kRowBuf];
    __shared__ int occ_s[kWarps][kMaxModes];
    __shared__ int n_s[kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const OpTables& T = *Tg;
    const int64_t warp0 = (int64_t)blockIdx.x * kWarps + w;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t j = warp0; j < d; j += nwarps) {
        if (lane == 0) {
            op_unrank(T, j, occ_s[w]);
            key[w][0] = j * (long long)(kMaxTerms + 1);      // the diagonal, first in term order
            v[w][0] = make_double2(0.0, 0.0);
            n_s[w] = 1;
        }
        __syncwarp();
        for (int t = lane; t < nterms; t += 32) {
            int o[kMaxModes];
            for (int l = 0; l < T.L; ++l) o[l] = occ_s[w][l];
            double prod = 1.0;
            bool ok = true;
            for (int q = toff[t + 1] - 1; q >= toff[t] && ok; --q) {   // rightmost acts first
                const int l = fmode[q];
                if (fdag[q]) {
                    o[l] += 1;
                    if (o[l] > T.cap[l]) ok = false;
                    else prod *= (double)o[l];
                } else {
                    if (o[l] == 0) ok = false;
                    else {
                        prod *= (double)o[l];
                        o[l] -= 1;
                    }
                }
            }
            if (!ok) continue;
            int tot = 0;
            for (int l = 0; l < T.L; ++l) tot += o[l];
            if (tot != T.N) continue;
            const long long i = op_rank(T, o);
            const double s = sqrt(prod);
            const double2 c = coef[t];
            const int pos = atomicAdd(&n_s[w], 1);
            if (pos < kRowBuf) {
                key[w][pos] = i * (long long)(kMaxTerms + 1) + 1 + t;
                v[w][pos] = make_double2(c.x * s, -c.y * s);
            }
        }
        __syncwarp();
        const int n = n_s[w];
        if (n > kRowBuf) {
            if (lane == 0) atomicExch(&flags[0], 1);
            __syncwarp();
            continue;
        }
        // bitonic sort of the keys (padded with the largest key) with their values
        int m2 = 1;
        while (m2 < n) m2 <<= 1;
        for (int i = n + lane; i < m2; i += 32) key[w][i] = 0x7fffffffffffffffLL;
        __syncwarp();
        for (int k = 2; k <= m2; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int i = lane; i < m2; i += 32) {
                    const int pr = i ^ jj;
                    if (pr > i) {
                        const bool up = (i & k) == 0;
                        const long long a = key[w][i], b = key[w][pr];
                        if ((a > b) == up) {
                            key[w][i] = b;
                            key[w][pr] = a;
                            const double2 tv = v[w][i];
                            v[w][i] = v[w][pr];
                            v[w][pr] = tv;
                        }
                    }
                }
                __syncwarp();
            }
        }
        if (lane == 0) {
            int64_t out = fill ? rowptr[j] : 0;
            int uniq = 0;
            int q = 0;
            while (q < n) {
                const long long c0 = key[w][q] / (kMaxTerms + 1);
                double2 s = make_double2(0.0, 0.0);            // contributions in term order
                for (; q < n && key[w][q] / (kMaxTerms + 1) == c0; ++q) {
                    s.x += v[w][q].x;
                    s.y += v[w][q].y;
                }
                if (fill) {
                    col[out] = (int32_t)c0;
                    val[out] = s;
                    ++out;
                }
                ++uniq;
            }
            if (!fill) cnt[j] = uniq;
        }
        __syncwarp();
    }
}

__global__ void k_op_occupation(const OpTables* __restrict__ Tg, int64_t d, int mode,
                                double* __restrict__ out) {
    int occ[kMaxModes];
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d;
         r += (int64_t)gridDim.x * blockDim.x) {
        op_unrank(*Tg, r, occ);
        out[r] = (double)occ[mode];
    }
}

te_status check_op(te_ctx* ctx, const te_operator_desc* o) {
    if (o->n_modes < 1 || o->n_modes > kMaxModes || o->n_particles < 0 || o->n_particles > kMaxN)
        return set_error(ctx, TE_ERR_INVALID_ARG, "need 1 <= n_modes <= 32 and 0 <= n_particles <= 64");
    if (o->n_terms < 0 || o->n_terms > kMaxTerms || (o->n_terms > 0 && (!o->term_len || !o->coef)))
        return set_error(ctx, TE_ERR_INVALID_ARG, "need 0 <= n_terms <= 4096 with term_len and coef");
    int64_t nf = 0;
    for (int t = 0; t < o->n_terms; ++t) {
        if (o->term_len[t] < 0 || o->term_len[t] > kMaxFactors)
            return set_error(ctx, TE_ERR_INVALID_ARG, "a term has more than 8 ladder operators");
        nf += o->term_len[t];
        if (!isfinite(o->coef[2 * t]) || !isfinite(o->coef[2 * t + 1]))
            return set_error(ctx, TE_ERR_NONFINITE, "non-finite coefficient");
    }
    if (nf > 0 && (!o->modes || !o->dagger)) return set_error(ctx, TE_ERR_INVALID_ARG, "NULL modes / dagger");
    for (int64_t q = 0; q < nf; ++q)
        if (o->modes[q] < 0 || o->modes[q] >= o->n_modes || (o->dagger[q] != 0 && o->dagger[q] != 1))
            return set_error(ctx, TE_ERR_INVALID_ARG, "operator mode or dagger flag out of range");
    return TE_OK;
}

int grid_rows(int64_t d, int num_sms) {
    const int64_t want = (d + kWarps - 1) / kWarps;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms * 16));
}

}  // namespace

extern "C" {

te_status te_build_operator(te_ctx* ctx, const te_operator_desc* o, te_matrix** out) {
    if (!ctx || !o || !out) return TE_ERR_INVALID_ARG;
    *out = nullptr;
    if (te_status s = check_op(ctx, o)) return s;
    cudaSetDevice(ctx->device);
    cudaGetLastError();
    OpTables T;
    op_tables(o, &T);
    const unsigned long long dd = T.cnt[0][T.N];
    if (dd == 0) return set_error(ctx, TE_ERR_INVALID_ARG, "no occupation tuple satisfies the caps");
    if (dd >= (1ull << 31)) return set_error(ctx, TE_ERR_UNSUPPORTED, "basis too large");
    const int64_t d = (int64_t)dd;
    const int nt = o->n_terms;
    std::vector<int32_t> toff(nt + 1, 0);
    for (int t = 0; t < nt; ++t) toff[t + 1] = toff[t] + o->term_len[t];
    const int nf = toff[nt];
    std::vector<double2> cf(std::max(nt, 1));
    for (int t = 0; t < nt; ++t) cf[t] = make_double2(o->coef[2 * t], o->coef[2 * t + 1]);
    cudaStream_t s = ctx->stream;
    OpTables* Td = nullptr;
    int32_t *dtoff = nullptr, *dmode = nullptr, *ddag = nullptr, *cnt = nullptr;
    double2* dcoef = nullptr;
    int* flags = nullptr;
    te_matrix* H = new te_matrix();
    H->ctx = ctx;
    auto cleanup = [&]() {
        for (void* q : {(void*)Td, (void*)dtoff, (void*)dmode, (void*)ddag, (void*)cnt, (void*)dcoef,
                        (void*)flags})
            if (q) dev_free(ctx, q);
    };
    auto fail = [&](te_status st) {
        cleanup();
        te_matrix_free(H);
        return st;
    };
    cudaError_t e = dev_alloc(ctx, &Td, sizeof(OpTables));
    if (e == cudaSuccess) e = dev_alloc(ctx, &dtoff, sizeof(int32_t) * (nt + 1));
    if (e == cudaSuccess) e = dev_alloc(ctx, &dmode, sizeof(int32_t) * std::max(nf, 1));
    if (e == cudaSuccess) e = dev_alloc(ctx, &ddag, sizeof(int32_t) * std::max(nf, 1));
    if (e == cudaSuccess) e = dev_alloc(ctx, &dcoef, sizeof(double2) * std::max(nt, 1));
    if (e == cudaSuccess) e = dev_alloc(ctx, &cnt, sizeof(int32_t) * d);
    if (e == cudaSuccess) e = dev_alloc(ctx, &flags, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Td, &T, sizeof(OpTables), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dtoff, toff.data(), sizeof(int32_t) * (nt + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nf > 0)
        e = cudaMemcpyAsync(dmode, o->modes, sizeof(int32_t) * nf, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nf > 0)
        e = cudaMemcpyAsync(ddag, o->dagger, sizeof(int32_t) * nf, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nt > 0)
        e = cudaMemcpyAsync(dcoef, cf.data(), sizeof(double2) * nt, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, sizeof(int) * 4, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(set_error(ctx, e == cudaErrorMemoryAllocation ? TE_ERR_OOM : TE_ERR_CUDA,
                              "allocating the operator builder"));
    }
    const int grid = grid_rows(d, ctx->num_sms);
    k_op_rows<<<grid, 32 * kWarps, 0, s>>>(Td, nt, dtoff, dmode, ddag, dcoef, d, 0, cnt, nullptr,
                                           nullptr, nullptr, flags);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_error(ctx, e, "k_op_rows (count)"));
    int hf[4] = {0, 0, 0, 0};
    e = cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(cuda_error(ctx, e, "operator builder"));
    if (hf[0]) return fail(set_error(ctx, TE_ERR_UNSUPPORTED, "a row has more than 256 contributions"));
    int32_t* rowptr = nullptr;
    if (dev_alloc(ctx, &rowptr, sizeof(int32_t) * (d + 1)) != cudaSuccess) {
        cudaGetLastError();
        return fail(set_error(ctx, TE_ERR_OOM, "row pointer"));
    }
    int64_t nnz = 0;
    te_status st = scan_counts(ctx, cnt, d, rowptr, &nnz, s);
    H->d = d;
    H->rowptr = rowptr;
    if (st) return fail(st);
    H->nnz = nnz;
    if (dev_alloc(ctx, &H->col, sizeof(int32_t) * std::max<int64_t>(nnz, 1)) != cudaSuccess ||
        dev_alloc(ctx, &H->val, sizeof(double2) * std::max<int64_t>(nnz, 1)) != cudaSuccess) {
        cudaGetLastError();
        return fail(set_error(ctx, TE_ERR_OOM, "device allocation of the CSR arrays failed"));
    }
    k_op_rows<<<grid, 32 * kWarps, 0, s>>>(Td, nt, dtoff, dmode, ddag, dcoef, d, 1, nullptr, rowptr,
                                           H->col, H->val, flags);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_error(ctx, e, "k_op_rows (fill)"));
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(cuda_error(ctx, e, "operator fill"));
    cleanup();
    Td = nullptr;
    dtoff = dmode = ddag = cnt = nullptr;
    dcoef = nullptr;
    flags = nullptr;
    st = finish_matrix_stats(ctx, H);
    if (st == TE_OK) st = build_sell(ctx, H);
    if (st) {
        te_matrix_free(H);
        return st;
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        H->id = ctx->next_matrix_id++;
    }
    *out = H;
    return TE_OK;
}

te_status te_operator_basis_index(const te_operator_desc* o, const int32_t* occ, int64_t* index) {
    if (!o || !occ || !index) return TE_ERR_INVALID_ARG;
    if (check_op(nullptr, o)) return TE_ERR_INVALID_ARG;
    OpTables T;
    op_tables(o, &T);
    int tot = 0;
    for (int l = 0; l < T.L; ++l) {
        if (occ[l] < 0 || occ[l] > T.cap[l]) return TE_ERR_INVALID_ARG;
        tot += occ[l];
    }
    if (tot != T.N) return TE_ERR_INVALID_ARG;
    *index = op_rank(T, occ);
    return TE_OK;
}

te_status te_operator_occupation(te_ctx* ctx, const te_operator_desc* o, int32_t mode, double* out,
                                 uint32_t flags) {
    if (!ctx || !o || !out) return TE_ERR_INVALID_ARG;
    if (te_status s = check_op(ctx, o)) return s;
    if (mode < 0 || mode >= o->n_modes) return set_error(ctx, TE_ERR_INVALID_ARG, "mode out of range");
    cudaSetDevice(ctx->device);
    cudaGetLastError();
    OpTables T;
    op_tables(o, &T);
    const int64_t d = (int64_t)T.cnt[0][T.N];
    cudaStream_t s = ctx->stream;
    const bool dev = (flags & TE_PTR_DEVICE) != 0;
    OpTables* Td = nullptr;
    double* dst = out;
    TE_CUDA_TRY(ctx, dev_alloc(ctx, &Td, sizeof(OpTables)));
    cudaError_t e = cudaMemcpyAsync(Td, &T, sizeof(OpTables), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !dev) e = dev_alloc(ctx, &dst, sizeof(double) * (size_t)std::max<int64_t>(d, 1));
    if (e == cudaSuccess) {
        const int64_t want = (d + TE_BLOCK - 1) / TE_BLOCK;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)ctx->num_sms * 8));
        k_op_occupation<<<grid, TE_BLOCK, 0, s>>>(Td, d, mode, dst);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !dev)
        e = cudaMemcpyAsync(out, dst, sizeof(double) * (size_t)d, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(ctx, Td);
    if (!dev && dst) dev_free(ctx, dst);
    if (e != cudaSuccess) return cuda_error(ctx, e, "te_operator_occupation");
    return TE_OK;
}

}  // extern "C"
