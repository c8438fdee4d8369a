// te_build.cu -- Hamiltonian matrices built on the device (Sec. 3 of arXiv 2205.15346).
//
// Sec. 3 forms H by applying the operator to every basis state and storing
// each coefficient at (state, image state), with the state -> index map held in
// a hash table (Sec. 4).  Here one thread builds one row: it applies the
// operator to its basis state, looks the image states up, sorts the row by
// column and writes it.  The stored matrix is the standard H[i,j] = <i|H|j>.
//
// Values are formed with explicitly rounded multiplies and adds in a fixed
// order (the definitions are stated in te.h), so the arrays are reproducible
// bit for bit by any implementation that follows the same definitions.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "te_internal.cuh"

namespace {

constexpr int kBoseMaxEntries = 1 + 15 * 15;   // diagonal + n_occupied (K - 1), K <= 16, N <= 15
constexpr int kMemMaxEntries = 3 + 15 * 15;    // diagonal, two boson hops, Nm (Q - Nm) qubit hops
constexpr unsigned long long kEmpty = ~0ull;

__device__ __forceinline__ double spin_sign(int64_t r, int i) {
    return 1.0 - 2.0 * (double)((r >> i) & 1);
}

// ---------------------------------------------------------------- TFIM

__global__ void k_build_tfim(int L, const double* __restrict__ J, const double* __restrict__ hx,
                             int64_t d, int32_t* __restrict__ rowptr, int32_t* __restrict__ col,
                             double2* __restrict__ val) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= d) return;
    const int64_t w = L + 1;
    rowptr[r] = (int32_t)(r * w);
    if (r == d - 1) rowptr[d] = (int32_t)(d * w);
    double acc = 0.0;
    for (int b = 0; b < L - 1; ++b)
        acc = __dadd_rn(acc, __dmul_rn(-J[b], spin_sign(r, b) * spin_sign(r, b + 1)));
    int64_t pos = r * w;
    for (int i = L - 1; i >= 0; --i)               // flips that lower the index, ascending
        if ((r >> i) & 1) {
            col[pos] = (int32_t)(r ^ (1ll << i));
            val[pos] = make_double2(-hx[i], 0.0);
            ++pos;
        }
    col[pos] = (int32_t)r;
    val[pos] = make_double2(acc, 0.0);
    ++pos;
    for (int i = 0; i < L; ++i)                    // flips that raise the index, ascending
        if (!((r >> i) & 1)) {
            col[pos] = (int32_t)(r ^ (1ll << i));
            val[pos] = make_double2(-hx[i], 0.0);
            ++pos;
        }
}

// ---------------------------------------------------------------- XXZ-DM

__global__ void k_count_xxzdm(int L, int nb, int64_t d, int32_t* __restrict__ cnt) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= d) return;
    int c = 1;
    for (int b = 0; b < nb; ++b) c += (int)(((r >> b) ^ (r >> ((b + 1) % L))) & 1);
    cnt[r] = c;
}

__global__ void k_fill_xxzdm(int L, int nb, double delta, const double* __restrict__ hre,
                             const double* __restrict__ him, const double* __restrict__ hz,
                             int64_t d, const int32_t* __restrict__ rowptr,
                             int32_t* __restrict__ col, double2* __restrict__ val) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= d) return;
    int32_t cs[32];
    double2 vs[32];
    double acc = 0.0;
    const double dq = delta * 0.25;
    for (int b = 0; b < nb; ++b)
        acc = __dadd_rn(acc, __dmul_rn(dq, spin_sign(r, b) * spin_sign(r, (b + 1) % L)));
    for (int i = 0; i < L; ++i) acc = __dadd_rn(acc, __dmul_rn(hz[i] * 0.5, spin_sign(r, i)));
    int n = 0;
    cs[n] = (int32_t)r;
    vs[n] = make_double2(acc, 0.0);
    ++n;
    for (int b = 0; b < nb; ++b) {
        const int a = b, c = (b + 1) % L;
        const int ba = (int)((r >> a) & 1), bc = (int)((r >> c) & 1);
        if (ba == bc) continue;
        const int64_t tgt = r ^ ((1ll << a) | (1ll << c));
        const double re = 0.5 * hre[b], im = 0.5 * him[b];
        cs[n] = (int32_t)tgt;
        vs[n] = (ba == 0) ? make_double2(re, im) : make_double2(re, -im);
        ++n;
    }
    for (int i = 1; i < n; ++i) {                   // insertion sort by column
        const int32_t kc = cs[i];
        const double2 kv = vs[i];
        int k = i - 1;
        while (k >= 0 && cs[k] > kc) {
            cs[k + 1] = cs[k];
            vs[k + 1] = vs[k];
            --k;
        }
        cs[k + 1] = kc;
        vs[k + 1] = kv;
    }
    const int64_t p = rowptr[r];
    for (int i = 0; i < n; ++i) {
        col[p + i] = cs[i];
        val[p + i] = vs[i];
    }
}

// ---------------------------------------------------------------- bosons

struct BoseTables {
    int K, N;
    unsigned long long comp[16][17];   // comp[n][k]: ways to put n bosons in k modes
};

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Occupations of basis index r (descending lexicographic order), packed 4 bits per mode.
__device__ unsigned long long bose_unrank(const BoseTables& T, int64_t r, int* occ) {
    int rem = T.N;
    unsigned long long key = 0;
    for (int p = 0; p < T.K - 1; ++p) {
        int a = rem;
        for (; a > 0; --a) {
            const unsigned long long cnt = T.comp[rem - a][T.K - 1 - p];
            if ((unsigned long long)r < cnt) break;
            r -= (int64_t)cnt;
        }
        occ[p] = a;
        key |= (unsigned long long)a << (4 * p);
        rem -= a;
    }
    occ[T.K - 1] = rem;
    key |= (unsigned long long)rem << (4 * (T.K - 1));
    return key;
}

__global__ void k_bose_insert(BoseTables T, int64_t d, unsigned long long* __restrict__ keys,
                              int32_t* __restrict__ vals, unsigned long long mask,
                              int32_t* __restrict__ cnt, int* __restrict__ err) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= d) return;
    int occ[16];
    const unsigned long long key = bose_unrank(T, r, occ);
    int nocc = 0;
    for (int i = 0; i < T.K; ++i) nocc += occ[i] > 0;
    cnt[r] = 1 + nocc * (T.K - 1);
    unsigned long long h = mix64(key) & mask;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
        const unsigned long long prev = atomicCAS(keys + h, kEmpty, key);
        if (prev == kEmpty || prev == key) {
            vals[h] = (int32_t)r;
            return;
        }
        h = (h + 1) & mask;
    }
    atomicExch(err, 1);                             // table full (cannot happen at load <= 1/2)
}

__device__ __forceinline__ int32_t bose_lookup(const unsigned long long* keys, const int32_t* vals,
                                               unsigned long long mask, unsigned long long key) {
    unsigned long long h = mix64(key) & mask;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
        const unsigned long long k = keys[h];
        if (k == key) return vals[h];
        if (k == kEmpty) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

__global__ void k_bose_fill(BoseTables T, const double* __restrict__ cre,
                            const double* __restrict__ cim, const double* __restrict__ U,
                            int64_t d, const unsigned long long* __restrict__ keys,
                            const int32_t* __restrict__ vals, unsigned long long mask,
                            const int32_t* __restrict__ rowptr, int32_t* __restrict__ col,
                            double2* __restrict__ val, int* __restrict__ err) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= d) return;
    int occ[16];
    const unsigned long long key = bose_unrank(T, r, occ);
    const int K = T.K;
    int32_t cs[kBoseMaxEntries];
    double2 vs[kBoseMaxEntries];
    double acc = 0.0;
    for (int i = 0; i < K; ++i) acc = __dadd_rn(acc, __dmul_rn(U[i], (double)(occ[i] * occ[i])));
    int n = 0;
    cs[n] = (int32_t)r;
    vs[n] = make_double2(acc, 0.0);
    ++n;
    for (int i = 0; i < K; ++i) {
        if (occ[i] == 0) continue;
        for (int j = 0; j < K; ++j) {
            if (j == i) continue;
            // source state n - e_i + e_j; <n| c_ij a_i^+ a_j |src> = c_ij sqrt(n_i) sqrt(n_j + 1)
            const unsigned long long src = key - (1ull << (4 * i)) + (1ull << (4 * j));
            const int32_t c = bose_lookup(keys, vals, mask, src);
            if (c < 0) {
                atomicExch(err, 2);
                return;
            }
            const double amp = __dmul_rn(sqrt((double)occ[i]), sqrt((double)(occ[j] + 1)));
            double re, im;
            if (i < j) {
                const int p = i * K - i * (i + 1) / 2 + (j - i - 1);
                re = cre[p];
                im = cim[p];
            } else {
                const int p = j * K - j * (j + 1) / 2 + (i - j - 1);
                re = cre[p];
                im = -cim[p];
            }
            cs[n] = c;
            vs[n] = make_double2(__dmul_rn(re, amp), __dmul_rn(im, amp));
            ++n;
        }
    }
    for (int i = 1; i < n; ++i) {
        const int32_t kc = cs[i];
        const double2 kv = vs[i];
        int k = i - 1;
        while (k >= 0 && cs[k] > kc) {
            cs[k + 1] = cs[k];
            vs[k + 1] = vs[k];
            --k;
        }
        cs[k + 1] = kc;
        vs[k + 1] = kv;
    }
    const int64_t p = rowptr[r];
    if (rowptr[r + 1] - p != n) {
        atomicExch(err, 3);
        return;
    }
    for (int i = 0; i < n; ++i) {
        col[p + i] = cs[i];
        val[p + i] = vs[i];
    }
}


// ---------------------------------------------------------------- the paper's example system

struct MemTables {
    int K, Q, Nm, N0;
    long long nq;                        // C(Q, Nm)
    long long C[32][32];                 // binomial coefficients C(n, k)
    double Nc, dNc, em, C0, Cm;
};

// Qubit tuple of rank qi (descending lexicographic: 1 before 0 at each position).
__device__ __host__ unsigned mem_unrank(const MemTables& T, long long qi) {
    unsigned mask = 0;
    int rem = T.Nm;
    for (int pos = 0; pos < T.Q && rem > 0; ++pos) {
        const long long with_one = T.C[T.Q - pos - 1][rem - 1];
        if (qi < with_one) {
            mask |= 1u << pos;
            --rem;
        } else {
            qi -= with_one;
        }
    }
    return mask;
}

__device__ __host__ long long mem_rank(const MemTables& T, unsigned mask) {
    long long r = 0;
    int rem = T.Nm;
    for (int pos = 0; pos < T.Q && rem > 0; ++pos) {
        if (mask & (1u << pos)) {
            --rem;
        } else {
            r += T.C[T.Q - pos - 1][rem - 1];
        }
    }
    return r;
}

__global__ void k_count_memory(MemTables T, int64_t d, int32_t* __restrict__ cnt) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= d) return;
    const long long b = r / T.nq;
    const int n0 = T.N0 - (int)b, m0 = (int)b;
    int c = 1 + (n0 >= 1) + (m0 >= 1) + T.Nm * (T.Q - T.Nm);
    cnt[r] = c;
}

__global__ void k_fill_memory(MemTables T, const double* __restrict__ f, int64_t d,
                              const int32_t* __restrict__ rowptr, int32_t* __restrict__ col,
                              double2* __restrict__ val, int* __restrict__ err) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= d) return;
    const long long b = r / T.nq, qi = r % T.nq;
    const int n0 = T.N0 - (int)b, m0 = (int)b;
    const unsigned mask = mem_unrank(T, qi);
    const int n1 = __popc(mask & ((1u << T.K) - 1u));
    const int n2 = __popc(mask) - n1;
    int32_t cs[kMemMaxEntries];
    double vs[kMemMaxEntries];
    const double t1 = __dmul_rn(__dmul_rn(T.em, __dsub_rn(1.0, __ddiv_rn((double)n0, T.Nc))), (double)n1);
    const double t2 = __dmul_rn(__dmul_rn(T.em, __dsub_rn(1.0, __ddiv_rn((double)n0, __dsub_rn(T.Nc, T.dNc)))),
                                (double)n2);
    int n = 0;
    cs[n] = (int32_t)r;
    vs[n] = __dadd_rn(t1, t2);
    ++n;
    if (n0 >= 1) {                           // a0^+ b0 brings (n0 - 1, m0 + 1) here
        cs[n] = (int32_t)((b + 1) * T.nq + qi);
        vs[n] = __dmul_rn(T.C0, __dmul_rn(sqrt((double)n0), sqrt((double)(m0 + 1))));
        ++n;
    }
    if (m0 >= 1) {                           // b0^+ a0 brings (n0 + 1, m0 - 1) here
        cs[n] = (int32_t)((b - 1) * T.nq + qi);
        vs[n] = __dmul_rn(T.C0, __dmul_rn(sqrt((double)m0), sqrt((double)(n0 + 1))));
        ++n;
    }
    for (int a = 0; a < T.Q; ++a) {
        for (int c = a + 1; c < T.Q; ++c) {
            const unsigned ba = (mask >> a) & 1u, bc = (mask >> c) & 1u;
            if (ba == bc) continue;
            const unsigned src = mask ^ (1u << a) ^ (1u << c);
            cs[n] = (int32_t)(b * T.nq + mem_rank(T, src));
            vs[n] = __dmul_rn(T.Cm, f[a * T.Q - a * (a + 1) / 2 + (c - a - 1)]);
            ++n;
        }
    }
    for (int i = 1; i < n; ++i) {
        const int32_t kc = cs[i];
        const double kv = vs[i];
        int k = i - 1;
        while (k >= 0 && cs[k] > kc) {
            cs[k + 1] = cs[k];
            vs[k + 1] = vs[k];
            --k;
        }
        cs[k + 1] = kc;
        vs[k + 1] = kv;
    }
    const int64_t p = rowptr[r];
    if (rowptr[r + 1] - p != n) {
        atomicExch(err, 1);
        return;
    }
    for (int i = 0; i < n; ++i) {
        col[p + i] = cs[i];
        val[p + i] = make_double2(vs[i], 0.0);
    }
}

void mem_tables(const te_model_desc* m, MemTables* T) {
    memset(T, 0, sizeof(*T));
    T->K = m->L;
    T->Q = m->L + m->L2;
    T->Nm = m->N;
    T->N0 = m->N2;
    for (int n = 0; n < 32; ++n) {
        T->C[n][0] = 1;
        for (int k = 1; k <= n; ++k) T->C[n][k] = T->C[n - 1][k - 1] + (k <= n - 1 ? T->C[n - 1][k] : 0);
    }
    T->nq = T->C[T->Q][T->Nm];
    T->Nc = m->p[0];
    T->dNc = m->p[1];
    T->em = m->p[2];
    T->C0 = m->p[3];
    T->Cm = m->p[4];
}

// ---------------------------------------------------------------- scan and stats

constexpr int kScanItems = 4;
constexpr int kScanTile = TE_BLOCK * kScanItems;

__global__ void k_scan_tiles(const int32_t* __restrict__ cnt, int64_t d, int64_t* __restrict__ tile_sum) {
    __shared__ int64_t sh[TE_BLOCK];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
    for (int q = 0; q < kScanItems; ++q)
        if (base + q < d) s += cnt[base + q];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = TE_BLOCK / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = sh[0];
}

// Exclusive scan within each tile plus the tile's offset (scanned on the host).
__global__ void k_scan_apply(const int32_t* __restrict__ cnt, int64_t d,
                             const int64_t* __restrict__ tile_off, int32_t* __restrict__ rowptr) {
    __shared__ int64_t sh[TE_BLOCK];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t loc[kScanItems];
    int64_t s = 0;
    for (int q = 0; q < kScanItems; ++q) {
        loc[q] = (base + q < d) ? cnt[base + q] : 0;
        s += loc[q];
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < TE_BLOCK; o <<= 1) {          // Hillis-Steele inclusive scan
        const int64_t v = (threadIdx.x >= (unsigned)o) ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = tile_off[blockIdx.x] + sh[threadIdx.x] - s;
    for (int q = 0; q < kScanItems; ++q) {
        if (base + q < d) rowptr[base + q] = (int32_t)run;
        run += loc[q];
    }
}

__global__ void k_row_stats(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const double2* __restrict__ val, int64_t d,
                            unsigned long long* __restrict__ max_sum_bits,
                            int* __restrict__ max_nnz, int* __restrict__ flags) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= d) return;
    const int b = rowptr[r], e = rowptr[r + 1];
    double s = 0.0;
    bool finite = true, inrange = (e >= b);
    for (int k = b; k < e; ++k) {
        const double2 v = val[k];
        finite &= isfinite(v.x) && isfinite(v.y);
        s += hypot(v.x, v.y);
        const int c = col[k];
        inrange &= (c >= 0) && (c < d);
    }
    if (!finite) atomicOr(flags, 1);
    if (!inrange) atomicOr(flags, 2);
    if (finite) atomicMax(max_sum_bits, (unsigned long long)__double_as_longlong(s));
    atomicMax(max_nnz, e - b);
}

template <typename T>
struct DevBuf {
    te_ctx* ctx = nullptr;
    T* p = nullptr;
    ~DevBuf() { if (p) dev_free(ctx, p); }
    cudaError_t alloc(te_ctx* c, size_t n) {
        ctx = c;
        return dev_alloc(c, &p, n * sizeof(T) + 16);
    }
};

int grid_for(int64_t n) { return (int)((n + TE_BLOCK - 1) / TE_BLOCK); }

te_status alloc_matrix(te_ctx* ctx, te_matrix* H, int64_t d, int64_t nnz) {
    if (nnz >= (1ll << 31) || d >= (1ll << 31))
        return set_error(ctx, TE_ERR_UNSUPPORTED, "matrix too large: nnz and d must stay below 2^31");
    H->d = d;
    H->nnz = nnz;
    if (dev_alloc(ctx, &H->rowptr, sizeof(int32_t) * (d + 1)) != cudaSuccess ||
        dev_alloc(ctx, &H->col, sizeof(int32_t) * (nnz > 0 ? nnz : 1)) != cudaSuccess ||
        dev_alloc(ctx, &H->val, sizeof(double2) * (nnz > 0 ? nnz : 1)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, TE_ERR_OOM, "device allocation of the CSR arrays failed");
    }
    return TE_OK;
}

template <typename T>
te_status upload(te_ctx* ctx, DevBuf<T>& buf, const T* host, size_t n, cudaStream_t s) {
    TE_CUDA_TRY(ctx, buf.alloc(ctx, n));
    TE_CUDA_TRY(ctx, cudaMemcpyAsync(buf.p, host, n * sizeof(T), cudaMemcpyHostToDevice, s));
    return TE_OK;
}

void bose_tables(int K, int N, BoseTables* T) {
    T->K = K;
    T->N = N;
    for (int n = 0; n < 16; ++n)
        for (int k = 0; k < 17; ++k) {
            // C(n + k - 1, k - 1) for k >= 1; no way to hold n > 0 bosons in 0 modes
            if (k == 0) {
                T->comp[n][k] = (n == 0) ? 1 : 0;
                continue;
            }
            unsigned long long c = 1;
            for (int i = 1; i <= k - 1; ++i) c = c * (unsigned long long)(n + i) / (unsigned long long)i;
            T->comp[n][k] = c;
        }
}

}  // namespace

// rowptr from per-row counts; returns the total through *nnz.
te_status scan_counts(te_ctx* ctx, const int32_t* cnt, int64_t d, int32_t* rowptr, int64_t* nnz,
                      cudaStream_t s) {
    const int64_t tiles = (d + kScanTile - 1) / kScanTile;
    DevBuf<int64_t> tsum;
    TE_CUDA_TRY(ctx, tsum.alloc(ctx, tiles));
    k_scan_tiles<<<(int)tiles, TE_BLOCK, 0, s>>>(cnt, d, tsum.p);
    TE_CUDA_TRY(ctx, cudaGetLastError());
    std::vector<int64_t> h(tiles);
    TE_CUDA_TRY(ctx, cudaMemcpyAsync(h.data(), tsum.p, sizeof(int64_t) * tiles,
                                     cudaMemcpyDeviceToHost, s));
    TE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    int64_t run = 0;
    for (int64_t t = 0; t < tiles; ++t) {
        const int64_t v = h[t];
        h[t] = run;
        run += v;
    }
    *nnz = run;
    if (run >= (1ll << 31))
        return set_error(ctx, TE_ERR_UNSUPPORTED, "matrix too large: nnz must stay below 2^31");
    TE_CUDA_TRY(ctx, cudaMemcpyAsync(tsum.p, h.data(), sizeof(int64_t) * tiles,
                                     cudaMemcpyHostToDevice, s));
    k_scan_apply<<<(int)tiles, TE_BLOCK, 0, s>>>(cnt, d, tsum.p, rowptr);
    TE_CUDA_TRY(ctx, cudaGetLastError());
    const int32_t last = (int32_t)run;
    TE_CUDA_TRY(ctx, cudaMemcpyAsync(rowptr + d, &last, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    TE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    return TE_OK;
}

te_status build_tfim(te_ctx* ctx, const te_model_desc* m, te_matrix* H) {
    const int L = m->L;
    if (L < 2 || L > 26 || !m->a || !m->b)
        return set_error(ctx, TE_ERR_INVALID_ARG, "TFIM needs 2 <= L <= 26 and the J, h arrays");
    cudaStream_t s = ctx->stream;
    const int64_t d = 1ll << L;
    te_status st = alloc_matrix(ctx, H, d, d * (L + 1));
    if (st) return st;
    DevBuf<double> J, hx;
    if ((st = upload(ctx, J, m->a, L - 1, s)) || (st = upload(ctx, hx, m->b, L, s))) return st;
    k_build_tfim<<<grid_for(d), TE_BLOCK, 0, s>>>(L, J.p, hx.p, d, H->rowptr, H->col, H->val);
    TE_CUDA_TRY(ctx, cudaGetLastError());
    TE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    return TE_OK;
}

te_status build_xxzdm(te_ctx* ctx, const te_model_desc* m, te_matrix* H) {
    const int L = m->L;
    const int nb = m->pbc ? L : L - 1;
    if (L < 2 || L > 30 || (m->pbc && L < 3) || !m->a || !m->b || !m->c)
        return set_error(ctx, TE_ERR_INVALID_ARG,
                         "XXZ-DM needs 2 <= L <= 30 (L >= 3 periodic) and the hop/field arrays");
    cudaStream_t s = ctx->stream;
    const int64_t d = 1ll << L;
    if (d >= (1ll << 31)) return set_error(ctx, TE_ERR_UNSUPPORTED, "dimension must stay below 2^31");
    DevBuf<int32_t> cnt;
    TE_CUDA_TRY(ctx, cnt.alloc(ctx, d));
    te_status st;
    DevBuf<double> hre, him, hz;
    if ((st = upload(ctx, hre, m->a, nb, s)) || (st = upload(ctx, him, m->b, nb, s)) ||
        (st = upload(ctx, hz, m->c, L, s)))
        return st;
    k_count_xxzdm<<<grid_for(d), TE_BLOCK, 0, s>>>(L, nb, d, cnt.p);
    TE_CUDA_TRY(ctx, cudaGetLastError());
    int32_t* rowptr = nullptr;
    TE_CUDA_TRY(ctx, dev_alloc(ctx, &rowptr, sizeof(int32_t) * (d + 1)));
    int64_t nnz = 0;
    if ((st = scan_counts(ctx, cnt.p, d, rowptr, &nnz, s))) {
        dev_free(ctx, rowptr);
        return st;
    }
    H->d = d;
    H->nnz = nnz;
    H->rowptr = rowptr;
    if (dev_alloc(ctx, &H->col, sizeof(int32_t) * nnz) != cudaSuccess ||
        dev_alloc(ctx, &H->val, sizeof(double2) * nnz) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, TE_ERR_OOM, "device allocation of the CSR arrays failed");
    }
    k_fill_xxzdm<<<grid_for(d), TE_BLOCK, 0, s>>>(L, nb, m->delta, hre.p, him.p, hz.p, d, rowptr,
                                                   H->col, H->val);
    TE_CUDA_TRY(ctx, cudaGetLastError());
    TE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    return TE_OK;
}

te_status build_bose(te_ctx* ctx, const te_model_desc* m, te_matrix* H) {
    const int K = m->L, N = m->N;
    if (K < 2 || K > 16 || N < 1 || N > 15 || !m->a || !m->b || !m->c)
        return set_error(ctx, TE_ERR_INVALID_ARG,
                         "bosons need 2 <= K <= 16 modes, 1 <= N <= 15 and the c, U arrays");
    BoseTables T;
    bose_tables(K, N, &T);
    const unsigned long long dd = T.comp[N][K];
    if (dd >= (1ull << 31)) return set_error(ctx, TE_ERR_UNSUPPORTED, "basis too large");
    const int64_t d = (int64_t)dd;
    cudaStream_t s = ctx->stream;
    unsigned long long cap = 1;
    while (cap < 2ull * dd) cap <<= 1;
    DevBuf<unsigned long long> keys;
    DevBuf<int32_t> vals, cnt;
    DevBuf<int> err;
    TE_CUDA_TRY(ctx, keys.alloc(ctx, cap));
    TE_CUDA_TRY(ctx, vals.alloc(ctx, cap));
    TE_CUDA_TRY(ctx, cnt.alloc(ctx, d));
    TE_CUDA_TRY(ctx, err.alloc(ctx, 1));
    TE_CUDA_TRY(ctx, cudaMemsetAsync(keys.p, 0xff, cap * sizeof(unsigned long long), s));
    TE_CUDA_TRY(ctx, cudaMemsetAsync(err.p, 0, sizeof(int), s));
    const int npair = K * (K - 1) / 2;
    te_status st;
    DevBuf<double> cre, cim, U;
    if ((st = upload(ctx, cre, m->a, npair, s)) || (st = upload(ctx, cim, m->b, npair, s)) ||
        (st = upload(ctx, U, m->c, K, s)))
        return st;
    k_bose_insert<<<grid_for(d), TE_BLOCK, 0, s>>>(T, d, keys.p, vals.p, cap - 1, cnt.p, err.p);
    TE_CUDA_TRY(ctx, cudaGetLastError());
    int32_t* rowptr = nullptr;
    TE_CUDA_TRY(ctx, dev_alloc(ctx, &rowptr, sizeof(int32_t) * (d + 1)));
    int64_t nnz = 0;
    if ((st = scan_counts(ctx, cnt.p, d, rowptr, &nnz, s))) {
        dev_free(ctx, rowptr);
        return st;
    }
    H->d = d;
    H->nnz = nnz;
    H->rowptr = rowptr;
    if (dev_alloc(ctx, &H->col, sizeof(int32_t) * nnz) != cudaSuccess ||
        dev_alloc(ctx, &H->val, sizeof(double2) * nnz) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, TE_ERR_OOM, "device allocation of the CSR arrays failed");
    }
    k_bose_fill<<<grid_for(d), TE_BLOCK, 0, s>>>(T, cre.p, cim.p, U.p, d, keys.p, vals.p, cap - 1,
                                                  rowptr, H->col, H->val, err.p);
    TE_CUDA_TRY(ctx, cudaGetLastError());
    int herr = 0;
    TE_CUDA_TRY(ctx, cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    TE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (herr) return set_error(ctx, TE_ERR_INTERNAL, "bosonic basis hash table lookup failed");
    return TE_OK;
}

te_status finish_matrix_stats(te_ctx* ctx, te_matrix* H) {
    cudaStream_t s = ctx->stream;
    DevBuf<unsigned long long> mx;
    DevBuf<int> mn, fl;
    TE_CUDA_TRY(ctx, mx.alloc(ctx, 1));
    TE_CUDA_TRY(ctx, mn.alloc(ctx, 1));
    TE_CUDA_TRY(ctx, fl.alloc(ctx, 1));
    TE_CUDA_TRY(ctx, cudaMemsetAsync(mx.p, 0, sizeof(unsigned long long), s));
    TE_CUDA_TRY(ctx, cudaMemsetAsync(mn.p, 0, sizeof(int), s));
    TE_CUDA_TRY(ctx, cudaMemsetAsync(fl.p, 0, sizeof(int), s));
    k_row_stats<<<grid_for(H->d), TE_BLOCK, 0, s>>>(H->rowptr, H->col, H->val, H->d, mx.p, mn.p, fl.p);
    TE_CUDA_TRY(ctx, cudaGetLastError());
    unsigned long long bits = 0;
    int maxnnz = 0, flags = 0;
    TE_CUDA_TRY(ctx, cudaMemcpyAsync(&bits, mx.p, sizeof(bits), cudaMemcpyDeviceToHost, s));
    TE_CUDA_TRY(ctx, cudaMemcpyAsync(&maxnnz, mn.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    TE_CUDA_TRY(ctx, cudaMemcpyAsync(&flags, fl.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    TE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (flags & 1) return set_error(ctx, TE_ERR_NONFINITE, "matrix has NaN or Inf entries");
    if (flags & 2) return set_error(ctx, TE_ERR_INVALID_ARG, "column index outside [0, d)");
    double n1;
    memcpy(&n1, &bits, sizeof(n1));
    H->norm1 = n1;
    H->max_row_nnz = maxnnz;
    H->lanes = spmv_lanes_for(H->d > 0 ? (double)H->nnz / (double)H->d : 0.0);
    return TE_OK;
}

int64_t bose_rank_host(int K, int N, const int32_t* occ) {
    BoseTables T;
    bose_tables(K, N, &T);
    int sum = 0;
    for (int i = 0; i < K; ++i) {
        if (occ[i] < 0) return -1;
        sum += occ[i];
    }
    if (sum != N) return -1;
    int64_t idx = 0;
    int rem = N;
    for (int p = 0; p < K - 1; ++p) {
        for (int a = rem; a > occ[p]; --a) idx += (int64_t)T.comp[rem - a][K - 1 - p];
        rem -= occ[p];
    }
    return idx;
}

te_status build_memory(te_ctx* ctx, const te_model_desc* m, te_matrix* H) {
    const int K = m->L, Kp = m->L2, Nm = m->N, N0 = m->N2;
    if (K < 1 || Kp < 1 || K + Kp > 30 || Nm < 0 || Nm > K + Kp || N0 < 0 || !m->a || !m->p ||
        (int64_t)Nm * (K + Kp - Nm) + 3 > kMemMaxEntries)
        return set_error(ctx, TE_ERR_INVALID_ARG,
                         "memory model needs K, K' >= 1, K + K' <= 30, 0 <= Nm <= K + K', N0 >= 0, "
                         "Nm (K + K' - Nm) <= 225, the f table and 5 scalar parameters");
    MemTables T;
    mem_tables(m, &T);
    const long long dd = (long long)(N0 + 1) * T.nq;
    if (dd >= (1ll << 31)) return set_error(ctx, TE_ERR_UNSUPPORTED, "basis too large");
    const int64_t d = dd;
    cudaStream_t s = ctx->stream;
    const int Q = K + Kp;
    DevBuf<double> f;
    DevBuf<int32_t> cnt;
    DevBuf<int> err;
    te_status st;
    if ((st = upload(ctx, f, m->a, (size_t)std::max(Q * (Q - 1) / 2, 1), s))) return st;
    TE_CUDA_TRY(ctx, cnt.alloc(ctx, d));
    TE_CUDA_TRY(ctx, err.alloc(ctx, 1));
    TE_CUDA_TRY(ctx, cudaMemsetAsync(err.p, 0, sizeof(int), s));
    k_count_memory<<<grid_for(d), TE_BLOCK, 0, s>>>(T, d, cnt.p);
    TE_CUDA_TRY(ctx, cudaGetLastError());
    int32_t* rowptr = nullptr;
    TE_CUDA_TRY(ctx, dev_alloc(ctx, &rowptr, sizeof(int32_t) * (d + 1)));
    int64_t nnz = 0;
    if ((st = scan_counts(ctx, cnt.p, d, rowptr, &nnz, s))) {
        dev_free(ctx, rowptr);
        return st;
    }
    H->d = d;
    H->nnz = nnz;
    H->rowptr = rowptr;
    if (dev_alloc(ctx, &H->col, sizeof(int32_t) * nnz) != cudaSuccess ||
        dev_alloc(ctx, &H->val, sizeof(double2) * nnz) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, TE_ERR_OOM, "device allocation of the CSR arrays failed");
    }
    k_fill_memory<<<grid_for(d), TE_BLOCK, 0, s>>>(T, f.p, d, rowptr, H->col, H->val, err.p);
    TE_CUDA_TRY(ctx, cudaGetLastError());
    int herr = 0;
    TE_CUDA_TRY(ctx, cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    TE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (herr) return set_error(ctx, TE_ERR_INTERNAL, "memory model row length mismatch");
    return TE_OK;
}

int64_t memory_rank_host(const te_model_desc* m, const int32_t* occ) {
    MemTables T;
    mem_tables(m, &T);
    const int n0 = occ[0], m0 = occ[1];
    if (n0 < 0 || m0 < 0 || n0 + m0 != T.N0) return -1;
    unsigned mask = 0;
    int ones = 0;
    for (int q = 0; q < T.Q; ++q) {
        if (occ[2 + q] != 0 && occ[2 + q] != 1) return -1;
        if (occ[2 + q]) {
            mask |= 1u << q;
            ++ones;
        }
    }
    if (ones != T.Nm) return -1;
    return (long long)(T.N0 - n0) * T.nq + mem_rank(T, mask);
}

// ---------------------------------------------------------------- occupations

namespace {

__global__ void k_occ_spin(int64_t d, int l, double* __restrict__ out) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d;
         r += (int64_t)gridDim.x * blockDim.x)
        out[r] = (double)((r >> l) & 1);
}

__global__ void k_occ_bose(BoseTables T, int64_t d, int l, double* __restrict__ out) {
    int occ[16];
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d;
         r += (int64_t)gridDim.x * blockDim.x) {
        bose_unrank(T, r, occ);
        out[r] = (double)occ[l];
    }
}

__global__ void k_occ_memory(MemTables T, int64_t d, int l, double* __restrict__ out) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d;
         r += (int64_t)gridDim.x * blockDim.x) {
        const long long b = r / T.nq;
        double v;
        if (l == 0) v = (double)(T.N0 - b);
        else if (l == 1) v = (double)b;
        else v = (double)((mem_unrank(T, r - b * T.nq) >> (l - 2)) & 1u);
        out[r] = v;
    }
}

}  // namespace

extern "C" te_status te_model_occupation(te_ctx* ctx, const te_model_desc* desc, int32_t mode,
                                         double* out, uint32_t flags) {
    if (!ctx || !desc || !out) return TE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaGetLastError();
    cudaStream_t s = ctx->stream;
    int64_t d = 0;
    int modes = 0;
    BoseTables BT;
    MemTables MT;
    switch (desc->model) {
        case TE_MODEL_TFIM:
        case TE_MODEL_XXZDM:
            if (desc->L < 2 || desc->L > 30) return set_error(ctx, TE_ERR_INVALID_ARG, "L outside 2..30");
            d = 1ll << desc->L;
            modes = desc->L;
            break;
        case TE_MODEL_BOSE:
            if (desc->L < 2 || desc->L > 16 || desc->N < 1 || desc->N > 15)
                return set_error(ctx, TE_ERR_INVALID_ARG, "bosons need 2 <= K <= 16, 1 <= N <= 15");
            bose_tables(desc->L, desc->N, &BT);
            d = (int64_t)BT.comp[desc->N][desc->L];
            modes = desc->L;
            break;
        case TE_MODEL_MEMORY:
            if (desc->L < 1 || desc->L2 < 1 || desc->L + desc->L2 > 30 || desc->N < 0 ||
                desc->N > desc->L + desc->L2 || desc->N2 < 0)
                return set_error(ctx, TE_ERR_INVALID_ARG, "invalid memory model sizes");
            mem_tables(desc, &MT);
            d = (int64_t)(desc->N2 + 1) * MT.nq;
            modes = 2 + desc->L + desc->L2;
            break;
        default:
            return set_error(ctx, TE_ERR_INVALID_ARG, "unknown model");
    }
    if (mode < 0 || mode >= modes) return set_error(ctx, TE_ERR_INVALID_ARG, "mode outside the model");
    const bool dev = (flags & TE_PTR_DEVICE) != 0;
    double* dst = out;
    if (!dev) TE_CUDA_TRY(ctx, dev_alloc(ctx, &dst, sizeof(double) * (size_t)d));
    const int grid = grid_for(d);
    switch (desc->model) {
        case TE_MODEL_TFIM:
        case TE_MODEL_XXZDM: k_occ_spin<<<grid, TE_BLOCK, 0, s>>>(d, mode, dst); break;
        case TE_MODEL_BOSE: k_occ_bose<<<grid, TE_BLOCK, 0, s>>>(BT, d, mode, dst); break;
        default: k_occ_memory<<<grid, TE_BLOCK, 0, s>>>(MT, d, mode, dst); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !dev)
        e = cudaMemcpyAsync(out, dst, sizeof(double) * (size_t)d, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (!dev) dev_free(ctx, dst);
    if (e != cudaSuccess) return cuda_error(ctx, e, "te_model_occupation");
    return TE_OK;
}
