// te_sell.cu -- sliced-ELLPACK (SELL-C-sigma) form of H and the SpMV that uses it.
//
// On GB300 the FP64 pipe executes 2 lanes per SM per cycle (1.26 TFLOP/s for
// the whole GPU), while a complex128 multiply-add costs 4 DFMA per stored entry
// of 20 bytes.  The product y = H x is therefore bound by FP64 issue, not by
// HBM, and the layout is chosen to waste no FP64 lane: one lane per row, 32
// rows per slice (a warp), every row of a slice padded to the slice's widest
// row, and rows sorted by length inside windows of kSigma rows so that padding
// is rare.  No lane idles inside the loop and no shuffle reduction is needed.
//
// The sort is a symmetric permutation of the basis: new index i holds old row
// perm[i], columns are renumbered through iperm, and the solver works on
// permuted vectors (copied in and out once per solve).  Entries of slice s
// are stored lane-interleaved: entry k of lane l sits at off[s] + 32 k + l, so
// each warp load is 32 consecutive values.  Padding entries hold 0 and point at
// the lane's own row.
//
// Each complex multiply-add costs three DFMA instead of four: for an entry
// h = a + ib and a vector element x + iy,
//     Re(h x) = a (x + y) - (a + b) y,   Im(h x) = a (x + y) + (b - a) x
// (Gauss's three-multiplication complex product; normwise stable, Higham, SIAM
// J. Matrix Anal. Appl. 13 (1992) 681).  The matrix keeps a and the pair
// (b - a, a + b) per entry, and the product reads the sums s = x + y of the
// vector from a companion array that the kernels writing Lanczos vectors fill.
// The three sums are accumulated separately over the row and combined at its
// end.  The gathers this adds go to the load/store path, which this kernel
// leaves mostly idle.
//
// Value-indexed form.  Hamiltonians built from a few couplings hold few
// distinct off-diagonal values (tens for spin chains, thousands for bosons),
// so the copy can store, per entry, the column and a 16-bit index into a table
// of (a, b - a, a + b) triples, with the (real) diagonal in an array of its own:
// 6 bytes per entry instead of 28, which leaves the product bound by FP64 issue
// alone.  The table is found on the device with a hash set keyed on the value's
// 128 bits; a matrix with a complex diagonal or more than 65535 distinct
// off-diagonal values keeps the full-value form.  When every off-diagonal
// value is real, the product uses the table's a alone: two DFMA per entry.
#include <algorithm>
#include <vector>

#include "te_internal.cuh"
#include "te_slices.cuh"

using te_slices::FullSlices;
using te_slices::IndexedSlices;
using te_slices::RealIndexedSlices;

namespace {

constexpr int kSigma = 1024;     // rows per sorting window (multiple of 32)
constexpr int kGroup = 256;      // tasks per group of the two-level Re<x, Hx> sum
constexpr int64_t kCtrMin = 4096; // partials the other reduction kernels may use from index 0
constexpr int kTaskEntries = 1536;   // stored entries per SpMV task (slices are grouped to this)

// The SpMV keeps per-group counters in its partials buffer, above what the other
// reduction kernels of a restart write (they use at most kCtrMin entries from 0),
// so they persist (at zero) from one launch to the next.
// Tasks: the first sell_big_tasks() take tpt slices each, the remaining slices
// (about the last eighth) go out one per task, which shortens the ragged end.
__host__ __device__ __forceinline__ int64_t sell_big_tasks(int64_t nslices, int tpt) {
    return tpt > 1 ? (nslices - nslices / 8) / tpt : 0;
}
__host__ __device__ __forceinline__ int64_t sell_ntasks(int64_t nslices, int tpt) {
    const int64_t nb = sell_big_tasks(nslices, tpt);
    return tpt > 1 ? nb + (nslices - nb * tpt) : nslices;
}

__host__ __device__ __forceinline__ int64_t sell_ctr_offset(int64_t ntasks) {
    const int64_t ngroups = (ntasks + kGroup - 1) / kGroup;
    return ntasks + ngroups > kCtrMin ? ntasks + ngroups : kCtrMin;
}

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

// ---------------------------------------------------------------- conversion

// Stored length of each row: all entries (full-value form) or the off-diagonal
// ones (value-indexed form, whose diagonal has an array of its own).
__global__ void k_row_len(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                          int64_t d, int offdiag, int32_t* __restrict__ len) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int b = rowptr[r], e = rowptr[r + 1];
        int l = e - b;
        if (offdiag)
            for (int q = b; q < e; ++q) l -= (col[q] == r);
        len[r] = l;
    }
}

// One block per window: rank of each row = rows that are longer, or equally
// long with a smaller index (a stable descending sort by length).
__global__ void __launch_bounds__(kSigma) k_sell_rank(const int32_t* __restrict__ rowlen, int64_t d,
                                                      int32_t* __restrict__ perm,
                                                      int32_t* __restrict__ iperm) {
    __shared__ int32_t len[kSigma];
    const int64_t base = (int64_t)blockIdx.x * kSigma;
    const int n = (int)((d - base) < kSigma ? (d - base) : kSigma);
    const int t = threadIdx.x;
    if (t < n) len[t] = rowlen[base + t];
    __syncthreads();
    if (t >= n) return;
    const int mine = len[t];
    int rank = 0;
    for (int q = 0; q < n; ++q) {
        const int l = len[q];
        rank += (l > mine) || (l == mine && q < t);
    }
    perm[base + rank] = (int32_t)(base + t);
    iperm[base + t] = (int32_t)(base + rank);
}

// Entries of slice s: 32 x (length of its first, longest row).
__global__ void k_sell_width(const int32_t* __restrict__ rowlen, const int32_t* __restrict__ perm,
                             int64_t nslices, int32_t* __restrict__ cnt) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nslices) return;
    cnt[s] = 32 * rowlen[perm[s * 32]];
}

// ---------------------------------------------------------------- value table

struct alignas(16) VKey {
    unsigned long long lo, hi;
};
constexpr int kDictBits = 17;
constexpr int kDictSlots = 1 << kDictBits;     // hash slots (load factor <= 1/2)
constexpr int kDictMax = 65535;                // distinct values (index 0 is the zero value)
constexpr int kProbeMax = 512;
constexpr unsigned long long kEmpty = ~0ull;   // a NaN pattern: never a stored value

__device__ __forceinline__ VKey vkey(double2 v) {
    VKey k;
    k.lo = (unsigned long long)__double_as_longlong(v.x);
    k.hi = (unsigned long long)__double_as_longlong(v.y);
    return k;
}

__device__ __forceinline__ unsigned int vhash(VKey k) {
    unsigned long long h = k.lo * 0x9E3779B97F4A7C15ull ^ (k.hi + 0x632BE59BD9B4E019ull) * 0xC2B2AE3D27D4EB4Full;
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 29;
    return (unsigned int)(h >> (64 - kDictBits));
}

// Read of a slot that may race with its insertion; a torn read is neither empty
// nor any finite value, so the caller treats it as "taken by another value".
__device__ __forceinline__ VKey read_slot(const VKey* slot) {
    const double2 raw = __ldcg(reinterpret_cast<const double2*>(slot));
    VKey k;
    k.lo = (unsigned long long)__double_as_longlong(raw.x);
    k.hi = (unsigned long long)__double_as_longlong(raw.y);
    return k;
}

// flags[0]: table full or probe limit hit; flags[1]: complex diagonal entry;
// flags[2]: distinct values inserted; flags[3]: an off-diagonal value with a
// nonzero imaginary part (the table is complex).  A value may land in two slots when two
// threads race on it (harmless: both hold the same value).
__global__ void k_dict_insert(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                              const double2* __restrict__ val, int64_t d, VKey* slots, int* flags) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d;
         r += (int64_t)gridDim.x * blockDim.x) {
        for (int q = rowptr[r]; q < rowptr[r + 1]; ++q) {
            const double2 v = val[q];
            if (col[q] == r) {
                if (v.y != 0.0) atomicExch(&flags[1], 1);
                continue;
            }
            if (v.y != 0.0) atomicExch(&flags[3], 1);
            const VKey key = vkey(v);
            unsigned int h = vhash(key);
            bool placed = false;
            for (int probe = 0; probe < kProbeMax && !placed; ++probe) {
                VKey cur = read_slot(slots + h);
                if (cur.lo == key.lo && cur.hi == key.hi) {
                    placed = true;
                } else if (cur.lo == kEmpty && cur.hi == kEmpty) {
                    VKey empty{kEmpty, kEmpty};
                    const VKey prev = atomicCAS(slots + h, empty, key);
                    if (prev.lo == kEmpty && prev.hi == kEmpty) {
                        atomicAdd(&flags[2], 1);
                        placed = true;
                    } else if (prev.lo == key.lo && prev.hi == key.hi) {
                        placed = true;
                    }
                }
                if (!placed) h = (h + 1) & (kDictSlots - 1);
            }
            if (!placed) atomicExch(&flags[0], 1);
        }
    }
}

// One block: dense index 1.. of every filled slot (in slot order) and the
// table of (a, b - a, a + b); index 0 is the zero value used by padding.
__global__ void __launch_bounds__(1024) k_dict_compact(const VKey* __restrict__ slots,
                                                       uint16_t* __restrict__ slot_idx,
                                                       double* __restrict__ ta,
                                                       double2* __restrict__ tpq) {
    __shared__ int part[1024];
    constexpr int per = kDictSlots / 1024;
    const int t = threadIdx.x;
    int n = 0;
    for (int i = 0; i < per; ++i) {
        const VKey k = slots[t * per + i];
        n += !(k.lo == kEmpty && k.hi == kEmpty);
    }
    part[t] = n;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {           // inclusive scan (Hillis-Steele)
        const int v = (t >= o) ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int idx = 1 + part[t] - n;
    for (int i = 0; i < per; ++i) {
        const VKey k = slots[t * per + i];
        if (k.lo == kEmpty && k.hi == kEmpty) continue;
        const double a = __longlong_as_double((long long)k.lo);
        const double b = __longlong_as_double((long long)k.hi);
        if (idx <= kDictMax) {
            slot_idx[t * per + i] = (uint16_t)idx;
            ta[idx] = a;
            tpq[idx] = make_double2(b - a, a + b);
        }
        ++idx;
    }
    if (t == 0) {
        ta[0] = 0.0;
        tpq[0] = make_double2(0.0, 0.0);
    }
}

__device__ __forceinline__ uint16_t dict_find(const VKey* slots, const uint16_t* slot_idx,
                                              double2 v, int* flags) {
    const VKey key = vkey(v);
    unsigned int h = vhash(key);
    for (int probe = 0; probe < kProbeMax; ++probe) {
        const VKey cur = slots[h];
        if (cur.lo == key.lo && cur.hi == key.hi) return slot_idx[h];
        h = (h + 1) & (kDictSlots - 1);
    }
    atomicExch(&flags[0], 1);
    return 0;
}

// Value-indexed slices: column and table index per off-diagonal entry, the real
// diagonal per (permuted) row.
__global__ void k_sellv_fill(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const double2* __restrict__ val, const int32_t* __restrict__ perm,
                             const int32_t* __restrict__ iperm, const int32_t* __restrict__ off,
                             int64_t d, int64_t nslices, const VKey* __restrict__ slots,
                             const uint16_t* __restrict__ slot_idx, int32_t* __restrict__ scol,
                             uint16_t* __restrict__ sidx, double* __restrict__ diag, int* flags) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nslices * 32) return;
    const int64_t s = i >> 5;
    const int lane = (int)(i & 31);
    const int64_t o = off[s];
    const int w = (off[s + 1] - off[s]) >> 5;
    const int32_t self = (int32_t)(i < d ? i : 0);
    int k = 0;
    double dg = 0.0;
    if (i < d) {
        const int64_t old = perm[i];
        for (int q = rowptr[old]; q < rowptr[old + 1]; ++q) {
            const double2 v = val[q];
            if (col[q] == old) {
                dg = v.x;
                continue;
            }
            if (k < w) {
                const int64_t p = o + 32ll * k + lane;
                scol[p] = iperm[col[q]];
                sidx[p] = dict_find(slots, slot_idx, v, flags);
            }
            ++k;
        }
        diag[i] = dg;
    }
    for (; k < w; ++k) {
        const int64_t p = o + 32ll * k + lane;
        scol[p] = self;
        sidx[p] = 0;
    }
}

__global__ void k_sell_fill(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const double2* __restrict__ val, const int32_t* __restrict__ perm,
                            const int32_t* __restrict__ iperm, const int32_t* __restrict__ off,
                            int64_t d, int64_t nslices, int32_t* __restrict__ scol,
                            double* __restrict__ sa, double2* __restrict__ spq) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nslices * 32) return;
    const int64_t s = i >> 5;
    const int lane = (int)(i & 31);
    const int64_t o = off[s];
    const int w = (off[s + 1] - off[s]) >> 5;
    int b = 0, len = 0;
    if (i < d) {
        const int64_t old = perm[i];
        b = rowptr[old];
        len = rowptr[old + 1] - b;
    }
    const int32_t self = (int32_t)(i < d ? i : 0);
    for (int k = 0; k < w; ++k) {
        const int64_t p = o + 32ll * k + lane;
        if (k < len) {
            const double2 v = val[b + k];
            scol[p] = iperm[col[b + k]];
            sa[p] = v.x;                                   // a
            spq[p] = make_double2(v.y - v.x, v.x + v.y);   // (b - a, a + b)
        } else {
            scol[p] = self;
            sa[p] = 0.0;
            spq[p] = make_double2(0.0, 0.0);
        }
    }
}

// ---------------------------------------------------------------- SpMV

// mode 0: Lanczos step j (y = sign scale[j] H u_j - beta[j-1] scale[j-1] u_{j-1},
// partial Re<u_j, y>, matvec count); mode 1: y = H x and Re<x, y>.  xs[i] must
// hold Re x_i + Im x_i.
//
// Each warp takes one task (tpt consecutive slices, about kTaskEntries stored
// entries; the last eighth of the slices one per task, so that the tasks still
// running at the end are short) at a time from an atomic counter, asking for the
// next one only when it is done with the current one (reserving ahead left every
// warp holding an unstarted task at the end and stretched the tail).  SMs that run slower simply
// take fewer tasks, and the kernel ends within about one task of perfect
// balance.  Re<x, y> is summed without atomics on values: every task
// stores its warp's partial; the warp that completes a group of kGroup tasks (a
// per-group counter tells it) adds the group's partials in task order; the last
// CTA to finish adds the group sums in group order.  The result does not depend
// on which warp took which task.
template <class Slices, int kAsync = 0, bool kPair = false>
__device__ __forceinline__ void spmv_sell_body(const Slices& M, const double2* __restrict__ x,
                                               const double* __restrict__ xs,
                                               const double2* __restrict__ xprev,
                                               double2* __restrict__ y, int64_t d, int64_t nslices,
                                               int tpt, DevState* st, int j, int mode,
                                               double* partials, unsigned char* stage = nullptr) {
    __shared__ double sh[32];
    __shared__ bool am_last;
    double cx = 1.0, bp = 0.0;
    if (mode == 0) {
        if (st->status != 0 || st->done != 0 || st->stop) return;
        cx = st->sign * st->scale[j];
        if (j > 0) bp = st->beta[j - 1] * st->scale[j - 1];
    }
    const int lane = threadIdx.x & 31;
    const int64_t ntasks = sell_ntasks(nslices, tpt);
    const int64_t nbig = sell_big_tasks(nslices, tpt);
    const int64_t ngroups = (ntasks + kGroup - 1) / kGroup;
    double* gpart = partials + ntasks;
    unsigned int* gctr = reinterpret_cast<unsigned int*>(partials + sell_ctr_offset(ntasks));
    unsigned int* next = &st->counter[6];
    unsigned int c = 0;
    if (lane == 0) c = atomicAdd(next, 1u);
    c = __shfl_sync(0xffffffffu, c, 0);
    while ((int64_t)c < ntasks) {
        const bool big = (int64_t)c < nbig;
        const int64_t s0 = big ? (int64_t)c * tpt : nbig * tpt + ((int64_t)c - nbig);
        const int64_t s1 = big ? s0 + tpt : s0 + 1;
        double acc = 0.0;
        // y of one row from its product hx; the alpha partial in slice order
        auto finish = [&](int64_t row, bool real_row, double2 xr, double2 hx) {
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
        };
        int64_t s = s0;
        if constexpr (kPair) {
#pragma unroll 1
            for (; s + 1 < s1; s += 2) {                  // two slices per pass
                const int64_t ra = s * 32 + lane, rb = ra + 32;
                const bool reala = ra < d, realb = rb < d;
                const double2 xa = reala ? __ldg(x + ra) : make_double2(0.0, 0.0);
                const double2 xb = realb ? __ldg(x + rb) : make_double2(0.0, 0.0);
                double2 ha, hb;
                M.row_pair(s, s + 1, lane, x, xs, reala ? ra : -1, realb ? rb : -1, xa, xb, &ha, &hb);
                finish(ra, reala, xa, ha);
                finish(rb, realb, xb, hb);
            }
        }
#pragma unroll 1
        for (; s < s1; ++s) {
            const int64_t row = s * 32 + lane;
            const bool real_row = row < d;
            const double2 xr = real_row ? __ldg(x + row) : make_double2(0.0, 0.0);
            double2 hx;
            if constexpr (kAsync > 0) {
                const te_slices::Staging<kAsync, 3> stg(
                    stage + (threadIdx.x >> 5) * te_slices::Staging<kAsync, 3>::kBytesPerWarp);
                hx = M.template row_async<kAsync>(s, lane, x, xs, real_row ? row : -1, xr, stg);
            } else {
                hx = M.row(s, lane, x, xs, real_row ? row : -1, xr);
            }
            finish(row, real_row, xr, hx);
        }
        acc = warp_sum(acc);
        unsigned int done = 0;
        const int64_t g = (int64_t)c / kGroup;
        if (lane == 0) {
            partials[c] = acc;
            __threadfence();
            done = atomicAdd(gctr + g, 1u);
        }
        done = __shfl_sync(0xffffffffu, done, 0);
        const int64_t gsize = (g + 1) * kGroup <= ntasks ? kGroup : ntasks - g * kGroup;
        if ((int64_t)done == gsize - 1) {             // this warp finished group g
            __threadfence();
            double v = 0.0;
            for (int64_t i = lane; i < gsize; i += 32) v += __ldcg(partials + g * kGroup + i);
            v = warp_sum(v);
            if (lane == 0) {
                gpart[g] = v;
                gctr[g] = 0;
                __threadfence();
            }
        }
        unsigned int cn = 0;
        if (lane == 0) cn = atomicAdd(next, 1u);
        c = __shfl_sync(0xffffffffu, cn, 0);
    }
    __syncthreads();
    unsigned int* ctr = &st->counter[1];
    if (threadIdx.x == 0) {
        __threadfence();
        am_last = (atomicAdd(ctr, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < ngroups; i += blockDim.x) v += __ldcg(gpart + i);
    const double tot = block_sum(v, sh);
    if (threadIdx.x == 0) {
        if (mode == 0) {
            const double a = st->scale[j] * tot;
            st->alpha[j] = a;
            st->as_cur = a * st->scale[j];
            st->matvecs += 1;
        } else {
            st->spmv_dot = tot;
        }
        *ctr = 0;
        *next = 0;
    }
}

__global__ void __launch_bounds__(TE_BLOCK, 4) k_spmv_sell(
    FullSlices M, const double2* __restrict__ x, const double* __restrict__ xs,
    const double2* __restrict__ xprev, double2* __restrict__ y, int64_t d, int64_t nslices,
    int tpt, DevState* st, int j, int mode, double* partials) {
    spmv_sell_body(M, x, xs, xprev, y, d, nslices, tpt, st, j, mode, partials);
}

__global__ void __launch_bounds__(TE_BLOCK, 4) k_spmv_sellv(
    IndexedSlices M, const double2* __restrict__ x, const double* __restrict__ xs,
    const double2* __restrict__ xprev, double2* __restrict__ y, int64_t d, int64_t nslices,
    int tpt, DevState* st, int j, int mode, double* partials) {
    spmv_sell_body(M, x, xs, xprev, y, d, nslices, tpt, st, j, mode, partials);
}

// The value-indexed product with its gathers staged through shared memory (te_slices.cuh
// row_async; kTrip entries per trip, three stages per warp).  The sums are the same as
// k_spmv_sellv's, added in the same order: the results are bitwise equal.
// The value-indexed product taking two slices per pass (te_slices.cuh row_pair): twice
// the independent gathers and FMA chains per lane for short rows; bitwise k_spmv_sellv's.
__global__ void __launch_bounds__(TE_BLOCK, 3) k_spmv_sellv_pair(
    IndexedSlices M, const double2* __restrict__ x, const double* __restrict__ xs,
    const double2* __restrict__ xprev, double2* __restrict__ y, int64_t d, int64_t nslices,
    int tpt, DevState* st, int j, int mode, double* partials) {
    spmv_sell_body<IndexedSlices, 0, true>(M, x, xs, xprev, y, d, nslices, tpt, st, j, mode, partials);
}

// (Four-entry trips take 72 KB of staging per block, so three blocks fit an SM and each
// thread may use up to 85 registers.)
template <int kTrip>
__global__ void __launch_bounds__(TE_BLOCK, kTrip == 4 ? 3 : 4) k_spmv_sellv_async(
    IndexedSlices M, const double2* __restrict__ x, const double* __restrict__ xs,
    const double2* __restrict__ xprev, double2* __restrict__ y, int64_t d, int64_t nslices,
    int tpt, DevState* st, int j, int mode, double* partials) {
    extern __shared__ __align__(16) unsigned char stage_smem[];
    spmv_sell_body<IndexedSlices, kTrip>(M, x, xs, xprev, y, d, nslices, tpt, st, j, mode, partials,
                                         stage_smem);
}

__global__ void __launch_bounds__(TE_BLOCK, 4) k_spmv_sellr(
    RealIndexedSlices M, const double2* __restrict__ x, const double* __restrict__ xs,
    const double2* __restrict__ xprev, double2* __restrict__ y, int64_t d, int64_t nslices,
    int tpt, DevState* st, int j, int mode, double* partials) {
    spmv_sell_body(M, x, xs, xprev, y, d, nslices, tpt, st, j, mode, partials);
}

// dst[i] = src[map[i]]  (map = perm: old -> new order; map = iperm: back);
// with dsum, also dsum[i] = Re dst[i] + Im dst[i] for the product's 3M form.
__global__ void k_gather(const double2* __restrict__ src, const int32_t* __restrict__ map,
                         int64_t d, double2* __restrict__ dst, double* __restrict__ dsum) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = src[map[i]];
        dst[i] = v;
        if (dsum) dsum[i] = v.x + v.y;
    }
}

}  // namespace

namespace {

// Try the value table: returns true (and the table in H) when the diagonal is
// real and the off-diagonal values fit a 16-bit index.
te_status build_dict(te_ctx* ctx, te_matrix* H, VKey** slots_out, uint16_t** slot_idx_out,
                     int** flags_out, bool* ok) {
    cudaStream_t s = ctx->stream;
    *ok = false;
    VKey* slots = nullptr;
    uint16_t* slot_idx = nullptr;
    int* flags = nullptr;
    TE_CUDA_TRY(ctx, dev_alloc(ctx, &slots, sizeof(VKey) * kDictSlots));
    *slots_out = slots;
    TE_CUDA_TRY(ctx, dev_alloc(ctx, &slot_idx, sizeof(uint16_t) * kDictSlots));
    *slot_idx_out = slot_idx;
    TE_CUDA_TRY(ctx, dev_alloc(ctx, &flags, sizeof(int) * 4));
    *flags_out = flags;
    TE_CUDA_TRY(ctx, cudaMemsetAsync(slots, 0xff, sizeof(VKey) * kDictSlots, s));
    TE_CUDA_TRY(ctx, cudaMemsetAsync(flags, 0, sizeof(int) * 4, s));
    const int64_t want = (H->d + TE_BLOCK - 1) / TE_BLOCK;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)ctx->num_sms * 8));
    k_dict_insert<<<grid, TE_BLOCK, 0, s>>>(H->rowptr, H->col, H->val, H->d, slots, flags);
    TE_CUDA_TRY(ctx, cudaGetLastError());
    int hf[4] = {0, 0, 0, 0};
    TE_CUDA_TRY(ctx, cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
    TE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (hf[0] || hf[1] || hf[2] > kDictMax) return TE_OK;
    TE_CUDA_TRY(ctx, dev_alloc(ctx, &H->dict_a, sizeof(double) * (size_t)(hf[2] + 1)));
    TE_CUDA_TRY(ctx, dev_alloc(ctx, &H->dict_pq, sizeof(double2) * (size_t)(hf[2] + 1)));
    k_dict_compact<<<1, 1024, 0, s>>>(slots, slot_idx, H->dict_a, H->dict_pq);
    TE_CUDA_TRY(ctx, cudaGetLastError());
    H->dict_n = hf[2];
    H->dict_real = hf[3] == 0;
    *ok = true;
    return TE_OK;
}

}  // namespace

te_status build_sell(te_ctx* ctx, te_matrix* H) {
    cudaStream_t s = ctx->stream;
    const int64_t d = H->d;
    const int64_t nslices = (d + 31) / 32;
    const int64_t windows = (d + kSigma - 1) / kSigma;
    VKey* slots = nullptr;
    uint16_t* slot_idx = nullptr;
    int* flags = nullptr;
    int32_t* rowlen = nullptr;
    int32_t* cnt = nullptr;
    auto cleanup = [&]() {
        for (void* q : {(void*)slots, (void*)slot_idx, (void*)flags, (void*)rowlen, (void*)cnt})
            if (q) dev_free(ctx, q);
    };
    bool dict = false;
    te_status st = build_dict(ctx, H, &slots, &slot_idx, &flags, &dict);
    if (st) {
        cleanup();
        return st;
    }
    if (!dict) {
        if (H->dict_a) dev_free(ctx, H->dict_a);
        if (H->dict_pq) dev_free(ctx, H->dict_pq);
        H->dict_a = nullptr;
        H->dict_pq = nullptr;
        H->dict_n = 0;
        H->dict_real = false;
    }
    cudaError_t e = dev_alloc(ctx, &H->perm, sizeof(int32_t) * (size_t)nslices * 32);
    if (e == cudaSuccess) e = dev_alloc(ctx, &H->iperm, sizeof(int32_t) * (size_t)d);
    if (e == cudaSuccess) e = dev_alloc(ctx, &H->sell_off, sizeof(int32_t) * (size_t)(nslices + 1));
    if (e == cudaSuccess) e = dev_alloc(ctx, &rowlen, sizeof(int32_t) * (size_t)d);
    if (e == cudaSuccess) e = dev_alloc(ctx, &cnt, sizeof(int32_t) * (size_t)nslices);
    // rows past d (in the last slice) map to row 0's length: give perm a valid entry there
    if (e == cudaSuccess) e = cudaMemsetAsync(H->perm, 0, sizeof(int32_t) * (size_t)nslices * 32, s);
    const int64_t want = (d + TE_BLOCK - 1) / TE_BLOCK;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)ctx->num_sms * 8));
    if (e == cudaSuccess) {
        k_row_len<<<grid, TE_BLOCK, 0, s>>>(H->rowptr, H->col, d, dict ? 1 : 0, rowlen);
        k_sell_rank<<<(int)windows, kSigma, 0, s>>>(rowlen, d, H->perm, H->iperm);
        k_sell_width<<<(int)((nslices + TE_BLOCK - 1) / TE_BLOCK), TE_BLOCK, 0, s>>>(rowlen, H->perm,
                                                                                    nslices, cnt);
        e = cudaGetLastError();
    }
    int64_t total = 0;
    if (e == cudaSuccess) st = scan_counts(ctx, cnt, nslices, H->sell_off, &total, s);
    if (e != cudaSuccess || st) {
        cleanup();
        return e != cudaSuccess ? cuda_error(ctx, e, "building the sliced copy") : st;
    }
    H->nslices = nslices;
    H->sell_nnz = total;
    {
        const double per_slice = (double)total / (double)nslices;
        const double t = per_slice > 0.0 ? kTaskEntries / per_slice : 16.0;
        // at most 4 slices: XXZ-DM L = 20 keeps only ~5 tasks per resident warp at 4
        H->sell_tpt = (int)std::min(4.0, std::max(1.0, floor(t + 0.5)));
    }
    const size_t tot1 = (size_t)std::max<int64_t>(total, 1);
    e = dev_alloc(ctx, &H->sell_col, sizeof(int32_t) * tot1);
    if (dict) {
        if (e == cudaSuccess) e = dev_alloc(ctx, &H->sell_idx, sizeof(uint16_t) * tot1);
        if (e == cudaSuccess) e = dev_alloc(ctx, &H->sell_diag, sizeof(double) * (size_t)d);
        if (e == cudaSuccess) {
            k_sellv_fill<<<(int)((nslices * 32 + TE_BLOCK - 1) / TE_BLOCK), TE_BLOCK, 0, s>>>(
                H->rowptr, H->col, H->val, H->perm, H->iperm, H->sell_off, d, nslices, slots,
                slot_idx, H->sell_col, H->sell_idx, H->sell_diag, flags);
            e = cudaGetLastError();
        }
    } else {
        if (e == cudaSuccess) e = dev_alloc(ctx, &H->sell_a, sizeof(double) * tot1);
        if (e == cudaSuccess) e = dev_alloc(ctx, &H->sell_pq, sizeof(double2) * tot1);
        if (e == cudaSuccess) {
            k_sell_fill<<<(int)((nslices * 32 + TE_BLOCK - 1) / TE_BLOCK), TE_BLOCK, 0, s>>>(
                H->rowptr, H->col, H->val, H->perm, H->iperm, H->sell_off, d, nslices, H->sell_col,
                H->sell_a, H->sell_pq);
            e = cudaGetLastError();
        }
    }
    int hf[4] = {0, 0, 0, 0};
    if (e == cudaSuccess && dict) e = cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) return cuda_error(ctx, e, "filling the sliced copy");
    if (dict && hf[0]) return set_error(ctx, TE_ERR_INTERNAL, "value table lookup failed");
    H->sell_grid = sell_grid(nslices, ctx->num_sms, dict ? (H->dict_real ? 2 : 1) : 0);
    return TE_OK;
}

int sell_grid(int64_t nslices, int num_sms, int form) {
    int nb = 0;
    if (form == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv_sellr, TE_BLOCK, 0);
    else if (form == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv_sellv, TE_BLOCK, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv_sell, TE_BLOCK, 0);
    if (nb < 1) nb = 1;
    const int64_t need = (nslices + (TE_BLOCK / 32) - 1) / (TE_BLOCK / 32);
    const int64_t full = (int64_t)nb * num_sms;
    return (int)std::max<int64_t>(1, std::min(need, full));
}

constexpr int async_smem(int trip) {
    return (TE_BLOCK / 32) * (trip == 4 ? te_slices::Staging<4, 3>::kBytesPerWarp
                                        : te_slices::Staging<2, 3>::kBytesPerWarp);
}

cudaError_t sell_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_spmv_sellv_async<4>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, async_smem(4));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_spmv_sellv_async<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 async_smem(2));
    return e;
}

int sell_async_grid(int64_t nslices, int num_sms, int trip) {
    int nb = 0;
    if (trip == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv_sellv_pair, TE_BLOCK, 0);
    else if (trip == 4)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv_sellv_async<4>, TE_BLOCK, async_smem(4));
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv_sellv_async<2>, TE_BLOCK, async_smem(2));
    if (nb < 1) nb = 1;
    const int64_t need = (nslices + (TE_BLOCK / 32) - 1) / (TE_BLOCK / 32);
    const int64_t full = (int64_t)nb * num_sms;
    return (int)std::max<int64_t>(1, std::min(need, full));
}

// partials must hold sell_partials(H) doubles (one per chunk of slices); xs holds
// Re x + Im x.
cudaError_t launch_spmv_sell(const te_matrix* H, const double2* x, const double* xs,
                             const double2* xprev, double2* y, DevState* st, int j, int mode,
                             double* partials, cudaStream_t s, int grid) {
    const int g = grid > 0 ? grid : H->sell_grid;
    if (H->sell_idx && H->dict_real) {
        const RealIndexedSlices M{H->sell_off, H->sell_col, H->sell_idx, H->dict_a, H->sell_diag};
        k_spmv_sellr<<<g, TE_BLOCK, 0, s>>>(M, x, xs, xprev, y, H->d, H->nslices,
                                                      H->sell_tpt, st, j, mode, partials);
    } else if (H->sell_idx) {
        const IndexedSlices M{H->sell_off, H->sell_col, H->sell_idx, H->dict_a, H->dict_pq,
                              H->sell_diag};
        if (H->sell_async == 1)
            k_spmv_sellv_pair<<<g, TE_BLOCK, 0, s>>>(M, x, xs, xprev, y, H->d, H->nslices,
                                                               H->sell_tpt, st, j, mode, partials);
        else if (H->sell_async == 4)
            k_spmv_sellv_async<4><<<g, TE_BLOCK, async_smem(4), s>>>(
                M, x, xs, xprev, y, H->d, H->nslices, H->sell_tpt, st, j, mode, partials);
        else if (H->sell_async == 2)
            k_spmv_sellv_async<2><<<g, TE_BLOCK, async_smem(2), s>>>(
                M, x, xs, xprev, y, H->d, H->nslices, H->sell_tpt, st, j, mode, partials);
        else
            k_spmv_sellv<<<g, TE_BLOCK, 0, s>>>(M, x, xs, xprev, y, H->d, H->nslices,
                                                          H->sell_tpt, st, j, mode, partials);
    } else {
        const FullSlices M{H->sell_off, H->sell_col, H->sell_a, H->sell_pq};
        k_spmv_sell<<<g, TE_BLOCK, 0, s>>>(M, x, xs, xprev, y, H->d, H->nslices,
                                                     H->sell_tpt, st, j, mode, partials);
    }
    return cudaGetLastError();
}

cudaError_t launch_gather(const double2* src, const int32_t* map, int64_t d, double2* dst,
                          double* dsum, int num_sms, cudaStream_t s) {
    const int64_t want = (d + TE_BLOCK - 1) / TE_BLOCK;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms * 8));
    k_gather<<<grid, TE_BLOCK, 0, s>>>(src, map, d, dst, dsum);
    return cudaGetLastError();
}

// partials the SpMV needs: per-slice and per-group sums, then the group counters
// (which must be zero before the first launch).
int64_t sell_partials(const te_matrix* H) {
    const int64_t ntasks = sell_ntasks(H->nslices, H->sell_tpt);
    return sell_ctr_offset(ntasks) + (ntasks + kGroup - 1) / kGroup;
}
