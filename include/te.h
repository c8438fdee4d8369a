/*
 * te.h -- C ABI of libte: restarted Krylov time evolution exp(-iHt)v on one GPU.
 *
 * The method is TimeEvolver's (arXiv 2205.15346): Lanczos vectors of a sparse
 * Hermitian H (Sec. 2.1, eq. arnoldi), the a-posteriori error bound of
 * eq. errorIntegral evaluated by adaptive tanh-sinh quadrature (Sec. 2.3, Sec. 4),
 * the largest step allowed by eqs. errorRate and stepSize, the Krylov exponential
 * of eq. krylovApproximation, and a restart from the result (Algorithm 1).
 * Everything is complex128 / float64.
 *
 * Conventions for every call:
 *   - Functions return te_status; 0 is TE_OK.  They never abort or throw.  After
 *     an error te_last_error(ctx) holds a message owned by the context.
 *   - Complex vectors are interleaved (re, im) float64 pairs, i.e. the memory
 *     layout of C99 double complex / cuDoubleComplex / torch.complex128.
 *   - Pointers are host pointers unless the call's flags contain TE_PTR_DEVICE,
 *     in which case they are device pointers on the context's device.  Caller
 *     buffers are borrowed for the duration of the call only (te_submit copies
 *     its input vector before it returns).
 *   - Work is issued on the context's stream.  Synchronous calls (te_build_*,
 *     te_evolve, te_spmv, te_matrix_export) have finished on the device when
 *     they return.
 *   - Matrices are stored as CSR with int32 row pointers and column indices and
 *     complex128 values (20 bytes per stored entry); nnz must stay below 2^31.
 *     The library also keeps a sliced-ELLPACK copy (32-row slices, rows sorted by
 *     length within windows of 1024) for its default SpMV; the sort is a
 *     symmetric permutation of the basis that te_evolve and te_spmv undo.
 */
#ifndef TE_H_
#define TE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t te_status;
#define TE_OK                  0
#define TE_PENDING             1   /* te_poll: request not finished yet */
#define TE_ERR_INVALID_ARG    -1   /* bad size, index out of range, bad option */
#define TE_ERR_CUDA           -2   /* a CUDA runtime call failed (message has the CUDA error) */
#define TE_ERR_OOM            -3   /* device or host allocation failed */
#define TE_ERR_NOT_HERMITIAN  -4   /* TE_CHECK_HERMITIAN found H[i,j] != conj(H[j,i]) */
#define TE_ERR_NOT_NORMALIZED -5   /* | ||v_in|| - 1 | > 1e-10 (Sec. 2.1 assumes ||v(0)|| = 1) */
#define TE_ERR_STEP_UNDERFLOW -6   /* no step >= min_step_rel*|t| meets the error rate (e.g. m = 1) */
#define TE_ERR_NONFINITE      -7   /* NaN or Inf in the input vector or in H */
#define TE_ERR_TIMEOUT        -8   /* a bounded wait gave up (scheduler, device waits) */
#define TE_ERR_CANCELLED      -9   /* request cancelled by te_cancel */
#define TE_ERR_UNSUPPORTED   -10   /* valid request outside this build's limits (nnz >= 2^31, m > TE_M_MAX) */
#define TE_ERR_INTERNAL      -11   /* eigensolver did not converge or another internal check failed */

/* flags for pointer arguments and builders */
#define TE_PTR_DEVICE        0x1u  /* pointer arguments are device pointers */
#define TE_CHECK_HERMITIAN   0x2u  /* te_build_csr: verify H == H^dagger (relative 1e-13 of max |H_ij|) */
#define TE_INPUT_IS_CSR      0x4u  /* te_build_csr: rows is a row pointer array of length d+1 */

/* te_stats.flags */
#define TE_WARN_ROUNDOFF     0x1u  /* d ||H||_1 eps exceeded a step's error integral (eq. numericalError, Sec. 2.4) */
#define TE_WARN_QUAD         0x2u  /* an error integral did not reach quad_rel_tol within quad_max_levels (Sec. 4) */
#define TE_FLAG_BREAKDOWN    0x4u  /* a lucky breakdown ended a Krylov space early (Sec. 2.4 step 1) */
#define TE_FLAG_FUSED_RETRY  0x8u  /* a grid barrier of the fused Lanczos loop gave up; that restart
                                      and the rest of the solve ran as separate launches */

#define TE_M_MAX 128               /* largest Krylov dimension m */

/* te_options.quad */
#define TE_QUAD_TANH_SINH 0        /* adaptive double-exponential rule (default, Sec. 2.3) */
#define TE_QUAD_GAUSS     1        /* non-adaptive Gauss-Legendre, gauss_n nodes (Sec. 4) */
/* te_options.reorth */
#define TE_REORTH_NONE 0           /* three-term recurrence of eq. arnoldi (default) */
#define TE_REORTH_FULL 1           /* also classical Gram-Schmidt twice against all earlier vectors */
/* te_options.small_exp: how exp(-i H_m tau) e_1 and the error integrand are evaluated */
#define TE_SMALLEXP_CHEB 0         /* Chebyshev/Bessel (Jacobi-Anger) series of the tridiagonal H_m (default) */
#define TE_SMALLEXP_EIG  1         /* diagonalisation of H_m, the paper's choice (Sec. 2.4) */
/* te_options.fused_lanczos */
#define TE_FUSED_AUTO 0            /* small matrices (d <= 1024 x SMs, 155,648 on GB300) run the m
                                      Lanczos steps of a restart as one cooperative kernel (default) */
#define TE_FUSED_OFF  1            /* always one launch per product and per orthogonalisation */
/* te_options.flags */
#define TE_OPT_TEST_FUSED_TIMEOUT 0x20u   /* test aid: one block of the first fused Lanczos loop
                                           leaves before its first grid barrier, so the others'
                                           bounded wait (1 s) runs out and the retry path runs */
#define TE_OPT_PROFILE 0x10u       /* time the fused SpMV of Lanczos step m/2 of every restart with
                                      CUDA events (te_stats.spmv_*; one event pair per restart; with
                                      a fused Lanczos loop the pair brackets that whole kernel) */

/*
 * Solver options.  te_default_options fills the defaults, which follow the
 * paper: first step guess 0.1 and a 0.97 shrink of the previous step
 * (Algorithm 1), tanh-sinh with relative tolerance 1e-3 and at most 15
 * refinements (Sec. 4).  n_substeps (the paper's N_SUBSTEPS) is 10.
 */
typedef struct te_options {
    int32_t  quad;             /* TE_QUAD_TANH_SINH or TE_QUAD_GAUSS */
    int32_t  gauss_n;          /* Gauss nodes per interval, 2..64 (default 20) */
    int32_t  n_substeps;       /* growth substeps per step, >= 1 (default 10) */
    int32_t  reorth;           /* TE_REORTH_NONE or TE_REORTH_FULL */
    double   t_step0;          /* first step guess (default 0.1) */
    double   shrink;           /* factor on the previous step, in (0,1] (default 0.97) */
    double   quad_rel_tol;     /* tanh-sinh stop: |I_k - I_{k-1}| <= tol |I_k| (default 1e-3) */
    int32_t  quad_max_levels;  /* tanh-sinh refinements, 3..20 (default 15) */
    int32_t  max_substeps;     /* cap on growth substeps per step (default 1000) */
    double   min_step_rel;     /* underflow when a step falls below this * |t| (default 1e-13) */
    uint32_t flags;            /* TE_PTR_DEVICE for v_in / v_out; TE_OPT_PROFILE */
    int32_t  spmv_lanes;       /* 0: sliced-ELLPACK SpMV, one lane per row (default);
                                  1..32 (power of 2): CSR SpMV with that many lanes per row */
    int32_t  small_exp;        /* TE_SMALLEXP_CHEB (default) or TE_SMALLEXP_EIG */
    int32_t  fused_lanczos;    /* TE_FUSED_AUTO (default) or TE_FUSED_OFF.  The fused loop applies
                                  to the sliced SpMV (spmv_lanes 0) without reorthogonalisation;
                                  it computes the same steps, summing alpha and beta in another
                                  order */
} te_options;

/* Per-solve report.  err_bound is the sum of the accepted step errors (the
 * a-posteriori bound on ||v_out - exp(-iHt)v_in|| up to roundoff and the
 * quadrature tolerance).  roundoff_est = restarts x d ||H||_1 2^-52: the estimate of
 * eq. numericalError, once per restart (compared with that restart's error integral). */
typedef struct te_stats {
    int64_t  restarts;         /* Krylov spaces built */
    int64_t  matvecs;          /* products H v */
    int64_t  breakdowns;       /* lucky breakdowns */
    int64_t  quad_warnings;    /* integrals stopped by quad_max_levels */
    double   err_bound;
    double   roundoff_est;
    double   t_reached;        /* signed time reached (t unless an error stopped the solve) */
    double   norm_in;          /* ||v_in|| */
    uint32_t flags;            /* TE_WARN_*, TE_FLAG_* */
    int32_t  m_used;           /* Krylov dimension used (min(m, d)) */
    double   spmv_ms;          /* TE_OPT_PROFILE: summed CUDA-event time of the timed SpMV launches */
    int64_t  spmv_launches;    /* TE_OPT_PROFILE: launches summed in spmv_ms (one per restart) */
    double   solve_ms;         /* host wall time of the call */
    int64_t  quad_integrals;   /* error integrals evaluated by the step search */
    int64_t  quad_nodes;       /* integrand evaluations in those integrals */
    double   eig_mcycles;      /* 1e6 SM cycles spent diagonalising H_m (all restarts) */
    double   search_mcycles;   /* 1e6 SM cycles spent in the step search and omega */
    int64_t  fused_restarts;   /* restarts whose Lanczos loop ran as one cooperative kernel */
} te_stats;

typedef struct te_matrix_info {
    int64_t d;                 /* dimension */
    int64_t nnz;               /* stored entries */
    double  norm1;             /* ||H||_1 = max absolute column sum (= max row sum for Hermitian H) */
    int32_t max_row_nnz;
    int32_t spmv_lanes;        /* lanes per row the CSR kernel would use for this matrix */
    int64_t sell_nnz;          /* entries of the sliced-ELLPACK copy, padding included */
    int32_t sell_dict;         /* distinct off-diagonal values of a value-indexed copy (column +
                                  16-bit table index per entry, real diagonal apart); 0 when the
                                  copy stores full values (complex diagonal or > 65535 values) */
    int32_t sell_tpt;          /* slices (of 32 rows) per work item of the sliced SpMV */
    int32_t sell_real;         /* 1 when the value table is real (every off-diagonal value has a
                                  zero imaginary part): the product then takes 2 DFMA per entry
                                  instead of 3 */
    int32_t sell_async;        /* complex value table: 0 when the product gathers x through
                                  registers one slice at a time; 1 when it takes two slices per
                                  pass; 2 or 4 when it stages the gathers of the next trip of
                                  that many entries in shared memory (cp.async); chosen by
                                  te_matrix_tune, bitwise the same result */
} te_matrix_info;

/* Synthetic model Hamiltonians built on the device (Sec. 3: the matrix of an
 * operator expression in a number-state basis).  Parameter arrays are host
 * pointers, read during the call. */
#define TE_MODEL_TFIM  1  /* H = -sum_{b<L-1} a[b] Z_b Z_{b+1} - sum_i b[i] X_i, open chain, d = 2^L */
#define TE_MODEL_XXZDM 2  /* H = sum_b [1/2 (e^{i phi_b} S+_b S-_{b+1} + h.c.) + delta Sz_b Sz_{b+1}]
                             + sum_i c[i] Sz_i; e^{i phi_b} = a[b] + i b[b]; pbc -> L bonds, else L-1 */
#define TE_MODEL_BOSE  3  /* H = sum_{i!=j} c_ij a_i^+ a_j + sum_i c[i] n_i^2 on K = L modes with N bosons;
                             c_ij = a[p] + i b[p] for i<j, p in (i-major, j-minor) order, c_ji = conj(c_ij) */
#define TE_MODEL_MEMORY 4 /* the paper's example system (Sec. 5, eq. fullHamiltonianSimple):
                             C0 (a0^+ b0 + h.c.) + em (1 - n0/Nc) sum_{k<=K} n_k
                             + em (1 - n0/(Nc - dNc)) sum_{k'} n'_k'
                             + Cm sum_{p<q} f(p,q) (a_p^+ a_q + h.c.) over all K + K' qubits;
                             L = K, L2 = K', N = Nm excitations, N2 = N0 bosons in a_0, b_0;
                             a = f(p,q) for p < q in (p-major, q-minor) order;
                             p = {Nc, dNc, em, C0, Cm}.  Real symmetric. */
typedef struct te_model_desc {
    int32_t model;             /* TE_MODEL_* */
    int32_t L;                 /* spins (chains, 3..30) or modes K (bosons, 2..16) */
    int32_t N;                 /* bosons: particles, 1..15 */
    int32_t pbc;               /* XXZ-DM: 1 periodic (needs L >= 3), 0 open */
    double  delta;             /* XXZ-DM anisotropy */
    const double* a;           /* see the model comments */
    const double* b;
    const double* c;
    int32_t L2;                /* TE_MODEL_MEMORY: K' */
    int32_t N2;                /* TE_MODEL_MEMORY: N0 */
    const double* p;           /* TE_MODEL_MEMORY: {Nc, dNc, em, C0, Cm} */
} te_model_desc;
/* Basis conventions: spin chains use index bit i = 1 for spin i down
 * (sigma^z_i = -1).  Bosonic states are occupation tuples (n_0..n_{K-1}) with
 * sum N, indexed in descending lexicographic order from (N,0,...,0); on the
 * device the tuple -> index map is a hash table (Sec. 4). */

typedef struct te_ctx te_ctx;
typedef struct te_matrix te_matrix;
typedef struct te_request te_request;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * owned by the caller (NULL: the context creates and owns a non-blocking
 * stream).  The context owns its device workspace (Krylov bases, reduction
 * scratch, captured CUDA graphs) and frees it in te_destroy. */
te_status te_create(te_ctx** out, int32_t device, void* cuda_stream);

/* A caller-supplied allocator for the library's device memory.  Sec. 2.1 of the
 * paper states the problem as (H, v, t, err_max, m) and says nothing about where
 * the solver's memory comes from; this hook lets a caller that owns device
 * memory through its own pool (a framework's caching allocator, a service with
 * a fixed budget) supply every device buffer the library uses: the CSR arrays
 * and sliced copies of its matrices, the Krylov bases and solver state of its
 * plans (the (m+1) d complex128 basis is the large one: 2.75 GB at d = 2^22,
 * m = 40), the buffers of asynchronous requests and the temporaries of the
 * builders.  Pinned host memory for the per-restart state copies still comes
 * from cudaMallocHost, and te_spmv_noalloc's fixed scratch is not allocated.
 *   alloc(user, bytes, device, stream): return `bytes` bytes of device memory
 *     on `device`, aligned to at least 256 bytes, or NULL (the calling function
 *     then fails with TE_ERR_OOM).  `stream` is the context's stream, on which
 *     the library orders its work (requests run on per-worker streams and
 *     synchronise them before their memory is released).
 *   free(user, ptr, device, stream): release a pointer that alloc returned.  The
 *     library synchronises the context's stream before every free, and frees
 *     only memory whose work has finished, so a pool may reuse it at once.
 * Both may be called from the calling thread and from the request scheduler's
 * worker threads (te_submit), never concurrently for the same pointer.  A
 * matrix or plan keeps using the allocator of the context that made it; free
 * matrices and requests before destroying their context. */
typedef struct te_allocator {
    void* (*alloc)(void* user, size_t bytes, int32_t device, void* stream);
    void (*free)(void* user, void* ptr, int32_t device, void* stream);
    void* user;
} te_allocator;

/* te_create with a caller-supplied device allocator (NULL, or alloc == NULL:
 * cudaMalloc / cudaFree as in te_create).  alloc and free must both be set or
 * both be NULL (else TE_ERR_INVALID_ARG).  The allocator is copied. */
te_status te_create_with_allocator(te_ctx** out, int32_t device, void* cuda_stream,
                                   const te_allocator* allocator);
void te_destroy(te_ctx* ctx);
const char* te_last_error(const te_ctx* ctx);
const char* te_status_string(te_status s);
void te_default_options(te_options* opt);
/* Version string of the library (static storage). */
const char* te_version(void);

/* ---- matrices ----------------------------------------------------------- */

/* Build H from COO triplets (row, col, value) -- or, with TE_INPUT_IS_CSR,
 * from CSR arrays where rows[0..d] is the row pointer and n_entries = rows[d].
 * Entries are ordered by (row, col); duplicates are added in input order;
 * explicit zeros are kept.  vals holds 2*n_entries doubles (re, im).
 * Errors: TE_ERR_INVALID_ARG (d < 1, an index outside [0, d), a non-monotone
 * row pointer), TE_ERR_NONFINITE, TE_ERR_NOT_HERMITIAN (with TE_CHECK_HERMITIAN),
 * TE_ERR_UNSUPPORTED (nnz >= 2^31 or d >= 2^31), TE_ERR_OOM.
 * The library owns the result; release it with te_matrix_free. */
te_status te_build_csr(te_ctx* ctx, int64_t d, int64_t n_entries, const int64_t* rows,
                       const int64_t* cols, const double* vals, uint32_t flags,
                       te_matrix** out);

/* Build a model Hamiltonian on the device (see TE_MODEL_*).  Rows hold ascending
 * columns with the diagonal always stored.  Errors: TE_ERR_INVALID_ARG,
 * TE_ERR_UNSUPPORTED (size limits), TE_ERR_OOM. */
te_status te_build_model(te_ctx* ctx, const te_model_desc* desc, te_matrix** out);

/* Index of an occupation tuple in a model basis (host-side ranking;
 * TE_ERR_INVALID_ARG if the tuple is not in the basis): TE_MODEL_BOSE takes
 * occ[0..K-1]; TE_MODEL_MEMORY takes (n0, m0, q_1..q_{K+K'}), its basis ordered
 * descending lexicographically (index = (N0 - n0) C(K+K', Nm) + rank of the
 * qubit tuple). */
te_status te_model_basis_index(const te_model_desc* desc, const int32_t* occ, int64_t* index);

te_status te_matrix_info_get(const te_matrix* H, te_matrix_info* info);

/* Copy the CSR arrays out: rowptr[d+1], col[nnz] (int32), val[2*nnz]
 * (host buffers, or device buffers with TE_PTR_DEVICE).  Any pointer may be
 * NULL to skip that array. */
te_status te_matrix_export(te_ctx* ctx, const te_matrix* H, int32_t* rowptr, int32_t* col,
                           double* val, uint32_t flags);

/* Free a matrix (and any cached solver plans built for it). */
void te_matrix_free(te_matrix* H);

/* Autotune the sliced SpMV of H on this GPU: times the product (CUDA events, the
 * best of `repeats` launches after one warm-up) for work items of 1, 2, 3, 4, 6 and
 * 8 slices, and for a complex value table also with two slices per pass and with
 * the gathers staged in shared memory two or four entries ahead, and keeps the
 * fastest (another form than the register-gather one only when it is at least 1 %
 * faster) (te_matrix_info.sell_tpt,
 * sell_async; every candidate gives bitwise the same product).  The initial choice
 * is a fixed rule (about 1.5K stored entries per item, at most 4 slices).  Cached
 * solver plans of H are dropped (their scratch depends on the item size); returns
 * TE_ERR_INVALID_ARG while a solve on H is running.  best_ms (may be NULL)
 * receives the fastest product time.  repeats: 1..100. */
te_status te_matrix_tune(te_ctx* ctx, te_matrix* H, int32_t repeats, double* best_ms);

/* Pin the sliced SpMV configuration that te_matrix_tune would choose:
 * slices_per_task 1..8, async_trip 0 (gathers through registers), 1 (two slices
 * per pass) or 2 / 4 (gathers staged in shared memory that many entries ahead);
 * 1, 2 and 4 exist for the complex value table only.
 * Every configuration gives bitwise the same product.  Cached plans of H are
 * dropped.  Errors: TE_ERR_INVALID_ARG (bad value, no sliced copy, staging asked
 * for another form, a solve on H running). */
te_status te_matrix_set_sell(te_ctx* ctx, te_matrix* H, int32_t slices_per_task, int32_t async_trip);

/* ---- measurement -------------------------------------------------------- */

/* The FP64 fused multiply-add rate the context's GPU sustains, in TFLOP/s
 * (2 FLOP per FMA), measured on independent FMA chains with no memory traffic:
 * the attainable ceiling of the solve's FP64-bound products (the SpMV of
 * Sec. 2.1, the orthogonalisation and the recombination of Algorithm 1).  Runs
 * for about 0.1 s on the context's stream after the caller's queued work,
 * allocates and frees a 1 MB scratch, and returns when the result is in
 * *tflops (host pointer).  Errors: TE_ERR_INVALID_ARG (NULL argument),
 * TE_ERR_CUDA. */
te_status te_measure_fp64(te_ctx* ctx, double* tflops);

/* The FP64 rate of the GPU's FP64 matrix instruction (mma.sync m8n8k4 on .f64
 * operands, 256 multiply-adds per warp instruction), in TFLOP/s, on independent
 * accumulator tiles with no memory traffic.  The paper has no counterpart: it
 * is the measurement that decides whether the recombination w = V_m omega or the
 * orthogonalisation of Algorithm 1, written as small dense products, could run
 * faster on it than on the FP64 vector pipe (te_measure_fp64).  Runs for about
 * 0.2 s on the context's stream after the caller's queued work, allocates and
 * frees a 1 MB scratch.  Errors: TE_ERR_INVALID_ARG (NULL argument), TE_ERR_CUDA. */
te_status te_measure_fp64_mma(te_ctx* ctx, double* tflops);

/* The grid barrier of the fused Lanczos loop (te_options.fused_lanczos), run
 * once over a cooperative grid of one 32-thread block per SM.  The paper has no
 * counterpart: this exists so that tests can see that the barrier's bounded
 * wait ends a wait that cannot complete with an error instead of a hang.
 * absent_block < 0: every block arrives; the call returns TE_OK with *passed =
 * the number of blocks.  absent_block = b (0 <= b < SMs): block b leaves without
 * arriving; the others give up after about one second, *passed = 0 and the call
 * returns TE_ERR_TIMEOUT, the status a solve reports when this happens inside
 * its fused loop.  *ms (host pointer or NULL) receives the kernel's time.  Runs
 * on the context's stream after the caller's queued work; allocates and frees
 * 16 bytes.  Errors: TE_ERR_INVALID_ARG, TE_ERR_UNSUPPORTED (no cooperative
 * launches), TE_ERR_CUDA. */
te_status te_fused_barrier_check(te_ctx* ctx, int32_t absent_block, int32_t* passed, double* ms);

/* ---- products and solves ------------------------------------------------ */

/* y = H x (Sec. 2.1: the sparse product that dominates each Lanczos step).
 * x, y: complex128 vectors of length d, distinct buffers.  If x_dot_y is not
 * NULL it receives Re <x, H x> (the energy of x).  Flags: TE_PTR_DEVICE. */
te_status te_spmv(te_ctx* ctx, const te_matrix* H, const double* x, double* y,
                  double* x_dot_y, uint32_t flags);

/* Largest dimension accepted by te_spmv_noalloc. */
#define TE_NOALLOC_MAX_D 8388608

/* y = H x and Re <x, H x>, like te_spmv, but without allocating anything.
 * The paper has no counterpart: this exists for callers that cannot allocate
 * device memory at the moment they need the product -- code whose framework
 * owns all device memory through its own pool (a stray cudaMalloc can fail or
 * fragment it), services that must keep their device footprint fixed once
 * started, and latency-critical loops that cannot afford cudaMalloc or the
 * device-wide synchronisation implied by cudaFree.  te_spmv, by contrast,
 * allocates staging buffers for host vectors.
 *   x, y: device pointers (flags must contain TE_PTR_DEVICE), distinct,
 *         complex128, length d; x_dot_y: host pointer or NULL.
 *   d must not exceed TE_NOALLOC_MAX_D (else TE_ERR_UNSUPPORTED, nothing runs).
 * The reduction scratch is a fixed device array inside libte (about 64 KB),
 * which every GPU that loads the library keeps until the process exits.  The
 * first call on a device is a set-up step: it looks up that array's device
 * address, and under CUDA's lazy module loading (the default) it is also when
 * the array and the kernel are loaded onto the device, which the driver may
 * allocate for.  Later calls allocate nothing.  So make the first call on each
 * device before any stream capture begins and before the caller's device
 * footprint must stay fixed.  All calls on a device share the array and it keeps the last
 * call's contents: the library clears the part that must start at zero on every
 * call, but calls that overlap on the GPU (from other streams or other host
 * threads) race on it and must be serialised by the caller.  The call waits
 * for the caller's stream, runs on the context's stream and returns when done. */
te_status te_spmv_noalloc(te_ctx* ctx, const te_matrix* H, const double* x, double* y,
                          double* x_dot_y, uint32_t flags);

/* v_out = exp(-i H t) v_in to within err_max = tol (Algorithm 1).
 * v_in must be normalised to 1e-10 (Sec. 2.1).  t < 0 evolves with -H for |t|
 * (the reversal of Sec. 5); t = 0 copies v_in.  m is the Krylov dimension,
 * 1 <= m <= TE_M_MAX, clamped to d.  tol > 0.  opt may be NULL (defaults);
 * opt->flags & TE_PTR_DEVICE says whether v_in / v_out are device pointers.
 * v_in and v_out may be the same buffer.  st may be NULL.
 * Errors: TE_ERR_INVALID_ARG, TE_ERR_NOT_NORMALIZED, TE_ERR_NONFINITE,
 * TE_ERR_STEP_UNDERFLOW (v_out then holds the state at st->t_reached),
 * TE_ERR_UNSUPPORTED (also: after a lucky breakdown, which takes the whole
 * remaining time in one step, the default Chebyshev small exponential splits
 * that step into pieces of a ||H_m|| tau <= 2048 and accepts at most 512 of
 * them; TE_SMALLEXP_EIG has no such limit), TE_ERR_INTERNAL, TE_ERR_CUDA,
 * TE_ERR_OOM. */
te_status te_evolve(te_ctx* ctx, const te_matrix* H, const double* v_in, double t, double tol,
                    int32_t m, const te_options* opt, double* v_out, te_stats* st);

/* ---- operator expressions (Sec. 3) ---------------------------------------- */

/* A Hermitian operator written in creation / annihilation operators of L modes
 * (Sec. 3), on the basis of all occupation tuples (n_1..n_L) with sum N
 * (eq. totalOccupationNumber) and n_l <= max_occ[l] (the fixed maximal
 * occupations of Sec. 4; max_occ = NULL: no cap), ordered descending
 * lexicographically.  The operator is sum_t coef_t * O_{t,1} ... O_{t,k_t} with
 * each O a_l (annihilation) or a_l^dagger (creation), applied right to left:
 * a_l |n> = sqrt(n_l) |n - 1_l>, a_l^dagger |n> = sqrt(n_l + 1) |n + 1_l>; a
 * result outside the basis (a cap exceeded, the total changed) contributes
 * nothing.  The caller must pass the terms of a Hermitian operator (each
 * non-Hermitian term together with its adjoint). */
typedef struct te_operator_desc {
    int32_t n_modes;            /* L, 1..32 */
    int32_t n_particles;        /* N, 0..64 */
    const int32_t* max_occ;     /* NULL or L maximal occupations */
    int32_t n_terms;            /* 0..4096 */
    const int32_t* term_len;    /* n_terms: ladder operators in each term, 0..8 (0: coef * identity) */
    const int32_t* modes;       /* sum of term_len: the mode of each operator, left to right */
    const int32_t* dagger;      /* sum of term_len: 1 creation, 0 annihilation */
    const double* coef;         /* 2 n_terms: (re, im) of each term's coefficient */
} te_operator_desc;

/* createMatrix (Sec. 3) on the device: H[j][i] = <j|H|i>, built row by row from
 * the terms applied to basis state j; contributions to one entry are added in
 * term order; every diagonal entry is stored; columns ascending.  The index map
 * (ind of eq. findIndices) is the rank in the basis order above, computed
 * combinatorially instead of with a hash table.  Host arrays, read during the
 * call.  Errors: TE_ERR_INVALID_ARG (sizes, modes, flags), TE_ERR_NONFINITE,
 * TE_ERR_UNSUPPORTED (d >= 2^31, a row with more than 256 contributions),
 * TE_ERR_OOM, TE_ERR_CUDA. */
te_status te_build_operator(te_ctx* ctx, const te_operator_desc* op, te_matrix** out);
/* Basis index of an occupation tuple (L int32) of the operator's basis. */
te_status te_operator_basis_index(const te_operator_desc* op, const int32_t* occ, int64_t* index);
/* Number operator of one mode over the operator's basis (as te_model_occupation). */
te_status te_operator_occupation(te_ctx* ctx, const te_operator_desc* op, int32_t mode,
                                 double* out, uint32_t flags);

/* v_out = exp(-i H t) v_in as te_evolve, plus the states at intermediate times
 * (the extension remarked in Sec. 2.4: inside a step, the restart's H_m and V_m
 * give the state at any time the step covers, so sampling costs no extra
 * restarts) and diagonal observables of those states.
 *   t_samples: n_samples >= 1 host doubles with the sign of t (or 0), |s| <= |t|,
 *     non-decreasing |s|.  A sample is evaluated in the first restart whose step
 *     reaches it.
 *   v_samples: NULL or n_samples complex128 vectors of length d one after another
 *     (device if opt->flags has TE_PTR_DEVICE, else host).
 *   obs: NULL or n_obs real diagonal observables of length d one after another
 *     (O_l[i] = <i|O_l|i>, same pointer kind as v_in); obs_out: host,
 *     n_samples x n_obs doubles, obs_out[s n_obs + l] = sum_i O_l[i] |v_s[i]|^2.
 *   sample_bounds: NULL or n_samples host doubles: the error bound accumulated
 *     through the step that produced each sample (eq. errorIntegral; it also
 *     covers the sample, whose integral is a part of the step's).
 *   v_out must not be NULL; opt->spmv_lanes must be 0.
 * Device memory: that of te_evolve plus n_samples d 16 bytes (the samples) and,
 * with observables, n_obs d 8 bytes.  Errors as te_evolve; samples the solve did
 * not reach are left at zero. */
te_status te_evolve_sampled(te_ctx* ctx, const te_matrix* H, const double* v_in, double t,
                            int32_t n_samples, const double* t_samples, double tol, int32_t m,
                            const te_options* opt, double* v_out, double* v_samples, int32_t n_obs,
                            const double* obs, double* obs_out, double* sample_bounds,
                            te_stats* st);

/* Number operator of one mode as a diagonal over the model's basis:
 * out[i] = <i| n_mode |i> for every basis index i (out: d doubles, device if
 * flags has TE_PTR_DEVICE, else host).  Spin chains: mode l is site l, n_l = 1
 * when spin l points down (bit l of the index).  Bosons: occupation of mode l.
 * The paper's example system (Sec. 5): mode 0 = a_0, mode 1 = b_0, modes 2.. =
 * the qubits a_1..a_K, a'_1..a'_K' -- the observables whose expectation values
 * the paper plots over time.  Errors: TE_ERR_INVALID_ARG (unknown model, mode
 * out of range), TE_ERR_CUDA, TE_ERR_OOM. */
te_status te_model_occupation(te_ctx* ctx, const te_model_desc* desc, int32_t mode, double* out,
                              uint32_t flags);

/* Largest number of vectors in one block product of te_evolve_batch; larger
 * batches run in consecutive groups of this size. */
#define TE_BATCH_MAX 64

/* nvec solves v_out[b] = exp(-i H t) v_in[b] under one H, each to within
 * err_max = tol (Algorithm 1 applied to every vector; the paper solves one
 * vector at a time and has no batched form).  The vectors keep separate Krylov
 * spaces, step sizes, breakdowns and restart counts; what they share is the
 * product with H, done as one block product per Lanczos step for up to
 * TE_BATCH_MAX vectors.
 *   v_in, v_out: nvec complex128 vectors of length d stored one after another
 *     (vector b at offset 2 b d doubles); device pointers if opt->flags has
 *     TE_PTR_DEVICE, else host; they may be the same buffer.
 *   t, tol, m, opt: as for te_evolve, shared by all vectors (opt->reorth must be
 *     TE_REORTH_NONE; spmv_lanes is ignored).  TE_OPT_PROFILE times the block
 *     products (spmv_ms is then the group's total, repeated in its vectors).
 *   st: NULL or nvec entries; status: NULL or nvec entries, each vector's own
 *     te_status (a failed vector does not stop the others).
 * Returns TE_OK when every vector succeeded, else the first vector's error, or
 * a call-level error (TE_ERR_INVALID_ARG, TE_ERR_UNSUPPORTED, TE_ERR_CUDA,
 * TE_ERR_OOM).  Device memory: (m + 1) d B 16 bytes plus d B 8 bytes for the
 * group width B (nvec rounded up to a power of two, at most TE_BATCH_MAX), and
 * 24 bytes per stored entry of H for a cached copy of its values. */
te_status te_evolve_batch(te_ctx* ctx, const te_matrix* H, int32_t nvec, const double* v_in,
                          double t, double tol, int32_t m, const te_options* opt, double* v_out,
                          te_stats* st, int32_t* status);

/* Largest number of problems advanced together by te_evolve_multi; more run in
 * consecutive groups of this size. */
#define TE_MULTI_MAX 256

/* n independent solves v_out[i] = exp(-i H[i] t[i]) v_in[i], each to within
 * err_max = tol (Algorithm 1 for every problem; the paper solves one problem at
 * a time and has no grouped form).  The problems may have different H (of any
 * dimension), v and t, and keep separate Krylov spaces, steps and restart
 * counts; what they share is the launches: each Lanczos step of all running
 * problems is one grouped kernel launch, and the restarts run as rounds of one
 * captured CUDA graph, so small problems do not pay a launch latency per step.
 *   H: n matrices of this context (the same matrix may appear several times);
 *   v_in, v_out: n complex128 vectors, v_in[i] / v_out[i] of length H[i]'s d;
 *     device pointers if opt->flags has TE_PTR_DEVICE, else host;
 *   t: n times (t = 0 returns v_in after checking its norm; t < 0 evolves with -H);
 *   tol, m, opt: shared; m is clamped to each problem's d; opt->reorth must be
 *     TE_REORTH_NONE; TE_OPT_PROFILE times the grouped SpMV launches (spmv_ms
 *     is then the group's total, repeated in its problems);
 *   st, status: NULL or n entries (per-problem statistics and te_status; a
 *     failed problem does not stop the others).
 * Returns TE_OK when every problem succeeded, else the first problem's error, or
 * a call-level error (TE_ERR_INVALID_ARG, TE_ERR_UNSUPPORTED, TE_ERR_CUDA,
 * TE_ERR_OOM).  Device memory: (m + 1) D 16 + D 8 bytes, D = sum of the
 * dimensions rounded up to multiples of 32. */
te_status te_evolve_multi(te_ctx* ctx, int32_t n, const te_matrix* const* H,
                          const double* const* v_in, const double* t, double tol, int32_t m,
                          const te_options* opt, double* const* v_out, te_stats* st,
                          int32_t* status);

/* ---- asynchronous requests --------------------------------------------- */

/* Queue a solve with the same meaning as te_evolve.  v_in is copied before the
 * call returns.  H must outlive the request.  How requests are served
 * (te_serve_config):
 *   TE_SERVE_BATCH (default): continuous batching.  Two serving loops per
 *     context (small requests, H with fewer than 2^21 stored entries, and
 *     medium ones, each on a stream of its own) keep the Krylov state of every
 *     running request on the device in an arena of slots and advance all of
 *     them together, one restart of Algorithm 1 per round, through the grouped
 *     kernels of te_evolve_multi (every Lanczos step of all running requests of
 *     a loop is one launch), so small requests go round in short rounds.  The restart
 *     boundary is the checkpoint: a queued request is admitted, in arrival
 *     order, at the next round boundary as soon as a slot of its size
 *     ((d rounded up to 32) elements of the arena) is free, and a finished
 *     request leaves at the end of its round.  The result equals te_evolve's
 *     within the same error bound (the same steps, reductions summed in another
 *     order).  Requests whose H holds at least the large-lane threshold of
 *     stored entries (default 2^24; one restart of such a request fills the
 *     GPU by itself) run in the large lane instead: one at a time, first come
 *     first served, as a solo solve on its own stream beside the batches (stream
 *     priorities: small batch highest, large lane next, medium batch lowest), so
 *     that large requests neither slow each other down nor wait behind small ones.
 *     The large lane's sparse products and the medium batch's run one block per
 *     SM below full occupancy, leaving the small batch room to start at once.  A
 *     large request is reported finished before the next one starts.  Requests
 *     with reorthogonalisation, the CSR kernel (spmv_lanes),
 *     TE_OPT_PROFILE, m above the arena depth or d above its capacity take
 *     the large lane too.
 *   TE_SERVE_SOLO: up to 8 worker threads each admit the oldest queued request
 *     once its device footprint ((m+1) d 16 bytes plus reduction scratch)
 *     fits the context's memory budget, and run it on their own stream, one
 *     restart graph at a time. */
te_status te_submit(te_ctx* ctx, const te_matrix* H, const double* v_in, double t, double tol,
                    int32_t m, const te_options* opt, te_request** out);
/* TE_PENDING while queued or running; otherwise the solve's status, with the
 * result copied to v_out (host unless the submit options had TE_PTR_DEVICE) and
 * stats to st (either may be NULL). */
te_status te_poll(te_request* req, double* v_out, te_stats* st);
/* Wait up to timeout_ms (< 0: no limit) for the request; returns as te_poll,
 * TE_PENDING on timeout. */
te_status te_wait(te_request* req, double timeout_ms, double* v_out, te_stats* st);
/* Ask the scheduler to stop the request at its next restart boundary. */
te_status te_cancel(te_request* req);
/* Free a finished request (waits for it if it is still running). */
void te_request_free(te_request* req);
/* Bytes of device memory the scheduler may hold for running requests
 * (default: 80% of the free memory at te_create). */
te_status te_set_memory_budget(te_ctx* ctx, int64_t bytes);

#define TE_SERVE_BATCH 0           /* continuous batching of requests (default) */
#define TE_SERVE_SOLO  1           /* one solve per worker thread and stream */
/* How te_submit serves requests.  m_max is the Krylov depth of the serving
 * arena (1..TE_M_MAX; 0: keep, default 40), capacity the number of vector
 * elements per Krylov column it holds (0: keep; default
 * min(2^24, budget / (16 (m_max + 1) + 8)) at first use) in the medium batch's
 * arena (the small batch's holds a quarter of it), large_nnz the large-lane
 * threshold on the stored entries of H (0: keep, default 2^24; negative: no large
 * lane) and small_nnz the small batch's (0: keep, default 2^21; negative: one
 * batch for everything below the large lane).  Each arena takes
 * (m_max + 1) capacity 16 + capacity 8 bytes once its first request arrives,
 * counts against the memory budget, and is released by te_destroy.
 * Allowed only while no request is queued or running (else
 * TE_ERR_INVALID_ARG). */
te_status te_serve_config(te_ctx* ctx, int32_t mode, int32_t m_max, int64_t capacity,
                          int64_t large_nnz, int64_t small_nnz);

#ifdef __cplusplus
}
#endif
#endif /* TE_H_ */
