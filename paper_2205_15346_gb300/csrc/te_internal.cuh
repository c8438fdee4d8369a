// te_internal.cuh -- shared declarations of libte's translation units.
//
// Device-side solver state, matrix and plan objects, and the host launchers of
// the kernels.  Kernel numbering follows the restart cycle of Algorithm 1 of
// arXiv 2205.15346:
//   K0  k_init_norm      ||v_in||, validation (Sec. 2.1 assumes ||v(0)|| = 1)
//   K1  k_spmv_lanczos   y = s H u_j - beta_{j-1} v_{j-1}, partial Re<v_j, y>   (eq. arnoldi a-c)
//   K2  k_orth_norm      w~ = y - alpha_j v_j, ||w~||, breakdown test          (eq. arnoldi d-f)
//   KR  k_reorth_*       optional full Gram-Schmidt (not in the paper)
//   K3  k_step           eigen-decomposition of H_m, error integral, step size, omega
//                         (Sec. 2.4 step 2, eqs. errorIntegral, errorRate, stepSize)
//   K4  k_recombine      w = V_m omega, ||w||                                   (Algorithm 1 step 3)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "te.h"

#define TE_BLOCK 256                 // threads per block of the streaming kernels
#define TE_STEP_THREADS 256          // threads of the single-CTA step kernel
#define TE_GAUSS_MAX 64
#define TE_FUSED_SLICES_PER_WARP 4   // slices (of 32 rows) a warp of the fused Lanczos loop holds

// Solver state in device memory, one per plan.  Written by the kernels of a
// restart, read back by the host after each restart (a copy of the struct).
struct DevState {
    // constants of a solve (set by the host before the first restart)
    double T;                // |t|
    double tol_rate;         // err_max / |t|  (eq. errorRate)
    double sign;             // +1: H, -1: -H (negative t)
    double t_step0;
    double shrink;
    double quad_rel_tol;
    double min_step;         // min_step_rel * |t|
    int32_t m;               // Krylov dimension (clamped to d)
    int32_t n_substeps;
    int32_t quad;
    int32_t gauss_n;
    int32_t quad_max_levels;
    int32_t max_substeps;
    int32_t smallexp;        // TE_SMALLEXP_*
    int32_t test_hold;       // TE_OPT_TEST_FUSED_TIMEOUT: one block of the fused loop skips a barrier
    // progress of the solve
    double t_now;
    double prev_step;
    double err_acc;
    int32_t first;
    int32_t done;
    int32_t status;          // te_status of the solve (0 while fine)
    int32_t last_m_eff;      // Krylov size used by the last finished restart
    int64_t restarts;
    int64_t matvecs;
    int64_t breakdowns;
    int64_t quad_warnings;
    int64_t quad_integrals;  // error integrals evaluated
    int64_t quad_nodes;      // integrand evaluations
    int64_t eig_cycles;      // SM cycles in the eigensolver (K3, summed over restarts)
    int64_t search_cycles;   // SM cycles in the step search and omega (K3)
    // state of the current restart
    int32_t stop;            // inner Lanczos loop ended (breakdown)
    int32_t m_eff;
    int32_t breakdown;
    int32_t active;          // K3 took a step in this restart (batched recombination)
    double beta0;            // ||w|| at the start of the restart
    double as_cur;           // alpha_j * scale_j, handed from K1 to K2
    double spmv_dot;         // te_spmv: Re <x, H x>
    double last_step;
    double last_err;
    double min_err_step;     // smallest accepted step error (roundoff comparison)
    double win_t0, win_t1;   // |t| at the start and end of the last step taken
    int32_t win_last;        // that step reached |t|
    int32_t samp_next;       // first intermediate sample not yet evaluated
    int32_t samp_lo, samp_hi;    // samples of the current window
    double scale[TE_M_MAX + 1];   // v_j = scale[j] * u_j (stored vectors are unnormalised)
    double alpha[TE_M_MAX];       // diagonal of H_m
    double beta[TE_M_MAX];        // beta[j] = h_{j+2,j+1} (0-based j); h = beta[m_eff-1]
    double2 coef[TE_M_MAX];       // recombination coefficients beta0 * scale[k] * omega_k
    double2 rcoef[TE_M_MAX];      // reorthogonalisation coefficients
    double gx[TE_GAUSS_MAX];      // Gauss-Legendre nodes on [-1, 1]
    double gw[TE_GAUSS_MAX];
    unsigned int counter[8];      // last-block counters of the reductions
};

struct te_matrix {
    te_ctx* ctx;
    int64_t d;
    int64_t nnz;
    int32_t* rowptr;         // device, d + 1
    int32_t* col;            // device, nnz
    double2* val;            // device, nnz
    double norm1;
    int32_t max_row_nnz;
    int32_t lanes;           // lanes per row for the CSR SpMV variant
    uint64_t id;
    // sliced-ELLPACK copy in a length-sorted basis (te_sell.cu)
    int32_t* perm = nullptr;     // new index -> old row (padded to a multiple of 32)
    int32_t* iperm = nullptr;    // old row -> new index
    int32_t* sell_off = nullptr; // slice offsets, nslices + 1
    int32_t* sell_col = nullptr;
    double* sell_a = nullptr;    // full-value form: Re h per stored entry
    double2* sell_pq = nullptr;  // full-value form: (Im h - Re h, Re h + Im h) (3M product)
    uint16_t* sell_idx = nullptr;    // value-indexed form: table index per off-diagonal entry
    double* sell_diag = nullptr;     // value-indexed form: Re h_ii per permuted row
    double* dict_a = nullptr;        // value table (index 0 = 0): Re h
    double2* dict_pq = nullptr;      // value table: (Im h - Re h, Re h + Im h)
    int32_t dict_n = 0;              // distinct off-diagonal values (0: full-value form)
    bool dict_real = false;          // every off-diagonal value is real (2-DFMA product)
    int64_t nslices = 0;
    int64_t sell_nnz = 0;        // stored entries including padding
    int sell_grid = 0;           // blocks of the SpMV grid (resident on all SMs at once)
    int sell_tpt = 1;            // slices per SpMV task (about 1.5K stored entries)
    int sell_async = 0;          // complex value table: gathers staged in shared memory, 2 or 4
                                 // entries per trip (0: through registers); set by te_matrix_tune
    // 3M form for the batched product (te_block.cu), built on first use:
    // m3[k] = a, m3[nnz + k] = b - a, m3[2 nnz + k] = a + b for val[k] = a + ib
    double* m3 = nullptr;
};

// One solve's device workspace and captured restart graph.
struct Plan {
    te_ctx* ctx = nullptr;           // owner: its allocator holds the device memory below
    const te_matrix* H = nullptr;
    // intermediate-time sampling (te_sample.cu); such plans are built per call
    int ns = 0;                      // sample times
    double* samp_ts = nullptr;       // device: |t_s|, non-decreasing
    double2* samp_coef = nullptr;    // device: ns x m coefficients
    double2* samp_buf = nullptr;     // device: ns x d sampled states (permuted basis)
    double* samp_bound = nullptr;    // device: ns bounds
    uint64_t matrix_id = 0;
    int m = 0;
    int reorth = 0;
    int profile = 0;
    int lanes = 0;                   // 0: SELL kernel in the permuted basis; > 0: CSR kernel
    int64_t d = 0;
    double2* V = nullptr;            // (m + 1) columns of length d, column-major
    double* S = nullptr;             // Re + Im of the Lanczos vector the next SpMV reads (SELL)
    DevState* st = nullptr;          // device
    DevState* st_host = nullptr;     // pinned: written by the graph's last node
    DevState* st_init = nullptr;     // pinned: source of the per-solve initial state
    double* partials = nullptr;      // per-block reduction scratch
    double* partials_r = nullptr;    // reorthogonalisation scratch
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphExec_t exec_unfused = nullptr;   // fused plans: the same restart as separate launches
                                              // (run when the fused loop's barrier gave up)
    std::vector<cudaEvent_t> ev;     // TE_OPT_PROFILE: start/stop per Lanczos step
    size_t bytes = 0;
    bool in_use = false;
    int grid_k1 = 0, grid_stream = 0, grid_reorth = 0;
    // 1: the plan of a large request served beside the batches; its SpMV leaves one
    // block slot per SM free (grid_k1 one block per SM below full occupancy), so the
    // batches' kernels start without waiting for the SpMV's resident blocks to end
    int share = 0;
    // fused Lanczos loop (te_fused.cu): one cooperative kernel per restart
    int fused = 0;
    int fused_grid = 0, fused_threads = 0;
    unsigned int* bar = nullptr;     // its grid-barrier words
};

struct te_ctx;

struct te_request {
    te_ctx* ctx = nullptr;
    const te_matrix* H = nullptr;
    double* v_in_dev = nullptr;      // library-owned copy of v_in
    double* v_out_dev = nullptr;
    double t = 0, tol = 0;
    int32_t m = 0;
    te_options opt{};
    te_stats stats{};
    size_t footprint = 0;
    std::atomic<int> state{0};       // 0 queued, 1 running, 2 finished
    std::atomic<int> cancel{0};
    te_status result = TE_PENDING;
    std::mutex mu;
    std::condition_variable cv;
    std::string err;                 // message of a failed request
};

struct te_ctx {
    int device = 0;
    te_allocator alloc{};            // caller's device allocator (alloc == NULL: cudaMalloc)
    cudaStream_t stream = nullptr;        // the context's own non-blocking stream
    cudaStream_t user_stream = nullptr;   // the caller's stream (may be the legacy default)
    cudaEvent_t user_ev = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    int coop = 0;                    // device supports cooperative launches (fused Lanczos loop)
    std::string err;
    std::mutex mu;                   // plans, matrices
    std::vector<Plan*> plans;
    uint64_t next_matrix_id = 1;
    // te_spmv scratch
    DevState* spmv_st = nullptr;
    DevState* spmv_st_host = nullptr;
    double* spmv_partials = nullptr;
    // scheduler
    std::mutex qmu;
    std::condition_variable qcv;
    std::deque<te_request*> queue;   // requests for the solo workers
    std::vector<std::thread> workers;
    std::deque<te_request*> bqueue[2];   // requests for the two serving loops (continuous
    std::thread batcher[2];              // batching): [0] small requests, [1] medium ones
    int serve_mode = TE_SERVE_BATCH;
    int serve_m = 40;                // Krylov depth of the serving arena
    int64_t serve_cap = 0;           // elements per arena column (0: from the budget at first use)
    int64_t pending = 0;             // requests submitted and not yet finished
    int64_t serve_large_nnz = 1ll << 24;   // batch mode: H with this many entries takes the large lane
    int64_t serve_small_nnz = 1ll << 21;   // batch mode: H with fewer entries joins the small batch
    int solo_running = 0;            // requests the solo workers are running
    bool stopping = false;
    int64_t budget = 0;
    int64_t in_use = 0;
    int max_workers = 8;
};

// continuous-batching serving loop (te_multi.cu)
// -1: the large lane (solo workers); 0: the small batch; 1: the medium batch
int serve_class(const te_ctx* ctx, const te_request* r);
int64_t serve_class_capacity(const te_ctx* ctx, int cls);
void serve_loop(te_ctx* ctx, int cls);

// ---- host launchers (kernels live in te_lanczos.cu, te_step.cu, te_build.cu)

int spmv_lanes_for(double avg_row_nnz);
// S (may be null) receives Re v + Im v of every vector these kernels write,
// for the three-multiplication product of the SELL kernel.
cudaError_t launch_init_norm(const double2* v, double* S, int64_t d, DevState* st,
                             double* partials, int grid, cudaStream_t s);
cudaError_t launch_spmv_lanczos(const te_matrix* H, int lanes, const double2* x,
                                const double2* xprev, double2* y, DevState* st, int j,
                                int mode, double* partials, int grid, cudaStream_t s);
cudaError_t launch_orth_norm(double2* w, double* S, const double2* u, int64_t d, DevState* st,
                             int j, int write, int decide, double* partials, int grid,
                             cudaStream_t s);
cudaError_t launch_reorth_dots(const double2* V, const double2* w, int64_t d, DevState* st,
                               int j, double* partials, int grid, cudaStream_t s);
cudaError_t launch_reorth_update(const double2* V, double2* w, double* S, int64_t d, DevState* st,
                                 int j, int decide, double* partials, int grid, cudaStream_t s);
cudaError_t launch_step(DevState* st, int m, cudaStream_t s);
cudaError_t launch_step_batch(DevState* st, int nvec, int m, cudaStream_t s);
cudaError_t launch_recombine(double2* V, double* S, int64_t d, DevState* st, double* partials,
                             int grid, cudaStream_t s);
int spmv_grid(int lanes, int64_t d, int num_sms);
int occupancy_grid_spmv(int lanes, int num_sms);
int step_smem_bytes(int m);
cudaError_t step_prepare();

// SELL form (te_sell.cu)
te_status build_sell(te_ctx* ctx, te_matrix* H);
int sell_grid(int64_t nslices, int num_sms, int form);   // 0 full, 1 indexed, 2 real indexed
int sell_async_grid(int64_t nslices, int num_sms, int trip);   // the staged indexed product
cudaError_t sell_prepare();                     // shared-memory limit of the staged product
int64_t sell_partials(const te_matrix* H);
// grid > 0 overrides H->sell_grid (the kernel takes its work from a counter, so any
// grid computes the same product)
cudaError_t launch_spmv_sell(const te_matrix* H, const double2* x, const double* xs,
                             const double2* xprev, double2* y, DevState* st, int j, int mode,
                             double* partials, cudaStream_t s, int grid = 0);
cudaError_t launch_gather(const double2* src, const int32_t* map, int64_t d, double2* dst,
                          double* dsum, int num_sms, cudaStream_t s);
// fused Lanczos loop (te_fused.cu): shape of its cooperative grid (false: H too
// large or without a sliced copy); the launch clears bar and runs m steps.
bool fused_shape(const te_matrix* H, int num_sms, int* grid, int* threads);
cudaError_t launch_lanczos_fused(const te_matrix* H, double2* V, double* S, DevState* st, int m,
                                 double* part, unsigned int* bar, int grid, int threads,
                                 cudaStream_t s);
te_status scan_counts(te_ctx* ctx, const int32_t* cnt, int64_t d, int32_t* rowptr, int64_t* nnz,
                      cudaStream_t s);

// builders
te_status build_tfim(te_ctx* ctx, const te_model_desc* desc, te_matrix* H);
te_status build_xxzdm(te_ctx* ctx, const te_model_desc* desc, te_matrix* H);
te_status build_bose(te_ctx* ctx, const te_model_desc* desc, te_matrix* H);
te_status build_memory(te_ctx* ctx, const te_model_desc* desc, te_matrix* H);
int64_t memory_rank_host(const te_model_desc* desc, const int32_t* occ);
te_status finish_matrix_stats(te_ctx* ctx, te_matrix* H);
int64_t bose_rank_host(int K, int N, const int32_t* occ);

// batched solves (te_block.cu)
cudaError_t block_prepare();
void block_plans_release(te_ctx* ctx, uint64_t matrix_id);    // matrix_id 0: all of ctx
te_status run_block_solve(te_ctx* ctx, const te_matrix* H, int nvec, const double* v_in, double t,
                          double tol, int m, const te_options& o, double* v_out, bool dev,
                          te_stats* stats, int32_t* status, cudaStream_t s);
// intermediate-time sampling (te_sample.cu)
int sample_omega_smem(int mcap);
cudaError_t sample_prepare();
cudaError_t launch_sample_kernels(DevState* st, const double* ts, int ns, int mcap, double2* coef,
                                  double* bound, const double2* V, const double* S, int64_t d,
                                  double2* out, int grid_stream, cudaStream_t s);
cudaError_t launch_gather_real(const double* src, const int32_t* map, int64_t d, double* dst,
                               int num_sms, cudaStream_t s);
cudaError_t launch_observables(const double2* W, int64_t d, int ns, const double* O, int nobs,
                               double* partials, int G, double* out, cudaStream_t s);

// grouped independent solves (te_multi.cu)
void multi_plans_release(te_ctx* ctx, uint64_t matrix_id);    // matrix_id 0: all of ctx
bool multi_plans_in_use(te_ctx* ctx, uint64_t matrix_id);
te_status run_multi_solve(te_ctx* ctx, int n, const te_matrix* const* H, const double* const* v_in,
                          const double* t, double tol, int m, const te_options& o,
                          double* const* v_out, bool dev, te_stats* stats, int32_t* status,
                          cudaStream_t s);
// Gauss-Legendre nodes and weights on [-1, 1] (te_capi.cu)
void gauss_legendre_table(int n, double* x, double* w);

te_status set_error(te_ctx* ctx, te_status s, const std::string& msg);

// Device memory of a context: the caller's allocator (te_create_with_allocator),
// else cudaMalloc / cudaFree.  dev_free first waits for the context's stream, so
// a caller's pool may hand the memory out again at once.
cudaError_t dev_alloc(te_ctx* ctx, void** p, size_t bytes);
void dev_free(te_ctx* ctx, void* p);
template <class T>
inline cudaError_t dev_alloc(te_ctx* ctx, T** p, size_t bytes) {
    return dev_alloc(ctx, reinterpret_cast<void**>(p), bytes);
}
// Device status TE_ERR_UNSUPPORTED from the step or sample kernel: exp(-i H_m tau) e_1
// after a lucky breakdown needed more series pieces than the build allows.
constexpr const char* kSeriesRangeMsg =
    "exp(-i H_m tau) e_1 beyond the Chebyshev series' range (a lucky breakdown with "
    "||H_m|| |t| above ~1e6); TE_SMALLEXP_EIG evaluates any tau";
te_status cuda_error(te_ctx* ctx, cudaError_t e, const char* what);

#define TE_CUDA_TRY(ctx, call)                                   \
    do {                                                         \
        cudaError_t _e = (call);                                 \
        if (_e != cudaSuccess) return cuda_error((ctx), _e, #call); \
    } while (0)
