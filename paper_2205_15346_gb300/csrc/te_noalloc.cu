// te_noalloc.cu -- te_spmv_noalloc: y = H x and Re <x, H x> without any allocation.
//
// Some callers cannot allocate device memory when they need a product: code
// that lives under a framework owning all device memory through its own pool
// (a stray cudaMalloc there can fail or fragment the pool), services that must
// keep their device footprint fixed once started, and latency-critical loops
// that must not pay for cudaMalloc or the implicit device-wide synchronisation
// of cudaFree.  For them this file offers a
// variant of the library's SpMV-with-energy kernel whose reduction scratch (one
// partial sum per thread block, an arrival counter and the result slot) lives
// in a fixed, file-scope device array instead of memory allocated per call.
//
// Under CUDA's lazy module loading (the default) the array and the kernel are
// loaded onto a device at the first call there: that first call, which also
// looks up the array's device address, may allocate through the driver and is
// the set-up step; later calls on the device allocate nothing.  The array then
// stays on the device until the process exits.  Its size caps the problem: one block covers
// kRowsPerBlock rows and the array has room for kMaxBlocks partials, so d may
// be at most TE_NOALLOC_MAX_D.  All calls on a device share the one array and
// it keeps the last call's contents, so the arrival counter is cleared on the
// stream before every launch; calls whose work overlaps on the GPU (other
// streams, other host threads) race on the array and must be serialised by the
// caller.
#include <mutex>

#include "te_internal.cuh"

namespace {

constexpr int kRowsPerBlock = 1024;
constexpr int kMaxBlocks = TE_NOALLOC_MAX_D / kRowsPerBlock;
constexpr int kMaxDevices = 64;

// [0]: arrival counter (as unsigned int in the first word); [1]: result;
// [2 .. 2 + kMaxBlocks): one partial per block.
static __device__ __align__(256) double g_noalloc_scratch[2 + kMaxBlocks];

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

// G lanes per CSR row; block b owns rows [b * kRowsPerBlock, (b+1) * kRowsPerBlock).
// scratch points at g_noalloc_scratch (its device address, looked up on the host).
template <int G>
__global__ void __launch_bounds__(TE_BLOCK) k_spmv_dot_static(
    const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const double2* __restrict__ val, const double2* __restrict__ x, double2* __restrict__ y,
    int64_t d, double* scratch) {
    __shared__ double sh[32];
    __shared__ bool am_last;
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch);
    double* result = scratch + 1;
    double* partials = scratch + 2;
    const int lane = threadIdx.x & 31, sub = lane & (G - 1);
    constexpr int RPW = 32 / G;
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t row0 = (int64_t)blockIdx.x * kRowsPerBlock;
    const int64_t row1 = row0 + kRowsPerBlock < d ? row0 + kRowsPerBlock : d;
    double acc = 0.0;
    for (int64_t base = row0 + (int64_t)warp * RPW; base < row1; base += (int64_t)nwarps * RPW) {
        const int64_t row = base + lane / G;
        double re = 0.0, im = 0.0;
        if (row < row1) {
            const int b = rowptr[row], e = rowptr[row + 1];
            for (int k = b + sub; k < e; k += G) {
                const double2 a = val[k];
                const double2 xv = __ldg(x + col[k]);
                re = fma(a.x, xv.x, re);
                re = fma(-a.y, xv.y, re);
                im = fma(a.x, xv.y, im);
                im = fma(a.y, xv.x, im);
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o, G);
            im += __shfl_xor_sync(0xffffffffu, im, o, G);
        }
        if (sub == 0 && row < row1) {
            y[row] = make_double2(re, im);
            const double2 xr = __ldg(x + row);
            acc += xr.x * re + xr.y * im;
        }
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s;
        __threadfence();
        am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double v = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += __ldcg(partials + i);
    const double tot = block_sum(v, sh);
    if (threadIdx.x == 0) {
        *result = tot;
        *counter = 0u;
    }
}

std::mutex g_setup_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on `device` (which must be current),
// looked up once per device.
te_status scratch_address(te_ctx* ctx, int device, double** out) {
    if (device < 0 || device >= kMaxDevices)
        return set_error(ctx, TE_ERR_UNSUPPORTED, "te_spmv_noalloc: device index above 63");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(ctx, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_ptr[device] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[device];
    return TE_OK;
}

}  // namespace

extern "C" te_status te_spmv_noalloc(te_ctx* ctx, const te_matrix* H, const double* x, double* y,
                                     double* x_dot_y, uint32_t flags) {
    if (!ctx || !H || !x || !y) return TE_ERR_INVALID_ARG;
    if (!(flags & TE_PTR_DEVICE))
        return set_error(ctx, TE_ERR_INVALID_ARG,
                         "te_spmv_noalloc: x and y must be device pointers (TE_PTR_DEVICE)");
    if (x == y) return set_error(ctx, TE_ERR_INVALID_ARG, "x and y must be distinct buffers");
    if (H->d > TE_NOALLOC_MAX_D)
        return set_error(ctx, TE_ERR_UNSUPPORTED,
                         "te_spmv_noalloc: d exceeds TE_NOALLOC_MAX_D (8,388,608 rows); "
                         "use te_spmv for larger matrices");
    cudaSetDevice(ctx->device);
    cudaGetLastError();
    double* scratch = nullptr;
    te_status st = scratch_address(ctx, ctx->device, &scratch);
    if (st) return st;
    cudaStream_t s = ctx->stream;
    TE_CUDA_TRY(ctx, cudaEventRecord(ctx->user_ev, ctx->user_stream));
    TE_CUDA_TRY(ctx, cudaStreamWaitEvent(s, ctx->user_ev, 0));
    // the arrival counter must start at zero (the array keeps the last call's contents)
    TE_CUDA_TRY(ctx, cudaMemsetAsync(scratch, 0, sizeof(double), s));
    const int grid = (int)((H->d + kRowsPerBlock - 1) / kRowsPerBlock);
    const double2* xd = reinterpret_cast<const double2*>(x);
    double2* yd = reinterpret_cast<double2*>(y);
#define TE_NA(G) \
    k_spmv_dot_static<G><<<grid, TE_BLOCK, 0, s>>>(H->rowptr, H->col, H->val, xd, yd, H->d, scratch)
    switch (H->lanes) {
        case 1: TE_NA(1); break;
        case 2: TE_NA(2); break;
        case 4: TE_NA(4); break;
        case 8: TE_NA(8); break;
        case 16: TE_NA(16); break;
        default: TE_NA(32); break;
    }
#undef TE_NA
    TE_CUDA_TRY(ctx, cudaGetLastError());
    double dot = 0.0;
    TE_CUDA_TRY(ctx, cudaMemcpyAsync(&dot, scratch + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    TE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (x_dot_y) *x_dot_y = dot;
    return TE_OK;
}
