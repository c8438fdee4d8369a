// te_probe.cu -- te_measure_fp64: the FP64 fused multiply-add rate the GPU sustains.
//
// On GB300 the products of the Krylov solve (the SpMV, the orthogonalisation and
// the recombination) are bound by FP64 issue, not by HBM.  Their roofline is the
// FP64 pipe rate derived from the unit counts (SMs x FMA lanes x 2 FLOP x clock).
// This kernel measures what the pipe delivers on pure, independent FMA chains --
// no memory traffic, no other instructions in the loop -- so that a kernel's FP64
// fraction can be read against both the derived and the attainable rate.
#include "te_internal.cuh"

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread
constexpr int kIters = 8192;    // FMAs per chain
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;

// The trip count is a run-time argument on purpose: the same loop with a
// compile-time count and an unroll pragma measured 16 % slower on GB300 (code
// generation, not the pipe), while this form reaches the derived pipe rate.
__global__ void __launch_bounds__(kThreads) k_dfma_rate(double* out, int iters, double a, double b) {
    double acc[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) acc[q] = 1e-9 * threadIdx.x + q;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < kChains; ++q) acc[q] = fma(acc[q], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += acc[q];
    out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

}  // namespace

extern "C" te_status te_measure_fp64(te_ctx* ctx, double* tflops) {
    if (!ctx || !tflops) return TE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaGetLastError();
    cudaStream_t s = ctx->stream;
    TE_CUDA_TRY(ctx, cudaEventRecord(ctx->user_ev, ctx->user_stream));
    TE_CUDA_TRY(ctx, cudaStreamWaitEvent(s, ctx->user_ev, 0));
    const int grid = ctx->num_sms * kBlocksPerSM;
    double* out = nullptr;
    TE_CUDA_TRY(ctx, dev_alloc(ctx, &out, sizeof(double) * (size_t)grid * kThreads));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = INFINITY;
    for (int r = 0; r < 4 && e == cudaSuccess; ++r) {              // r = 0 warms up
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) {
            k_dfma_rate<<<grid, kThreads, 0, s>>>(out, kIters, 0.999999999, 1e-12);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0 && ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(ctx, out);
    if (e != cudaSuccess) return cuda_error(ctx, e, "te_measure_fp64");
    const double flop = 2.0 * kChains * (double)kIters * grid * kThreads;
    *tflops = flop / (best * 1e-3) * 1e-12;
    return TE_OK;
}
