// te_probe.cu -- te_measure_fp64 / te_measure_fp64_mma: the FP64 rates the GPU
// sustains on its vector FMA pipe and on its FP64 matrix instruction (DMMA).
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

// FP64 matrix multiply-accumulate, D = A B + C on 8 x 8 x 4 tiles (mma.sync with
// .f64 operands: one element of A and of B and two of C / D per lane), 256 FMA per
// warp instruction.  kChains independent accumulator tiles per warp keep the
// instruction's latency covered.  This is the only FP64 matrix instruction the
// GPU offers (the tcgen05 tensor path has no FP64 kind); it decides whether a
// recombination or orthogonalisation written as small dense products could run
// faster than on the FP64 vector pipe.
__global__ void __launch_bounds__(kThreads) k_dmma_rate(double* out, int iters, double a, double b) {
    double c0[kChains], c1[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) {
        c0[q] = 1e-9 * threadIdx.x + q;
        c1[q] = 1e-9 * threadIdx.x - q;
    }
    const double av = a * (1.0 + 1e-6 * (threadIdx.x & 31));
    const double bv = b;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < kChains; ++q) {
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                         : "+d"(c0[q]), "+d"(c1[q])
                         : "d"(av), "d"(bv));
        }
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += c0[q] + c1[q];
    out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

// Times `launch` (after one warm-up) on the context's stream: the best of three.
template <class F>
cudaError_t best_of_three(cudaStream_t s, F launch, float* best_ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = INFINITY;
    for (int r = 0; r < 4 && e == cudaSuccess; ++r) {              // r = 0 warms up
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = launch();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0 && ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *best_ms = best;
    return e;
}

}  // namespace

extern "C" te_status te_measure_fp64_mma(te_ctx* ctx, double* tflops) {
    if (!ctx || !tflops) return TE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaGetLastError();
    cudaStream_t s = ctx->stream;
    TE_CUDA_TRY(ctx, cudaEventRecord(ctx->user_ev, ctx->user_stream));
    TE_CUDA_TRY(ctx, cudaStreamWaitEvent(s, ctx->user_ev, 0));
    const int grid = ctx->num_sms * kBlocksPerSM;
    constexpr int kMmaIters = 2048;
    double* out = nullptr;
    TE_CUDA_TRY(ctx, dev_alloc(ctx, &out, sizeof(double) * (size_t)grid * kThreads));
    float best = 0.f;
    cudaError_t e = best_of_three(s, [&]() {
        k_dmma_rate<<<grid, kThreads, 0, s>>>(out, kMmaIters, 0.999999999, 1e-12);
        return cudaGetLastError();
    }, &best);
    dev_free(ctx, out);
    if (e != cudaSuccess) return cuda_error(ctx, e, "te_measure_fp64_mma");
    // 8 x 8 x 4 multiply-adds (2 FLOP each) per warp instruction
    const double flop = 2.0 * 256.0 * kChains * (double)kMmaIters * grid * (kThreads / 32);
    *tflops = flop / (best * 1e-3) * 1e-12;
    return TE_OK;
}

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
