// probe.cu -- nl_fma_peak: the fused multiply-add throughput of this GPU in FP32 and FP64,
// the ALU roofline of the pair quadrature (FP32 path) and of the FP64 path.
//
// Every thread runs kChains independent FMA recurrences x <- x a + b for `iters` steps: with
// 1024 threads per SM and eight chains a thread there are far more independent FMAs in flight
// than the pipes' latency needs, so the time is the issue time of the FMAs alone.  The chains
// start at distinct values and a result depends on every step (stored only if it matches a
// value it never takes), so the compiler keeps all of them.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, T a, T b, T *sink)
{
    T x[kChains];
    for (int c = 0; c < kChains; c++) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) x[c] = fma(x[c], a, b);
    }
    T s = 0;
    for (int c = 0; c < kChains; c++) s += x[c];
    if (s == (T)-1.2345) sink[blockIdx.x] = s;   // never true: keeps the chains live
}

template <typename T>
nl_status probe(nl_ctx *ctx, double *tflops)
{
    int nsm = 0;
    NL_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    const int blocks = nsm * (2048 / kThreads);   // two full-size blocks' worth of threads per SM, 4 blocks
    const int iters = sizeof(T) == sizeof(float) ? 16384 : 1024;
    T *sink = nullptr;
    nl_temps tmp(ctx->stream);
    nl_status s = tmp.get(ctx, &sink, (size_t)blocks);
    if (s != NL_OK) return s;
    cudaEvent_t e0, e1;
    NL_CK(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return nl_cuda_fail(ctx, e, "cudaEventCreate");
    }
    // a warm-up launch, then the best of three timed launches
    float best = 0.0f;
    for (int r = 0; r < 4 && e == cudaSuccess; r++) {
        e = cudaEventRecord(e0, ctx->stream);
        k_fma_chains<T><<<blocks, kThreads, 0, ctx->stream>>>(iters, (T)0.999999, (T)1e-7, sink);
        ++ctx->launches;
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return nl_cuda_fail(ctx, e, "FMA probe");
    const double flop = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
    *tflops = best > 0.0f ? flop / (best * 1e-3) / 1e12 : 0.0;
    return NL_OK;
}

}  // namespace

extern "C" nl_status nl_fma_peak(nl_ctx *ctx, int32_t prec, double *tflops)
{
    if (!ctx) return NL_EINVAL;
    if (!tflops) return nl_fail(ctx, NL_EINVAL, "null output");
    NL_CK(cudaSetDevice(ctx->device));
    if (prec == NL_PREC_FP64) return probe<double>(ctx, tflops);
    if (prec == NL_PREC_FP32_COMP) return probe<float>(ctx, tflops);
    return nl_fail(ctx, NL_EINVAL, "bad precision");
}
