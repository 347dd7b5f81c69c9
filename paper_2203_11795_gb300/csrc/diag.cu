// Measurement helper: the sustained FP64 fused multiply-add rate of the current device.
//
// The complex128 transforms run their butterflies and twiddle products on the FP64 pipe, which
// on GB300 is narrow enough that they are bound by it rather than by HBM.  Their roofline
// therefore needs the FP64 rate of this device as measured, not a datasheet figure: this kernel
// keeps every SM's FP64 pipe busy with independent FMA chains and times it with CUDA events.
#include <cuda_runtime.h>

#include "fftu_internal.h"

namespace fftu {
namespace {

constexpr int kChains = 8;      // independent FMA chains per thread (hides the FMA latency)
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fp64_fma_kernel(double *sink, int iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0) sink[0] = s;  // never true for these operands; keeps the chains live
}

}  // namespace
}  // namespace fftu

extern "C" fftu_status fftu_measure_fp64_rate(int reps, double *gflops) {
    using namespace fftu;
    record_error("");
    if (!gflops || reps < 1 || reps > 100) {
        record_error("fftu_measure_fp64_rate: gflops must be non-NULL and reps in [1, 100]");
        return FFTU_ERR_ARG;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_fma_kernel, kThreads, 0);
    double *sink = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(double));
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    const int iters = 1 << 14;
    double best_ms = 0.0;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {  // r = 0 warms up
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            fp64_fma_kernel<<<blocks, kThreads, 0, st>>>(sink, iters, 0.9999999, 1e-7);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0 && (best_ms == 0.0 || ms < best_ms)) best_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess || best_ms <= 0.0) {
        cudaGetLastError();
        record_error("fftu_measure_fp64_rate: CUDA call failed");
        return FFTU_ERR_CUDA;
    }
    const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
    *gflops = flops / (best_ms * 1e-3) / 1e9;
    return FFTU_OK;
}
