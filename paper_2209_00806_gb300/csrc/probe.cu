// FP64 fused multiply-add throughput of the device: the ALU roofline of the
// FP64 form, whose term kernel is bound by GB300's FP64 pipe rather than by
// HBM.  Every thread runs kChains independent FMA chains (enough to cover
// the pipe's latency) for n_iter rounds; the grid fills every SM several
// times over.  Timed with CUDA events on a private stream.  Not part of the
// method: a measurement the benchmark reports its FP64 kernels against.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "tbpm_internal.cuh"

namespace tbpm {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_fp64_fma(int n_iter, double a, double b,
                                                            double *sink)
{
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (threadIdx.x + k) * 1e-3;
    for (int it = 0; it < n_iter; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 12345.678) sink[0] = s;        // keeps the chains alive, never true
}

}  // namespace
}  // namespace tbpm

using namespace tbpm;

extern "C" int tbpm_fp64_fma_rate(int device, int n_iter, double *tflops, double *ms)
{
    if (!tflops || n_iter < 1) {
        set_thread_error("tbpm_fp64_fma_rate: NULL output or n_iter < 1");
        return TBPM_E_INVALID_ARG;
    }
    cudaError_t e = cudaSetDevice(device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double *sink = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(double));
    const int blocks = sms * 8;
    float t = 0.f;
    if (e == cudaSuccess) {
        k_fp64_fma<<<blocks, kProbeThreads, 0, st>>>(n_iter / 8 + 1, 0.999999, 1e-7, sink);  // warm-up
        cudaEventRecord(e0, st);
        k_fp64_fma<<<blocks, kProbeThreads, 0, st>>>(n_iter, 0.999999, 1e-7, sink);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    }
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        set_thread_error(std::string("tbpm_fp64_fma_rate: ") + cudaGetErrorString(e));
        return TBPM_E_CUDA;
    }
    const double flops = 2.0 * (double)blocks * kProbeThreads * kChains * (double)n_iter;
    *tflops = flops / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return TBPM_OK;
}
