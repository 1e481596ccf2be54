// Pipe-rate diagnostic: the FP64 (DFMA) rate of this device, the roofline
// denominator of the FP64 form (whose word products run on the FP64 pipe).
// Eight independent fused multiply-add chains per thread, 1024 threads per
// SM, so the pipe, not the latency of one chain, bounds the loop.
#include <cuda_runtime.h>

#include "mwmm_internal.h"

namespace mwmm {
namespace {

__device__ double g_fp64_sink;

__global__ void __launch_bounds__(256) fp64_fma_loop(int64_t iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 1.0 + 1e-3 * (threadIdx.x + 37 * j);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = __fma_rn(x[j], a, b);
    }
    double s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == -1.0) g_fp64_sink = s;  // never true; keeps the loop
}

}  // namespace
}  // namespace mwmm

extern "C" mwmm_status mwmm_measure_fp64_rate(int64_t iters, double *gflops, void *stream) {
    if (!gflops || iters < 1 || iters > (int64_t(1) << 24)) return MWMM_ERR_ARG;
    *gflops = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = 4 * mwmm::tc_sm_count();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return MWMM_ERR_CUDA;
    }
    // one short warm-up launch, then the timed one
    mwmm::fp64_fma_loop<<<blocks, 256, 0, s>>>(iters / 16 + 1, 0.9999999, 1e-7);
    cudaEventRecord(e0, s);
    mwmm::fp64_fma_loop<<<blocks, 256, 0, s>>>(iters, 0.9999999, 1e-7);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || ms <= 0) return MWMM_ERR_CUDA;
    *gflops = 2.0 * 8.0 * (double)iters * (double)blocks * 256.0 / (ms * 1e-3) / 1e9;
    return MWMM_OK;
}
