// Pipe-rate diagnostic: the FP64 (DFMA) rate of this device, the roofline
// denominator of the FP64 form (whose word products run on the FP64 pipe).
// The loop body is the FP64 word-product kernel's: a 4 x 4 block of
// accumulators updated as acc[r][c] = fma(a[r], b[c], acc[r][c]) (sixteen
// independent chains per thread, operands in distinct registers; a
// self-dependent x = fma(x, a, b) measured 14% below this on B300), 1024
// threads per SM, so the pipe, not the latency of one chain, bounds it.  Exactly
// one block per SM: each block asks for more than half of the SM's shared
// memory (unused), so the block scheduler cannot stack two blocks on one SM
// and leave another idle.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "mwmm_internal.h"

namespace mwmm {
namespace {

__device__ double g_fp64_sink;

constexpr int kDiagThreads = 1024;
constexpr int kDiagSmem = 120 << 10;

__global__ void __launch_bounds__(kDiagThreads, 1) fp64_fma_loop(int64_t iters, double a0, double b0) {
    double a[4], b[4], acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        a[r] = a0 - 1e-9 * r;
        b[r] = b0 * (1 + r);
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 1.0 + 1e-3 * (threadIdx.x + 5 * r + c);
    }
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = __fma_rn(a[r], b[c], acc[r][c]);
    }
    double s = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) s += acc[r][c];
    if (s == -1.0) g_fp64_sink = s;  // never true; keeps the loop
}

}  // namespace
}  // namespace mwmm

extern "C" mwmm_status mwmm_measure_fp64_rate(int64_t iters, double *gflops, void *stream) {
    if (!gflops || iters < 1 || iters > (int64_t(1) << 24)) return MWMM_ERR_ARG;
    *gflops = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = mwmm::tc_sm_count();
    if (mwmm::set_smem_attr(reinterpret_cast<const void *>(mwmm::fp64_fma_loop), mwmm::kDiagSmem) != cudaSuccess)
        return MWMM_ERR_CUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return MWMM_ERR_CUDA;
    }
    // one short warm-up launch, then the timed one
    mwmm::fp64_fma_loop<<<blocks, mwmm::kDiagThreads, mwmm::kDiagSmem, s>>>(iters / 16 + 1, 0.9999999, 1e-7);
    cudaEventRecord(e0, s);
    mwmm::fp64_fma_loop<<<blocks, mwmm::kDiagThreads, mwmm::kDiagSmem, s>>>(iters, 0.9999999, 1e-7);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || ms <= 0) return MWMM_ERR_CUDA;
    *gflops = 2.0 * 16.0 * (double)iters * (double)blocks * mwmm::kDiagThreads / (ms * 1e-3) / 1e9;
    return MWMM_OK;
}

extern "C" mwmm_status mwmm_tc_residency(int32_t *sms, int32_t *ctas, int32_t *pair_clusters) {
    int s = 0, c = 0, p = 0;
    if (mwmm::tc_residency(&s, &c, &p) != 0) return MWMM_ERR_CUDA;
    if (sms) *sms = s;
    if (ctas) *ctas = c;
    if (pair_clusters) *pair_clusters = p;
    return MWMM_OK;
}
