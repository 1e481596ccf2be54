// Elementwise Alg. 1 and Alg. 2 (the reductions used inside the products),
// exposed so each can be checked on its own against x mod p and x y mod p.
#include "device_common.cuh"
#include "mwmm_internal.h"

namespace mwmm {

namespace {

__global__ void fmod_kernel(const double *x, int64_t count, double p, double q, double *out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = fmod_alg1(x[e], p, q);
}

__global__ void mulmod_kernel(const double *x, const double *y, int64_t count, double p, double q,
                              int big_p, double two26, double *out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (!big_p) {
            out[e] = mulmod_alg2(x[e], y[e], p, q);
        } else {
            // x 2^26 mod p by Alg. 2 (x 2^26 < 2^78), then the split form.
            const double x26 = mulmod_alg2(x[e], two26, p, q);
            out[e] = mulmod_split(x[e], x26, y[e], p, q);
        }
    }
}

// One thread waits, through the product kernels' bounded-wait routine, on a
// barrier phase that nothing completes; the wait gives up after `limit`
// cycles and raises err[0].
__global__ void wait_probe_kernel(long long limit, int *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    (void)mbar_wait_for(&bar, 0, err, limit);
}

int grid_for(int64_t count) {
    int64_t b = (count + 255) / 256;
    if (b > 148 * 16) b = 148 * 16;
    return (int)(b > 0 ? b : 1);
}

}  // namespace

int launch_fmod(const double *x, int64_t count, uint64_t p, double *out, void *stream) {
    if (count == 0) return 0;
    const double pd = (double)p;
    fmod_kernel<<<grid_for(count), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, count, pd, 1.0 / pd, out);
    return (int)cudaGetLastError();
}

int launch_wait_probe(int64_t cycles, int *err, void *stream) {
    wait_probe_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>((long long)cycles, err);
    return (int)cudaGetLastError();
}

int launch_mulmod(const double *x, const double *y, int64_t count, uint64_t p, double *out, void *stream) {
    if (count == 0) return 0;
    const double pd = (double)p;
    typedef unsigned __int128 u128;
    const int big_p = (u128)3 * (p - 1) * (p - 1) > ((u128)p << 52);
    mulmod_kernel<<<grid_for(count), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        x, y, count, pd, 1.0 / pd, big_p, 67108864.0, out);
    return (int)cudaGetLastError();
}

}  // namespace mwmm
