// Device helpers shared by the libmwmm kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mwmm {

// A bounded wait gives up after this many SM cycles (about 2 s at 2 GHz) and
// raises the plan's timeout flag instead of hanging the GPU.
constexpr long long kWaitCycles = 4000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete.  Returns false, and
// sets err[0], if it has not completed within `limit` SM clock cycles.
__device__ __forceinline__ bool mbar_wait_for(uint64_t *bar, uint32_t parity, int *err, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) {
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

// The product kernels' waits: limit kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err) {
    return mbar_wait_for(bar, parity, err, kWaitCycles);
}

// One bulk (TMA) copy of `bytes` contiguous bytes global -> shared, completing
// `bytes` transactions on `bar`.  Both addresses 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// Floating-point modular arithmetic of Sec. 2.1.  Every operation is written
// with an explicitly rounded intrinsic so the compiler cannot contract or
// reassociate it (the proofs assume each step is rounded to nearest).

// Alg. 1: d = x mod p for integer x in F with x <= 2^(t-2) p, 4 <= p < 2^52,
// q = fl(1/p)  (Prop. 2.1).
__device__ __forceinline__ double fmod_alg1(double x, double p, double q) {
    const double b = __dmul_rn(x, q);
    const double c = floor(b);
    double d = __fma_rn(-c, p, x);
    if (d >= p) d = __dsub_rn(d, p);
    if (d < 0.0) d = __dadd_rn(d, p);
    return d;
}

// Alg. 2: e = x y mod p for integers x, y in F with x y <= (2^52 / 3) p,
// p <= 2^52  (Prop. 2.2).  (h, l) is the error-free product h + l = x y.
__device__ __forceinline__ double mulmod_alg2(double x, double y, double p, double q) {
    const double h = __dmul_rn(x, y);
    const double l = __fma_rn(x, y, -h);
    const double b = __dmul_rn(h, q);
    const double c = floor(b);
    const double d = __fma_rn(-c, p, h);
    double e = __dadd_rn(d, l);
    if (e >= p) e = __dsub_rn(e, p);
    if (e < 0.0) e = __dadd_rn(e, p);
    return e;
}

// g y mod p for g, y in [0, p) when p may exceed 2^52 / 3: y = y_h 2^26 + y_l
// (exact), g y = g y_l + (g 2^26 mod p) y_h with both products < 2^78, which
// Prop. 2.2 covers for p > 2^52 / 3.  g26 = g 2^26 mod p is precomputed.
__device__ __forceinline__ double mulmod_split(double g, double g26, double y, double p, double q) {
    const double yh = floor(__dmul_rn(y, 0x1p-26));
    const double yl = __fma_rn(-yh, 0x1p26, y);
    double e = __dadd_rn(mulmod_alg2(g, yl, p, q), mulmod_alg2(g26, yh, p, q));
    if (e >= p) e = __dsub_rn(e, p);
    return e;
}

}  // namespace mwmm

#include <mutex>

namespace mwmm {
// Host-side caches of the launchers (attributes set, SM and cluster counts)
// are filled under this lock: plans on different threads may launch at once.
inline std::mutex &launch_cache_mutex() {
    static std::mutex mu;
    return mu;
}

// Raise a kernel's dynamic shared-memory limit (once per device and kernel;
// later calls are free, so a launch inside a stream capture makes no
// attribute call once the same launch ran outside it).
inline cudaError_t set_smem_attr(const void *func, int bytes) {
    struct Done { const void *f; int dev; };
    static Done done[64];
    static int ndone = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(launch_cache_mutex());
    for (int i = 0; i < ndone; ++i)
        if (done[i].f == func && done[i].dev == dev) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && ndone < 64) done[ndone++] = Done{func, dev};
    return e;
}
}  // namespace mwmm
