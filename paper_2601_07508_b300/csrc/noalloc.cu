// mwmm_matmul_noalloc: the INT8-form product with its scratch memory in a
// fixed, file-scope device array instead of memory the library or the caller
// allocates.
//
// Who needs it: code that must not allocate device memory while it runs --
// for example a caller whose allocator is owned by another framework and may
// not be bypassed, a long-running service that has to keep its device
// footprint fixed after start-up, or a process that runs under a memory
// limit where cudaMalloc can fail mid-job.  Such callers pass only the
// inputs and the output; the word matrices and the diagonal sums go into
// g_scratch below.
//
// Properties the caller must know:
//   - The scratch is kNoAllocScratchBytes (64 MiB).  A product whose words
//     and diagonal sums do not fit runs the fused form (sums kept on the
//     SM, n > 128), whose scratch is the words alone; one that does not fit
//     either (roughly m = n = k = 1500 at 52 bits, larger for smaller
//     primes) is rejected with MWMM_ERR_BUDGET before any work.
//   - The array belongs to this library's device code: once this code is
//     loaded on a GPU (at the latest on the first call on that GPU), the GPU
//     holds the 64 MiB until the process exits.
//   - The first call on each device looks up the array's device address
//     (cudaGetSymbolAddress, with that device current) and caches it.
//   - Every call uses the same array and it keeps the previous call's
//     contents.  The kernels rewrite every word and sum they later read
//     (padding included), and the error words are cleared at the start of
//     each call.  Calls whose work overlaps on the GPU (from several host
//     threads or streams) race on the array and give wrong results: issue
//     them one at a time per device.
//   - The call is synchronous: it returns after C is written, with the
//     device-side status (MWMM_ERR_TIMEOUT if a bounded wait expired).
//   - It calls no cudaMalloc, cudaFree or other allocating routine.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "mwmm_internal.h"

namespace mwmm {
namespace {

constexpr uint64_t kNoAllocScratchBytes = 64ull << 20;
constexpr uint64_t kErrBytes = 256;  // error words at the start of the array
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint8_t g_scratch[kNoAllocScratchBytes];

uint8_t *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_setup_mutex;

// Device address of g_scratch on the current device (looked up once per device).
mwmm_status scratch_ptr(uint8_t **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MWMM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return MWMM_ERR_CUDA;
        g_scratch_ptr[dev] = static_cast<uint8_t *>(p);
    }
    *out = g_scratch_ptr[dev];
    return MWMM_OK;
}

mwmm_status from_cuda(int e) { return e == 0 ? MWMM_OK : MWMM_ERR_CUDA; }

}  // namespace
}  // namespace mwmm

extern "C" mwmm_status mwmm_matmul_noalloc(int64_t m, int64_t n, int64_t k, uint64_t p, const uint64_t *dA,
                                           int64_t lda, const uint64_t *dB, int64_t ldb, uint64_t *dC,
                                           int64_t ldc, void *stream) {
    using namespace mwmm;
    Plan pl;  // on the stack: planning allocates nothing
    mwmm_plan_opts o0;
    std::memset(&o0, 0, sizeof(o0));
    o0.tc_fill = 1;  // no extra sum planes in the fixed scratch
    mwmm_status st = make_plan(&pl, m, n, k, p, 0, 0, MWMM_FORM_INT8, &o0);
    if (st != MWMM_OK) return st;
    if (m == 0 || n == 0) return MWMM_OK;
    if (!dC || (k > 0 && (!dA || !dB)) || lda < (k > 0 ? k : 1) || ldb < (n > 0 ? n : 1) || ldc < n)
        return MWMM_ERR_ARG;
    if (pl.ws_bytes > kNoAllocScratchBytes - kErrBytes && n > kTcBN / 2) {
        // Too large with the diagonal sums in the scratch: the fused form
        // keeps them on the SM and needs the words only (one K part, so no
        // partial planes either).
        mwmm_plan_opts o;
        std::memset(&o, 0, sizeof(o));
        o.tc_fused = 2;
        o.ksplit = 1;
        if ((st = make_plan(&pl, m, n, k, p, 0, 0, MWMM_FORM_INT8, &o)) != MWMM_OK) return st;
    }
    if (pl.ws_bytes > kNoAllocScratchBytes - kErrBytes) return MWMM_ERR_BUDGET;
    uint8_t *base = nullptr;
    st = scratch_ptr(&base);
    if (st != MWMM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (k == 0) {
        if (cudaMemset2DAsync(dC, (size_t)ldc * 8, 0, (size_t)n * 8, (size_t)m, s) != cudaSuccess)
            return MWMM_ERR_CUDA;
        return cudaStreamSynchronize(s) == cudaSuccess ? MWMM_OK : MWMM_ERR_CUDA;
    }
    int *err = reinterpret_cast<int *>(base);
    uint8_t *ws = base + kErrBytes;
    pl.err_dev = err;
    if (cudaMemsetAsync(err, 0, kErrBytes, s) != cudaSuccess) return MWMM_ERR_CUDA;
    if ((st = from_cuda(launch_split(pl, 0, dA, lda, ws + pl.A_off, stream, plan_sq(pl, ws, 0)))) != MWMM_OK) return st;
    if ((st = from_cuda(launch_split(pl, 1, dB, ldb, ws + pl.B_off, stream, plan_sq(pl, ws, 1)))) != MWMM_OK) return st;
    if ((st = from_cuda(launch_tensor_products(pl, ws, dC, ldc, err, stream))) != MWMM_OK) return st;
    int flags[2] = {0, 0};
    if (cudaMemcpyAsync(flags, err, sizeof(flags), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MWMM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MWMM_ERR_CUDA;
    return flags[0] ? MWMM_ERR_TIMEOUT : MWMM_OK;
}
