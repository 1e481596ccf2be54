// FP64 form of the multiword product, fused in one kernel.
//
// For each output tile and each word pair (i, j) (Alg. 5's double loop):
//   T = A_i B_j accumulated in FP64 with an Alg. 1 reduction every lambda
//       k-steps (Alg. 3; exact by Prop. 2.3 / Prop. 3.3 since the running
//       value stays <= lambda * alpha * beta + p - 1 <= 2^53),
//   e = gamma_ij T mod p with Alg. 2 (gamma_ij = alpha^i beta^j mod p),
//   C = C + e mod p.
// This is the workspace variant described in Sec. 3.2 before Alg. 5, with the
// workspace T held in registers: the result equals Alg. 5's (C is unique) and
// needs neither the modular inverses delta_ij nor extra passes over C.
//
// B300 mapping: the FP64 pipe (about 2 DFMA per clock per SM) bounds this
// form, so the kernel keeps the DFMA issue dense and everything else off the
// critical path: word tiles (64 rows x 16 k, 8 KB) arrive by bulk TMA copies
// into a 4-stage shared-memory ring, each thread owns a 4 x 4 output block.
#include <cstring>
#include <vector>

#include "device_common.cuh"
#include "mwmm_internal.h"

namespace mwmm {

namespace {

constexpr int BM = kF64BM, BN = kF64BN, KB = kF64KB;
constexpr int STAGES = 4;
constexpr int THREADS = 256;
constexpr uint32_t kTileA = BM * kTileBytes, kTileB = BN * kTileBytes;
static_assert(BM == 64 && BN == 64 && KB == 16, "thread mapping assumes 64 x 64 x 16");

struct F64Params {
    const uint8_t *Aw, *Bw;
    uint64_t *C;
    int64_t ldc, m, n, nkb, A_rows, B_rows, lambda;
    int u, v, big_p;
    double p, q;
    double gamma[kMaxWords * kMaxWords];
    double gamma26[kMaxWords * kMaxWords];
    int *err;
};

// element kk (0..15) of word-layout row r inside a 128-byte swizzled chunk
__device__ __forceinline__ double lds_word(const uint8_t *tile, int r, int kk) {
    return *reinterpret_cast<const double *>(tile + r * kTileBytes + (((kk >> 1) ^ (r & 7)) << 4) +
                                             ((kk & 1) << 3));
}

// One 64 x 64 output tile (row0, col0) of the product described by P.
__device__ __forceinline__ void fp64_tile(const F64Params &P, int64_t row0, int64_t col0, uint8_t *smem,
                                          uint64_t *full) {
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * kTileA;

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t total = (int64_t)P.u * P.v * P.nkb;  // virtual k-blocks: (pair, kb)

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int64_t vb) {
        const int slot = (int)(vb % STAGES);
        const int pair = (int)(vb / P.nkb);
        const int64_t kb = vb % P.nkb;
        const int i = pair / P.v, j = pair % P.v;
        const uint8_t *a = P.Aw + (((int64_t)i * P.nkb + kb) * P.A_rows + row0) * kTileBytes;
        const uint8_t *b = P.Bw + (((int64_t)j * P.nkb + kb) * P.B_rows + col0) * kTileBytes;
        mbar_arrive_expect_tx(&full[slot], kTileA + kTileB);
        bulk_g2s(sA + slot * kTileA, a, kTileA, &full[slot]);
        bulk_g2s(sB + slot * kTileB, b, kTileB, &full[slot]);
    };
    if (tid == 0)
        for (int64_t vb = 0; vb < STAGES - 1 && vb < total; ++vb) issue(vb);

    const double p = P.p, q = P.q;
    double acc[4][4], cres[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) cres[r][c] = 0.0;
    int64_t cnt = 0;

    for (int64_t vb = 0; vb < total; ++vb) {
        // The slot refilled here was last read in iteration vb - 1, which every
        // thread has left (barrier at the end of that iteration).
        if (tid == 0 && vb + STAGES - 1 < total) issue(vb + STAGES - 1);
        const int slot = (int)(vb % STAGES);
        const bool ok = mbar_wait(&full[slot], (uint32_t)((vb / STAGES) & 1), P.err);
        if (!__syncthreads_and(ok)) break;  // uniform exit after a timed-out wait

        const int64_t kb = vb % P.nkb;
        if (kb == 0) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
            cnt = 0;
        }
        const uint8_t *ta = sA + slot * kTileA;
        const uint8_t *tb = sB + slot * kTileB;
#pragma unroll 4
        for (int kk = 0; kk < KB; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = lds_word(ta, ty + 16 * r, kk);
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = lds_word(tb, tx + 16 * c, kk);
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = __fma_rn(a[r], b[c], acc[r][c]);
            if (++cnt == P.lambda) {  // Alg. 3: C = C mod p after each block of lambda steps
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] = fmod_alg1(acc[r][c], p, q);
                cnt = 0;
            }
        }
        if (kb == P.nkb - 1) {  // word pair (i, j) complete: recombine (Alg. 5 / Alg. 2)
            const int pair = (int)(vb / P.nkb);
            const double g = P.gamma[pair], g26 = P.gamma26[pair];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const double T = fmod_alg1(acc[r][c], p, q);
                    double e;
                    if (pair == 0) e = T;  // gamma_00 = 1
                    else if (!P.big_p) e = mulmod_alg2(g, T, p, q);
                    else e = mulmod_split(g, g26, T, p, q);
                    double s = __dadd_rn(cres[r][c], e);
                    if (s >= p) s = __dsub_rn(s, p);
                    cres[r][c] = s;
                }
        }
        __syncthreads();
    }

#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t row = row0 + ty + 16 * r;
        if (row >= P.m) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t col = col0 + tx + 16 * c;
            if (col < P.n) P.C[row * P.ldc + col] = (uint64_t)cres[r][c];
        }
    }
}

__global__ void __launch_bounds__(THREADS) gemm_fp64_kernel(const __grid_constant__ F64Params P) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[STAGES];
    fp64_tile(P, (int64_t)blockIdx.y * BM, (int64_t)blockIdx.x * BN, smem, full);
}

// Batched: block b computes tile (row block y, col block x) of problem
// probs[jobs[b].x] with jobs[b] = (problem, y, x, 0).
__global__ void __launch_bounds__(THREADS) gemm_fp64_batched_kernel(const F64Params *probs, const int4 *jobs) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[STAGES];
    const int4 j = jobs[blockIdx.x];
    fp64_tile(probs[j.x], (int64_t)j.y * BM, (int64_t)j.z * BN, smem, full);
}

F64Params make_f64_params(const Plan &pl, const void *Aw, const void *Bw, uint64_t *C, int64_t ldc, int *err) {
    F64Params P;
    P.Aw = static_cast<const uint8_t *>(Aw);
    P.Bw = static_cast<const uint8_t *>(Bw);
    P.C = C;
    P.ldc = ldc;
    P.m = pl.m;
    P.n = pl.n;
    P.nkb = pl.nkb;
    P.A_rows = pl.A_rows;
    P.B_rows = pl.B_rows;
    P.lambda = pl.lambda;
    P.u = pl.u;
    P.v = pl.v;
    P.big_p = pl.big_p;
    P.p = pl.pd;
    P.q = pl.q;
    for (int i = 0; i < kMaxWords * kMaxWords; ++i) {
        P.gamma[i] = pl.gamma[i];
        P.gamma26[i] = pl.gamma26[i];
    }
    P.err = err;
    return P;
}

}  // namespace

size_t fp64_job_bytes() { return sizeof(F64Params); }

int prepare_tc_attributes();

int prepare_kernel_attributes() {
    const int smem = STAGES * (kTileA + kTileB);
    cudaError_t e = set_smem_attr(reinterpret_cast<const void *>(gemm_fp64_kernel), smem);
    if (e == cudaSuccess) e = set_smem_attr(reinterpret_cast<const void *>(gemm_fp64_batched_kernel), smem);
    if (e != cudaSuccess) return (int)e;
    return prepare_tc_attributes();
}

void fp64_job(const Plan &pl, const void *Aw, const void *Bw, uint64_t *C, int64_t ldc, int *err, void *rec,
              int index, std::vector<int> &jobs) {
    const F64Params P = make_f64_params(pl, Aw, Bw, C, ldc, err);
    std::memcpy(rec, &P, sizeof(P));
    for (int64_t y = 0; y < pl.A_rows / BM; ++y)
        for (int64_t x = 0; x < pl.B_rows / BN; ++x) {
            jobs.push_back(index);
            jobs.push_back((int)y);
            jobs.push_back((int)x);
            jobs.push_back(0);
        }
}

int launch_gemm_fp64_batched(const void *probs, const int *jobs, int njobs, void *stream) {
    if (njobs == 0) return 0;
    const int smem = STAGES * (kTileA + kTileB);
    cudaError_t e = set_smem_attr(reinterpret_cast<const void *>(gemm_fp64_batched_kernel), smem);
    if (e != cudaSuccess) return (int)e;
    gemm_fp64_batched_kernel<<<njobs, THREADS, smem, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const F64Params *>(probs), reinterpret_cast<const int4 *>(jobs));
    return (int)cudaGetLastError();
}

int launch_gemm_fp64(const Plan &pl, const void *Aw, const void *Bw, uint64_t *C, int64_t ldc, int *err,
                     void *stream) {
    const F64Params P = make_f64_params(pl, Aw, Bw, C, ldc, err);
    const int smem = STAGES * (kTileA + kTileB);
    cudaError_t e = set_smem_attr(reinterpret_cast<const void *>(gemm_fp64_kernel), smem);
    if (e != cudaSuccess) return (int)e;
    dim3 grid((unsigned)(pl.B_rows / BN), (unsigned)(pl.A_rows / BM));
    gemm_fp64_kernel<<<grid, THREADS, smem, static_cast<cudaStream_t>(stream)>>>(P);
    return (int)cudaGetLastError();
}

}  // namespace mwmm
