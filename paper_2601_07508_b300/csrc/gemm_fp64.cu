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
//
// Concatenation (Alg. 6, narrow n): the 64 columns of a tile hold f64_vs word
// slots of w = 64 / f64_vs output columns each, i.e. the product
// A_i [B_0 ... B_{v-1}] restricted to w columns of C, so a tile is full even
// when n is 32 or 16.  B's words are then stored k-block major so the slots of
// one k-block are adjacent.  A thread owns columns tx + 16 c, i.e. word slot
// (tx + 16 c) / w; after scaling each T_ij by gamma_ij it adds up its own
// columns of the same output column (no data exchange).  When m is the narrow
// side, the A words are concatenated instead ([A_0; ...; A_{u-1}] B_j, Sec.
// 3.2): the 64 rows of a tile hold u slots of w rows, and a thread adds up its
// rows ty + 16 r of the same output row.
//
// K ranges (plan ksplit > 1): grid z splits the k-blocks so that narrow or
// small products still fill the GPU; each range writes its partial C (already
// reduced mod p) and a second kernel adds the ranges mod p.
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
    int64_t kbr;                   // k-blocks per K range
    int64_t b_wstride, b_kstride;  // B layout: rows between consecutive words / k-blocks
    int64_t a_wstride, a_kstride;  // A layout: the same for A
    uint64_t *part;                // ksplit > 1: partial C of range z at part + z m n (row stride n)
    int u, v, big_p, concat, w;  // concat: 0 none, 1 B words, 2 A words (slots of w)
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

// One output tile (row tile `rt`, column tile `ct`) over K range z of the
// product described by P.
__device__ __forceinline__ void fp64_tile(const F64Params &P, int64_t rt, int64_t ct, int64_t z, uint8_t *smem,
                                          uint64_t *full) {
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * kTileA;

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t kb0 = z * P.kbr;
    const int64_t kbn = P.nkb - kb0 < P.kbr ? P.nkb - kb0 : P.kbr;
    const bool catB = P.concat == 1, catA = P.concat == 2;
    // concatenated: one product per A word (B concatenated) or per B word (A concatenated)
    const int npairs = catB ? P.u : catA ? P.v : P.u * P.v;
    const int64_t total = (int64_t)npairs * kbn;  // virtual k-blocks: (pair, kb)
    const int64_t col0 = catB ? ct * P.w : ct * BN;  // first output column
    const int64_t row0 = catA ? rt * P.w : rt * BM;  // first output row

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int64_t vb) {
        const int slot = (int)(vb % STAGES);
        const int pair = (int)(vb / kbn);
        const int64_t kb = kb0 + vb % kbn;
        uint8_t *dst = sB + slot * kTileB;
        if (catA) {  // A slots i = 0 .. u-1 of w rows each, then the B word j = pair
            const uint32_t wbytes = (uint32_t)P.w * kTileBytes;
            const uint8_t *a = P.Aw + (kb * P.a_kstride + row0) * kTileBytes;
            const uint8_t *b = P.Bw + (pair * P.b_wstride + kb * P.b_kstride + col0) * kTileBytes;
            mbar_arrive_expect_tx(&full[slot], (uint32_t)P.u * wbytes + kTileB);
            uint8_t *da = sA + slot * kTileA;
            if (P.A_rows == P.w) {  // one row tile: the u slots are adjacent
                bulk_g2s(da, a, (uint32_t)P.u * wbytes, &full[slot]);
            } else {
                for (int i = 0; i < P.u; ++i) bulk_g2s(da + i * wbytes, a + i * P.a_wstride * kTileBytes, wbytes, &full[slot]);
            }
            bulk_g2s(dst, b, kTileB, &full[slot]);
            return;
        }
        const int i = catB ? pair : pair / P.v;
        const uint8_t *a = P.Aw + (i * P.a_wstride + kb * P.a_kstride + row0) * kTileBytes;
        if (!catB) {
            const int j = pair % P.v;
            const uint8_t *b = P.Bw + (j * P.b_wstride + kb * P.b_kstride + col0) * kTileBytes;
            mbar_arrive_expect_tx(&full[slot], kTileA + kTileB);
            bulk_g2s(sA + slot * kTileA, a, kTileA, &full[slot]);
            bulk_g2s(dst, b, kTileB, &full[slot]);
            return;
        }
        // slots j = 0 .. v-1 of w rows each; slots >= v stay unloaded (their
        // columns are never used)
        const uint32_t wbytes = (uint32_t)P.w * kTileBytes;
        const uint8_t *b = P.Bw + (kb * P.b_kstride + col0) * kTileBytes;
        mbar_arrive_expect_tx(&full[slot], kTileA + (uint32_t)P.v * wbytes);
        bulk_g2s(sA + slot * kTileA, a, kTileA, &full[slot]);
        if (P.B_rows == P.w) {  // one column tile: the v slots are adjacent
            bulk_g2s(dst, b, (uint32_t)P.v * wbytes, &full[slot]);
        } else {
            for (int j = 0; j < P.v; ++j) bulk_g2s(dst + j * wbytes, b + j * P.b_wstride * kTileBytes, wbytes, &full[slot]);
        }
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

        const int64_t kb = vb % kbn;  // k-block within the range
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
        if (kb == kbn - 1) {  // word pair(s) complete: recombine (Alg. 5 / Alg. 6 with Alg. 2)
            const int pair = (int)(vb / kbn);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    // gamma index i v + j: i or j from the row's / column's word slot when concatenated
                    const int i = catA ? (ty + 16 * r) / P.w : catB ? pair : pair / P.v;
                    const int j = catB ? (tx + 16 * c) / P.w : catA ? pair : pair % P.v;
                    if (i >= P.u || j >= P.v) continue;  // unused slot
                    const int gi = i * P.v + j;
                    const double g = P.gamma[gi], g26 = P.gamma26[gi];
                    const double T = fmod_alg1(acc[r][c], p, q);
                    double e;
                    if (gi == 0) e = T;  // gamma_00 = 1
                    else if (!P.big_p) e = mulmod_alg2(g, T, p, q);
                    else e = mulmod_split(g, g26, T, p, q);
                    double s = __dadd_rn(cres[r][c], e);
                    if (s >= p) s = __dsub_rn(s, p);
                    cres[r][c] = s;
                }
            }
        }
        __syncthreads();
    }

    uint64_t *out = P.C;
    int64_t ld = P.ldc;
    if (P.part) {  // partial result of K range z
        out = P.part + z * P.m * P.n;
        ld = P.n;
    }
    if (catA) {
        // row ty + 16 r is output row (ty + 16 r) mod w of word slot
        // (ty + 16 r) / w; add the slots of each output row (w = 32: r and
        // r + 2; w = 16: all four)
        const bool two = P.w == 32;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t col = col0 + tx + 16 * c;
            if (col >= P.n) continue;
            double s0 = 0.0, s1 = 0.0;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if ((ty + 16 * r) / P.w >= P.u) continue;
                if (two && (r & 1)) {
                    s1 = __dadd_rn(s1, cres[r][c]);
                    if (s1 >= p) s1 = __dsub_rn(s1, p);
                } else {
                    s0 = __dadd_rn(s0, cres[r][c]);
                    if (s0 >= p) s0 = __dsub_rn(s0, p);
                }
            }
            if (row0 + ty < P.m) out[(row0 + ty) * ld + col] = (uint64_t)s0;
            if (two && row0 + ty + 16 < P.m) out[(row0 + ty + 16) * ld + col] = (uint64_t)s1;
        }
        return;
    }
    if (catB) {
        // column tx + 16 c is output column (tx + 16 c) mod w of word slot
        // (tx + 16 c) / w; add the slots of each output column (w = 32: c and
        // c + 2; w = 16: all four)
        const bool two = P.w == 32;  // output columns per thread and row: 2 (w = 32) or 1 (w = 16)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t row = row0 + ty + 16 * r;
            if (row >= P.m) continue;
            double s0 = 0.0, s1 = 0.0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if ((tx + 16 * c) / P.w >= P.v) continue;
                if (two && (c & 1)) {
                    s1 = __dadd_rn(s1, cres[r][c]);
                    if (s1 >= p) s1 = __dsub_rn(s1, p);
                } else {
                    s0 = __dadd_rn(s0, cres[r][c]);
                    if (s0 >= p) s0 = __dsub_rn(s0, p);
                }
            }
            if (col0 + tx < P.n) out[row * ld + col0 + tx] = (uint64_t)s0;
            if (two && col0 + tx + 16 < P.n) out[row * ld + col0 + tx + 16] = (uint64_t)s1;
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t row = row0 + ty + 16 * r;
        if (row >= P.m) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t col = col0 + tx + 16 * c;
            if (col < P.n) out[row * ld + col] = (uint64_t)cres[r][c];
        }
    }
}

// C = sum over the K ranges of their partial results, mod p (exact integer
// additions of values < p).
__global__ void fp64_range_sum_kernel(const uint64_t *part, int ranges, int64_t m, int64_t n, uint64_t p,
                                      uint64_t *C, int64_t ldc) {
    const int64_t mn = m * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < mn; e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t s = 0;
        for (int z = 0; z < ranges; ++z) {
            s += __ldcs(part + z * mn + e);
            if (s >= p) s -= p;
        }
        const int64_t r = e / n, c = e - r * n;
        C[r * ldc + c] = s;
    }
}

__global__ void __launch_bounds__(THREADS) gemm_fp64_kernel(const __grid_constant__ F64Params P) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[STAGES];
    fp64_tile(P, blockIdx.y, blockIdx.x, blockIdx.z, smem, full);
}

// Batched: block b computes tile (row block y, col tile x) over K range z of
// problem probs[jobs[b].x] with jobs[b] = (problem, y, x, z).
__global__ void __launch_bounds__(THREADS) gemm_fp64_batched_kernel(const F64Params *probs, const int4 *jobs) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[STAGES];
    const int4 j = jobs[blockIdx.x];
    fp64_tile(probs[j.x], j.y, j.z, j.w, smem, full);
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
    P.kbr = pl.kbr;
    P.b_wstride = pl.B_wstride;
    P.b_kstride = pl.B_kstride;
    P.a_wstride = pl.A_wstride;
    P.a_kstride = pl.A_kstride;
    P.part = nullptr;
    P.u = pl.u;
    P.v = pl.v;
    P.concat = pl.f64_concat;
    P.w = pl.f64_w;
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

int64_t col_tiles(const Plan &pl) { return pl.f64_concat == 1 ? pl.B_rows / pl.f64_w : pl.B_rows / BN; }
int64_t row_tiles(const Plan &pl) { return pl.f64_concat == 2 ? pl.A_rows / pl.f64_w : pl.A_rows / BM; }

}  // namespace

size_t fp64_job_bytes() { return sizeof(F64Params); }

int prepare_tc_attributes();

int prepare_kernel_attributes() {
    const int smem = STAGES * (kTileA + kTileB);
    cudaError_t e = set_smem_attr(reinterpret_cast<const void *>(gemm_fp64_kernel), smem);
    if (e == cudaSuccess) e = set_smem_attr(reinterpret_cast<const void *>(gemm_fp64_batched_kernel), smem);
    if (e != cudaSuccess) return (int)e;
    e = (cudaError_t)prepare_tc_fused_attributes();
    if (e != cudaSuccess) return (int)e;
    return prepare_tc_attributes();
}

// Batched products run one K range (plans made with ksplit = 1).
void fp64_job(const Plan &pl, const void *Aw, const void *Bw, uint64_t *C, int64_t ldc, int *err, void *rec,
              int index, std::vector<int> &jobs) {
    const F64Params P = make_f64_params(pl, Aw, Bw, C, ldc, err);
    std::memcpy(rec, &P, sizeof(P));
    for (int64_t y = 0; y < row_tiles(pl); ++y)
        for (int64_t x = 0; x < col_tiles(pl); ++x) {
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

int launch_gemm_fp64(const Plan &pl, const void *Aw, const void *Bw, uint64_t *C, int64_t ldc, uint64_t *part,
                     int *err, void *stream) {
    F64Params P = make_f64_params(pl, Aw, Bw, C, ldc, err);
    if (pl.ksplit > 1) {
        if (!part) return (int)cudaErrorInvalidValue;
        P.part = part;
    }
    const int smem = STAGES * (kTileA + kTileB);
    cudaError_t e = set_smem_attr(reinterpret_cast<const void *>(gemm_fp64_kernel), smem);
    if (e != cudaSuccess) return (int)e;
    if (row_tiles(pl) > 65535) return (int)cudaErrorInvalidConfiguration;  // grid y limit: m <= 4194240
    dim3 grid((unsigned)col_tiles(pl), (unsigned)row_tiles(pl), (unsigned)pl.ksplit);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    gemm_fp64_kernel<<<grid, THREADS, smem, s>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess || pl.ksplit == 1) return (int)e;
    const int64_t mn = pl.m * pl.n;
    const int64_t blocks = (mn + 255) / 256 < 4 * 148 ? (mn + 255) / 256 : 4 * 148;
    fp64_range_sum_kernel<<<(unsigned)blocks, 256, 0, s>>>(part, pl.ksplit, pl.m, pl.n, pl.p, C, ldc);
    return (int)cudaGetLastError();
}

}  // namespace mwmm
