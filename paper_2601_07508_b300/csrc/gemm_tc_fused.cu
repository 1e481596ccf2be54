// INT8-word form with the reduction and the recombination fused into the
// word-product kernel: C = sum_s R^s S_s mod p (R the digit radix) is accumulated in the
// epilogue as each diagonal sum S_s = sum_{i+j=s} A_i B_j completes, so no
// sum ever leaves the SM (Alg. 5 scales and accumulates each word product as
// it completes; here the products of one diagonal are first summed exactly,
// then folded in).
//
// Recombination (Horner's rule, exact integer arithmetic).  A work unit owns
// a 256 x 128 output tile (a CTA pair, 128 rows each) over a range of k and
// visits the diagonals from the top one down:
//     r <- (R r + S_s) mod p,      s = u + v - 2, ..., 0,
// (R = 2^8 or 2^9, the digit radix) with r < p held in tensor memory beside
// the accumulators (two 32-bit columns per output), so after s = 0,
// r = sum_s R^s S_s mod p.  One step is y = R r + S_s + off,
// off = p ceil(2^31 / p) (so y >= 0 and y < 2^62), reduced by a Barrett
// quotient (at most two corrections).
//
// Segments.  The k-range of a unit is cut into segments of `seg` k-blocks and
// the unit runs segment by segment, every diagonal in each, so that the word
// tiles the ~74 concurrent units read at one time -- the A and B words of
// one segment -- stay in L2 while every diagonal that needs them runs.  Each
// segment's sums are folded in by the same rule; between segments the
// residue is divided by R^nsums mod p (Montgomery steps of <= 11 bits:
// r <- (r + t p) / 2^b with t = r (-p^-1) mod 2^b, exact and < p), because
// the next segment's Horner pass multiplies it by R^nsums again.  The
// INT32 sums S_s of one segment hold ni x seg x 64 products of magnitude
// <= 2^14 (2^16 for 9-bit digits; ni <= min(u, v) pairs), within the same
// INT32 bound as the unfused form's K-range.
//
// K parts.  When the output has too few tiles to fill the GPU, K is split
// into parts computed by separate units; each writes its residue to a plane
// of partial results and a last kernel adds them mod p.
//
// Exactness of the word products is that of the unfused kernel (gemm_tc.cu):
// digits of magnitude <= 128 in bf16 (<= 256 in fp16), FP32 tensor-memory
// chunks of at most 1024 (256) products, so partial sums stay <= 2^24,
// drained into INT32 registers.
//
// Warp roles (320 threads per CTA, two CTAs per cluster):
//   warp 0      (both CTAs) TMA producer: the CTA's 128 A rows (16 KB) and
//               its half of the 128 B rows (8 KB) per stage, 8 stages; the
//               bytes complete on the leader CTA's barrier;
//   warp 1      allocates 512 TMEM columns (both CTAs): accumulators at
//               [0, 128) and [128, 256), residue low / high words at
//               [256, 384) and [384, 512); in the leader, one lane issues
//               tcgen05.mma.cta_group::2 (256 x 128 x 16);
//   warps 2-9   (both CTAs) drain a finished chunk into INT32 registers
//               (warp w: TMEM lanes 32 (w mod 4) .., columns 64 ((w-2)/4) ..),
//               and at the end of a diagonal fold it into the residue; after
//               the last diagonal store C (or the K part's partial plane).
// Every wait is bounded; a timeout raises the error flag and all roles leave.
#include <cstring>

#include "mwmm_internal.h"
#include "tcgen05.cuh"

namespace mwmm {

namespace {

constexpr int FS = 8;                                   // pipeline stages
constexpr int FBM = 128;                                // rows per CTA (TMEM lanes)
constexpr int FBN = 128;                                // columns of a tile (MMA N)
constexpr int EPI = 8;                                  // epilogue warps per CTA
constexpr int FTHREADS = 32 * (2 + EPI);
constexpr uint32_t kTA = FBM * kTileBytes;              // 16 KB: the CTA's A rows
constexpr uint32_t kTB = (FBN / 2) * kTileBytes;        // 8 KB: the CTA's half of B
constexpr int kStg = 20;                                // staging row stride (32-bit words)
constexpr uint32_t kStgBytes = EPI * 32 * kStg * 4;     // 20 KB
constexpr int kSmem = FS * (kTA + kTB) + kStgBytes + 1024;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColRlo = 256, kColRhi = 384;
constexpr int64_t kGroupN = 8;                          // column tiles per raster group

struct FusedParams {
    int64_t nkb, A_rows, B_rows;  // word layout (plain, k-block minor)
    int64_t m, n, ldc, ldr;
    int u, v, nsums;
    int mt2_count, nt_count;      // 256-row and 128-column tiles
    int64_t ntiles, nunits;       // nunits = ntiles * kparts
    int64_t kbr;                  // k-blocks per K part
    int kparts, seg, chunk_blocks;
    int hop_bits;                 // rbits nsums
    int rbits;                    // digit width (radix 2^rbits)
    uint32_t idesc;               // MMA descriptor (bf16 or fp16 words)
    uint32_t pinv11;              // -p^-1 mod 2^11
    int vec_c;                    // C and ldc allow 16-byte stores of two outputs
    uint64_t p, mu, off;          // mu = floor((2^64 - 1) / p), off = p ceil(2^31 / p)
    uint64_t *C, *R;              // output; partial planes [kparts][m][ldr] when kparts > 1
    int *err;
};

struct Unit {
    int64_t mt2, nt, kb0, nkbu;
    int kpart;
};

__device__ __forceinline__ Unit unit_at(const FusedParams &P, int64_t idx) {
    Unit U;
    U.kpart = (int)(idx / P.ntiles);
    const int64_t tile = idx - (int64_t)U.kpart * P.ntiles;
    // raster in groups of kGroupN column tiles, rows first inside a group
    const int64_t gsz = (int64_t)P.mt2_count * kGroupN;
    const int64_t grp = tile / gsz, t = tile - grp * gsz;
    const int64_t left = P.nt_count - grp * kGroupN;
    const int64_t width = left < kGroupN ? left : kGroupN;
    U.mt2 = t / width;
    U.nt = grp * kGroupN + (t - U.mt2 * width);
    U.kb0 = (int64_t)U.kpart * P.kbr;
    const int64_t rest = P.nkb - U.kb0;
    U.nkbu = rest < P.kbr ? rest : P.kbr;
    return U;
}

__device__ __forceinline__ int pair_lo(const FusedParams &P, int s) { return s - (P.v - 1) > 0 ? s - (P.v - 1) : 0; }
__device__ __forceinline__ int pair_hi(const FusedParams &P, int s) { return s < P.u - 1 ? s : P.u - 1; }

// y mod p for y < 2^64: the Barrett quotient umulhi(y, mu) is short by at
// most 2.
__device__ __forceinline__ uint64_t reduce_barrett(uint64_t y, uint64_t p, uint64_t mu) {
    uint64_t r = y - __umul64hi(y, mu) * p;
    if (r >= p) r -= p;
    if (r >= p) r -= p;
    return r;
}

// One Horner step: (R r + S) mod p for r < p < 2^52, R = 2^rbits <= 2^9 and
// |S| < 2^31 (y < 2^61 + 2^53).
__device__ __forceinline__ uint64_t horner(uint64_t r, int32_t S, const FusedParams &P) {
    return reduce_barrett((r << P.rbits) + (uint64_t)((int64_t)S + (int64_t)P.off), P.p, P.mu);
}

// r 2^-bits mod p for r < p (odd p), in Montgomery steps of at most 11 bits.
__device__ __forceinline__ uint64_t div_pow2_mod(uint64_t r, const FusedParams &P) {
    for (int bits = P.hop_bits; bits > 0; bits -= 11) {
        const int b = bits < 11 ? bits : 11;
        const uint32_t mask = (1u << b) - 1u;
        const uint32_t t = (((uint32_t)r & mask) * P.pinv11) & mask;
        r = (r + (uint64_t)t * P.p) >> b;
    }
    return r;
}

// Store 8 residues of this lane's row (columns col0 .. col0 + 7, halves in
// lo / hi) through the warp's staging area: the block is written by rows and
// read back with four lanes per row, so a store instruction covers 8 rows x
// 64 contiguous bytes.  row0 = the warp's first output row.
__device__ __forceinline__ void store_residues(const FusedParams &P, const Unit &U, const uint32_t (&lo)[8],
                                               const uint32_t (&hi)[8], uint32_t *stg, int lane, int64_t row0,
                                               int64_t col0) {
    uint64_t *base;
    int64_t ld;
    bool vec;
    if (P.kparts == 1) {
        base = P.C;
        ld = P.ldc;
        vec = P.vec_c != 0;
    } else {
        base = P.R + (int64_t)U.kpart * P.m * P.ldr;
        ld = P.ldr;
        vec = true;  // ldr is even and the planes are 256-byte aligned
    }
    __syncwarp();  // the previous block's reads are done
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4 *>(stg + lane * kStg + 4 * q) =
            make_uint4(lo[2 * q], hi[2 * q], lo[2 * q + 1], hi[2 * q + 1]);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = i * 8 + (lane >> 2), g = lane & 3;
        const uint4 w = *reinterpret_cast<const uint4 *>(stg + r * kStg + 4 * g);
        const int64_t row = row0 + r, col = col0 + 2 * g;
        if (row >= P.m || col >= P.n) continue;
        const uint64_t a = ((uint64_t)w.y << 32) | w.x, b = ((uint64_t)w.w << 32) | w.z;
        uint64_t *out = base + row * ld + col;
        if (vec && col + 1 < P.n) {
            __stcs(reinterpret_cast<ulonglong2 *>(out), make_ulonglong2(a, b));
        } else {
            __stcs(out, a);
            if (col + 1 < P.n) __stcs(out + 1, b);
        }
    }
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(FTHREADS, 1)
    gemm_tc_fused_kernel(const __grid_constant__ FusedParams P, const __grid_constant__ CUtensorMap tmA,
                         const __grid_constant__ CUtensorMap tmB) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[FS], empty[FS], tfull[2], tempty[2], done;
    __shared__ uint32_t tmem_base_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    uint8_t *sA = smem_raw + pad;
    uint8_t *sB = sA + FS * kTA;
    uint32_t *sStage = reinterpret_cast<uint32_t *>(sB + FS * kTB);

    if (threadIdx.x == 0) {
        for (int s = 0; s < FS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 2 * EPI);  // both CTAs' epilogue warps (the leader's copy counts)
        }
        mbar_init(&done, 1);
        fence_mbar_init();
    }
    if (warp == 1) {  // one warp of each CTA of the pair allocates, collectively
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    cluster_sync_all();  // barriers of both CTAs initialised, TMEM allocated
    tc_fence_after();
    const uint32_t tmem_base = tmem_base_sh;
    const int64_t cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;

    if (warp == 0) {
        if (lane == 0) {  // ---------------- TMA producer (both CTAs)
            const uint32_t lead_full = peer_addr(&full[0], 0);
            uint64_t g = 0;
            bool alive = true;
            for (int64_t idx = cid; alive && idx < P.nunits; idx += ncl) {
                const Unit U = unit_at(P, idx);
                for (int64_t seg0 = 0; alive && seg0 < U.nkbu; seg0 += P.seg) {
                    const int64_t segl = U.nkbu - seg0 < P.seg ? U.nkbu - seg0 : P.seg;
                    for (int s = P.nsums - 1; alive && s >= 0; --s) {
                        const int hi = pair_hi(P, s);
                        for (int i = pair_lo(P, s); alive && i <= hi; ++i) {
                            // row coordinates of the tensor maps (the host checks they fit int32)
                            int32_t ya = (int32_t)(((int64_t)i * P.nkb + U.kb0 + seg0) * P.A_rows + U.mt2 * (2 * FBM) +
                                                   rank * FBM);
                            int32_t yb = (int32_t)(((int64_t)(s - i) * P.nkb + U.kb0 + seg0) * P.B_rows + U.nt * FBN +
                                                   rank * (FBN / 2));
                            for (int64_t kb = 0; kb < segl;
                                 ++kb, ++g, ya += (int32_t)P.A_rows, yb += (int32_t)P.B_rows) {
                                const int slot = (int)(g % FS);
                                if (!mbar_wait(&empty[slot], (uint32_t)(((g / FS) & 1) ^ 1), P.err)) {
                                    alive = false;
                                    break;
                                }
                                if (leader) mbar_arrive_expect_tx(&full[slot], 2 * (kTA + kTB));
                                const uint32_t bar = lead_full + (uint32_t)(slot * sizeof(uint64_t));
                                tma2_load_pair(sA + slot * kTA, &tmA, ya, bar);
                                tma2_load_pair(sB + slot * kTB, &tmB, yb, bar);
                            }
                        }
                    }
                }
            }
            // Before exit: the leader sees every byte of both CTAs land; both
            // wait for the leader's last commit to each slot.
            for (int s = 0; s < FS; ++s) {
                const uint64_t armed = g > (uint64_t)s ? (g - s + FS - 1) / FS : 0;
                if (!armed) continue;
                if (leader) mbar_wait(&full[s], (uint32_t)((armed - 1) & 1), P.err);
                mbar_wait(&empty[s], (uint32_t)((armed - 1) & 1), P.err);
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {  // ---------------- MMA issuer (leader)
            uint64_t g = 0, c = 0;
            bool alive = true;
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
            for (int64_t idx = cid; alive && idx < P.nunits; idx += ncl) {
                const Unit U = unit_at(P, idx);
                for (int64_t seg0 = 0; alive && seg0 < U.nkbu; seg0 += P.seg) {
                    const int64_t segl = U.nkbu - seg0 < P.seg ? U.nkbu - seg0 : P.seg;
                    for (int s = P.nsums - 1; alive && s >= 0; --s) {
                        const int64_t nvb = (int64_t)(pair_hi(P, s) - pair_lo(P, s) + 1) * segl;
                        for (int64_t t0 = 0; alive && t0 < nvb; t0 += P.chunk_blocks, ++c) {
                            const int buf = (int)(c & 1);
                            if (!mbar_wait(&tempty[buf], (uint32_t)(((c >> 1) & 1) ^ 1), P.err)) {
                                alive = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t dt = tmem_base + (uint32_t)(buf * FBN);
                            const int64_t tend = t0 + P.chunk_blocks < nvb ? t0 + P.chunk_blocks : nvb;
                            for (int64_t t = t0; t < tend; ++t, ++g) {
                                const int slot = (int)(g % FS);
                                if (!mbar_wait(&full[slot], (uint32_t)((g / FS) & 1), P.err)) {
                                    alive = false;
                                    break;
                                }
                                tc_fence_after();
                                const uint64_t ad = sdesc(a0 + slot * kTA), bd = sdesc(b0 + slot * kTB);
#pragma unroll
                                for (int kk = 0; kk < 4; ++kk)  // K = 16 per MMA: +32 bytes = +2 in the address field
                                    mma_bf16_pair(dt, ad + 2 * kk, bd + 2 * kk, P.idesc, (t > t0 || kk > 0) ? 1u : 0u);
                                mma_commit_pair(&empty[slot], 3);
                            }
                            mma_commit_pair(&tfull[buf], 3);
                        }
                    }
                }
            }
            mma_commit_pair(&done, 1);
            mbar_wait(&done, 0, P.err);
        }
    } else {  // -------------------------------- epilogue warps 2..9 (both CTAs)
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const uint32_t tl = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 64);
        const uint32_t lead_tempty = peer_addr(&tempty[0], 0);
        uint32_t *stg = sStage + (warp - 2) * (32 * kStg);
        uint64_t c = 0;
        bool alive = true;
        for (int64_t idx = cid; alive && idx < P.nunits; idx += ncl) {
            const Unit U = unit_at(P, idx);
            const int64_t row0 = U.mt2 * (2 * FBM) + rank * FBM + quarter * 32;
            bool first = true;
            for (int64_t seg0 = 0; alive && seg0 < U.nkbu; seg0 += P.seg) {
                const int64_t segl = U.nkbu - seg0 < P.seg ? U.nkbu - seg0 : P.seg;
                for (int s = P.nsums - 1; alive && s >= 0; --s) {
                    const int64_t nvb = (int64_t)(pair_hi(P, s) - pair_lo(P, s) + 1) * segl;
                    const int64_t nch = (nvb + P.chunk_blocks - 1) / P.chunk_blocks;
                    int32_t acc[64];
#pragma unroll
                    for (int e = 0; e < 64; ++e) acc[e] = 0;
                    int buf = 0;
                    for (int64_t ch = 0; ch < nch; ++ch, ++c) {
                        buf = (int)(c & 1);
                        const bool ok = mbar_wait(&tfull[buf], (uint32_t)((c >> 1) & 1), P.err);
                        if (!__all_sync(0xffffffffu, ok)) {
                            alive = false;
                            break;
                        }
                        tc_fence_after();
#pragma unroll
                        for (int jb = 0; jb < 2; ++jb) {
                            uint32_t r[32];
                            tmem_ld32(tl + (uint32_t)(buf * FBN + jb * 32), r);
#pragma unroll
                            for (int e = 0; e < 32; ++e) acc[jb * 32 + e] += __float2int_rn(__uint_as_float(r[e]));
                        }
                        if (ch + 1 < nch) {  // the last buffer is released after the fold below
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive_cluster(lead_tempty + (uint32_t)(buf * sizeof(uint64_t)));
                        }
                    }
                    if (!alive) break;
                    // Fold S_s into the residue (Horner).  S_s goes back into
                    // this warp's columns of the drained buffer (the MMAs
                    // fill the other one meanwhile), so the fold runs 8
                    // columns at a time from tensor memory with few live
                    // registers.
                    {
                        uint32_t w[32];
#pragma unroll
                        for (int e = 0; e < 32; ++e) w[e] = (uint32_t)acc[e];
                        tmem_st32(tl + (uint32_t)(buf * FBN), w);
#pragma unroll
                        for (int e = 0; e < 32; ++e) w[e] = (uint32_t)acc[32 + e];
                        tmem_st32(tl + (uint32_t)(buf * FBN + 32), w);
                        tmem_st_wait();
                    }
                    const bool hop = seg0 > 0 && s == P.nsums - 1;
                    const bool last = s == 0 && seg0 + segl >= U.nkbu;
#pragma unroll 1
                    for (int jb = 0; jb < 8; ++jb) {
                        uint32_t sv[8], lo[8], hi[8];
                        tmem_ld8(tl + (uint32_t)(buf * FBN + jb * 8), sv);
                        if (!first) {
                            tmem_ld8(tl + kColRlo + (uint32_t)(jb * 8), lo);
                            tmem_ld8(tl + kColRhi + (uint32_t)(jb * 8), hi);
                        }
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            uint64_t r = first ? 0 : (((uint64_t)hi[e] << 32) | lo[e]);
                            if (hop) r = div_pow2_mod(r, P);
                            r = horner(r, (int32_t)sv[e], P);
                            lo[e] = (uint32_t)r;
                            hi[e] = (uint32_t)(r >> 32);
                        }
                        if (last) {
                            store_residues(P, U, lo, hi, stg, lane, row0, U.nt * FBN + half * 64 + jb * 8);
                        } else {
                            tmem_st8(tl + kColRlo + (uint32_t)(jb * 8), lo);
                            tmem_st8(tl + kColRhi + (uint32_t)(jb * 8), hi);
                        }
                    }
                    if (!last) tmem_st_wait();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive_cluster(lead_tempty + (uint32_t)(buf * sizeof(uint64_t)));
                    first = false;
                }
            }
        }
    }

    tc_fence_before();
    cluster_sync_all();  // no CTA frees TMEM or exits while its peer may still signal it
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                     : "memory");
}

// C = sum of the K parts' residues mod p (each < p).
__global__ void __launch_bounds__(256) fused_part_sum_kernel(const uint64_t *R, int parts, int64_t m, int64_t n,
                                                             int64_t ldr, uint64_t p, uint64_t *C, int64_t ldc) {
    const int64_t plane = m * ldr;
    for (int64_t row = blockIdx.y; row < m; row += gridDim.y)
        for (int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; col < n;
             col += (int64_t)gridDim.x * blockDim.x) {
            uint64_t s = 0;
            for (int z = 0; z < parts; ++z) {
                s += __ldcs(R + z * plane + row * ldr + col);
                if (s >= p) s -= p;
            }
            C[row * ldc + col] = s;
        }
}

int fused_clusters() {
    static int cached[64] = {0};
    return max_clusters2(reinterpret_cast<const void *>(gemm_tc_fused_kernel), FTHREADS, kSmem, cached);
}

}  // namespace

int prepare_tc_fused_attributes() {
    cudaError_t e = set_smem_attr(reinterpret_cast<const void *>(gemm_tc_fused_kernel), kSmem);
    if (e == cudaSuccess) (void)fused_clusters();
    return (int)e;
}

int launch_gemm_tc_fused(const Plan &pl, const void *Aw, const void *Bw, uint64_t *C, int64_t ldc, uint64_t *R,
                         int *err, void *stream) {
    FusedParams P;
    std::memset(&P, 0, sizeof(P));
    P.nkb = pl.nkb;
    P.A_rows = pl.A_rows;
    P.B_rows = pl.B_rows;
    P.m = pl.m;
    P.n = pl.n;
    P.ldc = ldc;
    P.ldr = pl.tc_ldr;
    P.u = pl.u;
    P.v = pl.v;
    P.nsums = pl.nsums;
    P.mt2_count = (int)(pl.A_rows / (2 * FBM));
    P.nt_count = (int)(pl.B_rows / FBN);
    P.ntiles = (int64_t)P.mt2_count * P.nt_count;
    P.kparts = pl.ksplit;
    P.nunits = P.ntiles * P.kparts;
    P.kbr = pl.kbr;
    P.seg = pl.tc_seg;
    P.chunk_blocks = (int)(pl.tc_chunk / kTcKB);
    P.rbits = pl.digit_bits;
    P.hop_bits = pl.digit_bits * pl.nsums;
    P.idesc = pl.digit_bits == 9 ? idesc_f16(2 * FBM, FBN) : idesc_bf16(2 * FBM, FBN);
    P.p = pl.p;
    P.mu = ~uint64_t(0) / pl.p;
    P.off = pl.p * ((((uint64_t)1 << 31) + pl.p - 1) / pl.p);
    // -p^-1 mod 2^11 by Newton's iteration on the inverse (p odd)
    uint32_t inv = (uint32_t)pl.p;  // correct to 3 bits
    for (int it = 0; it < 4; ++it) inv *= 2u - (uint32_t)pl.p * inv;
    P.pinv11 = (0u - inv) & 0x7FFu;
    P.vec_c = ((reinterpret_cast<uintptr_t>(C) & 15) == 0 && (ldc & 1) == 0) ? 1 : 0;
    P.C = C;
    P.R = R;
    P.err = err;
    if (P.nunits == 0) return 0;
    cudaError_t e = set_smem_attr(reinterpret_cast<const void *>(gemm_tc_fused_kernel), kSmem);
    if (e != cudaSuccess) return (int)e;
    const int clusters = fused_clusters();
    if (clusters <= 0) return (int)cudaErrorLaunchOutOfResources;
    const int64_t ncl = P.nunits < clusters ? P.nunits : clusters;
    CUtensorMap tmA, tmB;
    int r = encode_rows_map(&tmA, Aw, (uint64_t)pl.u * pl.nkb * pl.A_rows, FBM);
    if (r == 0) r = encode_rows_map(&tmB, Bw, (uint64_t)pl.v * pl.nkb * pl.B_rows, FBN / 2);
    if (r != 0) return r;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    gemm_tc_fused_kernel<<<(unsigned)(2 * ncl), FTHREADS, kSmem, s>>>(P, tmA, tmB);
    e = cudaGetLastError();
    if (e != cudaSuccess || P.kparts == 1) return (int)e;
    const unsigned gx = (unsigned)((pl.n + 255) / 256);
    const unsigned gy = (unsigned)(pl.m < 4096 ? pl.m : 4096);
    fused_part_sum_kernel<<<dim3(gx, gy), 256, 0, s>>>(R, P.kparts, pl.m, pl.n, pl.tc_ldr, pl.p, C, ldc);
    return (int)cudaGetLastError();
}

}  // namespace mwmm
