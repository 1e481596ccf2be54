// INT8-word form on the tcgen05 tensor pipe (sm_103a).
//
// Computes the diagonal word sums S_s = sum_{i+j=s} A_i B_j (exact integers)
// of the INT8 digit decomposition; recombine.cu then forms
// C = sum_s 256^s S_s mod p.  This is the paper's second perspective (Sec. 6):
// narrower words, more of them, multiplied on tensor cores.
//
// Exactness.  sm_103a's tcgen05 has no INT8 kind, so the digits (integers of
// magnitude <= 128) are carried exactly in bf16 and multiplied with
// tcgen05.mma.kind::f16 into FP32 tensor memory.  Every product is an integer
// of magnitude <= 2^14, so as long as a chunk sums at most 1024 of them every
// partial sum is an integer of magnitude <= 2^24, which FP32 represents
// exactly whatever the order or alignment of the additions: the block
// condition of Prop. 2.3 with a 24-bit significand in place of 53 bits.  Each
// chunk is drained from tensor memory into INT32 registers (the K-chunking of
// Alg. 3, with the reduction postponed to the exact integer recombination).
//
// Schedule.  Work item = (128-row tile, 256-col tile, diagonal s, K-range kc);
// its k-loop runs over the virtual k-blocks (pair (i, s-i), 64-wide k-block):
// the pairs of one diagonal are concatenated along K (the K-dimension analogue
// of Alg. 6's concatenation).  A persistent grid of one CTA per SM claims
// items in order from a counter in the workspace (the producer warp claims
// and hands the index to the MMA and epilogue warps through a small ring in
// shared memory), so uneven item costs balance themselves.  Items go window
// by window, heaviest first (the kernel ends on its lightest items), every
// tile of a window in a raster of kGroupN column tiles; inside an item the
// k-block is the outer loop and the diagonal's pairs the inner one, so a
// wave of items walks through k in step and shares each k-slab of words in
// L2.
//
// Warp roles (320 threads):
//   warp 0      one lane issues bulk TMA copies of the pre-swizzled word tiles
//               (A 16 KB + B 32 KB per stage, 4 stages);
//   warp 1      allocates 512 TMEM columns (two 128 x 256 FP32 accumulators);
//               one lane issues 4 MMAs (128 x 256 x 16) per stage;
//   warps 2-9   drain a finished accumulator (warp w reads TMEM lanes
//               32 (w mod 4) .. +31, columns half (w-2)/4), convert to INT32,
//               sum the chunks of an item, store S_s.
// Every wait is bounded (device_common.cuh); a timeout raises the plan's
// error flag and all roles leave their loops.
#include <cuda_bf16.h>

#include <cstring>

#include "mwmm_internal.h"
#include "tcgen05.cuh"

namespace mwmm {

namespace {

constexpr int BM = kTcBM;  // 128
constexpr int BN = kTcBN;  // 256
constexpr int STAGES = 4;
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 32 * (3 + EPI_WARPS);       // one-CTA kernel: + the planner warp (warp 10)
constexpr int THREADS_PAIR = THREADS;              // pair kernel: the same roles
constexpr int PLANNER_WARP = 2 + EPI_WARPS;
constexpr int kCertBlocks = 8;  // certified chunk: 8 k-block x pair steps (512 products of 9-bit digits)
constexpr uint32_t kTileA = BM * kTileBytes;  // 16 KB
constexpr uint32_t kTileB = BN * kTileBytes;  // 32 KB
constexpr uint32_t kTmemCols = 2 * BN;        // 512: two accumulator buffers
// Epilogue staging: per epilogue warp, 32 rows x 16 columns of INT32 sums
// with a row stride of 20 words (80 bytes: 128-bit accesses by 8 lanes at a
// time, rows or columns, touch all 32 banks once).
constexpr int kStgStride = 20;
constexpr uint32_t kStageBytes = EPI_WARPS * 32 * kStgStride * 4;  // 20 KB
constexpr int kSmemBytes = STAGES * (kTileA + kTileB) + kStageBytes + 1024;
constexpr int64_t kGroupN = 8;  // column tiles per raster group
constexpr int kRing = 2;  // claimed items in flight (planner -> producer, MMA and epilogue warps)

struct TcParams {
    // computed items (one product)
    const uint8_t *Aw, *Bw;
    int32_t *S;
    int64_t nkb, A_rows, B_rows, kcb, nitems;
    int u, v, nsums, nkc, mt_count, nt_count, nb, b_wpad;
    int f16;       // words in fp16 (9-bit digits), else bf16
    int64_t m, n;  // valid rows and columns (sums outside are not stored)
    int64_t b_wstride, b_kstride;  // bytes between consecutive B words / k-blocks
    uint32_t *sched;  // item counter of the computed items, zero at launch
    // diagonal windows, heaviest first: window g covers diagonals
    // g_s0[g] .. g_s0[g] + g_nd[g] - 1 and A words g_i0[g] .. + g_ni[g] - 1;
    // its sums start at S plane g_plane[g] (the diagonal s0; the modulus i of
    // the CRT form, whose window is the single pair (i, i) with s0 = 2 i)
    int g_s0[kMaxWindows], g_nd[kMaxWindows], g_i0[kMaxWindows], g_ni[kMaxWindows], g_plane[kMaxWindows];
    // table items (batch): items[0 .. nitems), claimed in table order
    const TcItem *items;
    const int64_t *cta_off;
    int chunk_blocks;
    int *err;
    // certified chunks (computed items only): squared-digit maxima of the
    // splits ([word][k-block][64-row group]), nullptr: worst-case chunks
    const uint32_t *sqA, *sqB;
    int cert;  // some item may run certified chunks: the planner warp claims (else the producer lane)
    // computed items: every second run of `wave` claims (one per resident CTA
    // or CTA pair) walks its k-blocks last to first; 0: all first to last
    int64_t wave;
};

// One work item with everything the three roles need (see TcItem).
struct Item {
    const uint8_t *Aw, *Bw;
    int32_t *S;  // S of diagonal s0 at the item's tile origin, row stride B_rows
    int64_t A_rows, B_rows, nkb, kb0, nkbc, mt, nt, plane, b_wstride, b_kstride;
    int s0, ndiag, nb, i0, ni, v, b_wpad;
    int rv, cv;  // rows of the tile inside m (from its first row), columns of each diagonal block inside n
    int nn;      // MMA N: ndiag nb
    int f16;     // words in fp16, else bf16
    int chunk;   // worst-case FP32 chunk in k-block x pair steps (its digit width's)
    const uint32_t *sqA, *sqB;  // squared-digit maxima for certified chunks, or nullptr
    int krev;    // k-blocks last to first
};

// The k-block (from kb0) of an item's kb-th step in its k order.
__device__ __forceinline__ int64_t item_kb(const Item &it, int64_t kb) { return it.krev ? it.nkbc - 1 - kb : kb; }

// Claims that run while the previous `wave` claims finish walk K the other
// way, so they start on the k-slabs of the words (the column tiles a raster
// group shares) that those left in L2 last.
__device__ __forceinline__ int wave_krev(const TcParams &P, int64_t idx) {
    return P.wave > 0 ? (int)((idx / P.wave) & 1) : 0;
}

// MMA N of an item: a single-diagonal tile runs only its valid columns,
// rounded up to 16 (the MMA's N step for M = 128), so the last column tile
// of a ragged product copies and multiplies no more B rows than it needs.
__device__ __forceinline__ int item_n(int ndiag, int nb, int cv) {
    if (ndiag == 1 && cv < nb) return cv < 16 ? 16 : (cv + 15) & ~15;
    return ndiag * nb;
}

__device__ __forceinline__ Item computed_item(const TcParams &P, int64_t idx) {
    Item it;
    const int64_t mtc = P.mt_count;
    // item idx -> (tile, K-range kc, window grp_w): windows heaviest first,
    // every tile of a window before the next window, every second pass over
    // the tiles in reverse so that it starts on the tiles (and the words they
    // share) the pass before has just left in L2
    const int64_t ntiles = mtc * P.nt_count;
    const int64_t rest = idx / ntiles;
    const int64_t tile = (rest & 1) ? ntiles - 1 - idx % ntiles : idx % ntiles;
    const int kc = (int)(rest % P.nkc);
    const int grp_w = (int)(rest / P.nkc);
    it.s0 = P.g_s0[grp_w];
    it.ndiag = P.g_nd[grp_w];
    it.i0 = P.g_i0[grp_w];
    it.ni = P.g_ni[grp_w];
    it.nb = P.nb;
    it.v = P.v;
    it.f16 = P.f16;
    it.chunk = P.chunk_blocks;
    it.sqA = P.sqA;
    it.sqB = P.sqB;
    it.b_wstride = P.b_wstride;
    it.b_kstride = P.b_kstride;
    it.b_wpad = P.b_wpad;
    // Raster in groups of kGroupN column tiles, rows inside a group first: the
    // ~148 tiles running at once cover about 18 row tiles x 8 column tiles,
    // the aspect that minimises the words they read (a B column tile is twice
    // the bytes of an A row tile), so fewer word tiles are fetched twice.
    // Odd groups take their rows bottom up, so a group starts on the row
    // tiles the previous one ended on.
    const int64_t gsz = mtc * kGroupN;
    const int64_t grp = tile / gsz, t = tile % gsz;
    const int64_t width = P.nt_count - grp * kGroupN < kGroupN ? P.nt_count - grp * kGroupN : kGroupN;
    it.mt = (grp & 1) ? mtc - 1 - t / width : t / width;
    it.nt = grp * kGroupN + t % width;
    it.kb0 = (int64_t)kc * P.kcb;
    const int64_t left = P.nkb - it.kb0;
    it.nkbc = left < P.kcb ? left : P.kcb;
    it.Aw = P.Aw;
    it.Bw = P.Bw;
    it.A_rows = P.A_rows;
    it.B_rows = P.B_rows;
    it.nkb = P.nkb;
    it.plane = (int64_t)P.nkc * P.A_rows * P.B_rows;
    it.S = P.S + (((int64_t)P.g_plane[grp_w] * P.nkc + kc) * P.A_rows + it.mt * BM) * P.B_rows + it.nt * BN;
    const int64_t rv = P.m - it.mt * BM, cv = P.n - it.nt * P.nb;
    it.rv = (int)(rv < BM ? rv : BM);
    it.cv = (int)(cv < P.nb ? cv : P.nb);
    it.nn = item_n(it.ndiag, it.nb, it.cv);
    it.krev = wave_krev(P, idx);
    return it;
}

__device__ __forceinline__ Item table_item(const TcParams &P, int64_t pos) {
    const TcItem &d = P.items[pos];
    Item it;
    it.Aw = d.Aw;
    it.Bw = d.Bw;
    it.S = d.S;
    it.A_rows = d.A_rows;
    it.B_rows = d.B_rows;
    it.nkb = d.nkb;
    it.kb0 = d.kb0;
    it.nkbc = d.nkbc;
    it.mt = d.mt;
    it.nt = d.nt;
    it.plane = d.plane;
    it.s0 = d.s0;
    it.ndiag = d.ndiag;
    it.nb = d.nb;
    it.i0 = d.i0;
    it.ni = d.ni;
    it.v = d.v;
    it.b_wstride = d.b_wstride;
    it.b_kstride = d.b_kstride;
    it.b_wpad = d.b_wpad;
    it.rv = d.rv;
    it.cv = d.cv;
    it.nn = item_n(it.ndiag, it.nb, it.cv);
    it.f16 = d.f16;
    it.chunk = d.chunk;
    it.sqA = d.sqA;
    it.sqB = d.sqB;
    it.krev = 0;
    return it;
}

template <bool kTable>
__device__ __forceinline__ Item get_item(const TcParams &P, int64_t idx) {
    return kTable ? table_item(P, idx) : computed_item(P, idx);
}

// The item sequence of one CTA, seen identically by its roles: items
// (computed, or rows of a batch's table) are claimed one at a time from the
// counter and published with their FP32 chunk in a ring of kRing slots
// (full: 1 arrival, the publisher; empty: 2 + 8 arrivals, the producer lane,
// the MMA lane and every epilogue warp).  With certified chunks the planner
// warp claims and publishes, running up to kRing items ahead; otherwise the
// producer lane claims each item when it is ready to load it (the planner
// warp idles): claims made earlier spread the items running at once over
// more tiles and cost DRAM reads (measured: +10% at 8-bit digits, 1-2%
// slower).  -1 ends the sequence.
struct ItemRing {
    int64_t *idx;
    int32_t *chunk;  // the item's FP32 chunk in k-block x pair steps
    uint64_t *full, *empty;
};

// Certified chunk of a computed item (one 256-wide diagonal tile, 9-bit
// digits): its k-block x pair steps in the MMA order (k-block outer, pairs
// inner), in windows of kCertBlocks.  For an output (r, c) and a step
// (pair (i, j), k-block kb), Cauchy-Schwarz bounds the sum of any subset of
// the step's 64 products by sqrt(SA SB), SA = sum over the k-block of
// A_i[r][k]^2 <= the split's maximum over r's group of 64 rows, SB the same
// for B_j's column c; so every partial sum of a window's products -- what the
// FP32 accumulator holds, in whatever order the tensor core adds them -- is
// at most sum_t sqrt(SA_t SB_t) <= sqrt(L sum_t SA_t SB_t) for L <= kCertBlocks
// steps.  L sum_t SA_t SB_t <= 2^48 for every window keeps each partial sum
// within 2^24, where FP32 is exact: then the item runs chunks of kCertBlocks
// steps (512 products), else the worst-case chunk (256).  The whole warp
// takes the windows in turn; every operand is an integer (sums of squares
// <= 64 x 2^16 = 2^22).  kAG: 64-row groups per row tile (2 for 128 rows,
// 4 for the pair kernel's 256).
template <int kAG>
__device__ __forceinline__ int certified_chunk(const Item &it, int lane) {
    if (it.ndiag != 1 || !it.sqA || 2 * it.chunk != kCertBlocks) return it.chunk;
    const int64_t nvb = (int64_t)it.ni * it.nkbc;
    const int64_t nwin = (nvb + kCertBlocks - 1) / kCertBlocks;
    const int64_t ga = it.A_rows / 64, gb = it.B_rows / 64;
    bool ok = true;
    for (int64_t w = lane; w < nwin; w += 32) {
        uint64_t sum = 0;
#pragma unroll
        for (int t = 0; t < kCertBlocks; ++t) {
            const int64_t v = w * kCertBlocks + t;
            if (v < nvb) {
                const int64_t kb = it.kb0 + item_kb(it, v / it.ni);
                const int i = it.i0 + (int)(v % it.ni), jw = it.s0 - i;
                const uint32_t *pa = it.sqA + ((int64_t)i * it.nkb + kb) * ga + kAG * it.mt;
                const uint32_t *pb = it.sqB + ((int64_t)jw * it.nkb + kb) * gb + 4 * it.nt;
                uint32_t sa = __ldg(pa);
#pragma unroll
                for (int q = 1; q < kAG; ++q) sa = max(sa, __ldg(pa + q));
                const uint32_t sb = max(max(__ldg(pb), __ldg(pb + 1)), max(__ldg(pb + 2), __ldg(pb + 3)));
                sum += (uint64_t)sa * sb;
            }
        }
        if ((uint64_t)kCertBlocks * sum > (uint64_t(1) << 48)) ok = false;
    }
    return __all_sync(0xffffffffu, ok) ? kCertBlocks : it.chunk;
}

// The producer lane as publisher (no certified chunks): claim the j-th item,
// publish it with its worst-case chunk, and read it as one of the slot's
// consumers.
template <bool kTable>
__device__ __forceinline__ int64_t produce_item(const TcParams &P, const ItemRing &R, int64_t j, bool &alive) {
    const int slot = (int)(j % kRing);
    if (!mbar_wait(&R.empty[slot], (uint32_t)(((j / kRing) & 1) ^ 1), P.err)) {
        alive = false;
        return -1;
    }
    int64_t idx = (int64_t)atomicAdd(P.sched, 1u);
    if (idx >= P.nitems) idx = -1;
    R.idx[slot] = idx;
    R.chunk[slot] = idx >= 0 ? get_item<kTable>(P, idx).chunk : P.chunk_blocks;
    mbar_arrive(&R.full[slot]);   // release: the index is visible to the waiters of this phase
    mbar_arrive(&R.empty[slot]);  // the producer has read it too
    return idx;
}

// The planner warp: claim the j-th item, work out its chunk, publish both.
template <bool kTable>
__device__ __forceinline__ int64_t plan_item(const TcParams &P, const ItemRing &R, int64_t j, bool &alive,
                                             int lane) {
    const int slot = (int)(j % kRing);
    int ok = 1;
    int64_t idx = -1;
    if (lane == 0) {
        ok = mbar_wait(&R.empty[slot], (uint32_t)(((j / kRing) & 1) ^ 1), P.err) ? 1 : 0;
        if (ok) {
            idx = (int64_t)atomicAdd(P.sched, 1u);
            if (idx >= P.nitems) idx = -1;
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) {
        alive = false;
        return -1;
    }
    idx = __shfl_sync(0xffffffffu, idx, 0);
    int chunk = P.chunk_blocks;
    if (idx >= 0) chunk = certified_chunk<2>(get_item<kTable>(P, idx), lane);
    if (lane == 0) {
        R.idx[slot] = idx;
        R.chunk[slot] = chunk;
        mbar_arrive(&R.full[slot]);  // release: index and chunk are visible to the waiters of this phase
    }
    return idx;
}

// kWarp: the whole warp waits and reads; one lane releases the slot.
template <bool kWarp>
__device__ __forceinline__ int64_t consume_item(const TcParams &P, const ItemRing &R, int64_t j, bool &alive,
                                                int *chunk = nullptr) {
    const int slot = (int)(j % kRing);
    bool ok = mbar_wait(&R.full[slot], (uint32_t)((j / kRing) & 1), P.err);
    if (kWarp) ok = __all_sync(0xffffffffu, ok);
    if (!ok) {
        alive = false;
        return -1;
    }
    const int64_t idx = R.idx[slot];
    if (chunk) *chunk = R.chunk[slot];
    if (kWarp) {
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(&R.empty[slot]);
    } else {
        mbar_arrive(&R.empty[slot]);
    }
    return idx;
}

// Instruction descriptor of a one-CTA MMA: M = 128, N = n (a multiple of 16,
// at most 256), bf16 or fp16 words.
__device__ __forceinline__ uint32_t idesc_n(int n, int f16) { return f16 ? idesc_f16(BM, n) : idesc_bf16(BM, n); }

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

// Store this warp's 32 x 128 block of sums (row r held by lane r in acc)
// through its shared-memory staging area: each 16-column block is written by
// rows and read back with four lanes per row, so one global store
// instruction covers 8 rows x 64 contiguous bytes instead of 32 rows x 16
// bytes (measured: the row-per-lane stores cost the 512-instance batch a
// quarter of its replay time).  Tile rows row0 + r >= rv and, per diagonal
// block, columns >= cv (tile padding) are not stored; column c of the
// accumulator is column c mod nb of diagonal s0 + c / nb.
// Adds the 128 FP32 chunk sums of this thread's TMEM lane (columns t0..t0+127)
// to its INT32 diagonal sums: 16 columns per load, the next load in flight
// while the current block is converted and added.  Every value is an exact
// integer with |x| <= 2^24, so cvt.rni is exact.  The conversions (a
// quarter-rate instruction) spread the tensor-memory reads over most of the
// next chunk's MMAs; measured, drains that read faster (an FP32 add of
// 1.5 * 2^23 in place of the conversion, exact below 2^22) made the whole
// kernel slower.
__device__ __forceinline__ void drain_add(uint32_t t0, int32_t (&acc)[128]) {
    uint32_t ra[16], rb[16];
    tmem_ld16_async(t0, ra);
    tmem_wait_ld16(ra);
#pragma unroll
    for (int jb = 0; jb < 8; ++jb) {
        uint32_t(&cur)[16] = (jb & 1) ? rb : ra;
        uint32_t(&nxt)[16] = (jb & 1) ? ra : rb;
        if (jb + 1 < 8) tmem_ld16_async(t0 + (uint32_t)((jb + 1) * 16), nxt);
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[jb * 16 + e] += __float2int_rn(__uint_as_float(cur[e]));
        if (jb + 1 < 8) tmem_wait_ld16(nxt);
    }
}

__device__ __forceinline__ void store_sums(const Item &it, const int32_t (&acc)[128], int32_t *stg, int lane, int row0,
                                           int col0) {
#pragma unroll
    for (int cb = 0; cb < 8; ++cb) {
        __syncwarp();  // the previous block's reads are done
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<int4 *>(stg + lane * kStgStride + 4 * q) =
                make_int4(acc[cb * 16 + 4 * q], acc[cb * 16 + 4 * q + 1], acc[cb * 16 + 4 * q + 2],
                          acc[cb * 16 + 4 * q + 3]);
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = i * 8 + (lane >> 2), g = lane & 3;
            const int4 v = *reinterpret_cast<const int4 *>(stg + r * kStgStride + 4 * g);
            const int row = row0 + r, cc = col0 + cb * 16 + 4 * g;
            const int d = cc / it.nb;
            // streaming stores: the sums are read once, by the recombination,
            // so they should not displace word tiles from L2
            if (row < it.rv && d < it.ndiag && cc - d * it.nb < it.cv)
                __stcs(reinterpret_cast<int4 *>(it.S + (int64_t)row * it.B_rows + d * it.plane + (cc - d * it.nb)), v);
        }
    }
}

template <bool kTable>
__global__ void __launch_bounds__(THREADS, 1) gemm_tc_kernel(const __grid_constant__ TcParams P) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], tfull[2], tempty[2], done;
    __shared__ __align__(8) uint64_t rfull[kRing], rempty[kRing];
    __shared__ int64_t ring_idx[kRing];
    __shared__ int32_t ring_chunk[kRing];
    __shared__ uint32_t tmem_base_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    uint8_t *sA = smem_raw + pad;
    uint8_t *sB = sA + STAGES * kTileA;
    int32_t *sStage = reinterpret_cast<int32_t *>(sB + STAGES * kTileB);
    const ItemRing ring{ring_idx, ring_chunk, rfull, rempty};

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], EPI_WARPS);
        }
        for (int r = 0; r < kRing; ++r) {
            mbar_init(&rfull[r], 1);
            mbar_init(&rempty[r], 2 + EPI_WARPS);
        }
        mbar_init(&done, 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_base_sh;

    if (warp == 0) {
        if (lane == 0) {  // ---------------- TMA producer
            uint64_t g = 0;
            bool alive = true;
            for (int64_t j = 0; alive; ++j) {
                const int64_t idx =
                    P.cert ? consume_item<false>(P, ring, j, alive) : produce_item<kTable>(P, ring, j, alive);
                if (idx < 0) break;
                const Item it = get_item<kTable>(P, idx);
                // One thread issues every copy, so the per-stage work is kept to a
                // few adds: nested (k-block, word) loops and running addresses.
                // The window's B words B_{s0-i} .. B_{s0-i+ndiag-1} are contiguous
                // (k-block-major layout padded with zero words), so each stage is
                // two copies whatever the window.  The k-block is the outer loop
                // (every pair of the diagonal at k-block kb, then kb + 1): the
                // ~148 items of one wave then walk through k together and share
                // each k-slab of the words in L2 while it is needed.
                const uint32_t bbytes = (uint32_t)it.nn * kTileBytes;
                const uint32_t stage_bytes = kTileA + bbytes;
                const int64_t a_wstep = it.nkb * it.A_rows * kTileBytes;  // next A word, same k-block
                for (int64_t kb = 0; alive && kb < it.nkbc; ++kb) {
                    const uint8_t *a =
                        it.Aw + (((int64_t)it.i0 * it.nkb + it.kb0 + item_kb(it, kb)) * it.A_rows + it.mt * BM) *
                                    kTileBytes;
                    const uint8_t *b = it.Bw + (int64_t)(it.s0 - it.i0 + it.b_wpad) * it.b_wstride +
                                       (it.kb0 + item_kb(it, kb)) * it.b_kstride + it.nt * it.nb * kTileBytes;
                    for (int ii = 0; ii < it.ni; ++ii, ++g, a += a_wstep, b -= it.b_wstride) {
                        const int slot = (int)(g % STAGES);
                        if (!mbar_wait(&empty[slot], (uint32_t)(((g / STAGES) & 1) ^ 1), P.err)) {
                            alive = false;
                            break;
                        }
                        mbar_arrive_expect_tx(&full[slot], stage_bytes);
                        bulk_g2s(sA + slot * kTileA, a, kTileA, &full[slot]);
                        bulk_g2s(sB + slot * kTileB, b, bbytes, &full[slot]);
                    }
                }
            }
            // Let every copy into this CTA land before exit.
            for (int s = 0; s < STAGES; ++s) {
                const uint64_t armed = g > (uint64_t)s ? (g - s + STAGES - 1) / STAGES : 0;
                if (armed) mbar_wait(&full[s], (uint32_t)((armed - 1) & 1), P.err);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---------------- MMA issuer
            uint64_t g = 0, c = 0;
            bool alive = true;
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
            for (int64_t j = 0; alive; ++j) {
                int chunk = P.chunk_blocks;
                const int64_t idx = consume_item<false>(P, ring, j, alive, &chunk);
                if (idx < 0) break;
                const Item it = get_item<kTable>(P, idx);
                const int64_t nvb = (int64_t)it.ni * it.nkbc;
                const uint32_t idesc = idesc_n(it.nn, it.f16);
                for (int64_t t0 = 0; alive && t0 < nvb; t0 += chunk, ++c) {
                    const int buf = (int)(c & 1);
                    if (!mbar_wait(&tempty[buf], (uint32_t)(((c >> 1) & 1) ^ 1), P.err)) {
                        alive = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tmem_base + (uint32_t)(buf * BN);
                    const int64_t tend = t0 + chunk < nvb ? t0 + chunk : nvb;
                    for (int64_t t = t0; t < tend; ++t, ++g) {
                        const int slot = (int)(g % STAGES);
                        if (!mbar_wait(&full[slot], (uint32_t)((g / STAGES) & 1), P.err)) {
                            alive = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t ad = sdesc(a0 + slot * kTileA), bd = sdesc(b0 + slot * kTileB);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)  // K = 16 per MMA: +32 bytes = +2 in the address field
                            mma_bf16(dt, ad + 2 * kk, bd + 2 * kk, idesc, (t > t0 || kk > 0) ? 1u : 0u);
                        mma_commit(&empty[slot]);
                    }
                    mma_commit(&tfull[buf]);
                }
            }
            // All MMAs this lane issued have completed once `done` flips.
            mma_commit(&done);
            mbar_wait(&done, 0, P.err);
        }
    } else if (warp == PLANNER_WARP) {  // ---------------- planner: claims, certified chunks
        if (P.cert) {
            bool alive = true;
            for (int64_t j = 0; alive; ++j)
                if (plan_item<kTable>(P, ring, j, alive, lane) < 0) break;
        }
    } else {  // -------------------------------- epilogue warps 2..9
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const uint32_t tlane = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 128);
        uint64_t c = 0;
        bool alive = true;
        for (int64_t j = 0; alive; ++j) {
            int chunk = P.chunk_blocks;
            const int64_t idx = consume_item<true>(P, ring, j, alive, &chunk);
            if (idx < 0) break;
            const Item it = get_item<kTable>(P, idx);
            const int64_t nvb = (int64_t)it.ni * it.nkbc;
            const int64_t nch = (nvb + chunk - 1) / chunk;
            int32_t acc[128];
#pragma unroll
            for (int e = 0; e < 128; ++e) acc[e] = 0;
            for (int64_t ch = 0; ch < nch; ++ch, ++c) {
                const int buf = (int)(c & 1);
                const bool ok = mbar_wait(&tfull[buf], (uint32_t)((c >> 1) & 1), P.err);
                if (!__all_sync(0xffffffffu, ok)) {
                    alive = false;
                    break;
                }
                tc_fence_after();
                if (half * 128 < it.nn)  // this warp's columns hold products (warp-uniform)
                    drain_add(tlane + (uint32_t)(buf * BN), acc);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
            }
            if (!alive) break;
            store_sums(it, acc, sStage + (warp - 2) * (32 * kStgStride), lane, quarter * 32, half * 128);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                     : "memory");
}

// ---------------------------------------------------------------------------
// Pair kernel (opt-in, plan option tc_pair): a cluster of two CTAs on two SMs
// computes a 256 x 256 tile with tcgen05.mma.cta_group::2 (M = 256 split over
// the pair, each CTA holding its 128 rows of A and its 128-row half of B).
// Each SM then receives 32 KB of operands per 64-wide k-block instead of
// 48 KB, and 6 stages fit in shared memory.  Roles per CTA as in the one-CTA
// kernel; only the even CTA ("leader") issues MMAs.  Both CTAs load their
// halves with tensor TMA (.cta_group::2), whose completion lands directly on
// the leader's barrier, so the leader waits on one barrier per stage; its
// commits are multicast to both CTAs.  The word tiles are already in their
// shared-memory order, so the tensor maps describe them as plain 2-D arrays
// of 128-byte rows (no TMA swizzle).
//
// Items are claimed as in the one-CTA kernel, by the leader alone: its
// publisher (the planner warp with certified chunks, else its producer lane)
// writes each index and chunk into both CTAs' rings (the peer's through
// distributed shared memory, then a release arrive on the peer's barrier),
// and every consumer of both CTAs releases the slot on the leader's empty
// barrier.  Item order, k-block-outer loads and certified chunks follow the
// one-CTA kernel.
constexpr int P_STAGES = 6;
constexpr int BM2 = 256;
constexpr uint32_t kTileA2 = 128 * kTileBytes;  // own 128 rows of A: 16 KB
constexpr uint32_t kTileB2 = 128 * kTileBytes;  // own half of B: 16 KB
constexpr int kSmemPair = P_STAGES * (kTileA2 + kTileB2) + kStageBytes + 1024;
constexpr uint32_t kIdescPair = idesc_bf16(BM2, BN);
// consumers of a ring slot: both CTAs' producer lanes and epilogue warps, and
// the leader's MMA lane
constexpr int kPairRingConsumers = 2 * (1 + EPI_WARPS) + 1;

__device__ __forceinline__ Item pair_item(const TcParams &P, int64_t idx) {
    // tiles of 256 rows: mt counts 256-row tiles here; A_rows % 256 == 0
    Item it;
    const int64_t mt2 = P.mt_count / 2;
    const int64_t ntiles = mt2 * P.nt_count;
    const int64_t rest = idx / ntiles;
    // every second pass over the tiles in reverse, as in computed_item
    const int64_t tile = (rest & 1) ? ntiles - 1 - idx % ntiles : idx % ntiles;
    const int kc = (int)(rest % P.nkc);
    const int grp_w = (int)(rest / P.nkc);  // nb = 256: one diagonal per window
    it.s0 = P.g_s0[grp_w];
    it.ndiag = 1;
    it.nb = BN;
    it.i0 = P.g_i0[grp_w];
    it.ni = P.g_ni[grp_w];
    it.v = P.v;
    it.f16 = P.f16;
    it.chunk = P.chunk_blocks;
    it.sqA = P.sqA;
    it.sqB = P.sqB;
    const int64_t gsz = mt2 * kGroupN;
    const int64_t grp = tile / gsz, t = tile % gsz;
    const int64_t width = P.nt_count - grp * kGroupN < kGroupN ? P.nt_count - grp * kGroupN : kGroupN;
    it.mt = (grp & 1) ? mt2 - 1 - t / width : t / width;  // 256-row tile index; odd groups bottom up
    it.nt = grp * kGroupN + t % width;
    it.kb0 = (int64_t)kc * P.kcb;
    const int64_t left = P.nkb - it.kb0;
    it.nkbc = left < P.kcb ? left : P.kcb;
    it.Aw = P.Aw;
    it.Bw = P.Bw;
    it.A_rows = P.A_rows;
    it.B_rows = P.B_rows;
    it.nkb = P.nkb;
    it.plane = (int64_t)P.nkc * P.A_rows * P.B_rows;
    it.S = P.S + (((int64_t)P.g_plane[grp_w] * P.nkc + kc) * P.A_rows + it.mt * BM2) * P.B_rows + it.nt * BN;
    const int64_t rv = P.m - it.mt * BM2, cv = P.n - it.nt * BN;  // clipped to the 256 x 256 tile
    it.rv = (int)(rv < BM2 ? rv : BM2);
    it.cv = (int)(cv < BN ? cv : BN);
    it.nn = BN;
    it.krev = wave_krev(P, idx);
    return it;
}

// The ring of one CTA of a pair, with the cluster addresses the leader's
// publisher writes to (the peer's slots and full barriers) and the consumers
// release to (the leader's empty barriers).
struct PairRing {
    int64_t *idx;
    int32_t *chunk;
    uint64_t *full, *empty;  // empty: used in the leader only
    uint32_t peer_idx, peer_chunk, peer_full, lead_empty;
};

// Leader: claim the j-th item (lane 0), work out its chunk (the whole warp
// when kWarp, certified chunks), publish it to both CTAs.  The slot's
// previous readers in both CTAs have released it (acquire at cluster scope
// orders this lane's stores into the peer after the peer's reads).
template <bool kWarp>
__device__ __forceinline__ int64_t pair_publish(const TcParams &P, const PairRing &R, int64_t j, bool &alive,
                                                int lane) {
    const int slot = (int)(j % kRing);
    int ok = 1;
    int64_t idx = -1;
    if (lane == 0) {
        ok = mbar_wait_cluster(&R.empty[slot], (uint32_t)(((j / kRing) & 1) ^ 1), P.err) ? 1 : 0;
        if (ok) {
            idx = (int64_t)atomicAdd(P.sched, 1u);
            if (idx >= P.nitems) idx = -1;
        }
    }
    if (kWarp) {
        ok = __shfl_sync(0xffffffffu, ok, 0);
        idx = __shfl_sync(0xffffffffu, idx, 0);
    }
    if (!ok) {
        alive = false;
        return -1;
    }
    int chunk = P.chunk_blocks;
    if (kWarp && idx >= 0) chunk = certified_chunk<4>(pair_item(P, idx), lane);
    if (lane == 0) {
        R.idx[slot] = idx;
        R.chunk[slot] = chunk;
        st_cluster_u64(R.peer_idx + (uint32_t)(slot * sizeof(int64_t)), (uint64_t)idx);
        st_cluster_u32(R.peer_chunk + (uint32_t)(slot * sizeof(int32_t)), (uint32_t)chunk);
        mbar_arrive(&R.full[slot]);
        // release at cluster scope: the two stores above are visible to the
        // peer's waiters of this phase
        mbar_arrive_cluster(R.peer_full + (uint32_t)(slot * sizeof(uint64_t)));
    }
    return idx;
}

// Any role of either CTA: wait for the j-th item in this CTA's ring, read it,
// release the slot on the leader's empty barrier (one lane when kWarp).
template <bool kWarp>
__device__ __forceinline__ int64_t pair_consume(const TcParams &P, const PairRing &R, int64_t j, bool &alive,
                                                int *chunk) {
    const int slot = (int)(j % kRing);
    bool ok = mbar_wait_cluster(&R.full[slot], (uint32_t)((j / kRing) & 1), P.err);
    if (kWarp) ok = __all_sync(0xffffffffu, ok);
    if (!ok) {
        alive = false;
        return -1;
    }
    const int64_t idx = R.idx[slot];
    if (chunk) *chunk = R.chunk[slot];
    if (kWarp) __syncwarp();
    if (!kWarp || (threadIdx.x & 31) == 0) mbar_arrive_cluster(R.lead_empty + (uint32_t)(slot * sizeof(uint64_t)));
    return idx;
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(THREADS_PAIR, 1)
    gemm_tc_pair_kernel(const __grid_constant__ TcParams P, const __grid_constant__ CUtensorMap tmA,
                        const __grid_constant__ CUtensorMap tmB) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[P_STAGES], empty[P_STAGES], tfull[2], tempty[2], done;
    __shared__ __align__(8) uint64_t rfull[kRing], rempty[kRing];
    __shared__ int64_t ring_idx[kRing];
    __shared__ int32_t ring_chunk[kRing];
    __shared__ uint32_t tmem_base_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    uint8_t *sA = smem_raw + pad;
    uint8_t *sB = sA + P_STAGES * kTileA2;
    int32_t *sStage = reinterpret_cast<int32_t *>(sB + P_STAGES * kTileB2);
    const PairRing ring{ring_idx,
                        ring_chunk,
                        rfull,
                        rempty,
                        peer_addr(&ring_idx[0], 1),
                        peer_addr(&ring_chunk[0], 1),
                        peer_addr(&rfull[0], 1),
                        peer_addr(&rempty[0], 0)};

    if (threadIdx.x == 0) {
        for (int s = 0; s < P_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 2 * EPI_WARPS);  // both CTAs' epilogue warps (leader's copy)
        }
        for (int r = 0; r < kRing; ++r) {
            mbar_init(&rfull[r], 1);
            mbar_init(&rempty[r], kPairRingConsumers);  // leader's copy
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

    if (warp == 0) {
        if (lane == 0) {  // ---------------- TMA producer (both CTAs)
            const uint32_t lead_full = peer_addr(&full[0], 0);
            uint64_t g = 0;
            bool alive = true;
            for (int64_t j = 0; alive; ++j) {
                int64_t idx;
                if (leader && !P.cert) {  // the leader's producer publishes, then reads as a consumer
                    idx = pair_publish<false>(P, ring, j, alive, 0);
                    if (alive) mbar_arrive(&rempty[(int)(j % kRing)]);
                } else {
                    idx = pair_consume<false>(P, ring, j, alive, nullptr);
                }
                if (idx < 0) break;
                const Item it = pair_item(P, idx);
                // k-block outer, the diagonal's pairs inner (as in the one-CTA kernel)
                for (int64_t kb = 0; alive && kb < it.nkbc; ++kb) {
                    for (int ii = 0; ii < it.ni; ++ii, ++g) {
                        const int i = it.i0 + ii;
                        const int jw = it.s0 - i;
                        // row coordinates of the tensor maps (the host checks they fit int32)
                        const int64_t kbe = it.kb0 + item_kb(it, kb);
                        const int32_t ya = (int32_t)(((int64_t)i * it.nkb + kbe) * it.A_rows + it.mt * BM2 +
                                                     rank * 128);
                        const int32_t yb = (int32_t)(((int64_t)jw * it.nkb + kbe) * it.B_rows + it.nt * BN +
                                                     rank * 128);
                        const int slot = (int)(g % P_STAGES);
                        if (!mbar_wait(&empty[slot], (uint32_t)(((g / P_STAGES) & 1) ^ 1), P.err)) {
                            alive = false;
                            break;
                        }
                        // the leader's barrier counts both CTAs' bytes
                        if (leader) mbar_arrive_expect_tx(&full[slot], 2 * (kTileA2 + kTileB2));
                        const uint32_t bar = lead_full + (uint32_t)(slot * sizeof(uint64_t));
                        tma2_load_pair(sA + slot * kTileA2, &tmA, ya, bar);
                        tma2_load_pair(sB + slot * kTileB2, &tmB, yb, bar);
                    }
                }
            }
            // Before exit: the leader sees every byte of both CTAs land; both
            // wait for the leader's last commit to each slot (after which no
            // copy into, or signal to, this CTA is outstanding).
            for (int s = 0; s < P_STAGES; ++s) {
                const uint64_t armed = g > (uint64_t)s ? (g - s + P_STAGES - 1) / P_STAGES : 0;
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
            const uint32_t idesc_pair = P.f16 ? idesc_f16(BM2, BN) : kIdescPair;
            for (int64_t j = 0; alive; ++j) {
                int chunk = P.chunk_blocks;
                const int64_t idx = pair_consume<false>(P, ring, j, alive, &chunk);
                if (idx < 0) break;
                const Item it = pair_item(P, idx);
                const int64_t nvb = (int64_t)it.ni * it.nkbc;
                for (int64_t t0 = 0; alive && t0 < nvb; t0 += chunk, ++c) {
                    const int buf = (int)(c & 1);
                    if (!mbar_wait(&tempty[buf], (uint32_t)(((c >> 1) & 1) ^ 1), P.err)) {
                        alive = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tmem_base + (uint32_t)(buf * BN);
                    const int64_t tend = t0 + chunk < nvb ? t0 + chunk : nvb;
                    for (int64_t t = t0; t < tend; ++t, ++g) {
                        const int slot = (int)(g % P_STAGES);
                        const uint32_t par = (uint32_t)((g / P_STAGES) & 1);
                        if (!mbar_wait(&full[slot], par, P.err)) {
                            alive = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t ad = sdesc(a0 + slot * kTileA2), bd = sdesc(b0 + slot * kTileB2);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_bf16_pair(dt, ad + 2 * kk, bd + 2 * kk, idesc_pair, (t > t0 || kk > 0) ? 1u : 0u);
                        mma_commit_pair(&empty[slot], 3);
                    }
                    mma_commit_pair(&tfull[buf], 3);
                }
            }
            mma_commit_pair(&done, 1);
            mbar_wait(&done, 0, P.err);
        }
    } else if (warp == PLANNER_WARP) {  // ---------------- planner (leader, certified chunks)
        if (leader && P.cert) {
            bool alive = true;
            for (int64_t j = 0; alive; ++j)
                if (pair_publish<true>(P, ring, j, alive, lane) < 0) break;
        }
    } else {  // -------------------------------- epilogue warps 2..9 (both CTAs)
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const uint32_t tlane = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 128);
        const uint32_t lead_tempty = peer_addr(&tempty[0], 0);
        uint64_t c = 0;
        bool alive = true;
        for (int64_t j = 0; alive; ++j) {
            int chunk = P.chunk_blocks;
            const int64_t idx = pair_consume<true>(P, ring, j, alive, &chunk);
            if (idx < 0) break;
            const Item it = pair_item(P, idx);
            const int64_t nvb = (int64_t)it.ni * it.nkbc;
            const int64_t nch = (nvb + chunk - 1) / chunk;
            int32_t acc[128];
#pragma unroll
            for (int e = 0; e < 128; ++e) acc[e] = 0;
            for (int64_t ch = 0; ch < nch; ++ch, ++c) {
                const int buf = (int)(c & 1);
                const bool ok = mbar_wait(&tfull[buf], (uint32_t)((c >> 1) & 1), P.err);
                if (!__all_sync(0xffffffffu, ok)) {
                    alive = false;
                    break;
                }
                tc_fence_after();
                drain_add(tlane + (uint32_t)(buf * BN), acc);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(lead_tempty + (uint32_t)(buf * sizeof(uint64_t)));
            }
            if (!alive) break;
            store_sums(it, acc, sStage + (warp - 2) * (32 * kStgStride), lane, (int)rank * 128 + quarter * 32,
                       half * 128);
        }
    }

    tc_fence_before();
    cluster_sync_all();  // no CTA frees TMEM or exits while its peer may still signal it
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                     : "memory");
}

int pair_clusters() {
    static int cached[64] = {0};
    return max_clusters2(reinterpret_cast<const void *>(gemm_tc_pair_kernel), THREADS_PAIR, kSmemPair, cached);
}

}  // namespace

int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    std::lock_guard<std::mutex> lock(launch_cache_mutex());
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        cached[dev] = n;
    }
    return cached[dev];
}

int max_clusters2(const void *kernel, int threads, int smem, int (&cached)[64]) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (set_smem_attr(kernel, smem) != cudaSuccess) return 0;
    const int sms = sm_count();
    std::lock_guard<std::mutex> lock(launch_cache_mutex());
    if (!cached[dev]) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * (unsigned)(sms / 2), 1, 1);
        cfg.blockDim = dim3((unsigned)threads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = 2;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess || n <= 0) return 0;
        cached[dev] = n;
    }
    return cached[dev];
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link
// against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

int encode_rows_map(CUtensorMap *map, const void *base, uint64_t rows, uint32_t box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return (int)cudaErrorNotSupported;
    if (rows == 0 || rows > (uint64_t)INT32_MAX) return (int)cudaErrorInvalidValue;  // int32 coordinates
    const cuuint64_t dims[2] = {64, rows};
    const cuuint64_t strides[1] = {kTileBytes};
    const cuuint32_t box[2] = {64, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : (int)cudaErrorInvalidValue;
}


int launch_gemm_tc(const Plan &pl, const void *Aw, const void *Bw, int32_t *S, int *err, void *stream,
                   const uint32_t *sqA, const uint32_t *sqB) {
    TcParams P;
    std::memset(&P, 0, sizeof(P));
    P.Aw = static_cast<const uint8_t *>(Aw);
    P.Bw = static_cast<const uint8_t *>(Bw);
    P.S = S;
    P.nkb = pl.nkb;
    P.A_rows = pl.A_rows;
    P.B_rows = pl.B_rows;
    P.kcb = pl.kc / kTcKB;
    P.u = pl.u;
    P.v = pl.v;
    P.nsums = pl.nsums;
    P.nkc = pl.nkc;
    P.f16 = pl.form == MWMM_FORM_INT8 && pl.digit_bits == 9;
    P.chunk_blocks = (int)(pl.tc_chunk / kTcKB);
    P.mt_count = (int)(pl.A_rows / BM);
    P.nt_count = pl.tc_nb == BN ? (int)(pl.B_rows / BN) : 1;
    const int nwin = (pl.nsums + pl.tc_ndiag - 1) / pl.tc_ndiag;
    P.nitems = (int64_t)P.mt_count * P.nt_count * nwin * pl.nkc;
    P.err = err;
    P.items = nullptr;
    P.cta_off = nullptr;
    // diagonal windows of tc_ndiag diagonals, by decreasing number of A words
    // (heaviest items first)
    P.nb = pl.tc_nb;
    P.m = pl.m;
    P.n = pl.n;
    P.b_wpad = pl.B_wpad;
    P.b_wstride = pl.B_wstride * kTileBytes;
    P.b_kstride = pl.B_kstride * kTileBytes;
    int ng = 0;
    int gs0[kMaxWindows], gnd[kMaxWindows], gi0[kMaxWindows], gni[kMaxWindows], gpl[kMaxWindows],
        order[kMaxWindows];
    if (pl.form == MWMM_FORM_CRT8) {  // one window per modulus: the pair (i, i)
        for (; ng < pl.crt_s; ++ng) {
            gs0[ng] = 2 * ng;
            gnd[ng] = 1;
            gi0[ng] = ng;
            gni[ng] = 1;
            gpl[ng] = ng;
            order[ng] = ng;
        }
    } else {
        for (int s0 = 0; s0 < pl.nsums; s0 += pl.tc_ndiag, ++ng) {
            gs0[ng] = s0;
            gnd[ng] = pl.nsums - s0 < pl.tc_ndiag ? pl.nsums - s0 : pl.tc_ndiag;
            const int lo = s0 - (pl.v - 1) > 0 ? s0 - (pl.v - 1) : 0;
            const int hi = s0 + gnd[ng] - 1 < pl.u - 1 ? s0 + gnd[ng] - 1 : pl.u - 1;
            gi0[ng] = lo;
            gni[ng] = hi - lo + 1;
            gpl[ng] = s0;
            order[ng] = ng;
        }
    }
    for (int a = 1; a < ng; ++a)
        for (int b = a; b > 0 && gni[order[b]] > gni[order[b - 1]]; --b) {
            int t = order[b];
            order[b] = order[b - 1];
            order[b - 1] = t;
        }
    for (int g = 0; g < kMaxWindows; ++g) {
        P.g_s0[g] = g < ng ? gs0[order[g]] : 0;
        P.g_nd[g] = g < ng ? gnd[order[g]] : 0;
        P.g_i0[g] = g < ng ? gi0[order[g]] : 0;
        P.g_ni[g] = g < ng ? gni[order[g]] : 0;
        P.g_plane[g] = g < ng ? gpl[order[g]] : 0;
    }
    if (P.nitems == 0) return 0;
    P.sched = reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(S) + (pl.sched_off - pl.S_off));
    // certified chunks: twice the worst-case chunk, one 256-wide diagonal per item
    if (sqA && sqB && pl.tc_cert_chunk == kCertBlocks * kTcKB && 2 * P.chunk_blocks == kCertBlocks &&
        pl.tc_nb == BN && pl.tc_ndiag == 1) {
        P.sqA = sqA;
        P.sqB = sqB;
        P.cert = 1;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (pl.tc_pair) {
        P.nitems = (int64_t)(P.mt_count / 2) * P.nt_count * nwin * pl.nkc;
        cudaError_t e = set_smem_attr(reinterpret_cast<const void *>(gemm_tc_pair_kernel), kSmemPair);
        if (e != cudaSuccess) return (int)e;
        const int clusters = pair_clusters();
        if (clusters <= 0) return (int)cudaErrorLaunchOutOfResources;
        const int64_t ncl = P.nitems < clusters ? P.nitems : clusters;
        P.wave = ncl;
        CUtensorMap tmA, tmB;
        int r = encode_rows_map(&tmA, Aw, (uint64_t)pl.u * pl.nkb * pl.A_rows, 128);
        if (r == 0) r = encode_rows_map(&tmB, Bw, (uint64_t)pl.v * pl.nkb * pl.B_rows, 128);
        if (r != 0) return r;
        e = cudaMemsetAsync(P.sched, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) return (int)e;
        gemm_tc_pair_kernel<<<(unsigned)(2 * ncl), THREADS_PAIR, kSmemPair, s>>>(P, tmA, tmB);
        return (int)cudaGetLastError();
    }
    cudaError_t e = set_smem_attr(reinterpret_cast<const void *>(gemm_tc_kernel<false>), kSmemBytes);
    if (e != cudaSuccess) return (int)e;
    const int64_t sms = sm_count();
    e = cudaMemsetAsync(P.sched, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return (int)e;
    const unsigned grid = (unsigned)(P.nitems < sms ? P.nitems : sms);
    P.wave = grid;
    gemm_tc_kernel<false><<<grid, THREADS, kSmemBytes, s>>>(P);
    return (int)cudaGetLastError();
}

int tc_sm_count() { return sm_count(); }

int tc_pairs_fill_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();  // no device here: clear the error, answer unknown
        return -1;
    }
    const int clusters = pair_clusters();
    if (clusters <= 0) return -1;
    return 2 * clusters >= sm_count() ? 1 : 0;
}

int tc_residency(int *sms, int *ctas, int *clusters) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return (int)cudaErrorNoDevice;
    cudaError_t e = set_smem_attr(reinterpret_cast<const void *>(gemm_tc_kernel<false>), kSmemBytes);
    if (e != cudaSuccess) return (int)e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gemm_tc_kernel<false>, THREADS, kSmemBytes);
    if (e != cudaSuccess) return (int)e;
    *sms = sm_count();
    *ctas = per_sm * *sms;
    *clusters = pair_clusters();
    return *clusters > 0 ? 0 : (int)cudaErrorUnknown;
}

int prepare_tc_attributes() {
    cudaError_t e = set_smem_attr(reinterpret_cast<const void *>(gemm_tc_kernel<false>), kSmemBytes);
    if (e == cudaSuccess) e = set_smem_attr(reinterpret_cast<const void *>(gemm_tc_kernel<true>), kSmemBytes);
    if (e == cudaSuccess) {  // cache the cluster counts outside any capture
        (void)pair_clusters();
        (void)tensor_map_encoder();
    }
    return (int)e;
}

int launch_gemm_tc_table(const TcItem *items, int64_t *cta_off, int64_t nitems, int ctas, int chunk_blocks, int *err,
                         void *stream, int cert) {
    if (ctas <= 0 || nitems <= 0) return 0;
    TcParams P;
    std::memset(&P, 0, sizeof(P));
    P.items = items;
    P.cta_off = cta_off;
    P.nitems = nitems;
    P.sched = reinterpret_cast<uint32_t *>(cta_off + 2);
    P.chunk_blocks = chunk_blocks;  // each item carries its own chunk; this is a fallback only
    P.err = err;
    P.cert = cert;
    cudaError_t e = set_smem_attr(reinterpret_cast<const void *>(gemm_tc_kernel<true>), kSmemBytes);
    if (e != cudaSuccess) return (int)e;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(P.sched, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return (int)e;
    gemm_tc_kernel<true><<<ctas, THREADS, kSmemBytes, s>>>(P);
    return (int)cudaGetLastError();
}

}  // namespace mwmm
