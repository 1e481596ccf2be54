// Split kernels: uint64 matrices -> word matrices in the tiled layout.
//
// FP64 form: Alg. 4 (MW-Decomposition) with integer alpha = ceil(p^(1/u)):
//   T = M; for i < u-1 { R = floor(T / alpha); M_i = T - alpha R; T = R }; M_{u-1} = T.
// The quotient is taken in exact 64-bit integer arithmetic (a Barrett
// reciprocal of alpha plus a correction); Lemma 3.1 shows that the paper's
// floor(fl(T / alpha)) is the same integer, so the words are identical.
//
// INT8 form: the signed representative s of M mod p (M, or M - p when
// M > (p-1)/2) is written as base-2^8 digits, s = sum_i 256^i d_i: balanced
// digits in [-128, 127] and a top digit in [-128, 128] (the remainder); the
// digits are stored exactly as bf16.
//
// CRT form (multimodular comparison, Sec. 5.2): word i is the signed
// residue of M modulo the i-th modulus m_i < 256 (in [-(m_i-1)/2, (m_i-1)/2]),
// stored exactly as bf16 in the same layout.
//
// Output layout (see mwmm_plan_desc): word w, k-block kb, row r occupies the
// 128-byte chunk ((w * nkb + kb) * rows_pad + r); inside it the 16-byte
// granule g sits at position g ^ (r & 7), which is the 128-byte swizzle the
// tcgen05 shared-memory descriptors expect, and keeps the FP64 kernel's
// shared-memory reads spread over all banks.
#include <cuda_bf16.h>

#include <cstring>
#include <vector>

#include "device_common.cuh"
#include "mwmm_internal.h"

namespace mwmm {

namespace {

constexpr int kST = 64;  // tile: 64 word-layout rows x 64 k

struct SplitParams {
    const uint64_t *M;
    int64_t ld;
    int side;        // 0: M is rows x K (A); 1: M is K x rows (B, transposed on output)
    int64_t rows;    // m (A) or n (B)
    int64_t K;
    int64_t rows_pad, nkb;
    uint8_t *out;
    int words;
    int64_t wstride, kstride;  // rows between consecutive words / k-blocks
    int wpad;                  // zero words written before and after the words
    uint64_t p;
    uint64_t alpha, mu;  // FP64: radix and floor((2^64 - 1) / alpha)
    int validate;
    int *err;
    int64_t cbias;              // INT8 form: 128 (1 + 256 + ... + 256^(words-2))
    int crt;                    // CRT form: residues instead of digits
    uint32_t cm[kMaxCrt];       // moduli (odd primes below 256)
    uint32_t cM[kMaxCrt];       // floor(2^32 / m_i) + 1
    uint32_t c18[kMaxCrt], c36[kMaxCrt];  // 2^18 mod m_i, 2^36 mod m_i
    float cmh[kMaxCrt];         // 1.5 * 2^23 + (m_i - 1) / 2
};

// Small integers to bf16 without the conversion pipe.  For |v| < 2^22 the
// FP32 number with bit pattern 0x4B400000 + v is 1.5 * 2^23 + v exactly, and
// subtracting 1.5 * 2^23 leaves v exactly.  A value of magnitude <= 256 has
// at most 8 significant bits, so its bf16 is the upper half of that FP32
// pattern (no rounding): two of them pack into one word with one byte
// permutation.
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
__device__ __forceinline__ float small_int_float(int v) { return __int_as_float(0x4B400000 + v) - kMagic; }
// FP32 value byte_i(x) - 128 (i in 0..3): the byte is placed under the
// exponent of 1.5 * 2^23 by a byte permutation.
__device__ __forceinline__ float byte_digit_float(uint32_t x, int i) {
    return __int_as_float((int)__byte_perm(x, 0x4B400000u, 0x7650u | (uint32_t)i)) - (kMagic + 128.0f);
}
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632u);
}

// Signed residue of x < 2^52 modulo an odd m < 256, in [-(m-1)/2, (m-1)/2],
// with 32-bit operations only: from the 18-bit limbs x = x2 2^36 + x1 2^18
// + x0, z = x2 (2^36 mod m) + x1 (2^18 mod m) + x0 + (m-1)/2 < 2^27 is
// congruent to x + (m-1)/2.  q = umulhi(z, floor(2^32 / m) + 1) is floor(z / m)
// or one more (the multiplier exceeds 2^32 / m by less than 1, and
// z / 2^32 < 1/32), so z - q m is z mod m, or that minus m (then m is added
// back).  The residue minus (m-1)/2 is the signed one; its FP32 value comes
// from the magic exponent with the offset folded into the constant cmh.
__device__ __forceinline__ float signed_residue(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t m, uint32_t M,
                                                uint32_t c18, uint32_t c36, float cmh) {
    const uint32_t z = x2 * c36 + x1 * c18 + x0 + (m >> 1);
    int r = (int)(z - __umulhi(z, M) * m);
    r += (r >> 31) & (int)m;
    return __int_as_float(0x4B400000 + r) - cmh;
}

__device__ __forceinline__ uint64_t load_tile_elem(const SplitParams &P, int64_t r, int64_t l) {
    if (r >= P.rows || l >= P.K) return 0;
    return P.side == 0 ? P.M[r * P.ld + l] : P.M[l * P.ld + r];
}

// Read a 64 x 64 tile of M (coalesced along M's contiguous dimension) into
// shared memory as tile[row][k].
__device__ __forceinline__ void load_tile(const SplitParams &P, uint64_t (*tile)[kST + 1], int64_t r0,
                                          int64_t l0) {
    const int t = threadIdx.x;
    constexpr int kPer = (kST * kST) / 256;
    bool bad = false;
    uint64_t x[kPer];  // every load of the thread in flight before the first store
#pragma unroll
    for (int it = 0; it < kPer; ++it) {
        const int a = t / kST + it * (256 / kST), b = t % kST;
        // side 0: a = row offset, b = k offset (contiguous);  side 1: a = k, b = row
        const int rr = P.side == 0 ? a : b, ll = P.side == 0 ? b : a;
        x[it] = load_tile_elem(P, r0 + rr, l0 + ll);
    }
#pragma unroll
    for (int it = 0; it < kPer; ++it) {
        const int a = t / kST + it * (256 / kST), b = t % kST;
        const int rr = P.side == 0 ? a : b, ll = P.side == 0 ? b : a;
        bad |= (x[it] >= P.p);
        tile[rr][ll] = x[it];
    }
    if (P.validate && bad) atomicExch(P.err + 1, 1);
    __syncthreads();
}

// Next Alg. 4 word of the running value T (exact division by alpha through
// the reciprocal mu = floor((2^64 - 1) / alpha)); the last word is T itself.
__device__ __forceinline__ double alg4_next(uint64_t &T, uint64_t alpha, uint64_t mu, bool last) {
    if (last) return (double)T;
    uint64_t R = __umul64hi(T, mu);
    uint64_t rem = T - R * alpha;
    while (rem >= alpha) {  // at most two corrections
        ++R;
        rem -= alpha;
    }
    T = R;
    return (double)rem;
}

// INT8 digits through bytes: with c = 128 (1 + 256 + ... + 256^(u-2)),
// t = s + c = sum_{i<u-1} (d_i + 128) 256^i + d_{u-1} 256^(u-1), and every
// d_i + 128 lies in [0, 255], so the lower digits are the bytes of t minus
// 128 and the top digit is t >> 8 (u-1) (arithmetic shift).
__device__ __forceinline__ float int8_digit(int64_t t, int w, bool last) {
    if (last) return small_int_float((int)(t >> (8 * w)));
    const uint32_t half = w < 4 ? (uint32_t)t : (uint32_t)((uint64_t)t >> 32);
    return byte_digit_float(half, w & 3);
}

// FP64 form: a 64 x 64 tile covers 4 k-blocks of 16 doubles, 8 granules each.
__device__ __forceinline__ void split_fp64_tile(const SplitParams &P, uint64_t (*tile)[kST + 1], int64_t by,
                                                int64_t bx) {
    const int64_t r0 = by * kST, l0 = bx * kST;
    load_tile(P, tile, r0, l0);
    // units: (row, granule) with 32 granules (2 doubles) per row of the tile
    for (int unit = threadIdx.x; unit < kST * 32; unit += 256) {
        const int rr = unit / 32, gg = unit % 32;
        const int64_t kb = (l0 / kF64KB) + gg / 8;
        if (kb >= P.nkb) continue;
        const int g = gg % 8;
        uint64_t T0 = tile[rr][2 * gg], T1 = tile[rr][2 * gg + 1];
        const int64_t r = r0 + rr;
        if (r >= P.rows_pad) continue;  // a last row tile may be partial (rows_pad < 64)
        for (int w = 0; w < P.words; ++w) {
            const bool last = (w == P.words - 1);
            const double w0 = alg4_next(T0, P.alpha, P.mu, last);
            const double w1 = alg4_next(T1, P.alpha, P.mu, last);
            uint8_t *dst = P.out + ((int64_t)w * P.wstride + kb * P.kstride + r) * kTileBytes +
                           ((g ^ (int)(r & 7)) * 16);
            *reinterpret_cast<double2 *>(dst) = make_double2(w0, w1);
        }
    }
}

// INT8 form: a 64 x 64 tile is exactly one k-block of 64 bf16, 8 granules.
__device__ __forceinline__ void split_int8_tile(const SplitParams &P, uint64_t (*tile)[kST + 1], int64_t by,
                                                int64_t bx) {
    const int64_t r0 = by * kST, l0 = bx * kST;
    load_tile(P, tile, r0, l0);
    const int64_t kb = l0 / kTcKB;
    const uint64_t half = (P.p - 1) / 2;
    for (int unit = threadIdx.x; unit < kST * 8; unit += 256) {
        const int rr = unit / 8, g = unit % 8;
        const int64_t r = r0 + rr;
        if (r >= P.rows_pad) continue;  // a last row tile may be partial (rows_pad 16 or 32)
        // word w of the unit's 8 entries, packed bf16, to its swizzled 16-byte granule
        auto store = [&](int w, const float (&f)[8]) {
            uint8_t *dst = P.out + ((int64_t)(w + P.wpad) * P.wstride + kb * P.kstride + r) * kTileBytes +
                           ((g ^ (int)(r & 7)) * 16);
            *reinterpret_cast<uint4 *>(dst) = make_uint4(pack_bf16x2(f[0], f[1]), pack_bf16x2(f[2], f[3]),
                                                         pack_bf16x2(f[4], f[5]), pack_bf16x2(f[6], f[7]));
        };
        if (P.crt) {
            uint32_t x0[8], x1[8], x2[8];  // 18-bit limbs
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint64_t x = tile[rr][8 * g + e];
                x0[e] = (uint32_t)x & 0x3FFFFu;
                x1[e] = (uint32_t)(x >> 18) & 0x3FFFFu;
                x2[e] = (uint32_t)(x >> 36);
            }
            for (int w = 0; w < P.words; ++w) {
                const uint32_t m = P.cm[w], M = P.cM[w], c18 = P.c18[w], c36 = P.c36[w];
                const float cmh = P.cmh[w];
                float f[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) f[e] = signed_residue(x0[e], x1[e], x2[e], m, M, c18, c36, cmh);
                store(w, f);
            }
        } else {
            int64_t t[8];  // signed representative + digit bias
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint64_t x = tile[rr][8 * g + e];
                t[e] = ((x <= half) ? (int64_t)x : (int64_t)x - (int64_t)P.p) + P.cbias;
            }
            for (int w = 0; w < P.words; ++w) {
                const bool last = (w == P.words - 1);
                float f[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) f[e] = int8_digit(t[e], w, last);
                store(w, f);
            }
        }
        for (int z = 0; z < P.wpad; ++z) {  // the zero words on both sides
            const int64_t base = kb * P.kstride + r;
            const uint4 zero = make_uint4(0, 0, 0, 0);
            *reinterpret_cast<uint4 *>(P.out + ((int64_t)z * P.wstride + base) * kTileBytes + ((g ^ (int)(r & 7)) * 16)) = zero;
            *reinterpret_cast<uint4 *>(P.out + ((int64_t)(P.wpad + P.words + z) * P.wstride + base) * kTileBytes +
                                       ((g ^ (int)(r & 7)) * 16)) = zero;
        }
    }
}

__global__ void __launch_bounds__(256) split_fp64_kernel(const __grid_constant__ SplitParams P) {
    __shared__ uint64_t tile[kST][kST + 1];
    split_fp64_tile(P, tile, blockIdx.y, blockIdx.x);
}

__global__ void __launch_bounds__(256) split_int8_kernel(const __grid_constant__ SplitParams P) {
    __shared__ uint64_t tile[kST][kST + 1];
    split_int8_tile(P, tile, blockIdx.y, blockIdx.x);
}

// Batched: block b splits tile blocks[b] = (job, tile row, tile col) of jobs[job].
__global__ void __launch_bounds__(256) split_batched_kernel(const SplitParams *jobs, const int4 *blocks,
                                                            int fp64) {
    __shared__ uint64_t tile[kST][kST + 1];
    __shared__ __align__(16) SplitParams P;  // staged once (all threads copy): the loops read it many times
    const int4 bl = blocks[blockIdx.x];
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(jobs + bl.x);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&P);
        for (int w = threadIdx.x; w < (int)(sizeof(SplitParams) / 4); w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    if (fp64) split_fp64_tile(P, tile, bl.y, bl.z);
    else split_int8_tile(P, tile, bl.y, bl.z);
}

SplitParams make_split_params(const Plan &pl, int side, const uint64_t *M, int64_t ld, void *words) {
    SplitParams P;
    P.M = M;
    P.ld = ld;
    P.side = side;
    P.rows = side == 0 ? pl.m : pl.n;
    P.K = pl.k;
    P.rows_pad = side == 0 ? pl.A_rows : pl.B_rows;
    P.nkb = pl.nkb;
    P.out = static_cast<uint8_t *>(words);
    P.words = side == 0 ? pl.u : pl.v;
    P.wstride = side == 0 ? pl.A_wstride : pl.B_wstride;
    P.kstride = side == 0 ? pl.A_kstride : pl.B_kstride;
    P.wpad = side == 0 ? 0 : pl.B_wpad;
    P.p = pl.p;
    P.alpha = side == 0 ? pl.alpha : pl.beta;
    P.mu = P.alpha >= 2 ? (~uint64_t(0)) / P.alpha : 0;
    P.validate = pl.validate;
    P.err = pl.err_dev;
    P.crt = pl.form == MWMM_FORM_CRT8;
    P.cbias = 0;
    for (int i = 0; i + 1 < P.words && !P.crt && pl.form != MWMM_FORM_FP64; ++i) P.cbias += (int64_t)128 << (8 * i);
    for (int i = 0; i < kMaxCrt; ++i) {
        const uint32_t m = i < pl.crt_s ? pl.crt_m[i] : 3;
        P.cm[i] = m;
        P.cM[i] = (uint32_t)((uint64_t(1) << 32) / m + 1);
        P.c18[i] = (uint32_t)((uint64_t(1) << 18) % m);
        P.c36[i] = (uint32_t)((uint64_t(1) << 36) % m);
        P.cmh[i] = 12582912.0f + (float)(m >> 1);
    }
    return P;
}

}  // namespace

size_t split_job_bytes() { return sizeof(SplitParams); }

// Host side of the batched split: fill the job record for (plan, side) into
// `job` (sizeof(SplitParams) bytes) and append its tile blocks to `blocks`
// as (job index, tile row, tile col, 0).
void split_job(const Plan &pl, int side, const uint64_t *M, int64_t ld, void *words, void *job, int job_index,
               std::vector<int> &blocks) {
    SplitParams P = make_split_params(pl, side, M, ld, words);
    std::memcpy(job, &P, sizeof(P));
    if (pl.nkb == 0 || P.rows_pad == 0) return;
    const int64_t kcols = pl.nkb * pl.kb_elems;
    const int64_t gx = (kcols + kST - 1) / kST, gy = (P.rows_pad + kST - 1) / kST;
    for (int64_t y = 0; y < gy; ++y)
        for (int64_t x = 0; x < gx; ++x) {
            blocks.push_back(job_index);
            blocks.push_back((int)y);
            blocks.push_back((int)x);
            blocks.push_back(0);
        }
}

int launch_split_batched(const void *jobs, const int *blocks, int nblocks, int fp64, void *stream) {
    if (nblocks == 0) return 0;
    split_batched_kernel<<<nblocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const SplitParams *>(jobs), reinterpret_cast<const int4 *>(blocks), fp64);
    return (int)cudaGetLastError();
}

int launch_split(const Plan &pl, int side, const uint64_t *M, int64_t ld, void *words, void *stream) {
    const SplitParams P = make_split_params(pl, side, M, ld, words);
    if (pl.nkb == 0 || P.rows_pad == 0) return 0;
    const int64_t kcols = pl.nkb * pl.kb_elems;
    dim3 grid((unsigned)((kcols + kST - 1) / kST), (unsigned)((P.rows_pad + kST - 1) / kST));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (pl.form == MWMM_FORM_FP64) {
        // Words equal to the input when u == 1 (alpha = p): Alg. 4 has no loop.
        split_fp64_kernel<<<grid, 256, 0, s>>>(P);
    } else {
        split_int8_kernel<<<grid, 256, 0, s>>>(P);
    }
    return (int)cudaGetLastError();
}

}  // namespace mwmm
