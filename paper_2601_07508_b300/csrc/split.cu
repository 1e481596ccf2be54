// Split kernels: uint64 matrices -> word matrices in the tiled layout.
//
// FP64 form: Alg. 4 (MW-Decomposition) with integer alpha = ceil(p^(1/u)):
//   T = M; for i < u-1 { R = floor(T / alpha); M_i = T - alpha R; T = R }; M_{u-1} = T.
// The quotient is taken in exact 64-bit integer arithmetic (a Barrett
// reciprocal of alpha plus a correction); Lemma 3.1 shows that the paper's
// floor(fl(T / alpha)) is the same integer, so the words are identical.
//
// INT8 form: the signed representative s of M mod p (M, or M - p when
// M > (p-1)/2) is written as base-2^b digits, s = sum_i R^i d_i (R = 2^b,
// h = R / 2): balanced digits in [-h, h - 1] and a top digit in [-h, h] (the
// remainder).  b = 8: the digits are stored exactly as bf16; b = 9: exactly
// as fp16 (integers up to 2^11 are exact in fp16, 2^8 in bf16).
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
#include <cuda_fp16.h>

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
    int64_t cbias;              // INT8 form: h (1 + R + ... + R^(words-2))
    int bits;                   // INT8 form: digit width b (8: bf16 words, 9: fp16 words)
    int crt;                    // CRT form: residues instead of digits
    // 9-bit digits with certified chunks: per word w, k-block kb and group of
    // 64 rows g, the largest sum over the k-block of a row's squared digits,
    // at sq[(w nkb + kb) (rows_pad / 64) + g]; nullptr: not written
    uint32_t *sq;
    float cmf[kMaxCrt];         // moduli m_i (odd primes below 256)
    float cinv[kMaxCrt];        // fl(1 / m_i), correctly rounded
    float c11[kMaxCrt], c22[kMaxCrt], c33[kMaxCrt], c44[kMaxCrt];  // 2^(11 j) mod m_i
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
// Two small integers as fp16 x 2 without the conversion pipe: for |v| < 512
// the fp16 with bit pattern 0x6600 + v is 1536 + v exactly (binade
// [1024, 2048), unit spacing), so one packed fp16 subtraction of 1536 leaves
// v exactly in both halves.  lo and hi are the patterns 0x6600 + v.
__device__ __forceinline__ uint32_t f16x2_from_biased(uint32_t lo, uint32_t hi) {
    const uint32_t packed = __byte_perm(lo, hi, 0x5410u);
    const uint32_t k1536 = 0x66006600u;
    const __half2 h = __hsub2(*reinterpret_cast<const __half2 *>(&packed), *reinterpret_cast<const __half2 *>(&k1536));
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Signed residue of x < 2^52 modulo an odd m < 256, in [-(m-1)/2, (m-1)/2],
// on the FP32 pipe.  From the 11-bit limbs x = sum_{j<5} x_j 2^(11 j),
// z = x_0 + sum_{j>=1} x_j (2^(11 j) mod m) <= 2047 + 3 * 2047 * 250 + 255 * 250
// < 2^21 is congruent to x, and every partial sum is an integer that FP32
// holds exactly.  q = rint(z fl(1/m)) equals rint(z / m): fl(1/m) is within a
// relative 2^-24 of 1/m, so the product is within 2^21 2^-24 / m = 0.125 / m
// of z / m, while z / m (m odd) lies at least 0.5 / m from every
// half-integer.  r = z - q m is then exact in one FMA, and it is the residue
// of x nearest to zero, i.e. the balanced one.
__device__ __forceinline__ float signed_residue(const float (&xl)[5], float m, float inv, float c11, float c22,
                                                float c33, float c44) {
    const float z = __fmaf_rn(xl[4], c44, __fmaf_rn(xl[3], c33, __fmaf_rn(xl[2], c22, __fmaf_rn(xl[1], c11, xl[0]))));
    const float q = __fsub_rn(__fmaf_rn(z, inv, kMagic), kMagic);
    return __fmaf_rn(-q, m, z);
}
// The five 11-bit limbs of x as FP32 integers (2^23 + limb through the
// exponent pattern, minus 2^23).  The top limb takes every bit from 44 up, so
// an entry >= 2^52 (outside the preconditions) still yields finite values.
__device__ __forceinline__ void limbs11(uint64_t x, float (&xl)[5]) {
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    const uint32_t l[5] = {lo & 0x7FFu, (lo >> 11) & 0x7FFu, __funnelshift_r(lo, hi, 22) & 0x7FFu, (hi >> 1) & 0x7FFu,
                           hi >> 12};
#pragma unroll
    for (int j = 0; j < 5; ++j) xl[j] = __int_as_float(0x4B000000 | (int)l[j]) - 8388608.0f;
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
// 9-bit digits the same way (in split_int8_tile): c = 256 (1 + 512 + ... +
// 512^(u-2)), the lower digits are the 9-bit fields of t minus 256, the top
// one t >> 9 (u-1) (|digit| <= 256), each taken as the fp16 pattern
// 0x6600 + digit: a lower digit's field f gives 0x6600 + f - 256 = 0x6500 + f.

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
// kSq: also the squared-digit maxima (P.sq set; a separate instantiation
// keeps the other kernels' registers down)
template <bool kSq>
__device__ __forceinline__ void split_int8_tile(const SplitParams &P, uint64_t (*tile)[kST + 1], int64_t by,
                                                int64_t bx) {
    const int64_t r0 = by * kST, l0 = bx * kST;
    load_tile(P, tile, r0, l0);
    const int64_t kb = l0 / kTcKB;
    const uint64_t half = (P.p - 1) / 2;
    // squared-digit maxima of this tile's 64 rows, per word (kSq: its plans have rows_pad a multiple of 128, so no unit
    // below skips and every lane takes part in the shuffles)
    // (each unit stores its 8 digits' squares per word; one pass at the end
    // adds a row's 8 units and takes the largest row)
    __shared__ uint32_t s_sq[kSq ? kMaxWords * kST * 8 : 1];
    __shared__ uint32_t s_sqmax[kMaxWords];
    if (kSq) {
        if (threadIdx.x < kMaxWords) s_sqmax[threadIdx.x] = 0;
    }
    // Loop invariants read once per tile: in the batched kernels P sits in
    // shared memory, where every field read inside the loops below would be
    // a shared-memory load.
    const int words = P.words, wpad = P.wpad;
    const bool crt = P.crt != 0, nine = P.bits == 9;
    const int64_t rows_pad = P.rows_pad;
    const int64_t wbytes = P.wstride * kTileBytes;  // bytes between consecutive words
    uint8_t *const out_kb = P.out + kb * P.kstride * kTileBytes;
    const int64_t pm = (int64_t)P.p, cbias = P.cbias;
    for (int unit = threadIdx.x; unit < kST * 8; unit += 256) {
        const int rr = unit / 8, g = unit % 8;
        const int64_t r = r0 + rr;
        if (r >= rows_pad) continue;  // a last row tile may be partial (rows_pad 16 or 32)
        // the unit's 16-byte granule of word 0 (words follow every wbytes bytes);
        // each word holds the unit's 8 entries packed bf16 (or fp16)
        uint8_t *const gran = out_kb + r * kTileBytes + ((g ^ (int)(r & 7)) * 16);
        uint8_t *dst = gran + wpad * wbytes;
        auto store = [&](const float (&f)[8]) {
            *reinterpret_cast<uint4 *>(dst) = make_uint4(pack_bf16x2(f[0], f[1]), pack_bf16x2(f[2], f[3]),
                                                         pack_bf16x2(f[4], f[5]), pack_bf16x2(f[6], f[7]));
        };
        if (crt) {
            float xl[8][5];  // 11-bit limbs
#pragma unroll
            for (int e = 0; e < 8; ++e) limbs11(tile[rr][8 * g + e], xl[e]);
            for (int w = 0; w < words; ++w, dst += wbytes) {
                const float m = P.cmf[w], inv = P.cinv[w], c11 = P.c11[w], c22 = P.c22[w], c33 = P.c33[w],
                            c44 = P.c44[w];
                float f[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) f[e] = signed_residue(xl[e], m, inv, c11, c22, c33, c44);
                store(f);
            }
        } else {
            int64_t t[8];  // signed representative + digit bias
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int64_t x = (int64_t)tile[rr][8 * g + e];
                t[e] = ((uint64_t)x <= half ? x : x - pm) + cbias;
            }
            if (nine) {
                // digits from the bottom up: t >> 9 w kept in t (arithmetic
                // shift), so each word takes one constant shift per entry
                for (int w = 0; w < words; ++w, dst += wbytes) {
                    const bool last = (w == words - 1);
                    uint32_t h[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        h[e] = last ? 0x6600u + (uint32_t)(int)t[e] : 0x6500u + ((uint32_t)t[e] & 511u);
                        t[e] >>= 9;
                    }
                    *reinterpret_cast<uint4 *>(dst) =
                        make_uint4(f16x2_from_biased(h[0], h[1]), f16x2_from_biased(h[2], h[3]),
                                   f16x2_from_biased(h[4], h[5]), f16x2_from_biased(h[6], h[7]));
                    if (kSq) {  // this unit's squared digits (<= 8 x 2^16)
                        uint32_t q = 0;
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int d = (int)h[e] - 0x6600;
                            q += (uint32_t)(d * d);
                        }
                        s_sq[w * (kST * 8) + unit] = q;
                    }
                }
            } else {
                for (int w = 0; w < words; ++w, dst += wbytes) {
                    const bool last = (w == words - 1);
                    float f[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) f[e] = int8_digit(t[e], w, last);
                    store(f);
                }
            }
        }
        const uint4 zero = make_uint4(0, 0, 0, 0);
        for (int z = 0; z < wpad; ++z) {  // the zero words on both sides
            *reinterpret_cast<uint4 *>(gran + z * wbytes) = zero;
            *reinterpret_cast<uint4 *>(gran + (wpad + words + z) * wbytes) = zero;
        }
    }
    if (kSq) {
        __syncthreads();
        // row sums (<= 2^22), the largest per word: a warp covers 32 rows of one word
        for (int i = threadIdx.x; i < P.words * kST; i += blockDim.x) {
            const uint32_t *q = s_sq + i * 8;
            uint32_t row = q[0] + q[1] + q[2] + q[3] + q[4] + q[5] + q[6] + q[7];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) row = max(row, __shfl_xor_sync(0xffffffffu, row, o));
            if ((threadIdx.x & 31) == 0) atomicMax(&s_sqmax[i / kST], row);
        }
        __syncthreads();
        if ((int)threadIdx.x < P.words)
            P.sq[((int64_t)threadIdx.x * P.nkb + kb) * (P.rows_pad / kST) + by] = s_sqmax[threadIdx.x];
    }
}

__global__ void __launch_bounds__(256) split_fp64_kernel(const __grid_constant__ SplitParams P) {
    __shared__ uint64_t tile[kST][kST + 1];
    split_fp64_tile(P, tile, blockIdx.y, blockIdx.x);
}

template <bool kSq>
__global__ void __launch_bounds__(256, 4) split_int8_kernel(const __grid_constant__ SplitParams P) {
    __shared__ uint64_t tile[kST][kST + 1];
    split_int8_tile<kSq>(P, tile, blockIdx.y, blockIdx.x);
}

// Batched: CTA c splits the tiles blocks[c * per, c * per + per) (each
// (job, tile row, tile col) of jobs[job]; a job's tiles are consecutive in
// the list).  The job's parameters are staged into shared memory only when
// the job changes: a CTA per tile spent a good part of its short life on
// that copy and its barrier (measured: 4.3 TB/s against 6.2 for the
// single-product split).
constexpr int kSplitTilesPerCta = 8;

// kSq: jobs with P.sq set also write their squared-digit maxima (its own
// kernel, launched when some job of the batch does; held to 3 CTAs per SM,
// where 4 would spill)
template <bool kSq, bool kFp64>
__device__ __forceinline__ void split_batched_body(const SplitParams *jobs, const int4 *blocks, int nblocks) {
    __shared__ uint64_t tile[kST][kST + 1];
    __shared__ __align__(16) SplitParams P;  // the loops read it many times
    const int b0 = blockIdx.x * kSplitTilesPerCta;
    const int b1 = b0 + kSplitTilesPerCta < nblocks ? b0 + kSplitTilesPerCta : nblocks;
    int job = -1;
    for (int b = b0; b < b1; ++b) {
        const int4 bl = blocks[b];
        __syncthreads();  // every thread is done with the previous tile (and P)
        if (bl.x != job) {  // block-uniform
            const uint32_t *src = reinterpret_cast<const uint32_t *>(jobs + bl.x);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&P);
            for (int w = threadIdx.x; w < (int)(sizeof(SplitParams) / 4); w += blockDim.x) dst[w] = src[w];
            job = bl.x;
            __syncthreads();
        }
        if (kFp64)
            split_fp64_tile(P, tile, bl.y, bl.z);
        else if (kSq && P.sq)  // block-uniform: P is in shared memory
            split_int8_tile<kSq>(P, tile, bl.y, bl.z);
        else
            split_int8_tile<false>(P, tile, bl.y, bl.z);
    }
}

// One kernel per job kind, so that each carries only its own path's registers:
// FP64 words, INT8 digits / CRT residues, and the same with squared-digit maxima.
template <bool kFp64>
__global__ void __launch_bounds__(256, 4) split_batched_kernel(const SplitParams *jobs, const int4 *blocks,
                                                            int nblocks) {
    split_batched_body<false, kFp64>(jobs, blocks, nblocks);
}

__global__ void __launch_bounds__(256, 3) split_batched_sq_kernel(const SplitParams *jobs, const int4 *blocks,
                                                               int nblocks) {
    split_batched_body<true, false>(jobs, blocks, nblocks);
}

SplitParams make_split_params(const Plan &pl, int side, const uint64_t *M, int64_t ld, void *words) {
    SplitParams P;
    P.sq = nullptr;
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
    P.bits = pl.form == MWMM_FORM_INT8 ? pl.digit_bits : 8;
    P.cbias = 0;
    for (int i = 0; i + 1 < P.words && !P.crt && pl.form != MWMM_FORM_FP64; ++i)
        P.cbias += (int64_t)1 << (P.bits - 1 + P.bits * i);
    for (int i = 0; i < kMaxCrt; ++i) {
        const uint32_t m = i < pl.crt_s ? pl.crt_m[i] : 3;
        P.cmf[i] = (float)m;
        P.cinv[i] = 1.0f / (float)m;  // IEEE single division: correctly rounded
        P.c11[i] = (float)((uint64_t(1) << 11) % m);
        P.c22[i] = (float)((uint64_t(1) << 22) % m);
        P.c33[i] = (float)((uint64_t(1) << 33) % m);
        P.c44[i] = (float)((uint64_t(1) << 44) % m);
    }
    return P;
}

}  // namespace

size_t split_job_bytes() { return sizeof(SplitParams); }

// Host side of the batched split: fill the job record for (plan, side) into
// `job` (sizeof(SplitParams) bytes) and append its tile blocks to `blocks`
// as (job index, tile row, tile col, 0).
void split_job(const Plan &pl, int side, const uint64_t *M, int64_t ld, void *words, void *job, int job_index,
               std::vector<int> &blocks, uint32_t *sq) {
    SplitParams P = make_split_params(pl, side, M, ld, words);
    if (sq && pl.tc_cert_chunk && pl.form == MWMM_FORM_INT8 && pl.digit_bits == 9 && P.rows_pad % (2 * kST) == 0)
        P.sq = sq;
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

int launch_split_batched(const void *jobs, const int *blocks, int nblocks, int fp64, void *stream, int sq) {
    if (nblocks == 0) return 0;
    const int ctas = (nblocks + kSplitTilesPerCta - 1) / kSplitTilesPerCta;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const SplitParams *J = static_cast<const SplitParams *>(jobs);
    const int4 *blk = reinterpret_cast<const int4 *>(blocks);
    if (fp64)
        split_batched_kernel<true><<<ctas, 256, 0, s>>>(J, blk, nblocks);
    else if (sq)
        split_batched_sq_kernel<<<ctas, 256, 0, s>>>(J, blk, nblocks);
    else
        split_batched_kernel<false><<<ctas, 256, 0, s>>>(J, blk, nblocks);
    return (int)cudaGetLastError();
}

int launch_split(const Plan &pl, int side, const uint64_t *M, int64_t ld, void *words, void *stream, uint32_t *sq) {
    SplitParams P = make_split_params(pl, side, M, ld, words);
    // squared-digit maxima only for the certified-chunk plans' own layout
    if (sq && pl.tc_cert_chunk && pl.form == MWMM_FORM_INT8 && pl.digit_bits == 9 && P.rows_pad % (2 * kST) == 0)
        P.sq = sq;
    if (pl.nkb == 0 || P.rows_pad == 0) return 0;
    const int64_t kcols = pl.nkb * pl.kb_elems;
    dim3 grid((unsigned)((kcols + kST - 1) / kST), (unsigned)((P.rows_pad + kST - 1) / kST));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (pl.form == MWMM_FORM_FP64) {
        // Words equal to the input when u == 1 (alpha = p): Alg. 4 has no loop.
        split_fp64_kernel<<<grid, 256, 0, s>>>(P);
    } else {
        if (P.sq)
            split_int8_kernel<true><<<grid, 256, 0, s>>>(P);
        else
            split_int8_kernel<false><<<grid, 256, 0, s>>>(P);
    }
    return (int)cudaGetLastError();
}

}  // namespace mwmm
