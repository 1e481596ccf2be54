// Recombination of the INT8 form:
//   C = sum_{s=0}^{u+v-2} gamma_s S_s mod p,  gamma_s = R^s mod p,
//   S_s = sum_{i+j=s} A_i B_j,
// the alpha^i beta^j mod p recombination of Alg. 5 with alpha = beta = R
// (R = 256 for 8-bit digits, 512 for 9-bit ones) and the pairs of equal
// i + j grouped.  B300's FP64 pipe runs at 1/64 of its
// integer rate, so the arithmetic is exact integer arithmetic, not Alg. 1 /
// Alg. 2.
//
// One K-range (nkc = 1, every product with k <= ~18k): |S_s| < 2^31, so
// U_s = S_s + 2^31 is in [0, 2^32).  With gamma_s = gl_s + gh_s 2^26
// (gl_s, gh_s < 2^26) the two sums A0 = sum_s gl_s U_s and A1 = sum_s gh_s U_s
// are exact in 64 bits (at most 15 terms below 2^58), and
//   C = (A0 + 2^26 A1 - 2^31 sum_s gamma_s) mod p,
// which takes three Barrett-type reductions per output instead of one per
// diagonal.  Several K-ranges: Horner's rule X <- (R X + S_s) mod p from
// the top diagonal down (R X < 2^61, |sum of the ranges| < nkc 2^31, so
// y = R X + S_s + off with off = p ceil(2^31 nkc / p) lies in [0, 2^64)).
#include <cstring>
#include <vector>

#include "device_common.cuh"
#include "mwmm_internal.h"

namespace mwmm {

namespace {

struct RecParams {
    const int32_t *S;
    uint64_t *C;
    int64_t ldc, m, n, A_rows, B_rows;
    int nsums, nkc;
    int rbits;            // digit width: radix 2^rbits
    uint64_t p, mu, off;  // mu = floor((2^64 - 1) / p)
    uint64_t mu90;        // floor(2^90 / p) when p > 2^26, else 0 (then every gh_s = 0)
    uint64_t K;           // (-2^31 sum_s gamma_s) mod p
    uint32_t gl[2 * kMaxWords], gh[2 * kMaxWords];
    int vec;  // C 16-byte aligned with an even ldc: four outputs leave as two 16-byte stores
};

__device__ __forceinline__ uint64_t reduce_u64(uint64_t y, uint64_t p, uint64_t mu) {
    const uint64_t qh = __umul64hi(y, mu);  // floor(y / p) - {0, 1, 2}
    uint64_t r = y - qh * p;
    if (r >= p) r -= p;
    if (r >= p) r -= p;
    return r;
}

// (r 2^26) mod p for r < p, p > 2^26: q = floor(r 2^26 / p) < 2^26 is
// estimated as umulhi(r, floor(2^90 / p)) (too small by at most 1); the
// remainder is below 2p < 2^53, so 64-bit wrap-around arithmetic gives it exactly.
__device__ __forceinline__ uint64_t shl26_mod(uint64_t r, uint64_t p, uint64_t mu90) {
    const uint64_t q = __umul64hi(r, mu90);
    uint64_t rem = (r << 26) - q * p;
    if (rem >= p) rem -= p;
    return rem;
}

// Rows row0, row0 + rstep, ... < P.m of C; each thread produces 4
// consecutive outputs (columns c0 .. c0 + 3) of a row.
__device__ __forceinline__ void recombine_rows(const RecParams &P, int64_t c0, int64_t row0, int64_t rstep) {
    if (c0 >= P.n) return;
    const int64_t plane = P.A_rows * P.B_rows;
    if (P.nkc == 1) {
        for (int64_t row = row0; row < P.m; row += rstep) {
            uint64_t A0[4] = {0, 0, 0, 0}, A1[4] = {0, 0, 0, 0};
            const int32_t *src = P.S + row * P.B_rows + c0;
            // four planes per round: their loads are issued together
            for (int s0 = 0; s0 < P.nsums; s0 += 4) {
                int4 v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (s0 + j < P.nsums) v[j] = __ldcs(reinterpret_cast<const int4 *>(src + (int64_t)(s0 + j) * plane));
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (s0 + j >= P.nsums) break;
                    const uint32_t U[4] = {(uint32_t)v[j].x + 0x80000000u, (uint32_t)v[j].y + 0x80000000u,
                                           (uint32_t)v[j].z + 0x80000000u, (uint32_t)v[j].w + 0x80000000u};
                    const uint32_t gl = P.gl[s0 + j], gh = P.gh[s0 + j];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        A0[e] += (uint64_t)gl * U[e];  // 32 x 32 -> 64
                        A1[e] += (uint64_t)gh * U[e];
                    }
                }
            }
            uint64_t *out = P.C + row * P.ldc + c0;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                uint64_t r = reduce_u64(A0[e] + P.K, P.p, P.mu);
                if (P.mu90) {
                    r += shl26_mod(reduce_u64(A1[e], P.p, P.mu), P.p, P.mu90);
                    if (r >= P.p) r -= P.p;
                }
                if (c0 + e < P.n) out[e] = r;
            }
        }
        return;
    }
    for (int64_t row = row0; row < P.m; row += rstep) {
    uint64_t R[4] = {0, 0, 0, 0};
    for (int s = P.nsums - 1; s >= 0; --s) {
        int64_t x[4] = {0, 0, 0, 0};
        for (int kc = 0; kc < P.nkc; ++kc) {
            const int4 v = *reinterpret_cast<const int4 *>(P.S + ((int64_t)s * P.nkc + kc) * plane +
                                                           row * P.B_rows + c0);
            x[0] += v.x; x[1] += v.y; x[2] += v.z; x[3] += v.w;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e)
            R[e] = reduce_u64((R[e] << P.rbits) + (uint64_t)(x[e] + (int64_t)P.off), P.p, P.mu);
    }
    uint64_t *out = P.C + row * P.ldc + c0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (c0 + e < P.n) out[e] = R[e];
    }
}

__global__ void __launch_bounds__(256) recombine_kernel(const __grid_constant__ RecParams P) {
    recombine_rows(P, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4, blockIdx.y, gridDim.y);
}

// One K-range with S sums known at compile time (the common case), and kWide
// (p > 2^26) selecting the second accumulator, so the narrow primes carry no
// dead work.  Below 8 sums the loads of all S planes are issued together;
// from 8 sums on they go in groups of 4 and the kernel is held to 64
// registers (4 blocks per SM): measured on B300 at 4096^2 outputs, that
// occupancy hides more latency than the few spilled registers cost (9 sums:
// 0.138 vs 0.145 ms, 13 sums: 0.18-0.19 vs 0.20 ms; below 8 sums a
// register cap only adds spills and scheduling constraints).  Same arithmetic
// as the nkc == 1 branch of recombine_rows.
template <int S, bool kWide, int G>
__device__ __forceinline__ void recombine_quad_s(const RecParams &P, int64_t row, int64_t c0) {
    const int64_t plane = P.A_rows * P.B_rows;
    {
        const int32_t *src = P.S + row * P.B_rows + c0;
        uint64_t A0[4] = {0, 0, 0, 0}, A1[4] = {0, 0, 0, 0};
#pragma unroll
        for (int g = 0; g < S; g += G) {
            int4 v[G];
#pragma unroll
            for (int j = 0; j < G; ++j)
                if (g + j < S) v[j] = __ldcs(reinterpret_cast<const int4 *>(src + (int64_t)(g + j) * plane));
#pragma unroll
            for (int j = 0; j < G; ++j) {
                if (g + j >= S) break;
                const uint32_t U[4] = {(uint32_t)v[j].x + 0x80000000u, (uint32_t)v[j].y + 0x80000000u,
                                       (uint32_t)v[j].z + 0x80000000u, (uint32_t)v[j].w + 0x80000000u};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    A0[e] += (uint64_t)P.gl[g + j] * U[e];
                    if (kWide) A1[e] += (uint64_t)P.gh[g + j] * U[e];
                }
            }
            if (G < S) asm volatile("" ::: "memory");  // the next group's loads stay behind this group's
        }
        uint64_t r[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            r[e] = reduce_u64(A0[e] + P.K, P.p, P.mu);
            if (kWide) {
                r[e] += shl26_mod(reduce_u64(A1[e], P.p, P.mu), P.p, P.mu90);
                if (r[e] >= P.p) r[e] -= P.p;
            }
        }
        uint64_t *out = P.C + row * P.ldc + c0;
        if (P.vec && c0 + 4 <= P.n) {
            reinterpret_cast<ulonglong2 *>(out)[0] = make_ulonglong2(r[0], r[1]);
            reinterpret_cast<ulonglong2 *>(out)[1] = make_ulonglong2(r[2], r[3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (c0 + e < P.n) out[e] = r[e];
        }
    }
}

template <int S, bool kWide, int G>
__device__ __forceinline__ void recombine_rows_s(const RecParams &P) {
    const int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (c0 >= P.n) return;
    for (int64_t row = blockIdx.y; row < P.m; row += gridDim.y) recombine_quad_s<S, kWide, G>(P, row, c0);
}

template <int S, bool kWide>
__global__ void __launch_bounds__(256) recombine_kernel_s(const __grid_constant__ RecParams P) {
    recombine_rows_s<S, kWide, S>(P);
}

template <int S, bool kWide>
__global__ void __launch_bounds__(256, 4) recombine_kernel_s4(const __grid_constant__ RecParams P) {
    recombine_rows_s<S, kWide, 4>(P);
}

template <int S>
void launch_recombine_s(const RecParams &P, dim3 grid, cudaStream_t st) {
    if constexpr (S >= 8) {
        if (P.mu90)
            recombine_kernel_s4<S, true><<<grid, 256, 0, st>>>(P);
        else
            recombine_kernel_s4<S, false><<<grid, 256, 0, st>>>(P);
    } else {
        if (P.mu90)
            recombine_kernel_s<S, true><<<grid, 256, 0, st>>>(P);
        else
            recombine_kernel_s<S, false><<<grid, 256, 0, st>>>(P);
    }
}

// The (row, 4-column group) units of one batched block with the sum count
// known at compile time (the single-product kernels' arithmetic and loads).
template <int S, bool kWide>
__device__ __forceinline__ void batched_units_s(const RecParams &P, int64_t cb, int64_t y0, int64_t rows,
                                                int64_t groups) {
    for (int64_t u = threadIdx.x; u < rows * groups; u += blockDim.x)
        recombine_quad_s<S, kWide, (S < 5 ? S : 4)>(P, y0 + u / groups, cb + (u % groups) * 4);
}

template <int S>
__device__ __forceinline__ bool batched_try_s(const RecParams &P, int64_t cb, int64_t y0, int64_t rows,
                                              int64_t groups) {
    if (P.nsums != S) return false;
    if (P.mu90)
        batched_units_s<S, true>(P, cb, y0, rows, groups);
    else
        batched_units_s<S, false>(P, cb, y0, rows, groups);
    return true;
}

// Batched: block b handles columns [1024 z, 1024 z + 1024) of rows
// [y0, y0 + 8) of problem jobs[b] = (problem, y0, z, 0); its threads take the
// (row, 4-column group) units of that block in turn, so narrow problems keep
// every thread busy.  One K-range with an odd sum count of 3 to 15 (u = v
// digits) takes a path specialised on that count (block-uniform branch);
// anything else the generic loop.  Held to 64 registers like the
// single-product kernels from 8 sums on (4 blocks per SM).
__global__ void __launch_bounds__(256, 4) recombine_batched_kernel(const RecParams *probs, const int4 *jobs) {
    __shared__ __align__(16) RecParams P;  // staged once (all threads copy): the loops read it many times
    const int4 j = jobs[blockIdx.x];
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(probs + j.x);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&P);
        for (int w = threadIdx.x; w < (int)(sizeof(RecParams) / 4); w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    const int64_t cb = (int64_t)j.z * 1024;
    const int64_t width = P.n - cb < 1024 ? P.n - cb : 1024;
    const int64_t rows = P.m - j.y < 8 ? P.m - j.y : 8;
    const int64_t groups = (width + 3) / 4;
    if (P.nkc == 1 && (batched_try_s<3>(P, cb, j.y, rows, groups) || batched_try_s<5>(P, cb, j.y, rows, groups) ||
                       batched_try_s<7>(P, cb, j.y, rows, groups) || batched_try_s<9>(P, cb, j.y, rows, groups) ||
                       batched_try_s<11>(P, cb, j.y, rows, groups) || batched_try_s<13>(P, cb, j.y, rows, groups) ||
                       batched_try_s<15>(P, cb, j.y, rows, groups)))
        return;
    for (int64_t u = threadIdx.x; u < rows * groups; u += blockDim.x)
        recombine_rows(P, cb + (u % groups) * 4, j.y + u / groups, P.m);
}

RecParams make_rec_params(const Plan &pl, const int32_t *S, uint64_t *C, int64_t ldc) {
    RecParams P;
    P.S = S;
    P.C = C;
    P.ldc = ldc;
    P.m = pl.m;
    P.n = pl.n;
    P.A_rows = pl.A_rows;
    P.B_rows = pl.B_rows;
    P.nsums = pl.nsums;
    P.nkc = pl.nkc;
    P.rbits = pl.digit_bits;
    P.p = pl.p;
    P.vec = (reinterpret_cast<uintptr_t>(C) % 16 == 0 && ldc % 2 == 0) ? 1 : 0;
    P.mu = (~uint64_t(0)) / pl.p;
    const unsigned __int128 need = (unsigned __int128)pl.nkc << 31;
    P.off = (uint64_t)((need + pl.p - 1) / pl.p * pl.p);
    P.mu90 = pl.p > (uint64_t(1) << 26) ? (uint64_t)(((unsigned __int128)1 << 90) / pl.p) : 0;
    uint64_t g = 1 % pl.p, gsum = 0;
    for (int s = 0; s < 2 * kMaxWords; ++s) {
        P.gl[s] = (uint32_t)(g & ((1u << 26) - 1));
        P.gh[s] = (uint32_t)(g >> 26);
        if (s < pl.nsums) gsum = (gsum + g) % pl.p;
        g = mulmod_u64(g, uint64_t(1) << pl.digit_bits, pl.p);
    }
    const uint64_t bias = mulmod_u64(gsum, uint64_t(1) << 31, pl.p);
    P.K = (pl.p - bias) % pl.p;
    return P;
}

}  // namespace

size_t recombine_job_bytes() { return sizeof(RecParams); }

void recombine_job(const Plan &pl, const int32_t *S, uint64_t *C, int64_t ldc, void *rec, int index,
                   std::vector<int> &jobs) {
    const RecParams P = make_rec_params(pl, S, C, ldc);
    std::memcpy(rec, &P, sizeof(P));
    const int64_t cblocks = ((pl.n + 3) / 4 + 255) / 256;
    for (int64_t y = 0; y < pl.m; y += 8)
        for (int64_t c = 0; c < cblocks; ++c) {
            jobs.push_back(index);
            jobs.push_back((int)y);
            jobs.push_back((int)c);
            jobs.push_back(0);
        }
}

int launch_recombine_batched(const void *probs, const int *jobs, int njobs, void *stream) {
    if (njobs == 0) return 0;
    recombine_batched_kernel<<<njobs, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const RecParams *>(probs), reinterpret_cast<const int4 *>(jobs));
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CRT form (multimodular comparison, Sec. 5.2): from the exact sums
// S_i = sum_l a_l b_l over signed residues mod m_i (S_i = C mod m_i, where C
// is the integer product, 0 <= C < M / 2, M = prod m_i), rebuild C mod p:
//   x_i = (S_i mod m_i) y_i  (< m_i^2, not reduced),  y_i = (M / m_i)^-1 mod m_i,
//   C = sum_i x_i (M / m_i) - q M,   q = floor(sum_i x_i / m_i)
// (the textbook CRT formula with unreduced x_i: C / M = sum_i x_i / m_i - q
// lies in [0, 1/2)).  q < 2^13 is evaluated in FP32 as
// floor(0.25 + sum_i x_i fl(1/m_i)): the rounding error stays below 0.01 <<
// 1/4, so the offset makes the floor exact.  Then
//   C mod p = (sum_i x_i w_i - q W) mod p,  w_i = (M / m_i) mod p, W = M mod p,
// with w_i = wh_i 2^26 + wl_i: the sums of x_i wl_i and x_i wh_i (< 2^42
// each) are exact in 64 bits and are combined mod p once per output.
// Remainders by the small moduli take one 32-bit multiply-high: for
// 0 <= a < 2^32, q = umulhi(a, floor(2^32 / m) + 1) is floor(a / m) or one
// more (the multiplier exceeds 2^32 / m by less than 1), so a - q m is
// a mod m or that minus m, and m is added back when it is negative.  A sum
// S (|S| <= 131071 * 2^14 < 2^31 - 2^14) enters as S + O_i with
// O_i = m_i ceil((2^31 - 1) / m_i), which keeps it in [0, 2^32) and
// congruent to S.
namespace {

struct CrtParams {
    const int32_t *S;
    uint64_t *C;
    int64_t ldc, m, n, A_rows, B_rows;
    int s, nkc;
    uint64_t p, mu, mu90, W;  // mu90 = floor(2^90 / p) when p > 2^26, else 0
    uint32_t cm[kMaxCrt], cy[kMaxCrt];
    uint32_t cB[kMaxCrt];     // floor(2^32 / m_i) + 1
    uint32_t cO[kMaxCrt];     // m_i ceil((2^31 - 1) / m_i)
    uint32_t wl[kMaxCrt], wh[kMaxCrt];  // w_i = wh_i 2^26 + wl_i
    float rinv[kMaxCrt];
};

// a mod m for 0 <= a < 2^32 (see above); B = floor(2^32 / m) + 1.
__device__ __forceinline__ uint32_t mod_small(uint32_t a, uint32_t m, uint32_t B) {
    int r = (int)(a - __umulhi(a, B) * m);
    r += (r >> 31) & (int)m;
    return (uint32_t)r;
}

// FP32 value of an integer 0 <= x < 2^22 without the conversion pipe: the
// bit pattern 0x4B400000 + x is 1.5 * 2^23 + x.
__device__ __forceinline__ float small_uint_float(uint32_t x) {
    return __int_as_float(0x4B400000 + (int)x) - 12582912.0f;
}

// C mod p from the per-output sums a0 + 2^26 a1 = sum_i x_i w_i and the
// quotient estimate qf (see above).
__device__ __forceinline__ void crt_store(const CrtParams &P, const uint64_t (&a0)[4], const uint64_t (&a1)[4],
                                          const float (&qf)[4], uint64_t *out, int64_t c0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const uint64_t q = (uint64_t)floorf(qf[e]);  // < 2^13
        // sum_i x_i w_i = a0 + 2^26 a1, and q W = q Wl + 2^26 q Wh
        uint64_t lo = reduce_u64(a0[e], P.p, P.mu), hi = reduce_u64(a1[e], P.p, P.mu);
        const uint64_t qlo = reduce_u64(q * (P.W & ((1u << 26) - 1)), P.p, P.mu);
        const uint64_t qhi = reduce_u64(q * (P.W >> 26), P.p, P.mu);
        lo = lo >= qlo ? lo - qlo : lo + P.p - qlo;
        hi = hi >= qhi ? hi - qhi : hi + P.p - qhi;
        uint64_t v = lo;
        if (P.mu90) {
            v += shl26_mod(hi, P.p, P.mu90);
            if (v >= P.p) v -= P.p;
        }
        if (c0 + e < P.n) out[e] = v;
    }
}

// One K-range, S moduli known at compile time: the modulus loop unrolls and
// the per-modulus constants become immediate kernel-parameter operands.
template <int S>
__device__ __forceinline__ void crt_rows_s(const CrtParams &P, int64_t c0, int64_t row0, int64_t rstep) {
    if (c0 >= P.n) return;
    const int64_t plane = P.A_rows * P.B_rows;
    for (int64_t row = row0; row < P.m; row += rstep) {
        uint64_t a0[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0};
        float qf[4] = {0.25f, 0.25f, 0.25f, 0.25f};
        const int32_t *src = P.S + row * P.B_rows + c0;
#pragma unroll
        for (int i0 = 0; i0 < S; i0 += 4) {  // four moduli per round: their loads are issued together
            int4 v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (i0 + j < S) v[j] = __ldcs(reinterpret_cast<const int4 *>(src + (int64_t)(i0 + j) * plane));
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (i0 + j >= S) break;
                const int i = i0 + j;
                const int32_t vv[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const uint32_t r = mod_small((uint32_t)vv[e] + P.cO[i], P.cm[i], P.cB[i]);
                    const uint32_t xi = r * P.cy[i];  // < m_i^2 < 2^16
                    qf[e] = __fmaf_rn(small_uint_float(xi), P.rinv[i], qf[e]);
                    a0[e] += (uint64_t)xi * P.wl[i];  // 32 x 32 -> 64
                    a1[e] += (uint64_t)xi * P.wh[i];
                }
            }
        }
        crt_store(P, a0, a1, qf, P.C + row * P.ldc + c0, c0);
    }
}

// Held to 64 registers (4 CTAs per SM): measured on B300 at 4096^2 outputs,
// the occupancy outweighs the spills from about 10 moduli on (16 moduli:
// 0.305 vs 0.368 ms; 7 moduli: 0.145 vs 0.158 ms; 12 moduli: 2% slower).
template <int S>
__global__ void __launch_bounds__(256, 4) crt_kernel_s(const __grid_constant__ CrtParams P) {
    crt_rows_s<S>(P, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4, blockIdx.y, gridDim.y);
}

// One K-range and S moduli: the unrolled rows above, chosen at run time.
__device__ __forceinline__ bool crt_rows_dispatch(const CrtParams &P, int64_t c0, int64_t row0, int64_t rstep) {
    if (P.nkc != 1) return false;
    switch (P.s) {
#define MWMM_CRT_CASE(k) \
    case k: crt_rows_s<k>(P, c0, row0, rstep); return true;
        MWMM_CRT_CASE(1) MWMM_CRT_CASE(2) MWMM_CRT_CASE(3) MWMM_CRT_CASE(4) MWMM_CRT_CASE(5) MWMM_CRT_CASE(6)
        MWMM_CRT_CASE(7) MWMM_CRT_CASE(8) MWMM_CRT_CASE(9) MWMM_CRT_CASE(10) MWMM_CRT_CASE(11) MWMM_CRT_CASE(12)
        MWMM_CRT_CASE(13) MWMM_CRT_CASE(14) MWMM_CRT_CASE(15) MWMM_CRT_CASE(16) MWMM_CRT_CASE(17) MWMM_CRT_CASE(18)
        MWMM_CRT_CASE(19) MWMM_CRT_CASE(20) MWMM_CRT_CASE(21) MWMM_CRT_CASE(22) MWMM_CRT_CASE(23) MWMM_CRT_CASE(24)
#undef MWMM_CRT_CASE
        default: return false;
    }
}

// Any number of moduli and K-ranges, 32-bit arithmetic only: the residues
// of the ranges' sums (each below m_i) are added up (below nkc m_i < 2^24)
// and reduced once.  Rows row0, row0 + rstep, ... < P.m;
// columns c0 .. c0 + 3.
__device__ __forceinline__ void crt_rows(const CrtParams &P, int64_t c0, int64_t row0, int64_t rstep) {
    if (c0 >= P.n) return;
    const int64_t plane = P.A_rows * P.B_rows;
    for (int64_t row = row0; row < P.m; row += rstep) {
        uint64_t a0[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0};
        float qf[4] = {0.25f, 0.25f, 0.25f, 0.25f};
#pragma unroll 4
        for (int i = 0; i < P.s; ++i) {
            const uint32_t mi = P.cm[i], yi = P.cy[i], Bi = P.cB[i], Oi = P.cO[i];
            uint32_t r[4] = {0, 0, 0, 0};
            for (int kc = 0; kc < P.nkc; ++kc) {
                const int4 v = __ldcs(reinterpret_cast<const int4 *>(P.S + ((int64_t)i * P.nkc + kc) * plane +
                                                                     row * P.B_rows + c0));
                const int32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) r[e] += mod_small((uint32_t)vv[e] + Oi, mi, Bi);
            }
            const float ri = P.rinv[i];
            const uint32_t wl = P.wl[i], wh = P.wh[i];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t xi = (P.nkc == 1 ? r[e] : mod_small(r[e], mi, Bi)) * yi;  // one range: r < m_i
                qf[e] = __fmaf_rn(small_uint_float(xi), ri, qf[e]);
                a0[e] += (uint64_t)xi * wl;
                a1[e] += (uint64_t)xi * wh;
            }
        }
        crt_store(P, a0, a1, qf, P.C + row * P.ldc + c0, c0);
    }
}

__global__ void __launch_bounds__(256) crt_kernel(const __grid_constant__ CrtParams P) {
    crt_rows(P, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4, blockIdx.y, gridDim.y);
}

// Batched: block b handles columns [1024 z, 1024 z + 1024) of rows
// [y0, y0 + 8) of problem jobs[b] = (problem, y0, z, 0), like the batched
// recombination.
__global__ void __launch_bounds__(256) crt_batched_kernel(const CrtParams *probs, const int4 *jobs) {
    __shared__ __align__(16) CrtParams P;  // staged once (all threads copy): the loops read it many times
    const int4 j = jobs[blockIdx.x];
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(probs + j.x);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&P);
        for (int w = threadIdx.x; w < (int)(sizeof(CrtParams) / 4); w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    const int64_t cb = (int64_t)j.z * 1024;
    const int64_t width = P.n - cb < 1024 ? P.n - cb : 1024;
    const int64_t rows = P.m - j.y < 8 ? P.m - j.y : 8;
    const int64_t groups = (width + 3) / 4;
    for (int64_t u = threadIdx.x; u < rows * groups; u += blockDim.x) {
        const int64_t c0 = cb + (u % groups) * 4, row = j.y + u / groups;
        if (!crt_rows_dispatch(P, c0, row, P.m)) crt_rows(P, c0, row, P.m);
    }
}

CrtParams make_crt_params(const Plan &pl, const int32_t *S, uint64_t *C, int64_t ldc) {
    CrtParams P;
    std::memset(&P, 0, sizeof(P));
    P.S = S;
    P.C = C;
    P.ldc = ldc;
    P.m = pl.m;
    P.n = pl.n;
    P.A_rows = pl.A_rows;
    P.B_rows = pl.B_rows;
    P.s = pl.crt_s;
    P.nkc = pl.nkc;
    P.p = pl.p;
    P.mu = (~uint64_t(0)) / pl.p;
    P.mu90 = pl.p > (uint64_t(1) << 26) ? (uint64_t)(((unsigned __int128)1 << 90) / pl.p) : 0;
    P.W = pl.crt_W;
    for (int i = 0; i < pl.crt_s; ++i) {
        P.cm[i] = pl.crt_m[i];
        P.cy[i] = pl.crt_y[i];
        P.rinv[i] = 1.0f / (float)pl.crt_m[i];
        P.wl[i] = (uint32_t)(pl.crt_w[i] & ((1u << 26) - 1));
        P.wh[i] = (uint32_t)(pl.crt_w[i] >> 26);
        const uint64_t mi = pl.crt_m[i];
        P.cB[i] = (uint32_t)((uint64_t(1) << 32) / mi + 1);
        P.cO[i] = (uint32_t)(mi * ((((uint64_t)1 << 31) - 1 + mi - 1) / mi));
    }
    return P;
}

}  // namespace

size_t crt_job_bytes() { return sizeof(CrtParams); }

void crt_job(const Plan &pl, const int32_t *S, uint64_t *C, int64_t ldc, void *rec, int index, std::vector<int> &jobs) {
    const CrtParams P = make_crt_params(pl, S, C, ldc);
    std::memcpy(rec, &P, sizeof(P));
    const int64_t cblocks = ((pl.n + 3) / 4 + 255) / 256;
    for (int64_t y = 0; y < pl.m; y += 8)
        for (int64_t c = 0; c < cblocks; ++c) {
            jobs.push_back(index);
            jobs.push_back((int)y);
            jobs.push_back((int)c);
            jobs.push_back(0);
        }
}

int launch_crt_batched(const void *probs, const int *jobs, int njobs, void *stream) {
    if (njobs == 0) return 0;
    crt_batched_kernel<<<njobs, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const CrtParams *>(probs), reinterpret_cast<const int4 *>(jobs));
    return (int)cudaGetLastError();
}

static int launch_crt(const Plan &pl, const int32_t *S, uint64_t *C, int64_t ldc, void *stream) {
    const CrtParams P = make_crt_params(pl, S, C, ldc);
    const int64_t groups = (pl.n + 3) / 4;
    dim3 grid((unsigned)((groups + 255) / 256), (unsigned)(pl.m < 65535 ? pl.m : 65535));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (pl.nkc != 1 || pl.crt_s < 1 || pl.crt_s > kMaxCrt) {
        crt_kernel<<<grid, 256, 0, st>>>(P);
        return (int)cudaGetLastError();
    }
    switch (pl.crt_s) {
        case 1: crt_kernel_s<1><<<grid, 256, 0, st>>>(P); break;
        case 2: crt_kernel_s<2><<<grid, 256, 0, st>>>(P); break;
        case 3: crt_kernel_s<3><<<grid, 256, 0, st>>>(P); break;
        case 4: crt_kernel_s<4><<<grid, 256, 0, st>>>(P); break;
        case 5: crt_kernel_s<5><<<grid, 256, 0, st>>>(P); break;
        case 6: crt_kernel_s<6><<<grid, 256, 0, st>>>(P); break;
        case 7: crt_kernel_s<7><<<grid, 256, 0, st>>>(P); break;
        case 8: crt_kernel_s<8><<<grid, 256, 0, st>>>(P); break;
        case 9: crt_kernel_s<9><<<grid, 256, 0, st>>>(P); break;
        case 10: crt_kernel_s<10><<<grid, 256, 0, st>>>(P); break;
        case 11: crt_kernel_s<11><<<grid, 256, 0, st>>>(P); break;
        case 12: crt_kernel_s<12><<<grid, 256, 0, st>>>(P); break;
        case 13: crt_kernel_s<13><<<grid, 256, 0, st>>>(P); break;
        case 14: crt_kernel_s<14><<<grid, 256, 0, st>>>(P); break;
        case 15: crt_kernel_s<15><<<grid, 256, 0, st>>>(P); break;
        case 16: crt_kernel_s<16><<<grid, 256, 0, st>>>(P); break;
        case 17: crt_kernel_s<17><<<grid, 256, 0, st>>>(P); break;
        case 18: crt_kernel_s<18><<<grid, 256, 0, st>>>(P); break;
        case 19: crt_kernel_s<19><<<grid, 256, 0, st>>>(P); break;
        case 20: crt_kernel_s<20><<<grid, 256, 0, st>>>(P); break;
        case 21: crt_kernel_s<21><<<grid, 256, 0, st>>>(P); break;
        case 22: crt_kernel_s<22><<<grid, 256, 0, st>>>(P); break;
        case 23: crt_kernel_s<23><<<grid, 256, 0, st>>>(P); break;
        case 24: crt_kernel_s<24><<<grid, 256, 0, st>>>(P); break;
        default: crt_kernel<<<grid, 256, 0, st>>>(P); break;
    }
    return (int)cudaGetLastError();
}

int launch_recombine(const Plan &pl, const int32_t *S, uint64_t *C, int64_t ldc, void *stream) {
    if (pl.form == MWMM_FORM_CRT8) return pl.m == 0 || pl.n == 0 ? 0 : launch_crt(pl, S, C, ldc, stream);
    const RecParams P = make_rec_params(pl, S, C, ldc);
    if (pl.m == 0 || pl.n == 0) return 0;
    const int64_t groups = (pl.n + 3) / 4;
    dim3 grid((unsigned)((groups + 255) / 256), (unsigned)(pl.m < 65535 ? pl.m : 65535));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (pl.nkc != 1) {
        recombine_kernel<<<grid, 256, 0, st>>>(P);
        return (int)cudaGetLastError();
    }
    switch (pl.nsums) {
        case 1: launch_recombine_s<1>(P, grid, st); break;
        case 2: launch_recombine_s<2>(P, grid, st); break;
        case 3: launch_recombine_s<3>(P, grid, st); break;
        case 4: launch_recombine_s<4>(P, grid, st); break;
        case 5: launch_recombine_s<5>(P, grid, st); break;
        case 6: launch_recombine_s<6>(P, grid, st); break;
        case 7: launch_recombine_s<7>(P, grid, st); break;
        case 8: launch_recombine_s<8>(P, grid, st); break;
        case 9: launch_recombine_s<9>(P, grid, st); break;
        case 10: launch_recombine_s<10>(P, grid, st); break;
        case 11: launch_recombine_s<11>(P, grid, st); break;
        case 12: launch_recombine_s<12>(P, grid, st); break;
        case 13: launch_recombine_s<13>(P, grid, st); break;
        case 14: launch_recombine_s<14>(P, grid, st); break;
        case 15: launch_recombine_s<15>(P, grid, st); break;
        default: recombine_kernel<<<grid, 256, 0, st>>>(P); break;
    }
    return (int)cudaGetLastError();
}

}  // namespace mwmm
