/*
 * mwmm_oracle.c -- CPU oracle for the multiword modular matrix product.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or helper with
 * the CUDA path under paper_2601_07508_b300/.
 *
 * Every function is the plain definition of the quantity the GPU path
 * computes, written with exact integer arithmetic (unsigned __int128), so a
 * reader can check it against the paper by eye:
 *
 *   oracle_matmul_mod     C = A B mod p                      (Sec. 1, goal equation)
 *   oracle_matmul_entries selected entries of A B mod p      (Sec. 1)
 *   oracle_freivalds      C x == A (B x) mod p, row by row   (textbook check)
 *   oracle_split_alpha    base-alpha words, top word absorbs (Alg. 4, Prop. 3.2)
 *   oracle_split_signed8  INT8 words: balanced base-2^8 digits of the
 *                         signed representative of M mod p  (Sec. 6, second
 *                         perspective: narrower words for low-precision units)
 *   oracle_split_signed_bits  the same with base-2^bits digits (8 or 9 bits)
 *   oracle_diag_sums      S_s = sum_{i+j=s} A_i B_j, exact integers (Sec. 3.2)
 *   oracle_recombine_pow  sum_s r^s S_s mod p                (Sec. 1, product of decompositions)
 *   oracle_mod_vec        x mod p            (the value Alg. 1 must return)
 *   oracle_mulmod_vec     x y mod p          (the value Alg. 2 must return)
 *   oracle_ceil_root      smallest a with a^u >= p  (alpha = ceil(p^(1/u)), Alg. 4)
 *   oracle_lambda         block size from Prop. 3.3 ((1,1): Sec. 2.2)
 *
 * Parity pins (tests/test_oracle_pins.py): Python big-integer brute force on
 * tiny inputs, algebraic invariants (A I = A, linearity, transpose, all-(p-1)
 * matrices), Freivalds on larger inputs, exact reconstruction of the words,
 * and Table 1's bitsize limits.  Nothing here is "parity unpinned".
 */
#include <stdint.h>
#include <string.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;
typedef __int128 i128;

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* C[r][c] = (sum_l A[r][l] * B[l][c]) mod p, exact.  Entries of A and B are
 * < 2^63; each product is < 2^126, so the accumulator is reduced mod p every
 * term when p >= 2^52, and every 2^20 terms otherwise (2^20 * 2^104 < 2^127).
 * Rows are independent and distributed over threads.  Returns 0 on success. */
int oracle_matmul_mod_rows(int64_t r0, int64_t r1, int64_t n, int64_t k, uint64_t p,
                           const uint64_t *A, int64_t lda, const uint64_t *B, int64_t ldb,
                           uint64_t *C, int64_t ldc, int nthreads) {
    if (p < 2 || n < 0 || k < 0 || r1 < r0) return 1;
    set_threads(nthreads);
    const int big = p >= ((uint64_t)1 << 52);
    int fail = 0;
#pragma omp parallel
    {
        u128 *acc = (u128 *)malloc(sizeof(u128) * (size_t)(n > 0 ? n : 1));
        if (!acc) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t r = r0; r < r1; ++r) {
                memset(acc, 0, sizeof(u128) * (size_t)n);
                for (int64_t l = 0; l < k; ++l) {
                    const uint64_t a = A[r * lda + l];
                    const uint64_t *brow = B + l * ldb;
                    if (big) {
                        for (int64_t c = 0; c < n; ++c)
                            acc[c] = (acc[c] + (u128)a * brow[c]) % p;
                    } else {
                        for (int64_t c = 0; c < n; ++c) acc[c] += (u128)a * brow[c];
                        if (((l + 1) & ((1 << 20) - 1)) == 0)
                            for (int64_t c = 0; c < n; ++c) acc[c] %= p;
                    }
                }
                for (int64_t c = 0; c < n; ++c) C[r * ldc + c] = (uint64_t)(acc[c] % p);
            }
            free(acc);
        }
    }
    return fail;
}

int oracle_matmul_mod(int64_t m, int64_t n, int64_t k, uint64_t p,
                      const uint64_t *A, int64_t lda, const uint64_t *B, int64_t ldb,
                      uint64_t *C, int64_t ldc, int nthreads) {
    return oracle_matmul_mod_rows(0, m, n, k, p, A, lda, B, ldb, C, ldc, nthreads);
}

/* out[t] = (sum_l A[rows[t]][l] * B[l][cols[t]]) mod p for t < count. */
int oracle_matmul_entries(int64_t k, uint64_t p, const uint64_t *A, int64_t lda,
                          const uint64_t *B, int64_t ldb, const int64_t *rows,
                          const int64_t *cols, int64_t count, uint64_t *out, int nthreads) {
    if (p < 2) return 1;
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < count; ++t) {
        u128 acc = 0;
        for (int64_t l = 0; l < k; ++l) {
            acc += (u128)A[rows[t] * lda + l] * B[l * ldb + cols[t]];
            acc %= p;
        }
        out[t] = (uint64_t)acc;
    }
    return 0;
}

/* Freivalds' check: y = B x, z = A y, w = C x (all mod p); returns the number
 * of rows r with z[r] != w[r] (0 when C == A B mod p; a wrong C is caught with
 * probability >= 1 - 1/p per independent x).  x has n entries in [0, p). */
int64_t oracle_freivalds(int64_t m, int64_t n, int64_t k, uint64_t p,
                         const uint64_t *A, int64_t lda, const uint64_t *B, int64_t ldb,
                         const uint64_t *C, int64_t ldc, const uint64_t *x, int nthreads) {
    set_threads(nthreads);
    uint64_t *y = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(k > 0 ? k : 1));
    if (!y) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < k; ++l) {
        u128 acc = 0;
        for (int64_t c = 0; c < n; ++c) acc = (acc + (u128)B[l * ldb + c] * x[c]) % p;
        y[l] = (uint64_t)acc;
    }
    int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t r = 0; r < m; ++r) {
        u128 z = 0, w = 0;
        for (int64_t l = 0; l < k; ++l) z = (z + (u128)A[r * lda + l] * y[l]) % p;
        for (int64_t c = 0; c < n; ++c) w = (w + (u128)C[r * ldc + c] * x[c]) % p;
        bad += (z != w);
    }
    free(y);
    return bad;
}

/* Alg. 4 (MW-Decomposition) with integer alpha: T = M; for i < u-1:
 * R = floor(T / alpha), M_i = T - alpha R, T = R; M_{u-1} = T.
 * words is [u][count].  Lemma 3.1 shows that the paper's floating-point
 * floor(fl(T/alpha)) equals the integer quotient used here. */
int oracle_split_alpha(const uint64_t *M, int64_t count, uint64_t alpha, int u, uint64_t *words) {
    if (alpha < 2 || u < 1) return 1;
    for (int64_t e = 0; e < count; ++e) {
        uint64_t T = M[e];
        for (int i = 0; i < u - 1; ++i) {
            const uint64_t R = T / alpha;
            words[(int64_t)i * count + e] = T - alpha * R;
            T = R;
        }
        words[(int64_t)(u - 1) * count + e] = T;
    }
    return 0;
}

/* INT8 words.  The signed representative s of M mod p is M when
 * M <= (p-1)/2 and M - p otherwise (|s| <= (p-1)/2).  Its balanced base-2^8
 * digits satisfy s = sum_i 256^i d_i: d_0..d_{u-2} are balanced,
 * d_i = ((s + 128) mod 256) - 128 in [-128, 127], s <- (s - d_i) / 256, and
 * the last digit is what remains, allowed in [-128, 128] (magnitude <= 2^7,
 * like every other digit).  Returns 2 if that last digit leaves [-128, 128]
 * (u too small for p).  words is [u][count]. */
/* Balanced base-R digits (R = 2^bits, h = R / 2) of the signed
 * representative s of each entry (s = M or M - p, |s| <= (p-1)/2): the lower
 * u - 1 digits d = ((s + h) mod R) - h in [-h, h - 1], each followed by
 * s <- (s - d) / R (exact), and the top digit the remainder, which must lie
 * in [-h, h].  Then s = sum_i R^i d_i.  Returns 2 if u digits do not
 * suffice. */
int oracle_split_signed_bits(const uint64_t *M, int64_t count, uint64_t p, int u, int bits, int32_t *words) {
    if (u < 1 || bits < 2 || bits > 16) return 1;
    const int64_t R = (int64_t)1 << bits, h = R / 2;
    for (int64_t e = 0; e < count; ++e) {
        int64_t s = (M[e] <= (p - 1) / 2) ? (int64_t)M[e] : (int64_t)M[e] - (int64_t)p;
        for (int i = 0; i < u - 1; ++i) {
            int64_t r = (s + h) % R;
            if (r < 0) r += R;
            const int64_t d = r - h;
            words[(int64_t)i * count + e] = (int32_t)d;
            s = (s - d) / R;
        }
        if (s < -h || s > h) return 2;
        words[(int64_t)(u - 1) * count + e] = (int32_t)s;
    }
    return 0;
}

int oracle_split_signed8(const uint64_t *M, int64_t count, uint64_t p, int u, int32_t *words) {
    return oracle_split_signed_bits(M, count, p, u, 8, words);
}

/* S_s[r][c] = sum_{i+j=s} sum_l A_i[r][l] B_j[l][c] (exact, int64) for the
 * word matrices Aw = [u][m][k] and Bw = [v][k][n] (int32 words); out is
 * [u+v-1][m][n].  The product of two words is an integer, so the sums are
 * exact as long as they fit int64 (checked by the caller's bounds). */
int oracle_diag_sums(int64_t m, int64_t n, int64_t k, int u, int v,
                     const int32_t *Aw, const int32_t *Bw, int64_t *out, int nthreads) {
    set_threads(nthreads);
    const int ns = u + v - 1;
    memset(out, 0, sizeof(int64_t) * (size_t)(ns * m * n));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < m; ++r)
        for (int i = 0; i < u; ++i)
            for (int j = 0; j < v; ++j) {
                int64_t *o = out + ((int64_t)(i + j) * m + r) * n;
                for (int64_t l = 0; l < k; ++l) {
                    const int64_t a = Aw[((int64_t)i * m + r) * k + l];
                    const int32_t *brow = Bw + ((int64_t)j * k + l) * n;
                    for (int64_t c = 0; c < n; ++c) o[c] += a * brow[c];
                }
            }
    return 0;
}

/* out[e] = (sum_{s<ns} radix^s S[s][e]) mod p, exact with signed S. */
int oracle_recombine_pow(const int64_t *S, int ns, int64_t count, uint64_t radix, uint64_t p,
                         uint64_t *out) {
    for (int64_t e = 0; e < count; ++e) {
        i128 acc = 0;
        u128 pw = 1;
        for (int s = 0; s < ns; ++s) {
            i128 term = (i128)(S[(int64_t)s * count + e] % (int64_t)p);
            if (term < 0) term += p;
            acc = (acc + (i128)((u128)term * pw % p)) % (i128)p;
            pw = pw * radix % p;
        }
        out[e] = (uint64_t)acc;
    }
    return 0;
}

/* out[e] = x[e] mod p for every nonnegative integer-valued double x[e]
 * (any magnitude: x = M 2^E with integer M < 2^53 and E >= 0, so
 * x mod p = (M mod p) (2^E mod p) mod p).  Returns 1 on a negative,
 * non-finite or non-integer input. */
int oracle_mod_vec(const double *x, int64_t count, uint64_t p, uint64_t *out) {
    for (int64_t e = 0; e < count; ++e) {
        double v = x[e];
        if (!(v >= 0.0) || v > 1.7976931348623157e308) return 1;
        uint64_t M;
        int E = 0;
        if (v < 9007199254740992.0) { /* < 2^53: exact as an integer */
            M = (uint64_t)v;
            if ((double)M != v) return 1;
        } else {
            while (v >= 9007199254740992.0) { v *= 0.5; ++E; } /* exact: halving an even float */
            M = (uint64_t)v;
            if ((double)M != v) return 1;
        }
        u128 r = M % p, pw = 1 % p;
        for (int i = 0; i < E; ++i) pw = (pw * 2) % p;
        out[e] = (uint64_t)(r * pw % p);
    }
    return 0;
}

/* out[e] = (x[e] * y[e]) mod p for nonnegative integers < 2^64. */
int oracle_mulmod_vec(const uint64_t *x, const uint64_t *y, int64_t count, uint64_t p, uint64_t *out) {
    for (int64_t e = 0; e < count; ++e) out[e] = (uint64_t)((u128)x[e] * y[e] % p);
    return 0;
}

/* Smallest integer a >= 1 with a^u >= p, i.e. ceil(p^(1/u)) (Alg. 4, line 1). */
uint64_t oracle_ceil_root(uint64_t p, int u) {
    if (u <= 1) return p;
    uint64_t lo = 1, hi = 1;
    for (;;) { /* find hi with hi^u >= p */
        u128 pw = 1;
        int ok = 0;
        for (int i = 0; i < u; ++i) { pw *= hi; if (pw >= p) { ok = 1; break; } }
        if (ok) break;
        hi *= 2;
    }
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        u128 pw = 1;
        int ge = 0;
        for (int i = 0; i < u; ++i) { pw *= mid; if (pw >= p) { ge = 1; break; } }
        if (ge) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* Largest block size lambda with lambda * alpha * beta + p - 1 <= 2^t
 * (Prop. 3.3), or with (p-1)^2 in place of alpha*beta for the single-word
 * product (Sec. 2.2, lambda = floor((2^t - p + 1) / (p - 1)^2)).  Returns 0 when no lambda >= 1 exists. */
uint64_t oracle_lambda(uint64_t p, int u, int v, int t) {
    const u128 two_t = (u128)1 << t;
    u128 prod;
    if (u == 1 && v == 1) {
        prod = (u128)(p - 1) * (p - 1);
    } else {
        prod = (u128)oracle_ceil_root(p, u) * oracle_ceil_root(p, v);
    }
    if (two_t + 1 < (u128)p) return 0;
    const u128 num = two_t - p + 1;
    const u128 lam = num / prod;
    return lam > (u128)UINT64_MAX ? UINT64_MAX : (uint64_t)lam;
}
