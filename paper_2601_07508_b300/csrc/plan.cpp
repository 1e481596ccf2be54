// Planner: word counts, radices and block sizes of the multiword product.
//
// Pure host logic (no CUDA calls), so plans can be made and inspected on a
// machine without a GPU.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "mwmm_internal.h"

namespace mwmm {

typedef unsigned __int128 u128;

static int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
static uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

uint64_t mulmod_u64(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((u128)a * b % p); }

// Smallest a >= 1 with a^u >= p: alpha = ceil(p^(1/u)) of Alg. 4, in exact
// integer arithmetic (a floating pow() can round across an integer).
uint64_t ceil_root(uint64_t p, int u) {
    if (u <= 1) return p;
    auto ge = [&](uint64_t a) {
        u128 pw = 1;
        for (int i = 0; i < u; ++i) {
            pw *= a;
            if (pw >= p) return true;
        }
        return false;
    };
    uint64_t hi = 1;
    while (!ge(hi)) hi *= 2;
    uint64_t lo = hi / 2 + (hi == 1);
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (ge(mid)) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Largest lambda with lambda * max(A_i) * max(B_j) + p - 1 <= 2^53.
// (u,v) = (1,1): the matrices are not split and their entries are <= p - 1,
// so lambda = floor((2^t - p + 1) / (p - 1)^2)  (Sec. 2.2).
// Otherwise the word bounds alpha, beta of Prop. 3.2 give Prop. 3.3's
// lambda = floor((2^t - p + 1) / (alpha beta)).  Returns 0 when < 1.
uint64_t block_size(uint64_t p, int u, int v) {
    const u128 two_t = (u128)1 << 53;
    if ((u128)p > two_t + 1) return 0;
    u128 prod = (u == 1 && v == 1) ? (u128)(p - 1) * (p - 1)
                                   : (u128)ceil_root(p, u) * ceil_root(p, v);
    if (prod == 0) return UINT64_MAX;
    u128 lam = (two_t - p + 1) / prod;
    return lam > (u128)UINT64_MAX ? UINT64_MAX : (uint64_t)lam;
}

// Fewest base-2^b digits for every signed representative in
// [-(p-1)/2, (p-1)/2]: u - 1 balanced digits in [-h, h - 1] and a top digit
// in [-h, h] (h = 2^(b-1)), so every digit product stays <= 2^(2b-2) in
// magnitude.  With R = 2^b and B = R^(u-1) the largest value reached is
// h B + (h - 1) (B - 1) / (R - 1): u digits cover every prime below 2^(bu).
int signed_digits(uint64_t p, int bits) {
    const u128 half = (p - 1) / 2, R = (u128)1 << bits, h = R / 2;
    int u = 1;
    u128 B = 1;
    while (h * B + (h - 1) * (B - 1) / (R - 1) < half) {
        ++u;
        B *= R;
    }
    return u;
}

int int8_digits(uint64_t p) { return signed_digits(p, 8); }

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Cost model of the two tensor forms (seconds), calibrated on B300 on 4096^3
// products (7 to 16 moduli, 3 to 7 digits a side) and on the 512-instance
// batch (m, n, k in [128, 2048], 50-bit primes).  The word products take the
// longer of their tensor time (~1.5 PFLOP/s of 2 m n k per product; 9-bit
// digits drain their 256-product FP32 chunks four times as often, 12-15%
// more per product) and their own DRAM traffic at ~6 TB/s: the 16-bit words,
// read about 1.8 times over (measured on the batch), and the INT32 sums
// written once.  Small-k products of many moduli are bound by the latter
// (batch: the CRT instances' word products ran at 63% of the INT8 ones'
// tensor rate).  Then the INT8 split (8 B read + 2 B per digit written per
// entry) at ~5 TB/s and recombination (4 B per sum read + 8 B written per
// output) at ~6 TB/s; the CRT split at 8 B per entry plus ~0.5 ps per
// (entry, modulus), the CRT reconstruction at 8 B per output plus ~1.2 ps
// per (output, modulus).
static double tensor_form_cost(const Plan &pl) {
    const double mnk2 = 2.0 * pl.m * pl.n * pl.k, mk = (double)pl.m * pl.k, kn = (double)pl.k * pl.n,
                 mk_kn = mk + kn, mn = (double)pl.m * pl.n;
    constexpr double kTensor = 1.5e15, kHbm = 5.0e12, kHbmRec = 6.0e12, kHbmGemm = 6.0e12, kWordReads = 1.8;
    if (pl.form == MWMM_FORM_CRT8) {
        const double s = pl.crt_s;
        const double gemm = std::max(s * mnk2 / kTensor, (2.0 * s * mk_kn * kWordReads + 4.0 * s * mn * pl.nkc) / kHbmGemm);
        return gemm + mk_kn * (8.0 / kHbm + s * 0.5e-12) + mn * (8.0 / kHbm + s * (1.2e-12 + 4.0 * (pl.nkc - 1) / kHbm));
    }
    const double drain = pl.digit_bits == 9 ? 1.15 : 1.0;
    const double gemm = std::max((double)pl.u * pl.v * mnk2 * drain / kTensor,
                                 (2.0 * (mk * pl.u + kn * pl.v) * kWordReads + 4.0 * mn * pl.nsums * pl.nkc) / kHbmGemm);
    return gemm + mk_kn * (8.0 + 2.0 * pl.u) / kHbm + mn * (4.0 * pl.nsums * pl.nkc + 8.0) / kHbmRec;
}

// Primes below 256, largest first (moduli of the CRT form).
static int small_primes_desc(uint32_t *out, int cap) {
    int n = 0;
    for (uint32_t c = 255; c >= 3 && n < cap; --c) {
        bool prime = true;
        for (uint32_t d = 2; d * d <= c; ++d)
            if (c % d == 0) { prime = false; break; }
        if (prime) out[n++] = c;
    }
    return n;
}

static uint64_t inv_mod_small(uint64_t a, uint64_t m) {  // a^-1 mod m for gcd(a, m) = 1, m < 2^16
    int64_t t = 0, nt = 1, r = (int64_t)m, nr = (int64_t)(a % m);
    while (nr) {
        const int64_t q = r / nr;
        int64_t x = t - q * nt; t = nt; nt = x;
        x = r - q * nr; r = nr; nr = x;
    }
    return (uint64_t)(t < 0 ? t + (int64_t)m : t);
}

// Moduli of the CRT form: the fewest largest primes below 256 whose product
// M exceeds 2 k (p-1)^2 (then C = AB over the integers is below M / 2, which
// the reconstruction needs), with the constants of the reconstruction.
static mwmm_status crt_moduli(Plan &P, int64_t k, uint64_t p) {
    uint32_t primes[64];
    const int np = small_primes_desc(primes, 64);
    const u128 kk = (u128)(k > 0 ? k : 1);
    if (kk > ((u128)1 << 22)) return MWMM_ERR_ARG;  // 2 k (p-1)^2 must stay below 2^127
    const u128 target = 2 * kk * (u128)(p - 1) * (p - 1);
    u128 prod = 1;
    int s = 0;
    while (prod <= target) {
        if (s >= kMaxCrt || s >= np) return MWMM_ERR_ARG;
        const uint32_t mi = primes[s];
        if (prod > target / mi) {  // prod * mi > target: the last modulus needed
            P.crt_m[s++] = mi;
            break;
        }
        prod *= mi;
        P.crt_m[s++] = mi;
    }
    P.crt_s = s;
    // M mod p and (M / m_i) mod p by products of the other moduli; y_i by
    // products mod m_i
    uint64_t W = 1 % p;
    for (int i = 0; i < s; ++i) W = mulmod_u64(W, P.crt_m[i], p);
    P.crt_W = W;
    for (int i = 0; i < s; ++i) {
        uint64_t wi = 1 % p, mi_mod = 1;
        for (int j = 0; j < s; ++j) {
            if (j == i) continue;
            wi = mulmod_u64(wi, P.crt_m[j], p);
            mi_mod = mi_mod * P.crt_m[j] % P.crt_m[i];
        }
        P.crt_w[i] = wi;
        P.crt_y[i] = (uint32_t)inv_mod_small(mi_mod, P.crt_m[i]);
    }
    return MWMM_OK;
}

mwmm_status make_plan(Plan *pl, int64_t m, int64_t n, int64_t k, uint64_t p, int u, int v,
                      int form, const mwmm_plan_opts *opts) {
    if (m < 0 || n < 0 || k < 0 || u < 0 || v < 0 || u > kMaxWords || v > kMaxWords)
        return MWMM_ERR_ARG;
    if ((u == 0) != (v == 0)) return MWMM_ERR_ARG;
    // Alg. 1 needs p < 2^(t-1) (Prop. 2.1); the paper also assumes p >= 5.
    if (p < 5 || (p & 1) == 0 || p >= (uint64_t(1) << 52)) return MWMM_ERR_PRIME;
    if (form == MWMM_FORM_AUTO) form = MWMM_FORM_INT8;
    if (form != MWMM_FORM_FP64 && form != MWMM_FORM_INT8 && form != MWMM_FORM_CRT8) return MWMM_ERR_ARG;
    mwmm_plan_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;

    Plan P;
    P.m = m; P.n = n; P.k = k; P.p = p; P.form = form;
    P.pd = (double)p;
    P.q = 1.0 / (double)p;  // q = fl(1/p): IEEE division, round to nearest
    P.validate = o.validate != 0;

    if (form == MWMM_FORM_FP64) {
        if (u == 0) {
            // Least modelled cost: u*v word products of k steps, plus an
            // Alg. 1 reduction (about 6 FP64 operations) every lambda steps.
            static const int cand[6][2] = {{1, 1}, {1, 2}, {1, 3}, {1, 4}, {2, 2}, {2, 3}};
            double best = 0;
            for (auto &c : cand) {
                uint64_t lam = block_size(p, c[0], c[1]);
                if (lam < 1) continue;
                int64_t kk = k > 0 ? k : 1;
                int64_t nred = (lam >= (uint64_t)kk) ? 1 : ceil_div(kk, (int64_t)lam);
                double cost = (double)(c[0] * c[1]) * ((double)kk + 6.0 * (double)nred + 12.0);
                if (u == 0 || cost < best) { u = c[0]; v = c[1]; best = cost; }
            }
            if (u == 0) return MWMM_ERR_BOUND;
        }
        uint64_t lam = block_size(p, u, v);
        if (lam < 1) return MWMM_ERR_BOUND;
        P.u = u; P.v = v;
        P.alpha = ceil_root(p, u);
        P.beta = ceil_root(p, v);
        P.lambda_max = lam > (uint64_t)INT64_MAX ? INT64_MAX : (int64_t)lam;
        P.lambda = P.lambda_max;
        if (o.lambda != 0) {
            if (o.lambda < 1 || o.lambda > P.lambda_max) return MWMM_ERR_BOUND;
            P.lambda = o.lambda;
        }
        // gamma_ij = alpha^i beta^j mod p, and gamma_ij 2^26 mod p for the
        // split form of Alg. 2 used when p > 2^52 / 3.
        uint64_t ai = 1 % p;
        for (int i = 0; i < u; ++i) {
            uint64_t g = ai;
            for (int j = 0; j < v; ++j) {
                P.gamma[i * v + j] = (double)g;
                P.gamma26[i * v + j] = (double)mulmod_u64(g, uint64_t(1) << 26, p);
                g = mulmod_u64(g, P.beta % p, p);
            }
            ai = mulmod_u64(ai, P.alpha % p, p);
        }
        // Prop. 2.2 covers x y <= (2^52 / 3) p; with x, y <= p - 1 that holds
        // iff 3 (p-1)^2 <= 2^52 p.
        P.big_p = (u128)3 * (p - 1) * (p - 1) > ((u128)p << 52);
        P.kb_elems = kF64KB;
        P.nkb = ceil_div(k, kF64KB);
        // Alg. 6: concatenate B's words along n when n is narrow (a 64-column
        // tile then holds v word slots of 64 / f64_vs columns instead of one
        // mostly empty word), or A's words along m when m is the narrow side
        // (Sec. 3.2: concatenate the side whose outer dimension is smaller);
        // at most 4 slots.
        if (o.f64_concat < 0 || o.f64_concat > 3) return MWMM_ERR_ARG;
        int side = 0;  // 1: B, 2: A
        if (o.f64_concat == 2) side = 1;
        if (o.f64_concat == 3) side = 2;
        if (o.f64_concat == 0 && (m < kF64BM || n < kF64BN)) {
            if (n <= m && v >= 2 && v <= 4) side = 1;
            else if (m < n && u >= 2 && u <= 4) side = 2;
        }
        const int words = side == 1 ? v : u;
        if (side && (words < 2 || words > 4)) return MWMM_ERR_ARG;
        P.f64_concat = side;
        P.f64_vs = side ? (words <= 2 ? 2 : 4) : 1;
        P.f64_w = kF64BN / P.f64_vs;
        P.A_rows = round_up(m > 0 ? m : 1, side == 2 ? P.f64_w : kF64BM);
        P.B_rows = round_up(n > 0 ? n : 1, side == 1 ? P.f64_w : kF64BN);
        if (side == 1) {  // k-block major: the word slots of one k-block are adjacent
            P.B_wstride = P.B_rows;
            P.B_kstride = (int64_t)v * P.B_rows;
        } else {
            P.B_wstride = P.nkb * P.B_rows;
            P.B_kstride = P.B_rows;
        }
        if (side == 2) {
            P.A_wstride = P.A_rows;
            P.A_kstride = (int64_t)u * P.A_rows;
        } else {
            P.A_wstride = P.nkb * P.A_rows;
            P.A_kstride = P.A_rows;
        }
        // K ranges: enough CTAs that the last wave is nearly full.  The
        // planner is device independent and assumes 148 SMs x 2 resident CTAs.
        const int64_t tiles = (P.A_rows / (side == 2 ? P.f64_w : kF64BM)) * (P.B_rows / (side == 1 ? P.f64_w : kF64BN));
        const int64_t smax = std::max<int64_t>(1, std::min<int64_t>(64, P.nkb / 8));
        int64_t ks = 1;
        if (o.ksplit != 0) {
            if (o.ksplit < 1 || o.ksplit > 64) return MWMM_ERR_ARG;
            ks = std::min<int64_t>(o.ksplit, std::max<int64_t>(P.nkb, 1));
        } else {
            const int64_t cap = 2 * 148;
            double best = -1.0;
            for (int64_t s = 1; s <= smax; ++s) {
                const int64_t ctas = tiles * s;
                const double eff = (double)ctas / (double)(ceil_div(ctas, cap) * cap);
                if (eff > best + 1e-9) { best = eff; ks = s; }
                if (eff >= 0.9) break;  // smallest split that fills 90% of the last wave
            }
        }
        P.kbr = ceil_div(std::max<int64_t>(P.nkb, 1), ks);
        P.ksplit = (int)ceil_div(std::max<int64_t>(P.nkb, 1), P.kbr);  // no empty range
        uint64_t abytes = (uint64_t)u * P.nkb * P.A_rows * kTileBytes;
        uint64_t bbytes = (uint64_t)v * P.nkb * P.B_rows * kTileBytes;
        P.A_off = 0;
        P.B_off = align256(abytes);
        P.S_off = align256(P.B_off + bbytes);
        P.ws_bytes = P.ksplit > 1 ? align256(P.S_off + (uint64_t)P.ksplit * m * n * 8) : P.S_off;
    } else {
        if (form == MWMM_FORM_CRT8) {  // one word (residue) per modulus on each side
            if (u != 0 || v != 0) return MWMM_ERR_ARG;
            mwmm_status cs = crt_moduli(P, k, p);
            if (cs != MWMM_OK) return cs;
            u = v = P.crt_s;
        } else {
            // Digit width: 9-bit digits (in fp16) when they need fewer digits
            // than 8-bit ones (in bf16): u^2 word products against more,
            // shorter FP32 chunks (256 products instead of 1024), measured
            // faster on B300 whenever a digit is saved (26 and 52 bits:
            // 34% and 17% less word-product time at 4096^3).
            if (o.tc_digit_bits != 0 && o.tc_digit_bits != 8 && o.tc_digit_bits != 9) return MWMM_ERR_ARG;
            int bits = o.tc_digit_bits;
            if (bits == 0) bits = (u == 0 && signed_digits(p, 9) < signed_digits(p, 8)) ? 9 : 8;
            P.digit_bits = bits;
            const int need = signed_digits(p, bits);
            if (u == 0) { u = need; v = need; }
            if (u < need || v < need) return MWMM_ERR_BOUND;
        }
        P.u = u; P.v = v;
        P.alpha = form == MWMM_FORM_CRT8 ? 0 : (uint64_t(1) << P.digit_bits);
        P.beta = P.alpha;
        P.nsums = form == MWMM_FORM_CRT8 ? P.crt_s : u + v - 1;  // one sum per modulus / per diagonal
        // FP32 chunk: digit products of magnitude <= 2^(2b-2), every partial
        // sum of a chunk <= 2^24 (CRT residues: |r| <= 127, as 8-bit digits)
        const int64_t chunk_max = tc_chunk_limit(P.digit_bits);
        P.tc_chunk = chunk_max;
        if (o.tc_chunk != 0) {
            if (o.tc_chunk < 64 || o.tc_chunk > chunk_max || o.tc_chunk % 64) return MWMM_ERR_ARG;
            P.tc_chunk = o.tc_chunk;
        }
        // One INT32 sum S_s collects w = min(u,v) pairs (at most; one for the
        // CRT form) over kc k-steps, each product |d_a d_b| <= 2^(2b-2): need
        // kc * w <= floor((2^31 - 1) / 2^(2b-2)).
        const int w = form == MWMM_FORM_CRT8 ? 1 : (u < v ? u : v);
        int64_t kcmax = (int32_sum_limit(P.digit_bits) / w) / kTcKB * kTcKB;
        int64_t kc = kcmax;
        if (o.kc != 0) {
            if (o.kc < kTcKB || o.kc % kTcKB || o.kc > kcmax) return MWMM_ERR_ARG;
            kc = o.kc;
        }
        int64_t kpad = round_up(k, kTcKB);
        if (kc > kpad) kc = kpad > 0 ? kpad : kTcKB;
        P.kb_elems = kTcKB;
        P.nkb = ceil_div(k, kTcKB);
        // Under-filled products: the persistent kernel's time is at least
        // its longest item (a tile's diagonal window: up to min(u, v) pairs
        // x the K range's k-blocks; one pair for the CRT form), so shorter K
        // ranges (more items, more sum planes) can finish sooner, while the
        // extra planes cost recombination time.  The K-range count is the
        // argmin of a model fitted on B300 (48 shapes from 64 x 64 x 4096 to
        // 2048^2 x 1024, 20 and 52 bits, mean 2% and at most 19% slower than
        // the best count measured): word products max(longest item, an SM's
        // share of all items), with a fixed cost per item (its drain and
        // 128 KB store: 4 us INT8, 0.5 us CRT), plus reading the sum planes
        // (one K range: 5.7 / 3 TB/s; several, through the Horner path:
        // 1.5 / 0.5 TB/s for INT8 / CRT).
        if (o.tc_fill < 0 || o.tc_fill > 1) return MWMM_ERR_ARG;
        const bool fused_req = form == MWMM_FORM_INT8 && n > kTcBN / 2 && o.tc_fused == 2;
        if (o.kc == 0 && o.tc_fill == 0 && !fused_req && k > 0 && m > 0 && n > 0) {
            const bool crt = form == MWMM_FORM_CRT8;
            constexpr double kSms = 148.0;
            const double t_kb = 2.0 * kTcBM * kTcBN * kTcKB / (1.5e15 / kSms) * (P.digit_bits == 9 ? 1.15 : 1.0);
            const double c_item = crt ? 0.5e-6 : 4.0e-6, r_one = crt ? 3.0e12 : 5.7e12, r_many = crt ? 0.5e12 : 1.5e12;
            int64_t tiles = ceil_div(m, kTcBM), nwin = P.nsums;
            if (n > kTcBN / 2) {
                tiles *= ceil_div(n, kTcBN);
            } else if (!crt) {  // narrow n: 256 / nb diagonals side by side in one tile
                int64_t nb = 16;
                while (nb < n) nb *= 2;
                nwin = ceil_div(P.nsums, std::min<int64_t>(kTcBN / nb, P.nsums));
            }
            const double pairs = crt ? (double)P.crt_s : (double)u * v;
            const double total_kb = (double)tiles * pairs * (double)P.nkb, mn = (double)m * n;
            auto cost = [&](int64_t kcb) {  // kcb: k-blocks per K range
                const int64_t nr = ceil_div(P.nkb, kcb);
                const double items = (double)(tiles * nwin * nr);
                const double gemm = std::max(w * (double)kcb * t_kb + c_item, (total_kb * t_kb + items * c_item) / kSms);
                return gemm + (double)P.nsums * nr * mn * 4.0 / (nr == 1 ? r_one : r_many);
            };
            int64_t best_kb = kc / kTcKB;
            double best = cost(best_kb);
            for (int64_t nr = ceil_div(P.nkb, best_kb) + 1; nr <= 64 && nr <= P.nkb; ++nr) {
                const int64_t kcb = ceil_div(P.nkb, nr);
                if (ceil_div(P.nkb, kcb) != nr) continue;  // the same ranges as a smaller count
                const double c = cost(kcb);
                if (c < best) { best = c; best_kb = kcb; }
            }
            kc = best_kb * kTcKB;
        }
        P.kc = kc;
        P.nkc = k > 0 ? (int)ceil_div(k, kc) : 0;
        // Column tiles: 256 wide when n > 128; narrower n is padded to 16, 32,
        // 64 or 128 and one tile then carries 256 / nb diagonals side by side.
        P.tc_nb = kTcBN;
        if (n <= kTcBN / 2) {
            P.tc_nb = 16;
            while (P.tc_nb < n) P.tc_nb *= 2;
        }
        P.tc_ndiag = kTcBN / P.tc_nb < P.nsums ? kTcBN / P.tc_nb : P.nsums;
        if (form == MWMM_FORM_CRT8) P.tc_ndiag = 1;  // each modulus pairs A_i with B_i only: no windows
        // Tile kernel.  The two-CTA kernel (256 x 256 tiles on an SM pair)
        // runs on request (tc_pair = 1), never with tc_pair = -1, and by
        // default (0) for 8-bit digits and CRT residues (1024-product chunks)
        // on products large enough that 256-row tiles add at most 3% padding
        // and leave several waves of items, on a device whose SMs all pair up
        // (when one is present): measured on B300 at 4096^3, 3-4% faster than
        // the one-CTA kernel at 20 to 48 bits and 4% on the CRT form's
        // products at 32-52 bits.  With 9-bit digits (drains twice as often,
        // each finished on both SMs before the pair reuses an accumulator) it
        // was level at 52 bits and 2% slower at 26, so those keep one CTA.
        if (o.tc_pair < -1 || o.tc_pair > 1) return MWMM_ERR_ARG;
        bool pair = o.tc_pair == 1;
        const bool chunk1024 = (form == MWMM_FORM_INT8 && P.digit_bits == 8) || form == MWMM_FORM_CRT8;
        if (o.tc_pair == 0 && chunk1024 && P.tc_nb == kTcBN && m >= kPairMinM) {
            const int64_t rows1 = round_up(m, kTcBM), rows2 = round_up(m, 2 * kTcBM);
            const int64_t items = (rows2 / (2 * kTcBM)) * ceil_div(n, kTcBN) * P.nsums * P.nkc;
            pair = rows2 * 32 <= rows1 * 33 && items >= kPairMinItems && tc_pairs_fill_device() != 0;
        }
        P.tc_pair = (m > kTcBM && P.tc_nb == kTcBN && pair) ? 1 : 0;
        // Fused recombination (INT8 form, n > 128) on request (tc_fused = 2):
        // its 256 x 128 pair tiles run the word products at about 60% of the
        // one-CTA 128 x 256 kernel's rate on B300, so the default keeps the
        // diagonal sums in the workspace; it needs no sum planes, which is
        // what memory-bound callers want.
        if (o.tc_fused < 0 || o.tc_fused > 2 || o.tc_seg < 0) return MWMM_ERR_ARG;
        if (form == MWMM_FORM_INT8 && n > kTcBN / 2 && o.tc_fused == 2) {
            P.tc_fused = 1;
            P.tc_pair = 0;
            P.tc_nb = kTcBN;
            P.tc_ndiag = 1;
        }
        P.A_rows = round_up(m > 0 ? m : 1, (P.tc_pair || P.tc_fused) ? 2 * kTcBM : kTcBM);
        P.A_wstride = P.nkb * P.A_rows;
        P.A_kstride = P.A_rows;
        P.B_rows = P.tc_nb == kTcBN ? round_up(n > 0 ? n : 1, P.tc_fused ? kTcBN / 2 : kTcBN) : P.tc_nb;
        uint64_t abytes = (uint64_t)u * P.nkb * P.A_rows * kTileBytes;
        // Narrow n: B's words k-block major with zero words on both sides, so
        // the words B_{s0-i} .. B_{s0-i+ndiag-1} of any window are contiguous.
        P.B_wpad = P.tc_nb < kTcBN ? P.tc_ndiag - 1 : 0;
        if (P.tc_nb < kTcBN) {
            P.B_wstride = P.B_rows;
            P.B_kstride = (int64_t)(v + 2 * P.B_wpad) * P.B_rows;
        } else {
            P.B_wstride = P.nkb * P.B_rows;
            P.B_kstride = P.B_rows;
        }
        uint64_t bbytes = (uint64_t)(v + 2 * P.B_wpad) * P.nkb * P.B_rows * kTileBytes;
        uint64_t sbytes = (uint64_t)P.nsums * P.nkc * P.A_rows * P.B_rows * 4;
        if (P.tc_fused) {
            // Segments: k-blocks per INT32 sum (ni <= w pairs of seg * 64
            // products each: seg * 64 <= kcmax); 64 by default (measured:
            // 16-block segments, whose words stay in L2, saved less DRAM
            // time than their extra residue folds cost).
            int64_t seg = o.tc_seg ? o.tc_seg : kFusedSeg;
            if (seg * kTcKB > kcmax && !o.tc_seg) seg = kcmax / kTcKB;
            if (seg * kTcKB > kcmax) return MWMM_ERR_ARG;
            if (seg > P.nkb && P.nkb > 0) seg = P.nkb;
            P.tc_seg = (int)(seg > 0 ? seg : 1);
            P.kc = (int64_t)P.tc_seg * kTcKB;
            P.nkc = k > 0 ? (int)ceil_div(k, P.kc) : 0;
            // K parts: enough units (tiles x parts) that the last wave of CTA
            // pairs is nearly full; the planner assumes 74 pairs (148 SMs).
            const int64_t tiles = (P.A_rows / (2 * kTcBM)) * (P.B_rows / (kTcBN / 2));
            const int64_t nkb1 = std::max<int64_t>(P.nkb, 1);
            int64_t ks = 1;
            if (o.ksplit != 0) {
                if (o.ksplit < 1 || o.ksplit > 64) return MWMM_ERR_ARG;
                ks = std::min<int64_t>(o.ksplit, nkb1);
            } else {
                const int64_t cap = kFusedPairs;
                double best = -1.0;
                for (int64_t s = 1; s <= std::min<int64_t>(8, nkb1); ++s) {
                    const int64_t units = tiles * s;
                    const double eff = (double)units / (double)(ceil_div(units, cap) * cap);
                    if (eff > best + 1e-9) { best = eff; ks = s; }
                    if (eff >= 0.9) break;  // the fewest parts that fill 90% of the last wave
                }
            }
            P.kbr = ceil_div(nkb1, ks);
            P.ksplit = (int)ceil_div(nkb1, P.kbr);  // no empty part
            P.tc_ldr = round_up(n > 0 ? n : 1, 2);
            sbytes = P.ksplit > 1 ? (uint64_t)P.ksplit * m * P.tc_ldr * 8 : 0;
        }
        P.A_off = 0;
        P.B_off = align256(abytes);
        P.S_off = align256(P.B_off + bbytes);
        P.ws_bytes = align256(P.S_off + sbytes);
        if (!P.tc_fused) {  // the one-CTA kernel claims its items from a counter after the sums
            P.sched_off = P.ws_bytes;
            P.ws_bytes += 256;
        }
        // Certified 512-product chunks for 9-bit digits (twice the
        // worst-case 256) where each item is one 256-wide diagonal tile.
        // (Not with an explicit tc_chunk, which fixes the chunk.)
        if (form == MWMM_FORM_INT8 && P.digit_bits == 9 && !P.tc_fused && P.tc_nb == kTcBN && k > 0 &&
            o.tc_chunk == 0) {
            P.tc_cert_chunk = 2 * (int)P.tc_chunk;
            P.sq_off = P.ws_bytes;
            P.sqB_off = align256((uint64_t)u * P.nkb * (P.A_rows / 64) * 4);
            P.ws_bytes = align256(P.sq_off + P.sqB_off + (uint64_t)v * P.nkb * (P.B_rows / 64) * 4);
        }
    }
    if (m == 0 || n == 0) P.ws_bytes = 0;
    *pl = P;
    return MWMM_OK;
}

int choose_tensor_form(int64_t m, int64_t n, int64_t k, uint64_t p) {
    mwmm_plan_opts z;
    std::memset(&z, 0, sizeof(z));
    z.tc_fused = 1;  // batches and the serving loop run the diagonal sums through the workspace
    z.tc_fill = 1;   // ... and interleave many products in one launch
    Plan a, c;
    if (make_plan(&a, m, n, k, p, 0, 0, MWMM_FORM_INT8, &z) != MWMM_OK) return MWMM_FORM_INT8;
    if (make_plan(&c, m, n, k, p, 0, 0, MWMM_FORM_CRT8, &z) != MWMM_OK) return MWMM_FORM_INT8;
    return tensor_form_cost(c) < tensor_form_cost(a) ? MWMM_FORM_CRT8 : MWMM_FORM_INT8;
}

}  // namespace mwmm
