"""Pins of the CPU oracle against facts fixed outside it.

Each test checks an oracle function against something other than itself:
Python big-integer brute force, algebraic identities of the product, the
paper's printed tables (tests/golden/), exact reconstruction, a library
routine (sympy), or a simulation of the paper's floating-point algorithms
with exactly rounded IEEE arithmetic.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2601_07508_b300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
SWEEP_PRIMES = {b: inputs.largest_prime_below_pow2(b) for b in inputs.SWEEP_BITS}
EDGE_PRIMES = [5, 7, 11, 251, 257, 65521, (1 << 31) - 1, inputs.prev_prime(1 << 50),
               inputs.prev_prime(1 << 51), inputs.prev_prime(1 << 52)]


def brute(A, B, p):
    m, k = A.shape
    n = B.shape[1]
    C = np.zeros((m, n), dtype=np.uint64)
    for r in range(m):
        for c in range(n):
            C[r, c] = sum(int(A[r, l]) * int(B[l, c]) for l in range(k)) % p
    return C


def load_rows(name):
    rows = []
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- product
@pytest.mark.parametrize("p", EDGE_PRIMES + list(SWEEP_PRIMES.values()))
def test_matmul_bruteforce_tiny(oracle, p):
    for seed, (m, n, k) in enumerate([(1, 1, 1), (2, 3, 4), (5, 4, 7), (8, 8, 8), (3, 1, 6), (4, 5, 0)]):
        A, B = inputs.problem(seed, m, n, k, p)
        assert np.array_equal(oracle.matmul_mod(A, B, p), brute(A, B, p))


def test_matmul_all_max_entries(oracle):
    # all entries p - 1: (p-1)^2 = 1 mod p, so every entry of C is k mod p.
    for p in EDGE_PRIMES:
        for k in (1, 2, 7, 64, 300):
            A = np.full((3, k), p - 1, dtype=np.uint64)
            B = np.full((k, 4), p - 1, dtype=np.uint64)
            assert np.all(oracle.matmul_mod(A, B, p) == k % p)


@pytest.mark.parametrize("b", [20, 40, 52])
def test_matmul_invariants(oracle, b):
    p = SWEEP_PRIMES[b]
    m, n, k = 17, 13, 29
    A, B = inputs.problem(b, m, n, k, p)
    _, B2 = inputs.problem(b + 1000, m, n, k, p)
    I_k = np.eye(k, dtype=np.uint64)
    I_m = np.eye(m, dtype=np.uint64)
    # A I = A, I A = A
    assert np.array_equal(oracle.matmul_mod(A, I_k, p), A)
    assert np.array_equal(oracle.matmul_mod(I_m, A, p), A)
    # zero
    assert np.all(oracle.matmul_mod(A, np.zeros((k, n), np.uint64), p) == 0)
    # linearity: A (B + B2) = A B + A B2 (mod p)
    Bs = ((B.astype(object) + B2.astype(object)) % p).astype(np.uint64)
    lhs = oracle.matmul_mod(A, Bs, p)
    rhs = (oracle.matmul_mod(A, B, p).astype(object) + oracle.matmul_mod(A, B2, p).astype(object)) % p
    assert np.array_equal(lhs, rhs.astype(np.uint64))
    # transpose: (A B)^T = B^T A^T
    assert np.array_equal(oracle.matmul_mod(A, B, p).T, oracle.matmul_mod(B.T.copy(), A.T.copy(), p))


def test_matmul_entries_and_rows(oracle):
    p = SWEEP_PRIMES[48]
    A, B = inputs.problem(3, 40, 33, 57, p)
    C = oracle.matmul_mod(A, B, p)
    rows = np.array([0, 39, 7, 20], dtype=np.int64)
    cols = np.array([0, 32, 5, 11], dtype=np.int64)
    assert np.array_equal(oracle.matmul_entries(A, B, p, rows, cols), C[rows, cols])
    assert np.array_equal(oracle.matmul_mod_rows(A, B, p, 5, 19), C[5:19])


def test_freivalds_accepts_and_catches_planted_error(oracle):
    p = SWEEP_PRIMES[52]
    A, B = inputs.problem(9, 64, 48, 80, p)
    C = oracle.matmul_mod(A, B, p)
    x = inputs.uniform_mod(9, 77, 48, p)
    assert oracle.freivalds(A, B, C, p, x) == 0
    Cbad = C.copy()
    Cbad[10, 3] = (int(Cbad[10, 3]) + 1) % p
    assert oracle.freivalds(A, B, Cbad, p, x) == 1


# ---------------------------------------------------------------- words
@pytest.mark.parametrize("p", EDGE_PRIMES + list(SWEEP_PRIMES.values()))
@pytest.mark.parametrize("u", [1, 2, 3, 4])
def test_split_alpha_prop32(oracle, p, u):
    """Prop. 3.2: the words reconstruct M exactly; lower words are < alpha and
    the top word is <= floor((p-1)/alpha^(u-1)) <= alpha."""
    alpha = oracle.ceil_root(p, u)
    if u > 1 and alpha < 2:
        pytest.skip("alpha < 2")
    M = np.concatenate([inputs.uniform_mod(u, 5, 500, p),
                        np.array([0, 1, p - 1, p // 2, alpha - 1 if alpha <= p else 0], dtype=np.uint64)])
    W = oracle.split_alpha(M, alpha, u)
    rec = sum(int(alpha) ** i * W[i].astype(object) for i in range(u))
    assert np.array_equal(rec.astype(np.uint64), M)
    if u > 1:
        assert int(W[:-1].max()) <= alpha - 1
    top_bound = (p - 1) // alpha ** (u - 1)
    assert int(W[-1].max()) <= top_bound <= alpha


def _fl_div_floor(a: float, b: float) -> float:
    return math.floor(a / b)  # Python float division is IEEE round-to-nearest


@pytest.mark.parametrize("b", [26, 32, 40, 48, 52])
@pytest.mark.parametrize("u", [2, 3])
def test_split_alpha_matches_floating_point_alg4(oracle, b, u):
    """Alg. 4 run in IEEE doubles (R = floor(fl(T/alpha)), M_i = T - alpha R)
    gives the same words as the integer split (Lemma 3.1)."""
    p = SWEEP_PRIMES[b]
    alpha = oracle.ceil_root(p, u)
    M = np.concatenate([inputs.uniform_mod(b, 6, 300, p), np.array([p - 1, 0, alpha ** (u - 1)], dtype=np.uint64)])
    W = oracle.split_alpha(M, alpha, u)
    for e, x in enumerate(M):
        T = float(int(x))
        for i in range(u - 1):
            R = float(_fl_div_floor(T, float(alpha)))
            Mi = T - float(alpha) * R
            assert Mi == float(int(W[i, e]))
            T = R
        assert T == float(int(W[u - 1, e]))


def test_ceil_root_exact(oracle):
    for u in (1, 2, 3, 4, 5, 7):
        for a in (2, 3, 10, 255, 256, 1024, 1 << 13):
            if a ** u >= 1 << 63:
                continue
            assert oracle.ceil_root(a ** u, u) == a
            assert oracle.ceil_root(a ** u + 1, u) == a + 1
            assert oracle.ceil_root(a ** u - 1, u) == (a if u > 1 else a - 1)
    for p in EDGE_PRIMES:
        for u in (2, 3, 4):
            a = oracle.ceil_root(p, u)
            assert a ** u >= p and (a - 1) ** u < p


@pytest.mark.parametrize("p", EDGE_PRIMES + list(SWEEP_PRIMES.values()))
def test_split_signed8(oracle, p):
    u = oracle.int8_words(p)
    M = np.concatenate([inputs.uniform_mod(11, 7, 400, p),
                        np.array([0, 1, p - 1, (p - 1) // 2, (p + 1) // 2], dtype=np.uint64)])
    W = oracle.split_signed8(M, p, u)
    assert W.min() >= -128 and W[:u - 1].max(initial=0) <= 127 and W[u - 1].max() <= 128
    for e, x in enumerate(M):
        x = int(x)
        s = x if x <= (p - 1) // 2 else x - p
        assert sum(256 ** i * int(W[i, e]) for i in range(u)) == s
    # u is the fewest digits: the largest signed representative needs all u.
    if u > 1:
        with pytest.raises(ValueError):
            oracle.split_signed8(np.array([(p - 1) // 2], dtype=np.uint64), p, u - 1)


def test_int8_words_table():
    # digits per side for the sweep primes (largest prime below 2^b)
    from oracle import oracle as O
    got = {b: O.int8_words(SWEEP_PRIMES[b]) for b in inputs.SWEEP_BITS}
    # u - 1 balanced digits and a top digit of magnitude <= 128 reach
    # 128 B + 127 (B - 1) / 255 with B = 256^(u-1), about 2^(8u-1): every
    # prime below 2^(8u) needs at most u digits (checked with floats)
    for b, u in got.items():
        p = SWEEP_PRIMES[b]
        B = 256.0 ** (u - 1)
        assert (p - 1) / 2 <= (128 * B + 127 * (B - 1) / 255) * (1 + 1e-12)
        assert (p - 1) / 2 > 128 * B / 256 + 127 * (B / 256 - 1) / 255
        assert u == -(-b // 8)
    assert got == {20: 3, 23: 3, 26: 4, 32: 4, 40: 5, 48: 6, 52: 7}


def test_split_signed8_top_digit_128(oracle):
    # (p-1)/2 for p = 2^32 - 5 is 2^31 - 3 = 128 * 2^24 - 3: digits (-3, 0, 0, 128)
    p = SWEEP_PRIMES[32]
    W = oracle.split_signed8(np.array([(p - 1) // 2, (p + 1) // 2], dtype=np.uint64), p, 4)
    assert W[:, 0].tolist() == [-3, 0, 0, 128] and W[:, 1].tolist() == [3, 0, 0, -128]
    # brute force over every signed value of a 2-digit split: the covered
    # range is [-128 * 257, 128 * 256 + 127], the top digit reaching -128 and
    # +128 at its ends, and one more on either side needs a third digit
    top = 128 * 256 + 127
    s = np.arange(-top - 2, top + 2, dtype=np.int64)
    pp = 2 * (top + 2) + 1          # odd modulus with (pp - 1) / 2 = top + 2
    M = np.where(s >= 0, s, s + pp).astype(np.uint64)
    for bad in (0, len(s) - 1):
        with pytest.raises(ValueError):
            oracle.split_signed8(M[bad:bad + 1], pp, 2)
    ok = (s >= -top - 1) & (s <= top)
    W = oracle.split_signed8(M[ok], pp, 2)
    assert np.array_equal(W[0] + 256 * W[1], s[ok])
    assert W[1].min() == -128 and W[1].max() == 128 and W[0].min() == -128 and W[0].max() == 127


@pytest.mark.parametrize("p", EDGE_PRIMES + list(SWEEP_PRIMES.values()))
def test_split_signed_9bit_digits(oracle, p):
    """Balanced base-2^9 digits (the fp16-carried digits of the tensor form):
    lower digits in [-256, 255], the top one in [-256, 256], exact
    reconstruction of the signed representative, and the fewest digits."""
    u = oracle.digit_words(p, 9)
    M = np.concatenate([inputs.uniform_mod(12, 7, 400, p),
                        np.array([0, 1, p - 1, (p - 1) // 2, (p + 1) // 2], dtype=np.uint64)])
    W = oracle.split_signed(M, p, u, 9)
    assert W.min() >= -256 and W[:u - 1].max(initial=0) <= 255 and W[u - 1].max() <= 256
    for e, x in enumerate(M):
        x = int(x)
        s = x if x <= (p - 1) // 2 else x - p
        assert sum(512 ** i * int(W[i, e]) for i in range(u)) == s
    if u > 1:
        with pytest.raises(ValueError):
            oracle.split_signed(np.array([(p - 1) // 2], dtype=np.uint64), p, u - 1, 9)
    # the 8-bit path through the same routine is the INT8 split
    W8 = oracle.split_signed(M, p, oracle.int8_words(p), 8)
    assert np.array_equal(W8, oracle.split_signed8(M, p, oracle.int8_words(p)))


def test_9bit_digit_counts():
    """Digits per side for the sweep primes: u 9-bit digits reach about
    2^(9u-1), so a b-bit prime needs ceil(b / 9) of them (or one fewer when
    (p-1)/2 still fits); they save a digit over 8-bit ones at 26 and 52 bits."""
    from oracle import oracle as O
    got = {b: O.digit_words(SWEEP_PRIMES[b], 9) for b in inputs.SWEEP_BITS}
    assert got == {20: 3, 23: 3, 26: 3, 32: 4, 40: 5, 48: 6, 52: 6}
    for b, u in got.items():
        assert u == -(-b // 9)
    # brute force over every signed value of a 2-digit split: the covered
    # range is [-256 * 513, 256 * 512 + 255]; one more on either side needs a
    # third digit
    top = 256 * 512 + 255
    s = np.arange(-top - 2, top + 2, dtype=np.int64)
    pp = 2 * (top + 2) + 1
    M = np.where(s >= 0, s, s + pp).astype(np.uint64)
    for bad in (0, len(s) - 1):
        with pytest.raises(ValueError):
            O.split_signed(M[bad:bad + 1], pp, 2, 9)
    ok = (s >= -top - 1) & (s <= top)
    W = O.split_signed(M[ok], pp, 2, 9)
    assert np.array_equal(W[0] + 512 * W[1], s[ok])
    assert W[1].min() == -256 and W[1].max() == 256 and W[0].min() == -256 and W[0].max() == 255


def test_diag_sums_and_recombine_reproduce_product(oracle):
    """sum_s 256^s S_s mod p with S_s = sum_{i+j=s} A_i B_j equals A B mod p
    (the product of the two decompositions, Sec. 1 / Sec. 3.2)."""
    for b in (20, 40, 52):
        p = SWEEP_PRIMES[b]
        m, n, k = 9, 7, 23
        A, B = inputs.problem(b, m, n, k, p)
        u = oracle.int8_words(p)
        Aw = oracle.split_signed8(A, p, u)                  # [u][m][k]
        Bw = oracle.split_signed8(B, p, u)                  # [u][k][n]
        S = oracle.diag_sums(Aw, Bw)
        # brute force the diagonal sums
        for s in range(2 * u - 1):
            ref = np.zeros((m, n), dtype=object)
            for i in range(u):
                j = s - i
                if 0 <= j < u:
                    ref += Aw[i].astype(object).dot(Bw[j].astype(object))
            assert np.array_equal(S[s].astype(object), ref)
        C = oracle.recombine_pow(S, 256, p)
        assert np.array_equal(C, oracle.matmul_mod(A, B, p))
        # the same with 9-bit digits and radix 512
        u9 = oracle.digit_words(p, 9)
        S9 = oracle.diag_sums(oracle.split_signed(A, p, u9, 9), oracle.split_signed(B, p, u9, 9))
        assert np.array_equal(oracle.recombine_pow(S9, 512, p), oracle.matmul_mod(A, B, p))


def test_recombine_pow_bruteforce(oracle):
    p = SWEEP_PRIMES[52]
    S = inputs.uniform_mod(1, 9, 5 * 6, 1 << 40).astype(np.int64).reshape(5, 6) - (1 << 39)
    out = oracle.recombine_pow(S, 1000003, p)
    for e in range(6):
        assert int(out[e]) == sum(1000003 ** s * int(S[s, e]) for s in range(5)) % p


# ---------------------------------------------------------------- scalar ops
def test_mod_and_mulmod_vec(oracle):
    p = SWEEP_PRIMES[52]
    xs = np.array([0.0, 1.0, float(p - 1), float(p), float(p + 1), 2.0 ** 53, 2.0 ** 53 - 1,
                   float(2 ** 51 * p)], dtype=np.float64)
    ref = [int(x) % p for x in xs]
    assert [int(v) for v in oracle.mod_vec(xs, p)] == ref
    x = inputs.uniform_mod(2, 1, 1000, p)
    y = inputs.uniform_mod(2, 2, 1000, p)
    got = oracle.mulmod_vec(x, y, p)
    assert all(int(g) == int(a) * int(b) % p for g, a, b in zip(got, x, y))


# ---------------------------------------------------------------- block size
def test_lambda_reproduces_table1_bitsize_limits(oracle):
    """Table 1: the largest bitsize b for which the largest prime below 2^b
    still has a block size lambda >= 1 under Prop. 3.3."""
    for u, v, flops, limit in load_rows("table1_bitsize_limits.txt"):
        u, v, flops, limit = int(u), int(v), int(flops), int(limit)
        assert u * v == flops
        ok = [b for b in range(4, 53) if oracle.lam(inputs.prev_prime(1 << b), u, v) >= 1]
        assert max(ok) == limit
        assert ok == list(range(4, limit + 1))


def test_theory_variant_ranges_follow_from_the_block_sizes(oracle):
    """Sec. 3.3's predicted best variants (the bullet list after Table 1):
    for each bitsize, the variants of fewest word products u v among those
    with a block size lambda >= 1 for the largest prime below 2^b, out of
    (1,1), (1,2), (1,3), (1,4), (2,2) -- (2,3) is not in that list."""
    rows = load_rows("variant_ranges.txt")
    want = {}
    for row in rows:
        lo, hi, u, v = (int(x) for x in row[:4])
        for b in range(lo, hi + 1):
            want.setdefault(b, set()).add((u, v))
    assert sorted(want) == list(range(1, 53))
    variants = [(1, 1), (1, 2), (1, 3), (1, 4), (2, 2)]
    for b in range(4, 53):
        p = inputs.prev_prime(1 << b)
        ok = [uv for uv in variants if oracle.lam(p, *uv) >= 1]
        fewest = min(u * v for u, v in ok)
        assert {uv for uv in ok if uv[0] * uv[1] == fewest} == want[b], b


def test_lambda_single_word_corollary(oracle):
    """Sec. 2.2 corollary: the (1,1) block size is >= 1 exactly when
    p (p - 1) <= 2^t, and it equals floor((2^t - p + 1) / (p-1)^2)."""
    for p in EDGE_PRIMES + list(SWEEP_PRIMES.values()) + [inputs.prev_prime(1 << 27)]:
        lam = oracle.lam(p, 1, 1)
        assert (lam >= 1) == (p * (p - 1) <= 1 << 53)
        if p * (p - 1) <= 1 << 53:
            assert lam == ((1 << 53) - p + 1) // (p - 1) ** 2


def test_lambda_22_handles_every_52bit_prime(oracle):
    """Sec. 3.2: the (2,2)-product handles all p < 2^(t-1); the block size
    tends to 1 as p approaches 2^52."""
    assert oracle.lam(SWEEP_PRIMES[52], 2, 2) == 1
    assert oracle.lam(inputs.prev_prime(1 << 48), 2, 2) > 1


def test_lambda_close_to_readable_condition(oracle):
    """The readable condition (Sec. 3.2) drops the ceilings: it admits at least
    the block size of Prop. 3.3, and for large p the two agree within 1%."""
    for b in (32, 40, 48, 52):
        p = SWEEP_PRIMES[b]
        for u, v in ((1, 2), (1, 3), (2, 2), (2, 3)):
            lam = oracle.lam(p, u, v)
            readable = ((1 << 53) - p + 1) / p ** (1 / u + 1 / v)
            assert lam <= readable * (1 + 1e-9)
            if lam > 100:
                assert lam >= 0.99 * readable


def test_lambda_sweep_values(oracle):
    # values of Prop. 3.3 for the bound-selected variants of the sweep; checked
    # here against a direct big-integer evaluation with a different root routine
    for b, (u, v) in {20: (1, 1), 23: (1, 1), 26: (1, 1), 32: (1, 2), 40: (2, 2), 48: (2, 2), 52: (2, 2)}.items():
        p = SWEEP_PRIMES[b]
        if (u, v) == (1, 1):
            prod = (p - 1) ** 2
        else:
            a = round(p ** (1 / u))
            while a ** u < p:
                a += 1
            while (a - 1) ** u >= p:
                a -= 1
            c = round(p ** (1 / v))
            while c ** v < p:
                c += 1
            while (c - 1) ** v >= p:
                c -= 1
            prod = a * c
        assert oracle.lam(p, u, v) == ((1 << 53) - p + 1) // prod


# ---------------------------------------------------------------- primes
def test_primes_against_sympy():
    import sympy
    for b in list(inputs.SWEEP_BITS) + [50, 60, 63]:
        assert inputs.largest_prime_below_pow2(b) == sympy.prevprime(1 << b)
    p50 = inputs.primes_below(1 << 50, 64)
    assert p50[0] == sympy.prevprime(1 << 50)
    for a, b in zip(p50, p50[1:]):
        assert b == sympy.prevprime(a)


def test_is_prime_small_and_known():
    sieve = np.ones(20000, dtype=bool)
    sieve[:2] = False
    for i in range(2, 142):
        if sieve[i]:
            sieve[i * i::i] = False
    assert all(inputs.is_prime(i) == bool(sieve[i]) for i in range(20000))
    for q in ((1 << 31) - 1, (1 << 61) - 1, (1 << 64) - 59, (1 << 32) - 5):
        assert inputs.is_prime(q)
    for c in (3215031751, 2152302898747, 3474749660383, 341550071728321, 3825123056546413051):
        assert not inputs.is_prime(c)  # strong pseudoprimes to small base sets


# ---------------------------------------------------------------- paper algorithms
def _fl(x: Fraction) -> float:
    return float(x)  # correctly rounded, ties to even


def _fma(a: float, b: float, c: float) -> float:
    return _fl(Fraction(a) * Fraction(b) + Fraction(c))


def alg1(x: float, p: float, q: float) -> float:
    b = x * q
    c = math.floor(b)
    d = _fma(-c, p, x)
    if d >= p:
        d = d - p
    if d < 0:
        d = d + p
    return d


def alg2(x: float, y: float, p: float, q: float) -> float:
    h = x * y
    l = _fma(x, y, -h)
    b = h * q
    c = math.floor(b)
    d = _fma(-c, p, h)
    e = d + l
    if e >= p:
        e = e - p
    if e < 0:
        e = e + p
    return e


@pytest.mark.parametrize("p", [5, 7, 65521, SWEEP_PRIMES[26], SWEEP_PRIMES[40], SWEEP_PRIMES[50 if 50 in SWEEP_PRIMES else 48], SWEEP_PRIMES[52]])
def test_alg1_reading_returns_x_mod_p(p):
    """Prop. 2.1: Alg. 1 returns x mod p for integer x <= 2^(t-2) p."""
    q = 1.0 / p
    xs = [0, 1, p - 1, p, p + 1, 2 * p - 1, 2 ** 53, 2 ** 53 - 1] + \
         [int(v) for v in inputs.uniform_mod(p % 1000, 3, 300, 1 << 53)]
    for x in xs:
        xf = float(x)
        assert float(int(xf)) == xf
        assert alg1(xf, float(p), q) == float(int(xf) % p)


@pytest.mark.parametrize("b", [20, 32, 40, 48, 50])
def test_alg2_reading_returns_xy_mod_p(b):
    """Prop. 2.2: Alg. 2 returns x y mod p when x y <= (2^(t-1)/3) p."""
    p = inputs.largest_prime_below_pow2(b)
    q = 1.0 / p
    assert p <= (1 << 52) // 3
    xs = [int(v) for v in inputs.uniform_mod(b, 4, 200, p)] + [p - 1, p - 2, 1, 0]
    ys = [int(v) for v in inputs.uniform_mod(b, 5, 200, p)] + [p - 1, p - 1, p - 1, p - 1]
    for x, y in zip(xs, ys):
        assert alg2(float(x), float(y), float(p), q) == float(x * y % p)


# ---- CRT (multimodular) comparison form, Sec. 5.2 ----
from math import gcd, prod


@pytest.mark.parametrize("b", [20, 23, 26, 32, 40, 48, 52])
@pytest.mark.parametrize("k", [1, 64, 4096, 32768])
def test_crt_moduli_are_minimal_coprime_and_cover_the_product(oracle, b, k):
    p = inputs.largest_prime_below_pow2(b)
    ms = oracle.crt_moduli(p, k)
    assert all(3 <= m < 256 for m in ms) and ms == sorted(ms, reverse=True)
    assert all(gcd(a, c) == 1 for i, a in enumerate(ms) for c in ms[i + 1:])
    target = 2 * k * (p - 1) ** 2
    assert prod(ms) > target >= prod(ms[:-1])  # enough, and one fewer is not
    # Sec. 5.2: M > k (p-1)^2 needs at least (2 log2(p-1) + log2 k) / 8 moduli below 2^8
    assert len(ms) >= (2 * (p - 1).bit_length() - 2 + k.bit_length() - 1) / 8


def test_crt_reconstruction_against_brute_force(oracle):
    ms = [3, 5, 7]
    for x in range(105):  # every residue triple comes from exactly one x < 105
        r = [((x % m) + m // 2) % m - m // 2 for m in ms]  # signed residues
        assert oracle.crt_reconstruct(r, ms) == x
    rng = np.random.default_rng(3)
    ms = oracle.crt_moduli(inputs.largest_prime_below_pow2(52), 4096)
    M = prod(ms)
    for _ in range(200):
        x = int(rng.integers(0, 1 << 62)) * int(rng.integers(0, 1 << 62)) % M
        assert oracle.crt_reconstruct([x % m for m in ms], ms) == x


@pytest.mark.parametrize("b", [20, 40, 52])
def test_crt_pipeline_reaches_the_exact_product(oracle, b):
    """Residues of A and B, one integer product per modulus, reconstruction:
    the integer product AB itself (checked with Python integers), hence AB mod
    p as the oracle computes it."""
    p = inputs.largest_prime_below_pow2(b)
    A, B = inputs.problem(70 + b, 5, 4, 6, p)
    ms = oracle.crt_moduli(p, 6)
    RA, RB = oracle.crt_residues(A, ms), oracle.crt_residues(B, ms)
    for i, m in enumerate(ms):
        assert np.all(np.abs(RA[i]) <= (m - 1) // 2) and np.all((RA[i].astype(np.int64) - A.astype(object) % m) % m == 0)
    S = [RA[i].astype(np.int64) @ RB[i].astype(np.int64) for i in range(len(ms))]
    exact = [[sum(int(A[r, l]) * int(B[l, c]) for l in range(6)) for c in range(4)] for r in range(5)]
    for r in range(5):
        for c in range(4):
            x = oracle.crt_reconstruct([S[i][r, c] for i in range(len(ms))], ms)
            assert x == exact[r][c]
    C = np.array([[oracle.crt_reconstruct([S[i][r, c] for i in range(len(ms))], ms) % p for c in range(4)]
                  for r in range(5)], dtype=np.uint64)
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))
