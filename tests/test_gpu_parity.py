"""Bit-exact parity of the CUDA path with the CPU oracle (needs a B300).

Every call goes through libmwmm's C ABI (via the ctypes binding); every
expected value comes from oracle/ on the same seeded inputs."""
import numpy as np
import pytest

from paper_2601_07508_b300 import build, inputs
from layout import unpack_words

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
SWEEP = {b: inputs.largest_prime_below_pow2(b) for b in inputs.SWEEP_BITS}
P50 = inputs.largest_prime_below_pow2(50)
P51 = inputs.largest_prime_below_pow2(51)


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_2601_07508_b300 import mwmm
    mwmm.lib()
    return mwmm


def dev(x: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()


def host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def gpu_product(M, A, B, p, **kw):
    m, k = A.shape
    n = B.shape[1]
    plan = M.Plan(m, n, k, p, **kw)
    C = plan.matmul(dev(A), dev(B))
    assert plan.check() == 0
    return host(C), plan


# ------------------------------------------------------------------ whole product
@pytest.mark.parametrize("form", ["fp64", "int8"])
def test_small_config_256cube_40bit(M, oracle, form):
    """256^3, p = largest prime below 2^40, seed 0; (2,2) in the FP64 form."""
    p = SWEEP[40]
    A, B = inputs.problem(0, 256, 256, 256, p)
    kw = dict(u=2, v=2) if form == "fp64" else {}
    C, plan = gpu_product(M, A, B, p, form=form, **kw)
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))


SHAPES = [(1, 1, 1), (5, 3, 7), (64, 64, 16), (100, 70, 50), (129, 65, 33), (130, 300, 257)]
FP64_VARIANTS = [(1, 1), (1, 2), (1, 3), (1, 4), (2, 2), (2, 3)]


@pytest.mark.parametrize("b", [20, 26, 32, 40, 48, 52])
@pytest.mark.parametrize("uv", FP64_VARIANTS)
def test_fp64_variants_ragged(M, oracle, b, uv):
    p = SWEEP[b]
    if oracle.lam(p, *uv) < 1:
        pytest.skip("variant cannot handle this bitsize")
    for seed, (m, n, k) in enumerate(SHAPES):
        A, B = inputs.problem(100 * b + seed, m, n, k, p)
        C, _ = gpu_product(M, A, B, p, form="fp64", u=uv[0], v=uv[1])
        assert np.array_equal(C, oracle.matmul_mod(A, B, p)), (m, n, k)


@pytest.mark.parametrize("uv", [(1, 2), (1, 3), (1, 4), (2, 2), (2, 3)])
@pytest.mark.parametrize("b", [23, 32, 40, 52])
def test_fp64_concatenated_words_narrow_n(M, oracle, uv, b):
    """Alg. 6: B's words concatenated along n (64-column tiles of 2 or 4 word
    slots), for n across the slot widths 16 and 32 and beyond one tile, with
    and without K ranges; equals the non-concatenated product and the oracle."""
    p = SWEEP[b]
    if oracle.lam(p, *uv) < 1:
        pytest.skip("variant cannot handle this bitsize")
    for seed, (m, n, k) in enumerate([(70, 1, 50), (130, 15, 333), (65, 16, 100), (200, 17, 257),
                                      (129, 32, 500), (100, 33, 64), (64, 63, 1000)]):
        A, B = inputs.problem(300 * b + seed, m, n, k, p)
        ref = oracle.matmul_mod(A, B, p)
        C, plan = gpu_product(M, A, B, p, form="fp64", u=uv[0], v=uv[1])
        assert plan.info["f64_concat"] == 1 and plan.info["B_rows"] % (32 if uv[1] == 2 else 16) == 0
        assert np.array_equal(C, ref), (m, n, k)
        C1, plan1 = gpu_product(M, A, B, p, form="fp64", u=uv[0], v=uv[1], f64_concat=1, ksplit=3)
        nkb = -(-k // 16)
        assert plan1.info["f64_concat"] == 0 and plan1.info["ksplit"] == -(-nkb // -(-nkb // min(3, nkb)))
        assert np.array_equal(C1, ref), (m, n, k)
        C2, plan2 = gpu_product(M, A, B, p, form="fp64", u=uv[0], v=uv[1], ksplit=5)
        assert plan2.info["f64_concat"] == 1
        assert np.array_equal(C2, ref), (m, n, k)


@pytest.mark.parametrize("uv", [(2, 2), (2, 3)])
@pytest.mark.parametrize("b", [32, 40, 52])
def test_fp64_concatenated_a_words_narrow_m(M, oracle, uv, b):
    """Alg. 6 with the A words concatenated (the narrow side is m, Sec. 3.2):
    64-row tiles of 2 word slots, with and without K ranges; equals the
    plain product and the oracle."""
    p = SWEEP[b]
    if oracle.lam(p, *uv) < 1:
        pytest.skip("variant cannot handle this bitsize")
    for seed, (m, n, k) in enumerate([(1, 70, 50), (15, 130, 333), (32, 257, 100), (33, 100, 257), (63, 64, 1000)]):
        A, B = inputs.problem(400 * b + seed, m, n, k, p)
        ref = oracle.matmul_mod(A, B, p)
        C, plan = gpu_product(M, A, B, p, form="fp64", u=uv[0], v=uv[1])
        assert plan.info["f64_concat"] == 2 and plan.info["A_rows"] % 32 == 0
        assert np.array_equal(C, ref), (m, n, k)
        C2, plan2 = gpu_product(M, A, B, p, form="fp64", u=uv[0], v=uv[1], ksplit=4)
        assert plan2.info["f64_concat"] == 2
        assert np.array_equal(C2, ref), (m, n, k)
        C3, _ = gpu_product(M, A, B, p, form="fp64", u=uv[0], v=uv[1], f64_concat=1)
        assert np.array_equal(C3, ref), (m, n, k)


@pytest.mark.parametrize("ks", [1, 2, 3, 7, 64])
def test_fp64_k_ranges(M, oracle, ks):
    """K ranges (grid z) with their partial results added mod p by a second
    kernel: ragged last range, ranges of one k-block, more ranges than asked
    when k is short; lambda boundaries inside ranges."""
    p = SWEEP[48]
    for seed, (m, n, k, lam) in enumerate([(70, 90, 1000, 0), (129, 65, 33, 0), (64, 64, 16 * 64, 3),
                                           (300, 130, 777, 31)]):
        A, B = inputs.problem(500 + seed, m, n, k, p)
        C, plan = gpu_product(M, A, B, p, form="fp64", u=2, v=2, lam=lam, ksplit=ks)
        nkb = -(-k // 16)
        assert plan.info["ksplit"] == -(-nkb // -(-nkb // min(ks, nkb)))
        assert np.array_equal(C, oracle.matmul_mod(A, B, p)), (m, n, k, ks)


@pytest.mark.parametrize("b", [20, 23, 26, 32, 40, 48, 50, 52])
def test_crt_form_ragged(M, oracle, b):
    """Multimodular comparison form (Sec. 5.2): residues modulo the primes
    below 256, one tcgen05 product per modulus, CRT reconstruction mod p."""
    p = SWEEP.get(b, P50)
    for seed, (m, n, k) in enumerate(SHAPES + [(300, 520, 1000), (129, 20, 777), (260, 130, 64)]):
        A, B = inputs.problem(2000 + 10 * b + seed, m, n, k, p)
        C, plan = gpu_product(M, A, B, p, form="crt8")
        assert plan.info["u"] == len(oracle.crt_moduli(p, k))
        assert np.array_equal(C, oracle.matmul_mod(A, B, p)), (m, n, k)


@pytest.mark.parametrize("b", [26, 52])
def test_crt_form_extremes_and_k_ranges(M, oracle, b):
    """All entries p - 1 (the largest integer product k (p-1)^2 the moduli
    must cover) and INT32 K-ranges of 64 / 320 steps (several sums per
    modulus added in 64 bits before the residue is taken)."""
    p = SWEEP[b]
    A = np.full((130, 700), p - 1, dtype=np.uint64)
    B = np.full((700, 260), p - 1, dtype=np.uint64)
    for kc in (0, 64, 320):
        C, plan = gpu_product(M, A, B, p, form="crt8", kc=kc)
        assert np.all(C == (700 * (p - 1) ** 2) % p), kc
    A, B = inputs.problem(77, 200, 300, 1500, p)
    C, plan = gpu_product(M, A, B, p, form="crt8", kc=192)
    assert plan.info["nkc"] == -(-1500 // 192)
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))


@pytest.mark.parametrize("form", ["int8", "crt8"])
@pytest.mark.parametrize("b", [20, 26, 52])
@pytest.mark.parametrize("shape", [(512, 512, 2048), (64, 64, 4096), (200, 300, 1500)])
def test_underfilled_products_split_k(M, oracle, form, b, shape):
    """A product whose work items would not fill the SMs plans shorter K
    ranges (more items, more sum planes added by the recombination); the
    result equals the oracle's and the one-K-range plan's."""
    m, n, k = shape
    p = SWEEP[b]
    A, B = inputs.problem(b + k, m, n, k, p)
    C, plan = gpu_product(M, A, B, p, form=form)
    C1, plan1 = gpu_product(M, A, B, p, form=form, tc_fill=1)
    assert plan1.info["nkc"] == 1 and plan.info["nkc"] >= 1
    assert form == "crt8" or plan.info["nkc"] > 1  # a diagonal's pairs make INT8 items long
    want = oracle.matmul_mod(A, B, p)
    assert np.array_equal(C, want) and np.array_equal(C1, want)


@pytest.mark.parametrize("b", [20, 52])
def test_crt_form_int32_sums_at_their_bound(M, oracle, b):
    """k at the INT32 K-range limit with constant columns, so each sum
    S_i = k d_a d_b sits near +-2^31 (|d| up to 125): the residues of the
    sums are taken over the whole 32-bit range."""
    p = SWEEP[b]
    k = 131008
    plan = M.Plan(2, 3, k, p, form="crt8", tc_fill=1)  # one K range: no split for the SMs' sake
    assert plan.info["nkc"] == 1
    m0 = plan.info["crt_m"][0]
    cols = np.array([p - 1, (m0 + 1) // 2, (m0 - 1) // 2], dtype=np.uint64)  # d = -1, -(m0-1)/2, (m0-1)/2 mod m0
    A = np.full((2, k), p - 1, dtype=np.uint64)
    B = np.tile(cols, (k, 1))
    C = host(plan.matmul(dev(A), dev(B)))
    assert plan.check() == 0
    ref = np.array([[k * (p - 1) * int(c) % p for c in cols]] * 2, dtype=np.uint64)
    assert np.array_equal(C, ref)


def test_crt_residue_words_and_sums_match_oracle(M, oracle):
    p = SWEEP[48]
    m, n, k = 130, 260, 300
    A, B = inputs.problem(79, m, n, k, p)
    plan = M.Plan(m, n, k, p, form="crt8", tc_fill=1)
    ws = plan.alloc_workspace()
    plan.matmul(dev(A), dev(B))
    assert plan.check() == 0
    d = plan.info
    ms = d["crt_m"][:d["u"]]
    assert ms == oracle.crt_moduli(p, k)
    WA = unpack_words(ws[d["A_off"]:].cpu().numpy(), d["u"], d["nkb"], d["A_rows"], "int8")
    WB = unpack_words(ws[d["B_off"]:].cpu().numpy(), d["v"], d["nkb"], d["B_rows"], "int8")
    RA, RB = oracle.crt_residues(A, ms), oracle.crt_residues(B.T.copy(), ms)
    assert np.array_equal(WA[:, :m, :k], RA) and np.array_equal(WB[:, :n, :k], RB)
    S = ws[d["S_off"]:d["S_off"] + d["nsums"] * d["nkc"] * d["A_rows"] * d["B_rows"] * 4]
    S = S.cpu().numpy().view(np.int32).reshape(d["nsums"], d["nkc"], d["A_rows"], d["B_rows"])
    for i in range(len(ms)):
        ref = RA[i].astype(np.int64) @ RB[i].astype(np.int64).T
        assert np.array_equal(S[i, 0, :m, :n], ref), i


@pytest.mark.parametrize("lam", [1, 2, 3, 7, 16, 17])
def test_fp64_block_size_boundaries(M, oracle, lam):
    """Reductions at every lambda-th k-step (including inside a 16-wide k-block)."""
    p = SWEEP[48]
    A, B = inputs.problem(7, 70, 90, 100, p)
    C, _ = gpu_product(M, A, B, p, form="fp64", u=2, v=2, lam=lam)
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))


@pytest.mark.parametrize("b,uv", [(26, (1, 1)), (32, (1, 2)), (40, (2, 2)), (52, (2, 2)), (52, (2, 3))])
def test_fp64_all_max_entries(M, oracle, b, uv):
    """All entries p - 1: every word is at its maximum, so every chunk sum
    reaches the largest value Prop. 3.3 allows."""
    p = SWEEP[b]
    A = np.full((70, 300), p - 1, dtype=np.uint64)
    B = np.full((300, 90), p - 1, dtype=np.uint64)
    C, _ = gpu_product(M, A, B, p, form="fp64", u=uv[0], v=uv[1])
    assert np.all(C == 300 % p)


@pytest.mark.parametrize("b", list(inputs.SWEEP_BITS) + [50])
def test_int8_all_bitsizes_ragged(M, oracle, b):
    p = SWEEP.get(b, P50)
    for seed, (m, n, k) in enumerate(SHAPES + [(300, 520, 1000)]):
        A, B = inputs.problem(1000 + 10 * b + seed, m, n, k, p)
        C, _ = gpu_product(M, A, B, p, form="int8")
        assert np.array_equal(C, oracle.matmul_mod(A, B, p)), (m, n, k)


@pytest.mark.parametrize("bits,tc_chunk,kc", [(8, 64, 0), (8, 192, 0), (8, 1024, 64), (8, 512, 320),
                                               (9, 64, 0), (9, 192, 0), (9, 256, 64), (9, 128, 320)])
def test_int8_chunk_boundaries(M, oracle, bits, tc_chunk, kc):
    """FP32 chunks of 1..16 k-blocks (1..4 with 9-bit digits) and INT32
    K-ranges of 1..5 k-blocks."""
    p = SWEEP[52]
    A, B = inputs.problem(11, 200, 300, 777, p)
    C, _ = gpu_product(M, A, B, p, form="int8", tc_chunk=tc_chunk, kc=kc, tc_digit_bits=bits)
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))


def _extreme(p: int, u: int, digit: int):
    """(entry, L): the entry whose L lowest balanced digits all equal `digit`
    and whose other digits are 0, with L <= u - 1 as large as the signed range
    [-(p-1)/2, (p-1)/2] allows."""
    for L in range(u - 1, 0, -1):
        s = digit * (256 ** L - 1) // 255
        if abs(s) <= (p - 1) // 2:
            return (s if s >= 0 else s + p), L
    raise ValueError("no room for an extreme digit pattern")


@pytest.mark.parametrize("b", [20, 40, 52])
@pytest.mark.parametrize("da,db", [(-128, -128), (127, 127), (-128, 127)])
def test_int8_extreme_digits_fill_the_fp32_chunk(M, oracle, b, da, db):
    """Digits at the ends of [-128, 127] make every product +-2^14 (or -16256),
    so a full 1024-product chunk reaches |sum| = 2^24: the exactness limit of
    the FP32 tensor-memory accumulator."""
    p = SWEEP[b]
    u = oracle.int8_words(p)
    (a, La), (bb, Lb) = _extreme(p, u, da), _extreme(p, u, db)
    Aw = oracle.split_signed8(np.array([a], np.uint64), p, u)[:, 0]
    Bw = oracle.split_signed8(np.array([bb], np.uint64), p, u)[:, 0]
    assert list(Aw) == [da] * La + [0] * (u - La) and list(Bw) == [db] * Lb + [0] * (u - Lb)
    A = np.full((130, 1024 + 64), a, dtype=np.uint64)
    B = np.full((1024 + 64, 260), bb, dtype=np.uint64)
    C, _ = gpu_product(M, A, B, p, form="int8", tc_digit_bits=8)
    assert np.all(C == (a * bb * (1024 + 64)) % p)


@pytest.mark.parametrize("b", [32, 40, 48])
@pytest.mark.parametrize("sa,sb", [(1, 1), (-1, -1), (1, -1)])
def test_int8_top_digit_128_fills_the_fp32_chunk(M, oracle, b, sa, sb):
    """For the largest prime below 2^(8u), +-(p-1)/2 has top digit +-128:
    u digits suffice, and top x top products of +-2^14 fill a 1024-product
    chunk to |sum| = 2^24."""
    p = SWEEP[b]
    u = oracle.int8_words(p)
    assert u == b // 8
    half = (p - 1) // 2
    a, bb = (half if sa > 0 else p - half), (half if sb > 0 else p - half)
    Aw = oracle.split_signed8(np.array([a], np.uint64), p, u)[:, 0]
    Bw = oracle.split_signed8(np.array([bb], np.uint64), p, u)[:, 0]
    assert Aw[-1] == 128 * sa and Bw[-1] == 128 * sb
    A = np.full((130, 1024 + 64), a, dtype=np.uint64)
    B = np.full((1024 + 64, 260), bb, dtype=np.uint64)
    C, _ = gpu_product(M, A, B, p, form="int8")
    assert np.all(C == (a * bb * (1024 + 64)) % p)
    # every entry at +-(p-1)/2 or 0, mixed, against the oracle
    rng = np.random.default_rng(b)
    A = rng.choice(np.array([0, half, p - half], np.uint64), size=(200, 1500))
    B = rng.choice(np.array([0, half, p - half], np.uint64), size=(1500, 300))
    C, _ = gpu_product(M, A, B, p, form="int8")
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))


# ------------------------------------------------------------------ FP32 chunk at its bound, odd low bits
# The tensor form's exactness rests on one property of the device: FP32
# tensor-memory accumulation of integer digit products is exact while every
# partial sum stays within 2^24 (Prop. 2.3's block condition with a 24-bit
# significand; a chunk holds at most 1024 products of magnitude <= 2^14).
# The patterns below make each MMA (K = 16) add an odd integer, or a small one
# far below the running sum, while that sum climbs past 2^23.8: an
# accumulator that dropped even one low bit near 2^24 would change the
# result.  The expected values come from the oracle only.
CHUNK = 1024            # digit products per FP32 chunk (default plan)
KDIM = CHUNK + 64       # two chunks: one full, one k-block


def _chunk_partials(a_dig: np.ndarray, b_dig: np.ndarray) -> np.ndarray:
    """Running sum after each K = 16 slice, restarted every CHUNK positions,
    of sum_k a_dig[k] b_dig[k] (one diagonal with one word pair)."""
    prod = (a_dig.astype(np.int64) * b_dig.astype(np.int64)).reshape(-1, 16).sum(axis=1)
    return np.concatenate([np.cumsum(prod[i:i + CHUNK // 16]) for i in range(0, prod.size, CHUNK // 16)])


def _kernel(fused):
    """Plan options for the word-product kernel under test: 1 = one CTA per
    tile, "pair" = CTA pairs (256 x 256 tiles, cta_group::2), 2 = the fused
    form (256 x 128 tiles on CTA pairs, recombination in the epilogue)."""
    return dict(tc_fused=2) if fused == 2 else dict(tc_fused=1, tc_pair=(fused == "pair"))


def _kernel_ok(plan, fused) -> bool:
    d = plan.info
    return d["tc_fused"] == (fused == 2) and d["tc_pair"] == (fused == "pair")


def _odd_slices_patterns(pos: int, neg: int, rows: int, cols: int):
    """A (rows x KDIM) and B (KDIM x cols) over {0, pos, neg}: A row r has
    the value at 15 of every 16 k positions (0 at k % 16 == 15), with sign +
    for the first r % 65 slices of each chunk and - after, so rows range from
    all +, through a zero crossing at every slice, to all -; B columns are all
    + or all - (by column parity)."""
    k = np.arange(KDIM)
    A = np.zeros((rows, KDIM), np.uint64)
    for r in range(rows):
        t = r % 65
        plus = ((k % CHUNK) // 16) < t
        A[r] = np.where(k % 16 == 15, 0, np.where(plus, pos, neg))
    B = np.empty((KDIM, cols), np.uint64)
    B[:, 0::2] = pos
    B[:, 1::2] = neg
    return A, B


@pytest.mark.parametrize("b", [20, 40, 52])
@pytest.mark.parametrize("fused", [1, "pair", 2])
def test_int8_fp32_chunk_odd_increments_near_2_24(M, oracle, b, fused):
    """Digits +-127 at 15 of every 16 k positions against B digits +-127: every
    MMA adds +-15 x 16129 (odd), and a chunk's running sum walks up to
    +-64 x 241935 = +-15,483,840 (2^23.88), with zero crossings at every
    slice across the rows."""
    p = SWEEP[b]
    u = oracle.int8_words(p)
    A, B = _odd_slices_patterns(127, p - 127, 130, 260)
    Ad = oracle.split_signed8(A, p, u)
    Bd = oracle.split_signed8(B, p, u)
    assert np.all(Ad[1:] == 0) and np.all(Bd[1:] == 0)  # only digit 0: one diagonal, one pair
    peak = 0
    for r in (0, 1, 32, 64):
        for c in (0, 1):
            part = _chunk_partials(Ad[0, r], Bd[0, :, c])
            assert np.all(np.diff(part[:CHUNK // 16]) % 2 == 1) and np.all(np.abs(part) <= 2 ** 24)
            peak = max(peak, int(np.abs(part).max()))
    assert peak > 2 ** 23.85
    C, plan = gpu_product(M, A, B, p, form="int8", **_kernel(fused), tc_digit_bits=8)
    assert _kernel_ok(plan, fused)
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))


def _small_addend_patterns(big_pos, big_neg, one_pos, one_neg, sign):
    """A (129 x KDIM), B (KDIM x 257): in each chunk the first 960 k positions
    (60 slices) hold the large value, then each of the last 4 slices holds a
    single small value (positions 960, 976, 992, 1008) and zeros; B holds the
    large value, then the small one, with + and - columns.  Odd rows of A are
    the pattern one slice later (the last small value moves into the next
    chunk).  `sign` picks the sign of A's values."""
    k = np.arange(KDIM)
    pos = k % CHUNK
    big, one = (big_pos, one_pos) if sign > 0 else (big_neg, one_neg)
    row = np.where(pos < 960, big, 0).astype(np.uint64)
    row[(pos >= 960) & (pos % 16 == 0)] = one
    A = np.tile(row, (129, 1))
    A[1::2] = np.roll(row, 16)
    B = np.empty((KDIM, 257), np.uint64)
    B[:, 0::2] = np.where(pos < 960, big_pos, one_pos)[:, None]
    B[:, 1::2] = np.where(pos < 960, big_neg, one_neg)[:, None]
    return A, B


@pytest.mark.parametrize("b", [20, 52])
@pytest.mark.parametrize("sign", [1, -1])
@pytest.mark.parametrize("fused", [1, "pair", 2])
def test_int8_fp32_chunk_small_addend_below_large_sum(M, oracle, b, sign, fused):
    """A chunk first sums 960 products of +-16129 (reaching +-15,483,840,
    2^23.88), then four MMAs that each add +-1 (one product 1 x 1 in 16): the
    small addends sit 24 bits below the accumulator."""
    p = SWEEP[b]
    u = oracle.int8_words(p)
    A, B = _small_addend_patterns(127, p - 127, 1, p - 1, sign)
    Ad = oracle.split_signed8(A, p, u)
    Bd = oracle.split_signed8(B, p, u)
    assert np.all(Ad[1:] == 0) and np.all(Bd[1:] == 0)
    part = _chunk_partials(Ad[0, 0], Bd[0, :, 0])
    last = part[CHUNK // 16 - 5:CHUNK // 16]
    assert list(np.diff(last)) == [sign] * 4 and abs(int(last[0])) == 960 * 16129
    assert np.all(np.abs(part) <= 2 ** 24) and np.abs(part).max() > 2 ** 23.85
    C, plan = gpu_product(M, A, B, p, form="int8", **_kernel(fused), tc_digit_bits=8)
    assert _kernel_ok(plan, fused)
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))


@pytest.mark.parametrize("b", [20, 40, 52])
@pytest.mark.parametrize("fused", [1, "pair", 2])
def test_int8_fp32_chunk_odd_increments_in_a_two_pair_diagonal(M, oracle, b, fused):
    """Digits 0 and 1 both at +-127 (entries +-(127 + 127 x 256)): diagonal 1
    concatenates the pairs (0,1) and (1,0) along K, so its chunks span both
    pairs; every slice still adds an odd multiple of 16129."""
    p = SWEEP[b]
    u = oracle.int8_words(p)
    e = 127 + 127 * 256
    A, B = _odd_slices_patterns(e, p - e, 130, 260)
    Ad = oracle.split_signed8(A, p, u)
    assert np.all(np.abs(Ad[:2]) <= 127) and np.all(Ad[2:] == 0) and int(Ad[1, 64, 0]) == 127
    C, plan = gpu_product(M, A, B, p, form="int8", **_kernel(fused), tc_digit_bits=8)
    assert _kernel_ok(plan, fused)
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))


# 9-bit digits (fp16): products of magnitude <= 2^16, FP32 chunks of 256.
CHUNK9 = 256
KDIM9 = 2 * CHUNK9 + 64   # two full chunks and one k-block


def _chunk_partials9(a_dig, b_dig):
    prod = (a_dig.astype(np.int64) * b_dig.astype(np.int64)).reshape(-1, 16).sum(axis=1)
    return np.concatenate([np.cumsum(prod[i:i + CHUNK9 // 16]) for i in range(0, prod.size, CHUNK9 // 16)])


@pytest.mark.parametrize("b", [26, 40, 52])
@pytest.mark.parametrize("da,db", [(-256, -256), (255, 255), (-256, 255)])
@pytest.mark.parametrize("fused", [1, "pair", 2])
def test_f16_extreme_digits_fill_the_fp32_chunk(M, oracle, b, da, db, fused):
    """9-bit digits at the ends of [-256, 255]: every product is +-2^16 (or
    -65280, 65025), so a full 256-product chunk reaches |sum| = 2^24."""
    p = SWEEP[b]
    u = oracle.digit_words(p, 9)
    a, bb = (da if da >= 0 else p + da), (db if db >= 0 else p + db)
    Aw = oracle.split_signed(np.array([a], np.uint64), p, u, 9)[:, 0]
    Bw = oracle.split_signed(np.array([bb], np.uint64), p, u, 9)[:, 0]
    assert list(Aw) == [da] + [0] * (u - 1) and list(Bw) == [db] + [0] * (u - 1)
    A = np.full((130, KDIM9), a, dtype=np.uint64)
    B = np.full((KDIM9, 260), bb, dtype=np.uint64)
    C, plan = gpu_product(M, A, B, p, form="int8", tc_digit_bits=9, **_kernel(fused))
    assert plan.info["tc_chunk"] == CHUNK9 and _kernel_ok(plan, fused)
    assert np.all(C == (a * bb * KDIM9) % p)


@pytest.mark.parametrize("b", [26, 52])
@pytest.mark.parametrize("fused", [1, "pair", 2])
def test_f16_fp32_chunk_odd_increments_near_2_24(M, oracle, b, fused):
    """9-bit digits +-255 at 15 of every 16 k positions against B digits
    +-255: every MMA adds +-15 x 65025 (odd), a chunk's running sum walks to
    +-16 x 975375 = +-15,606,000 (2^23.9), with zero crossings across rows."""
    p = SWEEP[b]
    u = oracle.digit_words(p, 9)
    k = np.arange(KDIM9)
    A = np.zeros((130, KDIM9), np.uint64)
    for r in range(130):
        t = r % 17
        plus = ((k % CHUNK9) // 16) < t
        A[r] = np.where(k % 16 == 15, 0, np.where(plus, 255, p - 255))
    B = np.empty((KDIM9, 260), np.uint64)
    B[:, 0::2] = 255
    B[:, 1::2] = p - 255
    Ad = oracle.split_signed(A, p, u, 9)
    Bd = oracle.split_signed(B, p, u, 9)
    assert np.all(Ad[1:] == 0) and np.all(Bd[1:] == 0)
    peak = 0
    for r in (0, 1, 8, 16):
        for c in (0, 1):
            part = _chunk_partials9(Ad[0, r], Bd[0, :, c])
            assert np.all(np.diff(part[:CHUNK9 // 16]) % 2 == 1) and np.all(np.abs(part) <= 2 ** 24)
            peak = max(peak, int(np.abs(part).max()))
    assert peak > 2 ** 23.89
    C, plan = gpu_product(M, A, B, p, form="int8", tc_digit_bits=9, **_kernel(fused))
    assert plan.info["tc_chunk"] == CHUNK9 and _kernel_ok(plan, fused)
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))


@pytest.mark.parametrize("b", [26, 52])
@pytest.mark.parametrize("sign", [1, -1])
def test_f16_fp32_chunk_small_addend_below_large_sum(M, oracle, b, sign):
    """12 slices of products +-255 x 255 (+-12,484,800, 2^23.57) then four MMAs
    each adding +-1 inside the same 256-product chunk."""
    p = SWEEP[b]
    u = oracle.digit_words(p, 9)
    k = np.arange(KDIM9)
    pos = k % CHUNK9
    big, one = (255, 1) if sign > 0 else (p - 255, p - 1)
    row = np.where(pos < 192, big, 0).astype(np.uint64)
    row[(pos >= 192) & (pos % 16 == 0)] = one
    A = np.tile(row, (129, 1))
    A[1::2] = np.roll(row, 16)
    B = np.empty((KDIM9, 257), np.uint64)
    B[:, 0::2] = np.where(pos < 192, 255, 1)[:, None]
    B[:, 1::2] = np.where(pos < 192, p - 255, p - 1)[:, None]
    Ad = oracle.split_signed(A, p, u, 9)
    Bd = oracle.split_signed(B, p, u, 9)
    part = _chunk_partials9(Ad[0, 0], Bd[0, :, 0])
    last = part[CHUNK9 // 16 - 5:CHUNK9 // 16]
    assert list(np.diff(last)) == [sign] * 4 and abs(int(last[0])) == 192 * 65025
    C, _ = gpu_product(M, A, B, p, form="int8", tc_digit_bits=9)
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))


def _sq_regions(d):
    """Byte offsets of the squared-digit maxima (A, B) in a certified plan's
    workspace: after the sums and the 256-byte item counter."""
    sums = d["nsums"] * d["nkc"] * d["A_rows"] * d["B_rows"] * 4
    a = (d["S_off"] + sums + 255) // 256 * 256 + 256
    return a, a + (d["u"] * d["nkb"] * (d["A_rows"] // 64) * 4 + 255) // 256 * 256


def _sq_expected(dig, rows_pad, nkb):
    """Per word, k-block and group of 64 rows: the largest sum over the
    k-block of a row's squared digits (dig: [words][rows][k] signed)."""
    w, r, k = dig.shape
    full = np.zeros((w, rows_pad, nkb * 64), np.int64)
    full[:, :r, :k] = dig
    sq = (full ** 2).reshape(w, rows_pad, nkb, 64).sum(-1)          # [w][row][kb]
    return sq.reshape(w, rows_pad // 64, 64, nkb).max(axis=2).transpose(0, 2, 1)  # [w][kb][group]


@pytest.mark.parametrize("b", [26, 52])
@pytest.mark.parametrize("pair", [False, True])
def test_f16_squared_digit_maxima_match_oracle(M, oracle, b, pair):
    """The splits of a certified plan write, per word, k-block and 64-row
    group, the largest row sum of squared digits: recomputed from the
    oracle's digits (A's rows, B's columns), ragged tiles included (128- and
    256-row tiles)."""
    p = SWEEP[b]
    m, n, k = 300, 700, 1000
    A, B = inputs.problem(b + 31, m, n, k, p)
    plan = M.Plan(m, n, k, p, form="int8", tc_pair=pair)
    d = plan.info
    assert d["tc_cert_chunk"] == 512 and d["tc_pair"] == pair
    ws = plan.alloc_workspace()
    C = host(plan.matmul(dev(A), dev(B)))
    assert plan.check() == 0 and np.array_equal(C, oracle.matmul_mod(A, B, p))
    oa, ob = _sq_regions(d)
    u, v, nkb = d["u"], d["v"], d["nkb"]
    raw = ws.cpu().numpy()
    got_a = raw[oa:oa + u * nkb * (d["A_rows"] // 64) * 4].view(np.uint32).reshape(u, nkb, -1)
    got_b = raw[ob:ob + v * nkb * (d["B_rows"] // 64) * 4].view(np.uint32).reshape(v, nkb, -1)
    Ad = oracle.split_signed(A, p, u, 9).astype(np.int64)
    Bd = oracle.split_signed(B.T.copy(), p, v, 9).astype(np.int64)
    assert np.array_equal(got_a, _sq_expected(Ad, d["A_rows"], nkb))
    assert np.array_equal(got_b, _sq_expected(Bd, d["B_rows"], nkb))


@pytest.mark.parametrize("b", [26, 52])
@pytest.mark.parametrize("digit", [181, 183, -181])
@pytest.mark.parametrize("pair", [False, True])
def test_f16_certified_chunk_at_its_bound(M, oracle, b, digit, pair):
    """Constant digits d (odd): every product is d^2 (odd), and a 512-product
    chunk of them sums to 512 d^2.  For |d| = 181 that is 16,773,632 (just
    below 2^24) and the certificate 8 x 8 (64 d^2)^2 <= 2^48 holds exactly
    at its bound, so the certified chunk runs with partial sums up to
    2^23.9996; for 183 it fails (512 d^2 > 2^24) and the 256-product chunk
    must run -- a wrong decision would round an odd partial sum above 2^24.
    Both the one-CTA and the pair kernel (256-row tiles)."""
    p = SWEEP[b]
    a = digit % p
    k = 2 * 512 + 64 + 37
    A = np.full((150, k), a, np.uint64)
    B = np.full((k, 300), a, np.uint64)
    u = oracle.digit_words(p, 9)
    assert list(oracle.split_signed(np.array([a], np.uint64), p, u, 9)[:, 0]) == [digit] + [0] * (u - 1)
    C, plan = gpu_product(M, A, B, p, form="int8", tc_pair=pair)
    assert plan.info["tc_cert_chunk"] == 512 and plan.info["tc_pair"] == pair
    assert np.all(C == (digit * digit * k) % p)
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))


@pytest.mark.parametrize("b", [26, 52])
@pytest.mark.parametrize("pair", [False, True])
def test_f16_certified_and_worst_case_items_mixed(M, oracle, b, pair):
    """Random digits (certified items) next to a row tile and a column tile
    of constant 183s (items whose certificate fails): every item exact."""
    p = SWEEP[b]
    m, n, k = 600, 600, 1200
    A, B = inputs.problem(b + 77, m, n, k, p)
    A[:128] = 183
    B[:, :256] = 183
    C, plan = gpu_product(M, A, B, p, form="int8", tc_pair=pair)
    assert plan.info["tc_cert_chunk"] == 512 and plan.info["tc_pair"] == pair
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))


@pytest.mark.parametrize("b", [26, 40, 48, 52])
def test_f16_digits_match_oracle_and_8bit_digits(M, oracle, b):
    """9-bit digits (fp16 words) on ragged shapes through several chunks,
    K-ranges and the pair and fused kernels: equal to the oracle and to the
    8-bit digits."""
    p = SWEEP[b]
    for seed, (m, n, k) in enumerate([(129, 300, 777), (300, 40, 1100), (257, 260, 5500), (1, 129, 64)]):
        A, B = inputs.problem(1200 + b + seed, m, n, k, p)
        ref = oracle.matmul_mod(A, B, p)
        for kw in ({}, {"tc_pair": True}, {"tc_fused": 2}, {"kc": 320, "tc_chunk": 128}):
            C, plan = gpu_product(M, A, B, p, form="int8", tc_digit_bits=9, **kw)
            assert plan.info["tc_digit_bits"] == 9
            assert np.array_equal(C, ref), (m, n, k, kw)
        C8, _ = gpu_product(M, A, B, p, form="int8", tc_digit_bits=8)
        assert np.array_equal(C8, ref)


@pytest.mark.parametrize("b", [20, 40, 52])
@pytest.mark.parametrize("pair", [False, True])
def test_crt_fp32_chunk_odd_increments_near_2_24(M, oracle, b, pair):
    """The CRT form's chunks: entries with residue +-125 modulo 251 (the
    first modulus; 125 and 126 = 251 - 125) at 15 of every 16 k positions,
    so the modulus-251 product adds +-15 x 15625 (odd) per slice and climbs
    to +-15,000,000 (2^23.84); the other moduli see other odd-heavy
    residues."""
    p = SWEEP[b]
    moduli = oracle.crt_moduli(p, KDIM)
    assert moduli[0] == 251
    A, B = _odd_slices_patterns(125, 126, 130, 260)
    R = oracle.crt_residues(A, moduli)
    Rb = oracle.crt_residues(B, moduli)
    part = _chunk_partials(R[0, 64], Rb[0, :, 0])
    assert np.all(np.diff(part[:CHUNK // 16]) % 2 == 1) and np.abs(part).max() > 2 ** 23.8
    assert np.all(np.abs(part) <= 2 ** 24)
    C, plan = gpu_product(M, A, B, p, form="crt8", tc_pair=pair)
    assert plan.info["crt_m"][0] == 251 and plan.info["tc_chunk"] == CHUNK and plan.info["tc_pair"] == pair
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))


@pytest.mark.parametrize("b", [20, 52])
@pytest.mark.parametrize("sign", [1, -1])
@pytest.mark.parametrize("pair", [False, True])
def test_crt_fp32_chunk_small_addend_below_large_sum(M, oracle, b, sign, pair):
    """CRT residues modulo 251: 960 products of +-125 x 125 (15,000,000,
    2^23.84), then four MMAs adding +-1 (residues 1 x 1) in the same chunk;
    126 and 250 are the residues -125 and -1."""
    p = SWEEP[b]
    moduli = oracle.crt_moduli(p, KDIM)
    assert moduli[0] == 251
    A, B = _small_addend_patterns(125, 126, 1, 250, sign)
    R = oracle.crt_residues(A, moduli)
    Rb = oracle.crt_residues(B, moduli)
    part = _chunk_partials(R[0, 0], Rb[0, :, 0])
    last = part[CHUNK // 16 - 5:CHUNK // 16]
    assert list(np.diff(last)) == [sign] * 4 and abs(int(last[0])) == 960 * 15625
    assert np.all(np.abs(part) <= 2 ** 24)
    C, plan = gpu_product(M, A, B, p, form="crt8", tc_pair=pair)
    assert plan.info["tc_pair"] == pair
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))


@pytest.mark.parametrize("form", ["fp64", "int8", "crt8"])
def test_leading_dimensions_and_degenerate_shapes(M, oracle, form):
    p = SWEEP[32]
    A, B = inputs.problem(5, 40, 30, 20, p)
    Abig = np.zeros((40, 33), np.uint64)
    Abig[:, :20] = A
    Bbig = np.zeros((20, 35), np.uint64)
    Bbig[:, :30] = B
    plan = M.Plan(40, 30, 20, p, form=form)
    Cbig = torch.zeros((40, 41), dtype=torch.int64, device="cuda")
    M.mwmm_matmul(plan.handle, dev(Abig)[:, :20], dev(Bbig)[:, :30], Cbig[:, :30], stream=None)
    assert plan.check() == 0
    got = host(Cbig)
    assert np.array_equal(got[:, :30], oracle.matmul_mod(A, B, p))
    assert np.all(got[:, 30:] == 0)
    # k = 0: empty sum
    plan0 = M.Plan(7, 9, 0, p, form=form)
    C0 = plan0.matmul(torch.zeros((7, 1), dtype=torch.int64, device="cuda"),
                      torch.zeros((1, 9), dtype=torch.int64, device="cuda"),
                      torch.full((7, 9), 5, dtype=torch.int64, device="cuda"))
    assert plan0.check() == 0 and int(C0.abs().sum()) == 0
    # m = 0 or n = 0: nothing to compute, nothing written, no workspace
    for m, n in ((0, 9), (7, 0), (0, 0)):
        pe = M.Plan(m, n, 5, p, form=form)
        assert pe.workspace_bytes == 0
        Ce = pe.matmul(torch.zeros((max(m, 1), 5), dtype=torch.int64, device="cuda")[:m],
                       torch.zeros((5, max(n, 1)), dtype=torch.int64, device="cuda")[:, :n])
        assert pe.check() == 0 and tuple(Ce.shape) == (m, n)


@pytest.mark.parametrize("form", ["fp64", "int8", "crt8"])
def test_host_entry_point(M, oracle, form):
    p = SWEEP[48]
    A, B = inputs.problem(21, 150, 140, 130, p)
    plan = M.Plan(150, 140, 130, p, form=form)
    C = plan.matmul_host(A, B)
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))


@pytest.mark.parametrize("form", ["fp64", "int8", "crt8"])
@pytest.mark.parametrize("shape", [(1100, 70, 300), (4100, 33, 200), (2048, 260, 129)])
def test_host_entry_point_row_block_pipeline(M, oracle, form, shape):
    """m >= 1024: row blocks on three streams (A in, compute, C out); strided
    host matrices; equal to the one-stream order (taken when timing is on)."""
    m, n, k = shape
    p = SWEEP[32] if form == "fp64" else SWEEP[52]
    A, B = inputs.problem(23 + m, m, n, k, p)
    ref = oracle.matmul_mod(A, B, p)
    plan = M.Plan(m, n, k, p, form=form)
    assert np.array_equal(plan.matmul_host(A, B), ref)
    # leading dimensions larger than the rows
    Ap = np.zeros((m, k + 3), np.uint64)
    Ap[:, :k] = A
    Bp = np.zeros((k, n + 5), np.uint64)
    Bp[:, :n] = B
    Cp = np.full((m, n + 2), 7, np.uint64)
    M.mwmm_matmul_host_ptr(plan.handle, Ap.ctypes.data, k + 3, Bp.ctypes.data, n + 5, Cp.ctypes.data, n + 2)
    assert np.array_equal(Cp[:, :n], ref) and np.all(Cp[:, n:] == 7)
    M.mwmm_plan_set_timing(plan.handle, True)  # one-stream path
    assert np.array_equal(plan.matmul_host(A, B), ref)


def test_host_async_products_on_separate_streams(M, oracle):
    """Enqueued host-buffer products of several plans on several streams
    (page-locked buffers) all complete with the oracle's results."""
    p = SWEEP[48]
    shapes = [(1500, 300, 200), (700, 64, 333), (2100, 20, 100)]
    jobs = []
    for i, (m, n, k) in enumerate(shapes):
        A, B = inputs.problem(60 + i, m, n, k, p)
        hA = torch.from_numpy(A.view(np.int64)).pin_memory()
        hB = torch.from_numpy(B.view(np.int64)).pin_memory()
        hC = torch.empty((m, n), dtype=torch.int64).pin_memory()
        plan = M.Plan(m, n, k, p, form="int8" if i != 1 else "fp64")
        st = torch.cuda.Stream()
        M.mwmm_matmul_host_async_ptr(plan.handle, hA.data_ptr(), k, hB.data_ptr(), n, hC.data_ptr(), n, stream=st)
        jobs.append((plan, st, hC, A, B))
    for plan, st, hC, A, B in jobs:
        assert plan.check(st) == 0
        assert np.array_equal(hC.numpy().view(np.uint64), oracle.matmul_mod(A, B, p))


def test_host_pipeline_reports_out_of_range_entries(M, oracle):
    p = SWEEP[40]
    m, n, k = 2000, 40, 100
    A, B = inputs.problem(5, m, n, k, p)
    A[1500, 7] = p  # in the second row block
    plan = M.Plan(m, n, k, p, form="int8", validate=True)
    with pytest.raises(M.MwmmError) as e:
        plan.matmul_host(A, B)
    assert e.value.status == 4  # MWMM_ERR_RANGE
    A[1500, 7] = 0
    assert np.array_equal(plan.matmul_host(A, B), oracle.matmul_mod(A, B, p))


def test_validation_reports_entries_out_of_range(M):
    p = SWEEP[40]
    A, B = inputs.problem(3, 64, 64, 64, p)
    A[3, 5] = p  # not in F_p
    plan = M.Plan(64, 64, 64, p, form="int8", validate=True)
    plan.matmul(dev(A), dev(B))
    assert plan.check() == 4  # MWMM_ERR_RANGE
    A[3, 5] = 0
    plan.matmul(dev(A), dev(B))
    assert plan.check() == 0


# ------------------------------------------------------------------ single steps
@pytest.mark.parametrize("form,b,uv,n", [("fp64", 40, (2, 2), 90), ("fp64", 52, (2, 3), 90), ("fp64", 32, (1, 4), 90),
                                         ("fp64", 32, (1, 2), 40), ("fp64", 40, (1, 4), 20), ("fp64", 52, (2, 3), 33),
                                         ("fp64", 40, (2, 2), 300),
                                         ("int8", 52, None, 290), ("int8", 23, None, 290), ("int8", 52, None, 90),
                                         ("int8", 40, None, 20), ("int8", 26, None, 290), ("int8", 52, None, 33),
                                         ("int8", 40, "f16", 290)])
def test_split_words_match_oracle(M, oracle, form, b, uv, n):
    p = SWEEP[b]
    m, k = 70, 150
    if form == "fp64" and n == 300:
        m = 20  # narrow m: the A words are concatenated (k-block major)
    A, B = inputs.problem(31, m, n, k, p)
    kw = dict(u=uv[0], v=uv[1]) if isinstance(uv, tuple) else ({"tc_digit_bits": 9} if uv == "f16" else {})
    plan = M.Plan(m, n, k, p, form=form, **kw)
    d = plan.info
    bits = d["tc_digit_bits"]
    for side, Mx, rows in ((0, A, m), (1, B, n)):
        words = d["u"] if side == 0 else d["v"]
        rows_pad = d["A_rows"] if side == 0 else d["B_rows"]
        wpad = d["B_wpad"] if side == 1 else 0
        buf = torch.full(((words + 2 * wpad) * d["nkb"] * rows_pad * 128,), 0x5A, dtype=torch.uint8, device="cuda")
        M.mwmm_split(plan.handle, side, dev(Mx), buf)
        torch.cuda.synchronize()
        kmajor = (side == 1 and d["f64_concat"] == 1) or (side == 0 and d["f64_concat"] == 2)
        W = unpack_words(buf.cpu().numpy(), words, d["nkb"], rows_pad, "f16" if bits == 9 else form, wpad,
                         kmajor=kmajor)
        src = Mx if side == 0 else Mx.T.copy()       # rows x k
        if form == "fp64":
            ref = oracle.split_alpha(src, d["alpha"] if side == 0 else d["beta"], words).astype(np.float64)
        else:
            ref = oracle.split_signed(src, p, words, bits).astype(np.float64)
        assert np.array_equal(W[:, :rows, :k], ref)
        assert np.all(W[:, rows:, :] == 0) and np.all(W[:, :, k:] == 0)


@pytest.mark.parametrize("b,bits", [(20, 0), (52, 0), (52, 8), (40, 9)])
def test_int8_diagonal_sums_match_oracle(M, oracle, b, bits):
    """S_s = sum_{i+j=s} A_i B_j read from the workspace after a product
    (8- or 9-bit digits), and C = sum_s R^s S_s mod p."""
    p = SWEEP[b]
    m, n, k = 130, 260, 700
    A, B = inputs.problem(41, m, n, k, p)
    plan = M.Plan(m, n, k, p, form="int8", kc=256, tc_digit_bits=bits)
    ws = plan.alloc_workspace()
    plan.matmul(dev(A), dev(B))
    assert plan.check() == 0
    d = plan.info
    S = ws[d["S_off"]:d["S_off"] + d["nsums"] * d["nkc"] * d["A_rows"] * d["B_rows"] * 4]
    S = S.cpu().numpy().view(np.int32).reshape(d["nsums"], d["nkc"], d["A_rows"], d["B_rows"])
    u, db = d["u"], d["tc_digit_bits"]
    assert db == (bits or (9 if b == 52 else 8))
    Aw = oracle.split_signed(A, p, u, db)
    Bw = oracle.split_signed(B, p, u, db)
    total = np.zeros((d["nsums"], m, n), np.int64)
    for kc in range(d["nkc"]):
        sl = slice(kc * d["kc"], min(k, (kc + 1) * d["kc"]))
        ref = oracle.diag_sums(np.ascontiguousarray(Aw[:, :, sl]), np.ascontiguousarray(Bw[:, sl, :]))
        assert np.array_equal(S[:, kc, :m, :n].astype(np.int64), ref)
        total += ref
    assert np.array_equal(oracle.recombine_pow(total, 2 ** db, p), oracle.matmul_mod(A, B, p))


@pytest.mark.parametrize("p", [5, 7, 65521, SWEEP[26], SWEEP[40], P50, P51, SWEEP[52]])
def test_fmod_alg1_matches_x_mod_p(M, oracle, p):
    xs = np.concatenate([
        inputs.uniform_mod(p % 997, 1, 20000, 1 << 53).astype(np.float64),
        np.array([0, 1, p - 1, p, p + 1, 2 * p - 1, 2.0 ** 53, 2.0 ** 53 - 1, float(p) * 2.0 ** 51], np.float64),
        (np.arange(1, 2001, dtype=np.float64) * 2.0 ** 40)])
    xs = xs[xs <= float(p) * 2.0 ** 51]
    out = torch.empty(xs.size, dtype=torch.float64, device="cuda")
    M.mwmm_fmod(torch.from_numpy(xs).cuda(), p, out)
    got = out.cpu().numpy()
    assert np.array_equal(got.astype(np.uint64), oracle.mod_vec(xs, p))
    assert np.all(got == np.floor(got))


@pytest.mark.parametrize("p", [5, 7, 65521, SWEEP[26], SWEEP[40], P50, P51, SWEEP[52]])
def test_mulmod_alg2_matches_xy_mod_p(M, oracle, p):
    x = np.concatenate([inputs.uniform_mod(3, 1, 20000, p), np.array([p - 1, p - 1, 0, 1], np.uint64)])
    y = np.concatenate([inputs.uniform_mod(3, 2, 20000, p), np.array([p - 1, 1, p - 1, p - 1], np.uint64)])
    out = torch.empty(x.size, dtype=torch.float64, device="cuda")
    M.mwmm_mulmod(torch.from_numpy(x.astype(np.float64)).cuda(), torch.from_numpy(y.astype(np.float64)).cuda(),
                  p, out)
    assert np.array_equal(out.cpu().numpy().astype(np.uint64), oracle.mulmod_vec(x, y, p))


@pytest.mark.parametrize("shape", [(129, 300, 257), (256, 256, 64), (700, 520, 1100), (1000, 90, 333),
                                   (100, 300, 200), (385, 20, 900)])
@pytest.mark.parametrize("b", [20, 40, 52])
def test_int8_pair_and_single_cta_kernels(M, oracle, shape, b):
    """The two-CTA kernel (256-row tiles on an SM pair, tcgen05 cta_group::2,
    tensor TMA completing on the leader's barrier) and the one-CTA kernel (the
    default) both match the oracle."""
    m, n, k = shape
    p = SWEEP[b]
    A, B = inputs.problem(60 + b, m, n, k, p)
    ref = oracle.matmul_mod(A, B, p)
    for pair in (False, True):
        C, plan = gpu_product(M, A, B, p, form="int8", tc_pair=pair)
        assert plan.info["tc_pair"] == (1 if pair and n > 128 and m > 128 else 0)  # pairs need 256-wide tiles
        assert plan.info["A_rows"] % (256 if plan.info["tc_pair"] else 128) == 0
        assert np.array_equal(C, ref), pair


@pytest.mark.parametrize("form,b", [("int8", 20), ("int8", 40), ("int8", 52), ("crt8", 32), ("crt8", 52)])
@pytest.mark.parametrize("kc", [0, 320])
def test_pair_kernel_k_ranges_and_forms(M, oracle, form, b, kc):
    """The pair kernel on ragged shapes (partial 256-row and 256-column
    tiles) with the planner's K ranges or explicit ones (kc = 320: 5 k-blocks
    per range, a last short range), 8-bit digits, 9-bit digits with certified
    chunks, and CRT residues: equal to the oracle and to the one-CTA kernel."""
    p = SWEEP[b]
    m, n, k = 515, 700, 1500
    A, B = inputs.problem(7000 + b + kc, m, n, k, p)
    ref = oracle.matmul_mod(A, B, p)
    kw = dict(kc=kc) if kc else {}
    C1, plan1 = gpu_product(M, A, B, p, form=form, tc_pair=True, **kw)
    C0, plan0 = gpu_product(M, A, B, p, form=form, tc_pair=False, **kw)
    assert plan1.info["tc_pair"] == 1 and plan0.info["tc_pair"] == 0
    if kc:
        assert plan1.info["nkc"] == -(-k // kc)  # else the planner's fill model picks the ranges
    assert np.array_equal(C1, ref) and np.array_equal(C0, ref)


def test_tc_residency_and_pipe_rate_diagnostics(M):
    """The residency diagnostic: the device's SM count, one resident CTA of
    the word-product kernel per SM, and between one and sms / 2 pair
    clusters; the FP64 rate diagnostic returns a positive rate below the
    nominal 2 flops x 2 DFMA per clock per SM at 2.5 GHz."""
    import torch
    r = M.mwmm_tc_residency()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert r["sms"] == sms and r["ctas"] == sms
    assert 1 <= r["pair_clusters"] <= sms // 2
    g = M.mwmm_measure_fp64_rate(1 << 12)
    assert 0 < g < 4 * sms * 2.5


# ------------------------------------------------------------------ fused recombination (INT8 form)
FUSED_SHAPES = [(129, 129, 65), (257, 300, 777), (700, 520, 1100), (513, 385, 64), (300, 1000, 2000)]


@pytest.mark.parametrize("b", [20, 23, 40, 52])
def test_int8_fused_matches_oracle(M, oracle, b):
    """Word products, reduction and the Horner recombination in one kernel
    (256 x 128 tiles on CTA pairs), on ragged shapes spanning several tiles,
    one or several segments and K parts; equals the oracle and the unfused
    kernels bit for bit."""
    p = SWEEP[b]
    for seed, (m, n, k) in enumerate(FUSED_SHAPES):
        A, B = inputs.problem(900 + 10 * b + seed, m, n, k, p)
        ref = oracle.matmul_mod(A, B, p)
        C, plan = gpu_product(M, A, B, p, form="int8", tc_fused=2)
        d = plan.info
        assert d["tc_fused"] == 1 and d["A_rows"] % 256 == 0 and d["B_rows"] % 128 == 0
        assert np.array_equal(C, ref), (m, n, k, d["ksplit"])
        C1, plan1 = gpu_product(M, A, B, p, form="int8", tc_seg=16, tc_fused=2)  # several segments
        assert plan1.info["tc_fused"] == 1 and np.array_equal(C1, ref), (m, n, k)


@pytest.mark.parametrize("seg,parts", [(1, 1), (3, 1), (16, 1), (2, 3), (5, 2), (1, 7), (64, 4)])
@pytest.mark.parametrize("b", [20, 52])
def test_int8_fused_segments_and_k_parts(M, oracle, b, seg, parts):
    """Segment lengths of 1..64 k-blocks (between segments the residue is
    divided by 2^(8 nsums) mod p) and 1..7 K parts (residue planes added mod
    p by a second kernel), with k not a multiple of 64."""
    p = SWEEP[b]
    m, n, k = 300, 260, 1500
    A, B = inputs.problem(950 + seg + 10 * parts, m, n, k, p)
    C, plan = gpu_product(M, A, B, p, form="int8", tc_fused=2, tc_seg=seg, ksplit=parts)
    d = plan.info
    nkb = d["nkb"]
    assert d["tc_fused"] == 1 and d["tc_seg"] == min(seg, nkb)
    assert d["ksplit"] == -(-nkb // -(-nkb // parts))  # parts of ceil(nkb / parts) k-blocks, none empty
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))


@pytest.mark.parametrize("p", [5, 7, 251, 257, 65521, 65537, (1 << 31) - 1])
def test_int8_fused_small_and_odd_primes(M, oracle, p):
    """Primes with one digit (nsums = 1: every Horner pass is one step, the
    segment hop divides by 2^8) and two or four digits."""
    m, n, k = 260, 200, 1100
    A, B = inputs.problem(p % 1000, m, n, k, p)
    for seg in (16, 3):
        C, plan = gpu_product(M, A, B, p, form="int8", tc_fused=2, tc_seg=seg)
        assert plan.info["tc_fused"] == 1
        assert np.array_equal(C, oracle.matmul_mod(A, B, p)), seg


@pytest.mark.parametrize("b", [26, 48])
def test_int8_fused_narrow_m_and_leading_dimensions(M, oracle, b):
    """tc_fused = 2 fuses m <= 128 too (a 256-row tile with padding); C with
    an odd leading dimension and a C that starts 8 bytes past a 16-byte
    boundary take the single-output stores; entries outside C stay untouched."""
    p = SWEEP[b]
    for m, n, k in ((1, 129, 70), (100, 300, 300), (129, 257, 500)):
        A, B = inputs.problem(960 + m, m, n, k, p)
        ref = oracle.matmul_mod(A, B, p)
        plan = M.Plan(m, n, k, p, form="int8", tc_fused=2)
        assert plan.info["tc_fused"] == 1
        for ldc, off in ((n, 0), (n + 1, 0), (n + 3, 1)):
            buf = torch.full((m * ldc + off + 8,), 7, dtype=torch.int64, device="cuda")
            Cv = buf[off:off + m * ldc].view(m, ldc)[:, :n]
            M.mwmm_matmul(plan.handle, dev(A), dev(B), Cv, stream=None)
            assert plan.check() == 0
            got = buf.cpu().numpy().view(np.uint64)
            body = got[off:off + m * ldc].reshape(m, ldc)
            assert np.array_equal(body[:, :n], ref), (m, n, k, ldc, off)
            assert np.all(body[:, n:] == 7) and np.all(got[:off] == 7) and np.all(got[off + m * ldc:] == 7)


@pytest.mark.parametrize("shape", [(1100, 300, 300), (2048, 260, 1500), (1537, 129, 64)])
def test_int8_fused_host_row_block_pipeline(M, oracle, shape):
    """Host entry point with the fused form: row blocks (sub-plans sharing B's
    words, every block fused, the last one down to one row) on three streams,
    and the one-stream order."""
    m, n, k = shape
    p = SWEEP[52]
    A, B = inputs.problem(990 + m, m, n, k, p)
    ref = oracle.matmul_mod(A, B, p)
    plan = M.Plan(m, n, k, p, form="int8", tc_fused=2)
    assert plan.info["tc_fused"] == 1
    assert np.array_equal(plan.matmul_host(A, B), ref)
    M.mwmm_plan_set_timing(plan.handle, True)  # one-stream path
    assert np.array_equal(plan.matmul_host(A, B), ref)


def test_int8_fused_extreme_digits_and_all_max_entries(M, oracle):
    """Every entry p - 1 (the largest residues) and every entry (p-1)/2 (top
    digit 128), through several segments and K parts at 40 and 52 bits."""
    for b in (40, 52):
        p = SWEEP[b]
        for val in (p - 1, (p - 1) // 2, (p + 1) // 2):
            A = np.full((260, 2100), val, dtype=np.uint64)
            B = np.full((2100, 300), val, dtype=np.uint64)
            for parts in (0, 3):
                C, plan = gpu_product(M, A, B, p, form="int8", tc_fused=2, tc_seg=16, ksplit=parts)
                assert plan.info["tc_fused"] == 1
                assert np.all(C == (val * val * 2100) % p), (b, val, parts)


@pytest.mark.parametrize("n", [1, 15, 16, 17, 32, 40, 64, 65, 100, 128])
@pytest.mark.parametrize("b", [23, 40, 52])
def test_int8_narrow_n_diagonal_windows(M, oracle, n, b):
    """n <= 128: one work item carries 256 / nb diagonals, the B words of a
    window concatenated along N (Alg. 6), zero slices where j is out of range."""
    p = SWEEP[b]
    m, k = 300, 777
    A, B = inputs.problem(70 + n, m, n, k, p)
    C, plan = gpu_product(M, A, B, p, form="int8")
    nb = plan.info["B_rows"]
    assert nb >= n and nb in (16, 32, 64, 128)
    assert np.array_equal(C, oracle.matmul_mod(A, B, p))
    C2, _ = gpu_product(M, A, B, p, form="int8", tc_chunk=128, kc=256)  # chunks and K-ranges inside windows
    assert np.array_equal(C2, C)


def test_int8_windowed_diagonal_sums_match_oracle(M, oracle):
    p = SWEEP[52]
    m, n, k = 130, 40, 500
    A, B = inputs.problem(43, m, n, k, p)
    plan = M.Plan(m, n, k, p, form="int8", kc=192)
    ws = plan.alloc_workspace()
    plan.matmul(dev(A), dev(B))
    assert plan.check() == 0
    d = plan.info
    assert d["B_rows"] == 64
    S = ws[d["S_off"]:d["S_off"] + d["nsums"] * d["nkc"] * d["A_rows"] * d["B_rows"] * 4]
    S = S.cpu().numpy().view(np.int32).reshape(d["nsums"], d["nkc"], d["A_rows"], d["B_rows"])
    u = d["u"]
    Aw = oracle.split_signed(A, p, u, d["tc_digit_bits"])
    Bw = oracle.split_signed(B, p, u, d["tc_digit_bits"])
    for kc in range(d["nkc"]):
        sl = slice(kc * d["kc"], min(k, (kc + 1) * d["kc"]))
        ref = oracle.diag_sums(np.ascontiguousarray(Aw[:, :, sl]), np.ascontiguousarray(Bw[:, sl, :]))
        assert np.array_equal(S[:, kc, :m, :n].astype(np.int64), ref)


@pytest.mark.parametrize("form", ["int8", "fp64"])
def test_reuse_a_words_across_products(M, oracle, form):
    """A decomposed once, then products with new B only (Sec. 4.1's unbalanced
    scenario); each result matches the oracle."""
    p = SWEEP[40]
    m, n, k = 300, 32, 2000
    A, B1 = inputs.problem(81, m, n, k, p)
    plan = M.Plan(m, n, k, p, form=form)
    dA = dev(A)
    C1 = plan.matmul(dA, dev(B1))
    assert plan.check() == 0
    assert np.array_equal(host(C1), oracle.matmul_mod(A, B1, p))
    for t in range(3):
        _, B2 = inputs.problem(82 + t, m, n, k, p)
        C2 = plan.matmul_reuse_a(dev(B2))
        assert plan.check() == 0
        assert np.array_equal(host(C2), oracle.matmul_mod(A, B2, p))


def test_concurrent_plans_on_separate_streams(M, oracle):
    """Plans of every form, each with its own workspace, launched together on
    separate streams (their kernels overlap on the device): every result
    equals the oracle, and rerunning them one at a time gives the same bits."""
    cases = [(300, 260, 700, 52, "int8"), (257, 300, 513, 40, "crt8"), (190, 70, 1000, 26, "int8"),
             (128, 129, 300, 32, "fp64"), (400, 64, 260, 48, "crt8"), (333, 111, 222, 20, "fp64")]
    plans, data, outs = [], [], []
    for i, (m, n, k, b, form) in enumerate(cases):
        p = inputs.largest_prime_below_pow2(b)
        A, B = inputs.problem(7700 + i, m, n, k, p)
        plans.append(M.Plan(m, n, k, p, form=form))
        data.append((A, B, p, dev(A), dev(B)))
        outs.append(torch.full((m, n), -1, dtype=torch.int64, device="cuda"))
    streams = [torch.cuda.Stream() for _ in cases]
    torch.cuda.synchronize()
    for rep in range(3):
        for pl, (_, _, _, dA, dB), C, st in zip(plans, data, outs, streams):
            pl.matmul(dA, dB, C, stream=st)
    torch.cuda.synchronize()
    for pl, (A, B, p, dA, dB), C in zip(plans, data, outs):
        assert pl.check() == 0
        assert np.array_equal(host(C), oracle.matmul_mod(A, B, p))
        assert torch.equal(pl.matmul(dA, dB), C)


_THREADS_SCRIPT = r'''
import sys, threading
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2601_07508_b300 import inputs, mwmm
out = sys.argv[2]
mwmm.lib()
cases = [(300, 260, 700, 52, "int8", False), (257, 300, 513, 40, "crt8", False), (400, 300, 500, 48, "int8", True),
         (128, 129, 300, 32, "fp64", False)]
go = threading.Barrier(len(cases))
errors = []

def run(i):
    try:
        m, n, k, b, form, pair = cases[i]
        p = inputs.largest_prime_below_pow2(b)
        A, B = inputs.problem(7800 + i, m, n, k, p)
        dA = torch.from_numpy(A.view(np.int64)).cuda()
        dB = torch.from_numpy(B.view(np.int64)).cuda()
        st = torch.cuda.Stream()
        plan = mwmm.Plan(m, n, k, p, form=form, tc_pair=pair)
        go.wait()  # the first launches (and the launchers' cache fills) start together
        with torch.cuda.stream(st):
            C = plan.matmul(dA, dB, stream=st)
            for _ in range(3):
                plan.matmul(dA, dB, C, stream=st)
        assert plan.check(st) == 0
        np.save("%s/c%d.npy" % (out, i), C.cpu().numpy().view(np.uint64))
    except Exception as e:  # reported by the parent
        errors.append(repr(e))

th = [threading.Thread(target=run, args=(i,)) for i in range(len(cases))]
for t in th: t.start()
for t in th: t.join()
if errors:
    print(errors); sys.exit(1)
'''


def test_plans_on_host_threads_launching_together_in_a_fresh_process(M, oracle, tmp_path):
    """Four host threads, each with its own plan (one-CTA and pair tcgen05
    kernels, CRT, FP64) and stream, make their first calls at the same
    moment in a fresh process, so the launchers' host-side caches (kernel
    attributes, SM and cluster counts) are filled concurrently; every result
    equals the oracle."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _THREADS_SCRIPT, root, str(tmp_path)], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    cases = [(300, 260, 700, 52), (257, 300, 513, 40), (400, 300, 500, 48), (128, 129, 300, 32)]
    for i, (m, n, k, b) in enumerate(cases):
        p = inputs.largest_prime_below_pow2(b)
        A, B = inputs.problem(7800 + i, m, n, k, p)
        assert np.array_equal(np.load(tmp_path / ("c%d.npy" % i)), oracle.matmul_mod(A, B, p)), i


@pytest.mark.parametrize("form,b,pair", [("int8", 20, False), ("int8", 52, False), ("crt8", 40, False),
                                         ("int8", 20, True)])
def test_ragged_last_column_tile_widths(M, oracle, form, b, pair):
    """The one-CTA kernel runs a last column tile of c < 256 valid columns
    at N = c rounded up to 16 (MMA width and B rows copied), alone and as a
    batch's table item; c on both sides of each multiple of 16.  The pair
    kernel keeps full 256-wide tiles; it runs the same shapes."""
    p = SWEEP[b]
    m, k = 150, 200
    items, refs = [], []
    for i, c in enumerate((1, 15, 16, 17, 112, 127, 129, 241, 255)):
        n = 256 + c
        A, B = inputs.problem(1700 + 10 * b + i, m, n, k, p)
        ref = oracle.matmul_mod(A, B, p)
        C, plan = gpu_product(M, A, B, p, form=form, tc_pair=pair)
        assert plan.info["tc_pair"] == (1 if pair else 0)
        assert np.array_equal(C, ref), (form, b, n)
        if not pair:
            items.append((dev(A), dev(B), torch.full((m, n), -1, dtype=torch.int64, device="cuda"), p))
            refs.append(ref)
    if items:
        bt = M.Batch(items, form=form)
        bt.run()
        assert bt.check() == 0
        for (_, _, C, _), ref in zip(items, refs):
            assert np.array_equal(host(C), ref), (form, b, C.shape)
