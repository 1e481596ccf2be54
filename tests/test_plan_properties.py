"""Property-based checks of the planner (host logic, no GPU): for random
primes, shapes and variants, every plan satisfies the bounds that make its
products exact, and matches the oracle's independent definitions."""
import pytest
from hypothesis import HealthCheck, given, settings, strategies as st

from paper_2601_07508_b300 import inputs

SETTINGS = settings(max_examples=150, deadline=None, suppress_health_check=[HealthCheck.function_scoped_fixture])


@pytest.fixture(scope="module")
def M():
    from paper_2601_07508_b300 import build
    build.build()
    from paper_2601_07508_b300 import mwmm
    mwmm.lib()
    return mwmm


primes = st.integers(min_value=3, max_value=52).flatmap(
    lambda b: st.integers(min_value=1 << (b - 1), max_value=(1 << b) - 1)).map(
    lambda x: inputs.prev_prime(x + 1) if x > 5 else 5)
dims = st.integers(min_value=1, max_value=5000)
kdims = st.integers(min_value=0, max_value=200000)


@SETTINGS
@given(p=primes, m=dims, n=dims, k=kdims,
       uv=st.sampled_from([(1, 1), (1, 2), (1, 3), (1, 4), (2, 2), (2, 3), (0, 0)]))
def test_fp64_plans_keep_every_chunk_exact(M, oracle, p, m, n, k, uv):
    if p < 5:
        return
    try:
        h = M.mwmm_plan(m, n, k, p, uv[0], uv[1], "fp64")
    except M.MwmmError as e:
        assert e.status == 3 and uv != (0, 0) and oracle.lam(p, *uv) < 1  # only an impossible variant fails
        return
    d = M.mwmm_plan_info(h)
    M.mwmm_plan_destroy(h)
    u, v, lam = d["u"], d["v"], d["lambda"]
    assert lam == oracle.lam(p, u, v) >= 1
    # Prop. 3.3 (Sec. 2.2 for (1,1)): lambda max|A_i| max|B_j| + p - 1 <= 2^53
    amax = p - 1 if u == 1 else d["alpha"]
    bmax = p - 1 if v == 1 else d["beta"]
    assert lam * amax * bmax + p - 1 <= 2 ** 53
    assert d["alpha"] == oracle.ceil_root(p, u) and d["beta"] == oracle.ceil_root(p, v)
    assert 1 <= d["ksplit"] <= 64 and d["workspace_bytes"] >= d["B_off"]
    if d["f64_concat"]:
        assert min(m, n) < 64


@SETTINGS
@given(p=primes, m=dims, n=dims, k=kdims)
def test_int8_plans_keep_fp32_chunks_and_int32_sums_exact(M, oracle, p, m, n, k):
    if p < 5:
        return
    h = M.mwmm_plan(m, n, k, p, 0, 0, "int8")
    d = M.mwmm_plan_info(h)
    M.mwmm_plan_destroy(h)
    u = d["u"]
    bits = d["tc_digit_bits"]
    # 9-bit digits exactly when they save a digit over 8-bit ones
    assert bits == (9 if oracle.digit_words(p, 9) < oracle.digit_words(p, 8) else 8)
    assert d["alpha"] == d["beta"] == 2 ** bits
    assert u == d["v"] == oracle.digit_words(p, bits)
    R, h = 2 ** bits, 2 ** (bits - 1)
    B = R ** (u - 1)  # u - 1 balanced digits, top digit in [-h, h]
    assert h * B + (h - 1) * (B - 1) // (R - 1) >= (p - 1) // 2  # every signed representative is reached
    assert u <= -(-(p.bit_length()) // bits)  # at most ceil(b / bits) digits for a b-bit prime
    if u > 1:  # and the fewest: u - 1 digits miss the largest signed representative
        B //= R
        assert h * B + (h - 1) * (B - 1) // (R - 1) < (p - 1) // 2
    assert d["tc_chunk"] * h * h <= 2 ** 24  # FP32 chunk: every partial sum exact
    assert d["kc"] * min(u, u) * h * h <= 2 ** 31 - 1 or k == 0  # INT32 sum of one K-range
    assert d["nkc"] == (-(-k // d["kc"]) if k else 0)
    assert d["A_rows"] >= m and d["B_rows"] >= n and d["A_rows"] % 128 == 0


@SETTINGS
@given(p=primes, k=st.integers(min_value=0, max_value=1 << 22))
def test_crt_plans_cover_the_integer_product(M, oracle, p, k):
    if p < 5:
        return
    h = M.mwmm_plan(64, 64, k, p, 0, 0, "crt8")
    d = M.mwmm_plan_info(h)
    M.mwmm_plan_destroy(h)
    ms = d["crt_m"][:d["u"]]
    assert ms == oracle.crt_moduli(p, k)
    prod = 1
    for m in ms:
        prod *= m
    assert prod > 2 * max(k, 1) * (p - 1) ** 2
    assert d["kc"] * 127 * 127 < 2 ** 31  # one residue product per INT32 sum
