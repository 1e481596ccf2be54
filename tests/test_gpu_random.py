"""Seeded randomized parity sweep: random forms, primes, shapes and plan
options, each product equal to the oracle's bit for bit."""
import numpy as np
import pytest

from paper_2601_07508_b300 import build, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_2601_07508_b300 import mwmm
    mwmm.lib()
    return mwmm


def _case(rng, oracle):
    b = int(rng.integers(4, 53))
    lo = max(5, 1 << (b - 1))
    p = inputs.prev_prime(int(rng.integers(lo, (1 << b))) + 1)
    if p < 5:
        p = 5
    m, n = (int(x) for x in rng.integers(1, 600, size=2))
    k = int(rng.integers(0, 3000))
    form = ["int8", "fp64", "crt8"][int(rng.integers(0, 3))]
    kw = {}
    if form == "fp64":
        ok = [uv for uv in [(1, 1), (1, 2), (1, 3), (1, 4), (2, 2), (2, 3)] if oracle.lam(p, *uv) >= 1]
        u, v = ok[int(rng.integers(0, len(ok)))]
        kw = dict(u=u, v=v, lam=int(rng.integers(1, oracle.lam(p, u, v) + 1)) if rng.random() < 0.3 else 0,
                  f64_concat=int(rng.integers(0, 2)), ksplit=int(rng.integers(0, 5)))
        kw["lam"] = min(kw["lam"], 10 ** 6)
    else:
        nine = False
        if form == "int8":
            bits = [0, 8, 9][int(rng.integers(0, 3))]
            kw["tc_digit_bits"] = bits
            nine = bits == 9 or (bits == 0 and oracle.digit_words(p, 9) < oracle.digit_words(p, 8))
        if rng.random() < 0.3:
            kw["kc"] = 64 * int(rng.integers(1, 8))
        if rng.random() < 0.3:
            kw["tc_chunk"] = 64 * int(rng.integers(1, 5 if nine else 17))  # FP32 chunk limit 256 / 1024
        if rng.random() < 0.25:
            kw["tc_pair"] = True
        if form == "int8" and rng.random() < 0.2:
            kw["tc_fused"] = 2
    return b, p, m, n, k, form, kw


@pytest.mark.parametrize("case", range(64))
def test_random_products_match_oracle(M, oracle, case):
    rng = np.random.default_rng(1000 + case)
    b, p, m, n, k, form, kw = _case(rng, oracle)
    A, B = inputs.problem(7000 + case, m, n, k, p)
    plan = M.Plan(m, n, k, p, form=form, **kw)
    C = plan.matmul(torch.from_numpy(A.view(np.int64)).cuda(), torch.from_numpy(B.view(np.int64)).cuda())
    assert plan.check() == 0
    got = C.cpu().numpy().view(np.uint64)
    assert np.array_equal(got, oracle.matmul_mod(A, B, p)), (b, p, m, n, k, form, kw)
