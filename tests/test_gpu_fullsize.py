"""Parity at the configured full sizes, in the launch configuration bench.py
times: the 4096^3 bitsize sweep and the three 50-bit shapes.  The oracle
computes sampled entries exactly and checks the whole result with Freivalds'
test (C x == A (B x) mod p for random x); the two forms are compared entry by
entry on the device."""
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


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()


def _check_with_oracle(oracle, A, B, C, p, seed):
    m, k = A.shape
    n = B.shape[1]
    rng = np.random.default_rng(seed)
    rows = np.concatenate([[0, m - 1, m // 2], rng.integers(0, m, 61)]).astype(np.int64)
    cols = np.concatenate([[0, n - 1, n // 2], rng.integers(0, n, 61)]).astype(np.int64)
    assert np.array_equal(C[rows, cols], oracle.matmul_entries(A, B, p, rows, cols))
    for t in range(2):
        x = inputs.uniform_mod(seed, 900 + t, n, p)
        assert oracle.freivalds(A, B, C, p, x) == 0


def fp64_bound_rule(oracle, p):
    for uv in ((1, 1), (1, 2), (2, 2)):
        if oracle.lam(p, *uv) >= 1:
            return uv


@pytest.mark.parametrize("b", inputs.SWEEP_BITS)
def test_sweep_4096_both_forms(M, oracle, b):
    n = 4096
    p = inputs.largest_prime_below_pow2(b)
    A, B = inputs.problem(b, n, n, n, p)
    dA, dB = _dev(A), _dev(B)
    Ci = M.Plan(n, n, n, p, form="int8").matmul(dA, dB)
    uv = fp64_bound_rule(oracle, p)
    Cf = M.Plan(n, n, n, p, uv[0], uv[1], form="fp64").matmul(dA, dB)
    torch.cuda.synchronize()
    assert torch.equal(Ci, Cf)
    _check_with_oracle(oracle, A, B, Ci.cpu().numpy().view(np.uint64), p, b)


@pytest.mark.parametrize("shape,seed", [((8192, 8192, 512), 1), ((8192, 64, 8192), 2), ((8192, 8192, 8192), 3)])
def test_shapes_50bit_int8_vs_fp64(M, oracle, shape, seed):
    m, n, k = shape
    p = inputs.largest_prime_below_pow2(50)
    A, B = inputs.problem(seed, m, n, k, p)
    dA, dB = _dev(A), _dev(B)
    Ci = M.Plan(m, n, k, p, form="int8").matmul(dA, dB)
    for uv in ((2, 2), (2, 3)):
        Cf = M.Plan(m, n, k, p, uv[0], uv[1], form="fp64").matmul(dA, dB)
        torch.cuda.synchronize()
        assert torch.equal(Ci, Cf), uv
        del Cf
    _check_with_oracle(oracle, A, B, Ci.cpu().numpy().view(np.uint64), p, seed)
