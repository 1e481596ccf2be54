"""Parity at the configured full sizes, in the launch configuration bench.py
times: the 4096^3 bitsize sweep (all three forms), the three 50-bit shapes
and the serving workload's request mix.  The oracle
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
    Cc = M.Plan(n, n, n, p, form="crt8").matmul(dA, dB)
    torch.cuda.synchronize()
    assert torch.equal(Ci, Cf) and torch.equal(Ci, Cc)
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


def test_serve_request_mix_full_size(M, oracle):
    """The first 256 requests of the serving workload (m, n, k log-uniform in
    [64, 4096], bitsize uniform in [20, 52], seed 5) through the serving loop
    as bench.py runs it (40 GB budget, 3 streams, <= 64 requests per batch,
    form per request): every result passes Freivalds' test, with sampled
    entries exact, and both tensor forms occur."""
    spec = inputs.serve_requests(count=256)
    forms = {M.mwmm_tensor_form(m, n, k, p) for (m, n, k, p) in spec}
    assert forms == {"int8", "crt8"}
    host, dev = [], []
    for i, (m, n, k, p) in enumerate(spec):
        A, B = inputs.problem(5000 + i, m, n, k, p)
        host.append((A, B, p))
        dev.append((_dev(A), _dev(B), torch.full((m, n), -1, dtype=torch.int64, device="cuda"), p))
    torch.cuda.synchronize()
    srv = M.Server(40 << 30, max_inflight=3, max_batch=64)
    tickets = []
    for d in dev:
        st, t = srv.submit(*d)
        assert st == 0
        tickets.append(t)
    for t in tickets:
        assert srv.wait(t, 300000) == 0
    assert srv.stats()["completed"] == len(spec)
    srv.close()
    for i, ((A, B, p), (_, _, C, _)) in enumerate(zip(host, dev)):
        Ch = C.cpu().numpy().view(np.uint64)
        x = inputs.uniform_mod(5, 7000 + i, B.shape[1], p)
        assert oracle.freivalds(A, B, Ch, p, x) == 0, i
        r = np.array([0, A.shape[0] - 1, A.shape[0] // 2], dtype=np.int64)
        c = np.array([B.shape[1] - 1, 0, B.shape[1] // 3], dtype=np.int64)
        assert np.array_equal(Ch[r, c], oracle.matmul_entries(A, B, p, r, c)), i
