"""Batched products (one CUDA-graph replay for many problems of different
shapes and primes): bit-exact against the oracle and identical to the same
products computed one at a time."""
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


def _mixed_problems(seed, count, lo, hi, bits_lo=20, bits_hi=52):
    dims = inputs.loguniform_dims(seed, inputs.STREAM_SHAPES, 3 * count, lo, hi).reshape(count, 3)
    bits = inputs.draws(seed, 77, np.arange(count, dtype=np.uint64)) % np.uint64(bits_hi - bits_lo + 1)
    out = []
    for i in range(count):
        b = int(bits[i]) + bits_lo
        p = inputs.random_prime_of_bitsize(seed, 78, i, b)
        m, n, k = (int(x) for x in dims[i])
        A, B = inputs.problem(seed * 1000 + i, m, n, k, p)
        out.append((A, B, p))
    return out


@pytest.mark.parametrize("form", ["int8", "fp64", "crt8", "auto"])
def test_batch_of_mixed_shapes_and_primes(M, oracle, form):
    probs = _mixed_problems(3, 24, 1, 300)
    items = [(_dev(A), _dev(B), torch.full((A.shape[0], B.shape[1]), -1, dtype=torch.int64, device="cuda"), p)
             for A, B, p in probs]
    batch = M.Batch(items, form=form)
    batch.run()
    assert batch.check() == 0
    for (A, B, p), (_, _, C, _) in zip(probs, items):
        assert np.array_equal(C.cpu().numpy().view(np.uint64), oracle.matmul_mod(A, B, p))


def test_auto_batch_mixes_int8_and_crt_problems(M, oracle):
    """Under "auto" every problem gets its tensor form from the planner's
    cost model; INT8 and CRT problems share the word-product launch and each
    form's recombination runs after it (4 launches).  Every C equals the
    oracle and the same product planned alone in that form."""
    shapes = [(1024, 1024, 1024, 52), (1100, 900, 1000, 48), (300, 200, 500, 52), (130, 70, 1500, 40),
              (1024, 1100, 900, 50), (64, 300, 64, 23)]
    probs = []
    for i, (m, n, k, b) in enumerate(shapes):
        p = inputs.random_prime_of_bitsize(21, 78, i, b)
        A, B = inputs.problem(2100 + i, m, n, k, p)
        probs.append((A, B, p))
    want = [M.mwmm_tensor_form(A.shape[0], B.shape[1], A.shape[1], p) for A, B, p in probs]
    assert "crt8" in want and "int8" in want
    items = [(_dev(A), _dev(B), torch.full((A.shape[0], B.shape[1]), -1, dtype=torch.int64, device="cuda"), p)
             for A, B, p in probs]
    batch = M.Batch(items, form="auto")
    assert batch.info["launches"] == 4
    got = [{2: "int8", 3: "crt8"}[batch.problem_info(i)["form"]] for i in range(len(items))]
    assert got == want
    batch.run()
    assert batch.check() == 0
    for (A, B, p), (dA, dB, C, _), f in zip(probs, items, want):
        Ch = C.cpu().numpy().view(np.uint64)
        if A.shape[0] * B.shape[1] * A.shape[1] <= 1 << 27:
            assert np.array_equal(Ch, oracle.matmul_mod(A, B, p))
        else:  # large: Freivalds over the whole result plus sampled entries
            x = inputs.uniform_mod(21, 7, B.shape[1], p)
            assert oracle.freivalds(A, B, Ch, p, x) == 0
            r = np.arange(0, A.shape[0], 37, dtype=np.int64)
            c = (r * 13) % B.shape[1]
            assert np.array_equal(Ch[r, c], oracle.matmul_entries(A, B, p, r, c))
        alone = M.Plan(A.shape[0], B.shape[1], A.shape[1], p, form=f).matmul(dA, dB)
        assert torch.equal(C, alone)


def test_batch_equals_products_alone_and_reruns_on_new_inputs(M, oracle):
    probs = _mixed_problems(5, 16, 50, 600)
    items = [(_dev(A), _dev(B), torch.empty((A.shape[0], B.shape[1]), dtype=torch.int64, device="cuda"), p)
             for A, B, p in probs]
    batch = M.Batch(items, form="int8")
    info = batch.info
    assert info["count"] == 16 and info["launches"] == 3 and info["ctas"] >= 1
    batch.run()
    assert batch.check() == 0
    for (A, B, p), (dA, dB, C, _) in zip(probs, items):
        alone = M.Plan(A.shape[0], B.shape[1], A.shape[1], p, form="int8").matmul(dA, dB)
        assert torch.equal(C, alone)
    # new contents in the bound A, B: the replay recomputes from them
    for i, (A, B, p) in enumerate(probs):
        A2, B2 = inputs.problem(900 + i, A.shape[0], B.shape[1], A.shape[1], p)
        items[i][0].copy_(_dev(A2))
        items[i][1].copy_(_dev(B2))
        probs[i] = (A2, B2, p)
    batch.run()
    assert batch.check() == 0
    for (A, B, p), (_, _, C, _) in zip(probs, items):
        assert np.array_equal(C.cpu().numpy().view(np.uint64), oracle.matmul_mod(A, B, p))


def test_batch_one_call_entry_point(M, oracle):
    probs = _mixed_problems(9, 6, 10, 200)
    items = [(_dev(A), _dev(B), torch.empty((A.shape[0], B.shape[1]), dtype=torch.int64, device="cuda"), p)
             for A, B, p in probs]
    M.mwmm_matmul_batched(items, form="int8")
    for (A, B, p), (_, _, C, _) in zip(probs, items):
        assert np.array_equal(C.cpu().numpy().view(np.uint64), oracle.matmul_mod(A, B, p))


def test_multi_prime_batch_512_instances(M, oracle):
    """512 instances over the 64 largest primes below 2^50, m, n, k
    log-uniform in [128, 2048], seed 4; each checked by Freivalds' test and
    sampled entries; the FP64-form batch gives the same results."""
    spec = inputs.batch_instances()
    items, host = [], []
    for i, (m, n, k, p) in enumerate(spec):
        A, B = inputs.problem(4000 + i, m, n, k, p)
        host.append((A, B, p))
        items.append((_dev(A), _dev(B), torch.empty((m, n), dtype=torch.int64, device="cuda"), p))
    batch = M.Batch(items, form="int8")
    batch.run()
    assert batch.check() == 0
    rng = np.random.default_rng(4)
    for i, ((A, B, p), (_, _, C, _)) in enumerate(zip(host, items)):
        Ch = C.cpu().numpy().view(np.uint64)
        x = inputs.uniform_mod(4, 500 + i, B.shape[1], p)
        assert oracle.freivalds(A, B, Ch, p, x) == 0, i
        if i % 16 == 0:
            r = rng.integers(0, A.shape[0], 8).astype(np.int64)
            c = rng.integers(0, B.shape[1], 8).astype(np.int64)
            assert np.array_equal(Ch[r, c], oracle.matmul_entries(A, B, p, r, c))
    ref = [C.clone() for (_, _, C, _) in items]
    fitems = [(dA, dB, torch.empty_like(C), p) for (dA, dB, C, p) in items]
    fb = M.Batch(fitems, form="fp64")
    fb.run()
    assert fb.check() == 0
    for (_, _, C, _), R in zip(fitems, ref):
        assert torch.equal(C, R)


@pytest.mark.parametrize("digit", [255, -255, 181])
def test_batch_9bit_items_chunk_exactly(M, oracle, digit):
    """Table items of 9-bit digits d at 15 of every 16 k positions (0 at the
    16th): every K = 16 MMA adds an odd 15 d^2 (up to 975375) over K of
    1300, so every FP32 chunk must stay within 2^24 (256 products; 512 when
    certified, as for 181 but not 255), else a partial sum above 2^24
    rounds.  Wide and narrow column tiles, next to an 8-bit-digit problem in
    the same batch; every C equals the oracle."""
    probs = []
    for (m, n, k, b) in [(300, 400, 1300, 52), (150, 90, 1300, 26), (200, 300, 1300, 20)]:
        p = inputs.largest_prime_below_pow2(b)
        a = digit % p
        A = np.full((m, k), a, np.uint64)
        A[:, np.arange(k) % 16 == 15] = 0
        probs.append((A, np.full((k, n), a, np.uint64), p))
    items = [(_dev(A), _dev(B), torch.full((A.shape[0], B.shape[1]), -1, dtype=torch.int64, device="cuda"), p)
             for A, B, p in probs]
    batch = M.Batch(items, form="int8")
    batch.run()
    assert batch.check() == 0
    for (A, B, p), (_, _, C, _) in zip(probs, items):
        assert np.array_equal(C.cpu().numpy().view(np.uint64), oracle.matmul_mod(A, B, p))
