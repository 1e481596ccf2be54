"""Serving loop (continuous batching): every result equals the same product
computed alone and the oracle's; requests are admitted against the memory
budget; stats report latency percentiles."""
import threading
import time

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


def _requests(seed, count, lo, hi):
    dims = inputs.loguniform_dims(seed, inputs.STREAM_SHAPES, 3 * count, lo, hi).reshape(count, 3)
    bz = inputs.draws(seed, inputs.STREAM_PRIMES, np.arange(count, dtype=np.uint64)) % np.uint64(33)
    out = []
    for i in range(count):
        p = inputs.random_prime_of_bitsize(seed, 104, i, 20 + int(bz[i]))
        m, n, k = (int(x) for x in dims[i])
        A, B = inputs.problem(seed * 10000 + i, m, n, k, p)
        out.append((A, B, p))
    return out


@pytest.mark.parametrize("form", ["auto", "crt8", "int8", "fp64"])
def test_serve_results_equal_alone_and_oracle(M, oracle, form):
    reqs = _requests(21, 120, 8, 400)
    dev = [(_dev(A), _dev(B), torch.full((A.shape[0], B.shape[1]), -1, dtype=torch.int64, device="cuda"), p)
           for A, B, p in reqs]
    torch.cuda.synchronize()
    srv = M.Server(2 << 30, max_inflight=2, max_batch=16, form=form)
    tickets = []
    for dA, dB, C, p in dev:  # a burst: later requests arrive while earlier batches run
        st, t = srv.submit(dA, dB, C, p)
        assert st == 0
        tickets.append(t)
    for t in tickets:
        assert srv.wait(t, 60000) == 0
    s = srv.stats()
    assert s["completed"] == 120 and s["status"] == 0
    assert s["batches"] >= 120 // 16 and s["mean_batch"] > 1.0
    assert s["peak_inflight"] >= 1 and 0 < s["p50_ms"] <= s["p99_ms"] <= s["max_ms"]
    srv.close()
    for (A, B, p), (dA, dB, C, _) in zip(reqs, dev):
        alone = M.Plan(A.shape[0], B.shape[1], A.shape[1], p, form="int8").matmul(dA, dB)
        assert torch.equal(C, alone)  # the result is unique: any form alone gives it
        assert np.array_equal(C.cpu().numpy().view(np.uint64), oracle.matmul_mod(A, B, p))


def test_serve_auto_form_mixes_int8_and_crt(M, oracle):
    """Under "auto" each request takes the planner's tensor form; large
    high-bitsize requests run as CRT, the others as INT8, in shared batches."""
    specs = [(900, 800, 1000, 52), (64, 64, 64, 30), (1000, 1000, 700, 48), (200, 300, 100, 21), (700, 900, 1024, 50),
             (128, 128, 2048, 26)]
    reqs = []
    for i, (m, n, k, b) in enumerate(specs):
        p = inputs.random_prime_of_bitsize(23, 104, i, b)
        A, B = inputs.problem(2300 + i, m, n, k, p)
        reqs.append((A, B, p))
    forms = [M.mwmm_tensor_form(A.shape[0], B.shape[1], A.shape[1], p) for A, B, p in reqs]
    assert "crt8" in forms and "int8" in forms
    dev = [(_dev(A), _dev(B), torch.full((A.shape[0], B.shape[1]), -1, dtype=torch.int64, device="cuda"), p)
           for A, B, p in reqs]
    torch.cuda.synchronize()
    srv = M.Server(4 << 30, max_inflight=2, max_batch=8)
    tickets = []
    for d in dev:
        st, t = srv.submit(*d)
        assert st == 0
        tickets.append(t)
    for t in tickets:
        assert srv.wait(t, 60000) == 0
    assert srv.stats()["completed"] == len(reqs)
    srv.close()
    for (A, B, p), (dA, dB, C, _), f in zip(reqs, dev, forms):
        alone = M.Plan(A.shape[0], B.shape[1], A.shape[1], p, form=f).matmul(dA, dB)
        assert torch.equal(C, alone)
        Ch = C.cpu().numpy().view(np.uint64)
        x = inputs.uniform_mod(23, 9, B.shape[1], p)
        assert oracle.freivalds(A, B, Ch, p, x) == 0
        r = np.arange(0, A.shape[0], 29, dtype=np.int64)
        c = (r * 7) % B.shape[1]
        assert np.array_equal(Ch[r, c], oracle.matmul_entries(A, B, p, r, c))


@pytest.mark.parametrize("form", ["int8", "crt8"])
def test_serve_batch_holds_table_and_direct_requests(M, oracle, form):
    """Requests of at most 32 tcgen05 work items go through the batched
    tables, larger ones through the single-product kernels of a plan.  The
    shapes straddle that line with work within 4x of each other, so a burst
    puts both kinds in one batch; every result equals the oracle's."""
    shapes = [(64, 64, 64), (128, 256, 1000), (256, 256, 512), (256, 512, 512), (200, 300, 600), (512, 768, 1024)]
    reqs = []
    for i in range(2 * len(shapes)):
        m, n, k = shapes[i % len(shapes)]
        p = inputs.random_prime_of_bitsize(31, 104, i, 52 - (i % 3))
        A, B = inputs.problem(3100 + i, m, n, k, p)
        reqs.append((A, B, p))
    dev = [(_dev(A), _dev(B), torch.full((A.shape[0], B.shape[1]), -1, dtype=torch.int64, device="cuda"), p)
           for A, B, p in reqs]
    torch.cuda.synchronize()
    items = [M.Batch([d], form=form).info["items"] for d in dev]
    table = [(A.shape[0] * B.shape[1] * A.shape[1], it) for (A, B, _), it in zip(reqs, items)]
    assert min(items) <= 32 < max(items)
    assert any(w1 <= w2 <= 4 * w1 for w1, i1 in table if i1 <= 32 for w2, i2 in table if i2 > 32)
    srv = M.Server(4 << 30, max_inflight=2, max_batch=16, form=form)
    tickets = []
    for d in dev:
        st, t = srv.submit(*d)
        assert st == 0
        tickets.append(t)
    for t in tickets:
        assert srv.wait(t, 60000) == 0
    s = srv.stats()
    assert s["completed"] == len(reqs) and s["status"] == 0 and s["mean_batch"] > 1.0
    srv.close()
    for (A, B, p), (_, _, C, _) in zip(reqs, dev):
        assert np.array_equal(C.cpu().numpy().view(np.uint64), oracle.matmul_mod(A, B, p))


def test_serve_poisson_stream_from_two_client_threads(M, oracle):
    reqs = _requests(22, 80, 16, 300)
    dev = [(_dev(A), _dev(B), torch.empty((A.shape[0], B.shape[1]), dtype=torch.int64, device="cuda"), p)
           for A, B, p in reqs]
    torch.cuda.synchronize()
    srv = M.Server(1 << 30, max_inflight=3, max_batch=8)
    arrivals = inputs.poisson_arrivals(22, len(reqs), 2000.0)
    tickets = [0] * len(reqs)
    t0 = srv.now()

    def client(idx):
        for i in idx:
            while srv.now() - t0 < arrivals[i]:
                time.sleep(0.0001)
            st, tk = srv.submit(*dev[i], t_arrival=t0 + arrivals[i])
            assert st == 0
            tickets[i] = tk

    th = [threading.Thread(target=client, args=(range(j, len(reqs), 2),)) for j in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for tk in tickets:
        assert srv.wait(tk, 60000) == 0
        assert srv.latency(tk) >= 0
    s = srv.stats()
    assert s["completed"] == len(reqs)
    srv.close()
    for (A, B, p), (_, _, C, _) in zip(reqs, dev):
        assert np.array_equal(C.cpu().numpy().view(np.uint64), oracle.matmul_mod(A, B, p))


def test_serve_admission_against_budget(M, oracle):
    p = inputs.largest_prime_below_pow2(52)
    # each 700^3 52-bit request needs ~47 MB of workspace in the INT8 form;
    # the arena holds one at a time
    budget = 2 * (32 << 20) + (60 << 20)
    srv = M.Server(budget, max_inflight=2, max_batch=4, form="int8")
    reqs = [inputs.problem(300 + i, 700, 700, 700, p) for i in range(5)]
    dev = [(_dev(A), _dev(B), torch.empty((700, 700), dtype=torch.int64, device="cuda")) for A, B in reqs]
    tickets = []
    for dA, dB, C in dev:
        st, t = srv.submit(dA, dB, C, p)
        assert st == 0
        tickets.append(t)
    # a request whose workspace can never fit is rejected at once
    big = torch.zeros((3000, 3000), dtype=torch.int64, device="cuda")
    st, _ = srv.submit(big, big, big, p)
    assert st == 6  # MWMM_ERR_BUDGET
    for t in tickets:
        assert srv.wait(t, 60000) == 0
    s = srv.stats()
    assert s["completed"] == 5 and s["rejected"] == 1
    assert s["peak_bytes"] <= budget - 2 * (32 << 20)
    assert s["mean_batch"] == 1.0  # memory admits one request at a time
    srv.close()
    for (A, B), (_, _, C) in zip(reqs, dev):
        assert np.array_equal(C.cpu().numpy().view(np.uint64), oracle.matmul_mod(A, B, p))


def test_serve_9bit_table_requests_chunk_exactly(M, oracle):
    """Small requests (batched table items) of 9-bit digits 255 at 15 of
    every 16 k positions against -255: every K = 16 MMA adds an odd
    -15 x 65025, so over K of 1300 each FP32 chunk is exact only at 256
    products; every result equals the oracle."""
    reqs = []
    for (m, n, k, b) in [(100, 300, 1300, 52), (150, 90, 1300, 26), (120, 260, 1300, 35)]:
        p = inputs.largest_prime_below_pow2(b)
        A = np.full((m, k), 255, np.uint64)
        A[:, np.arange(k) % 16 == 15] = 0
        reqs.append((A, np.full((k, n), p - 255, np.uint64), p))
    dev = [(_dev(A), _dev(B), torch.full((A.shape[0], B.shape[1]), -1, dtype=torch.int64, device="cuda"), p)
           for A, B, p in reqs]
    torch.cuda.synchronize()
    srv = M.Server(2 << 30, max_inflight=2, max_batch=16, form="int8")
    tickets = []
    for dA, dB, C, p in dev:
        st, t = srv.submit(dA, dB, C, p)
        assert st == 0
        tickets.append(t)
    for t in tickets:
        assert srv.wait(t, 60000) == 0
    srv.close()
    for (A, B, p), (_, _, C, _) in zip(reqs, dev):
        assert np.array_equal(C.cpu().numpy().view(np.uint64), oracle.matmul_mod(A, B, p))
