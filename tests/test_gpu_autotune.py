"""Autotuned plans and batches: whatever configuration the timing picks, the
product equals the oracle's; the cache answers repeated requests."""
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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()


@pytest.mark.parametrize("form,b,shape", [("int8", 52, (700, 520, 1100)), ("fp64", 40, (300, 40, 2000)),
                                          ("auto", 26, (256, 256, 256)), ("fp64", 32, (513, 300, 129)),
                                          ("auto", 52, (1024, 768, 1024))])
def test_autotuned_plan_matches_oracle_and_caches(M, oracle, form, b, shape):
    m, n, k = shape
    p = inputs.largest_prime_below_pow2(b)
    A, B = inputs.problem(800 + b, m, n, k, p)
    dA, dB = dev(A), dev(B)
    M.mwmm_autotune_cache_clear()
    plan = M.Plan.autotuned(m, n, k, p, form, dA, dB)
    d = plan.info
    assert d["tuned_tried"] >= 1 and d["tuned_ms"] > 0
    if form != "auto":
        assert d["form"] == {"int8": 2, "fp64": 1}[form]
    else:
        assert d["form"] in (1, 2, 3)  # FP64, INT8-word or CRT form, whichever timed fastest
    C = plan.matmul(dA, dB)
    assert plan.check() == 0
    assert np.array_equal(C.cpu().numpy().view(np.uint64), oracle.matmul_mod(A, B, p))
    assert M.mwmm_autotune_cache_entries() == 1
    again = M.Plan.autotuned(m, n, k, p, form)  # same bucket: answered by the cache
    assert again.info["tuned_tried"] == 0 and again.info["u"] == d["u"] and again.info["form"] == d["form"]


def test_autotune_cache_file_from_environment(M, oracle, tmp_path, monkeypatch):
    p = inputs.largest_prime_below_pow2(48)
    path = tmp_path / "tune.jsonl"
    M.mwmm_autotune_cache_clear()
    plan = M.Plan.autotuned(640, 640, 640, p, "int8")
    M.mwmm_autotune_cache_save(str(path))
    assert path.read_text().count("\n") == 1
    M.mwmm_autotune_cache_clear()
    M.mwmm_autotune_cache_load(str(path))
    again = M.Plan.autotuned(640, 640, 640, p, "int8")
    assert again.info["tuned_tried"] == 0 and again.info["tc_pair"] == plan.info["tc_pair"]
    M.mwmm_autotune_cache_clear()


@pytest.mark.parametrize("form", ["int8", "fp64", "crt8", "auto"])
def test_autotuned_batch_matches_oracle(M, oracle, form):
    rng = np.random.default_rng(9)
    items, refs, forms = [], [], set()
    for i in range(12):
        b = (40, 50, 26)[i % 3]
        p = inputs.largest_prime_below_pow2(b) if i % 2 else inputs.prev_prime(inputs.largest_prime_below_pow2(b))
        m, n, k = (int(x) for x in rng.integers(60, 400, size=3))
        if form == "auto" and i < 3:  # large enough for the CRT form
            m, n, k = 1100, 1000, 1200
        A, B = inputs.problem(900 + i, m, n, k, p)
        items.append((dev(A), dev(B), torch.empty((m, n), dtype=torch.int64, device="cuda"), p))
        refs.append(oracle.matmul_mod(A, B, p))
        forms.add((b, M.mwmm_tensor_form(m, n, k, p) if form == "auto" else form))
    M.mwmm_autotune_cache_clear()
    batch = M.Batch(items, form=form, autotune=True)
    assert batch.info["tuned_groups"] == len(forms)  # one per (bitsize, form)
    if form == "auto":
        assert {f for _, f in forms} == {"int8", "crt8"}
    batch.run()
    assert batch.check() == 0
    for (_, _, C, _), ref in zip(items, refs):
        assert np.array_equal(C.cpu().numpy().view(np.uint64), ref)
    M.mwmm_autotune_cache_clear()
