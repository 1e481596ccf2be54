"""mwmm_matmul_noalloc: the product for callers that cannot allocate device
memory (scratch in the library's static device array).  Checked through the
C ABI against mwmm_matmul and against the CPU oracle on the same inputs, on
two calls in a row so the second call runs over what the first left in the
shared array.

Kept in its own file, collected last, so a run that stops at the first
failure has already run every other test."""
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


def test_noalloc_matches_matmul_on_two_calls_in_a_row(M, oracle):
    # first a larger problem with a wide prime, then a smaller ragged one with
    # a narrow prime: the second call's words and sums land on the first's.
    cases = [(700, 760, 730, inputs.largest_prime_below_pow2(52), 1),
             (129, 300, 77, inputs.largest_prime_below_pow2(20), 2)]
    for m, n, k, p, seed in cases:
        A, B = inputs.problem(seed, m, n, k, p)
        dA, dB = _dev(A), _dev(B)
        ref = M.Plan(m, n, k, p, form="int8").matmul(dA, dB)
        torch.cuda.synchronize()
        C = torch.full((m, n), -1, dtype=torch.int64, device="cuda")
        st = M.mwmm_matmul_noalloc(dA, dB, C, p)
        assert st == 0, M.mwmm_status_str(st)
        assert torch.equal(C, ref), (m, n, k)
        # and bit for bit against the CPU oracle (a fault the two library
        # paths shared would pass the first comparison)
        got = C.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, oracle.matmul_mod(A, B, p)), (m, n, k)


def test_noalloc_runs_the_fused_form_when_the_sums_do_not_fit(M, oracle):
    # 900 x 1000 x 1100 at 52 bits: words 32 MB and diagonal sums 54 MB exceed
    # the 64 MiB scratch together, the words alone do not; two calls in a row
    p = inputs.largest_prime_below_pow2(52)
    m, n, k = 900, 1000, 1100
    h = M.mwmm_plan(m, n, k, p, 0, 0, "int8")
    assert M.mwmm_workspace_size(h) > 64 << 20
    M.mwmm_plan_destroy(h)
    for seed in (3, 4):
        A, B = inputs.problem(seed, m, n, k, p)
        dA, dB = _dev(A), _dev(B)
        ref = M.Plan(m, n, k, p, form="int8").matmul(dA, dB)
        torch.cuda.synchronize()
        C = torch.full((m, n), -1, dtype=torch.int64, device="cuda")
        st = M.mwmm_matmul_noalloc(dA, dB, C, p)
        assert st == 0, M.mwmm_status_str(st)
        assert torch.equal(C, ref)
        assert np.array_equal(C.cpu().numpy().view(np.uint64), oracle.matmul_mod(A, B, p))


def test_noalloc_rejects_products_larger_than_its_scratch(M):
    p = inputs.largest_prime_below_pow2(52)
    A = torch.zeros((2048, 2048), dtype=torch.int64, device="cuda")
    C = torch.zeros((2048, 2048), dtype=torch.int64, device="cuda")
    st = M.mwmm_matmul_noalloc(A, A, C, p)
    assert st == 6  # MWMM_ERR_BUDGET
