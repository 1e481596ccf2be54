"""Failure detection on the device without a fault: every barrier wait of the
product kernels is bounded, gives up by raising an error flag, and leaves the
context usable.  The wait is made to run out on a barrier that nothing
completes (a one-thread self-test kernel); no test traps, faults or hangs."""
import time

import numpy as np
import pytest

from paper_2601_07508_b300 import build, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TIMEOUT = 8  # MWMM_ERR_TIMEOUT


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_2601_07508_b300 import mwmm
    mwmm.lib()
    return mwmm


def _small_product(M, oracle, seed):
    p = inputs.largest_prime_below_pow2(40)
    A, B = inputs.problem(seed, 100, 70, 300, p)
    plan = M.Plan(100, 70, 300, p, form="int8")
    C = plan.matmul(torch.from_numpy(A.view(np.int64)).cuda(), torch.from_numpy(B.view(np.int64)).cuda())
    assert plan.check() == 0
    assert np.array_equal(C.cpu().numpy().view(np.uint64), oracle.matmul_mod(A, B, p))


@pytest.mark.parametrize("cycles", [1, 1 << 20, 20_000_000])
def test_bounded_wait_times_out_and_context_survives(M, oracle, cycles):
    t0 = time.perf_counter()
    assert M.mwmm_selftest_wait_timeout(cycles) == TIMEOUT
    assert time.perf_counter() - t0 < 10.0  # 2e7 cycles is ~10 ms at B300 clocks
    _small_product(M, oracle, 900 + cycles % 97)  # the context still runs kernels correctly
    stream = torch.cuda.Stream()
    assert M.mwmm_selftest_wait_timeout(cycles, stream) == TIMEOUT  # on a side stream too
    _small_product(M, oracle, 901)


def test_timeout_does_not_leak_into_plans(M, oracle):
    """A timed-out self-test raises its own flag only: a plan's status stays OK."""
    assert M.mwmm_selftest_wait_timeout(1 << 16) == TIMEOUT
    _small_product(M, oracle, 902)
