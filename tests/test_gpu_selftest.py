"""The bounded device waits give up and report instead of hanging: a wait
that nothing will end (an mbarrier no thread arrives at, a grid barrier
sized for two CTAs in a launch of one) runs out after a short limit, the
call returns RANDUTV_ETIMEOUT after about that limit, and the CUDA context
stays usable (a factorization right after it is checked against the
oracle).  This is the failure path every wait of the library relies on;
nothing here faults or hangs the GPU."""
import time
import numpy as np
import pytest
import synth
import oracle
from oracle import checks
from gpu_util import require_gpu, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    require_gpu()
    import paper_1703_00998_gb300 as R
    return R


@pytest.mark.parametrize("kind", [0, 1])
def test_wait_times_out_and_context_survives(R, kind):
    from paper_1703_00998_gb300 import native
    lib = native.lib()
    limit = 0.05
    t0 = time.perf_counter()
    st = lib.randutv_selftest_wait(kind, limit)
    dt = time.perf_counter() - t0
    assert st == native.ETIMEOUT, (st, lib.randutv_last_error())
    assert b"timed out" in lib.randutv_last_error()
    assert limit <= dt < 2.0, dt
    # the context still works: a small factorization against the oracle
    m = n = 96
    A = synth.make_matrix("exp50", m, n, 1703001)
    g = synth.gaussian_stream(998, m, n, 32)
    out = R.factor(dev(A), b=32, q=1, g_inject=dev(g))
    U, T, V = host(out.U), host(out.T), host(out.V)
    assert checks.residual(A, U, T, V) <= 1e-13
    _, To, _, _ = oracle.randutv(A, 32, 1, lambda i, k, b: synth.step_gaussian(998, i, k, b))
    d, do = np.abs(np.diag(T)), np.abs(np.diag(To))
    assert np.max(np.abs(d - do) / do) <= 1e-10
