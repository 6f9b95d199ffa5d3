"""randutv_small_svd_noalloc: the small-block SVD for callers that may not
allocate device memory (its scratch is a fixed array inside the library).
Called through the C ABI and checked against randutv_small_svd on two calls
in a row; this file is collected last."""
import ctypes
import numpy as np
import pytest
import synth
from gpu_util import require_gpu, dev, host

pytestmark = pytest.mark.gpu


def _call(lib, name, M, max_sweeps=30):
    import torch
    p = M.shape[0]
    Mst = dev(M).t().contiguous()            # column-major storage
    Us = torch.empty((p, p), dtype=torch.float64, device="cuda")
    Vs = torch.empty((p, p), dtype=torch.float64, device="cuda")
    d = torch.empty(p, dtype=torch.float64, device="cuda")
    lib.randutv_set_stream(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    st = getattr(lib, name)(p, Mst.data_ptr(), p, Us.data_ptr(), d.data_ptr(), Vs.data_ptr(), max_sweeps)
    torch.cuda.synchronize()
    return st, host(Us.t()), host(d), host(Vs.t())


def test_noalloc_matches_allocating_entry_point_twice():
    require_gpu()
    from paper_1703_00998_gb300 import native
    lib = native.lib()
    # upper triangular blocks, like the R11 factors the factorization passes
    mats = [np.linalg.qr(synth.make_matrix("exp50", 128, 128, 21))[1],
            np.linalg.qr(synth.make_matrix("exp5", 200, 200, 22))[1]]
    for M in mats:                               # two calls in a row
        st0, U0, d0, V0 = _call(lib, "randutv_small_svd", M)
        st1, U1, d1, V1 = _call(lib, "randutv_small_svd_noalloc", M)
        assert st0 == native.OK and st1 == native.OK
        p = M.shape[0]
        np.testing.assert_allclose(d1, d0, rtol=1e-13, atol=1e-15 * d0[0])
        np.testing.assert_allclose(U1, U0, atol=1e-12)
        np.testing.assert_allclose(V1, V0, atol=1e-12)
        np.testing.assert_allclose(U1 @ np.diag(d1) @ V1.T, M, atol=1e-14 * p * d0[0])


def test_noalloc_rejects_blocks_above_its_limit():
    require_gpu()
    from paper_1703_00998_gb300 import native
    lib = native.lib()
    st, _, _, _ = _call(lib, "randutv_small_svd_noalloc", np.eye(257))
    assert st == native.EUNSUPPORTED
    assert b"256" in lib.randutv_last_error()
