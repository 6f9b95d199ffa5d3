"""randutv_small_svd_noalloc: the small-block SVD for callers that may not
allocate device memory (its scratch is a fixed array inside the library).
Called through the C ABI and checked against randutv_small_svd on two calls
in a row, the second also for the absence of any device allocation during
the call; this file is collected last."""
import ctypes
import numpy as np
import pytest
import synth
from gpu_util import require_gpu, dev, host

pytestmark = pytest.mark.gpu


def _call(lib, name, M, max_sweeps=30, marks=None):
    """Run entry point `name` on M (after its buffers exist); with `marks` a list, append the
    device-memory marks taken right before and right after the call itself."""
    import torch
    p = M.shape[0]
    Mst = dev(M).t().contiguous()            # column-major storage
    Us = torch.empty((p, p), dtype=torch.float64, device="cuda")
    Vs = torch.empty((p, p), dtype=torch.float64, device="cuda")
    d = torch.empty(p, dtype=torch.float64, device="cuda")
    lib.randutv_set_stream(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    if marks is not None:
        _reset_pool_high(_device_memory_marks()[3])
        marks.append(_device_memory_marks())
    st = getattr(lib, name)(p, Mst.data_ptr(), p, Us.data_ptr(), d.data_ptr(), Vs.data_ptr(), max_sweeps)
    torch.cuda.synchronize()
    if marks is not None:
        marks.append(_device_memory_marks())
    return st, host(Us.t()), host(d), host(Vs.t())


def _device_memory_marks():
    """(free device bytes, used high-water mark of the device's default memory pool) after a
    reset of the mark: an allocation by cudaMalloc moves the first, one by cudaMallocAsync the
    second."""
    import torch
    from gpu_util import cudart
    rt = cudart()
    free, total = ctypes.c_size_t(), ctypes.c_size_t()
    assert rt.cudaMemGetInfo(ctypes.byref(free), ctypes.byref(total)) == 0
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    used, high = ctypes.c_uint64(), ctypes.c_uint64()
    USED_CURRENT, USED_HIGH = 7, 8          # cudaMemPoolAttrUsedMemCurrent, cudaMemPoolAttrUsedMemHigh
    assert rt.cudaMemPoolGetAttribute(pool, USED_CURRENT, ctypes.byref(used)) == 0
    assert rt.cudaMemPoolGetAttribute(pool, USED_HIGH, ctypes.byref(high)) == 0
    return free.value, used.value, high.value, pool


def _reset_pool_high(pool):
    from gpu_util import cudart
    zero = ctypes.c_uint64(0)
    assert cudart().cudaMemPoolSetAttribute(pool, 8, ctypes.byref(zero)) == 0


def test_noalloc_matches_allocating_entry_point_twice():
    require_gpu()
    from paper_1703_00998_gb300 import native
    lib = native.lib()
    # upper triangular blocks, like the R11 factors the factorization passes
    mats = [np.linalg.qr(synth.make_matrix("exp50", 128, 128, 21))[1],
            np.linalg.qr(synth.make_matrix("exp5", 200, 200, 22))[1]]
    for call, M in enumerate(mats):              # two calls in a row
        st0, U0, d0, V0 = _call(lib, "randutv_small_svd", M)
        # the second call (the first may load the library's module on this device) allocates
        # nothing: free device memory and the default pool's used high-water mark stay put
        marks = [] if call == 1 else None
        st1, U1, d1, V1 = _call(lib, "randutv_small_svd_noalloc", M, marks=marks)
        if marks:
            (free0, used0, _, _), (free1, used1, high1, _) = marks
            assert free1 == free0 and used1 == used0 and high1 <= used0, (free0, free1, used0, used1, high1)
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
