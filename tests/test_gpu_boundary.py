"""The boundary's own calls on the GPU against the oracle (config: 500 x 500,
sigma_j = exp(-j/50), b = 32, q = 1): randutv_factor (library-allocated U,
T, V released with randutv_free), randutv_factor_host (host buffers, copies
inside), the g_capture option (the Philox G a run used, given to the
oracle), and the mixed form's one-product TF32 sketch (sketch_prec)."""
import ctypes
import numpy as np
import pytest
import synth
import oracle
from oracle import checks
from gpu_util import require_gpu, dev, host, device_to_host

pytestmark = pytest.mark.gpu
SEED = 998
M = N = 500
B, Q = 32, 1


@pytest.fixture(scope="module")
def R():
    require_gpu()
    import paper_1703_00998_gb300 as R
    return R


@pytest.fixture(scope="module")
def A():
    return synth.make_matrix("exp50", M, N, 1703001)


@pytest.fixture(scope="module")
def ref(A):
    # the oracle on the host Philox/Box-Muller stream (libm normals; the device's agree to a few ulp)
    return oracle.randutv(A, B, Q, lambda i, k, b: synth.step_gaussian(SEED, i, k, b))


def check_against(ref, A, U, T, V, k, tol=1e-9):
    Uo, To, Vo, ko = ref
    assert k == ko == min(A.shape)
    d, do = np.abs(np.diag(T)), np.abs(np.diag(To))
    assert float(np.max(np.abs(d - do) / do)) <= 1e-10
    assert checks.residual(A, U, T, V) <= 1e-13
    assert checks.orth_err(U) <= 1e-13 and checks.orth_err(V) <= 1e-13
    assert checks.lower_max(T) == 0.0
    # the same conventions (reflector signs, small-SVD order and signs): entry by entry
    assert np.max(np.abs(T - To)) <= tol
    assert np.max(np.abs(U - Uo)) <= tol
    assert np.max(np.abs(V - Vo)) <= tol


def test_randutv_factor_library_allocated(R, A, ref):
    import torch
    from paper_1703_00998_gb300 import native
    lib = native.lib()
    Ad = dev(np.asfortranarray(A).T.copy())       # column-major storage: (n, m) contiguous
    lib.randutv_set_stream(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    pu, pt, pv = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    kr = ctypes.c_int64(-1)
    st = lib.randutv_factor(M, N, Ad.data_ptr(), M, B, Q, 0.0, ctypes.byref(pu), ctypes.byref(pt), ctypes.byref(pv),
                            ctypes.byref(kr))
    assert st == native.OK, native.strerror(st)
    try:
        U = device_to_host(pu.value, (M, M))
        T = device_to_host(pt.value, (M, N))
        V = device_to_host(pv.value, (N, N))
    finally:
        for ptr in (pu, pt, pv):
            lib.randutv_free(ptr)
    check_against(ref, A, U, T, V, kr.value)
    # A is not modified
    np.testing.assert_array_equal(host(Ad).T, A)


def test_randutv_factor_library_allocated_rejects(R):
    from paper_1703_00998_gb300 import native
    lib = native.lib()
    pu, pt, pv = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    kr = ctypes.c_int64(0)
    assert lib.randutv_factor(M, N, None, M, B, Q, 0.0, ctypes.byref(pu), ctypes.byref(pt), ctypes.byref(pv),
                              ctypes.byref(kr)) == -3
    lib.randutv_free(None)   # NULL is ignored


def test_randutv_factor_host(R, A, ref):
    import torch
    Ah = torch.from_numpy(np.ascontiguousarray(A.T)).pin_memory().t()   # pinned, column-major
    out = R.factor_host(Ah, b=B, q=Q, seed=SEED)
    U, T, V = (x.numpy() for x in (out.U, out.T, out.V))
    check_against(ref, A, U, T, V, out.k_reached)


def test_g_capture_records_the_stream_used(R, A):
    import torch
    layout = synth.stream_layout(M, N, B)
    cap = torch.full((layout[1],), float("nan"), dtype=torch.float64, device="cuda")
    f = R.factor(dev(A), b=B, q=Q, seed=SEED, g_capture=cap)
    g = host(cap)
    gh = synth.gaussian_stream(SEED, M, N, B)
    # the device normals agree with the host definition to a few ulp
    assert np.all(np.isfinite(g))
    assert np.max(np.abs(g - gh)) <= 64 * 2.0 ** -52 * np.max(np.abs(gh))
    # the oracle on the captured G reproduces the run entry by entry
    offs = {step: off for step, _, off in layout[0]}

    def gauss(i, k, b):
        o = offs[i]
        return g[o:o + k * b].reshape(b, k).T
    Uo, To, Vo, ko = oracle.randutv(A, B, Q, gauss)
    U, T, V = host(f.U), host(f.T), host(f.V)
    assert f.k_reached == ko
    assert np.max(np.abs(T - To)) <= 1e-9
    assert np.max(np.abs(U - Uo)) <= 1e-9
    assert np.max(np.abs(V - Vo)) <= 1e-9
    # and g_inject of the captured stream gives the same factorization again
    f2 = R.factor(dev(A), b=B, q=Q, g_inject=cap)
    assert float((f2.T - f.T).abs().max()) <= 1e-12


def test_mixed_g_capture_and_tf32_sketch(R, A):
    import torch
    A32 = A.astype(np.float32)
    cap = torch.zeros(synth.stream_layout(M, N, B)[1], dtype=torch.float64, device="cuda")
    m3 = R.factor_mixed(dev(A32), b=B, q=Q, seed=SEED, g_capture=cap)
    np.testing.assert_allclose(host(cap), synth.gaussian_stream(SEED, M, N, B), rtol=0, atol=1e-12)
    m1 = R.factor_mixed(dev(A32), b=B, q=Q, seed=SEED, sketch_prec=2)
    A64 = A32.astype(np.float64)
    for f in (m3, m1):
        U, T, V = (host(x).astype(np.float64) for x in (f.U, f.T, f.V))
        assert checks.residual(A64, U, T, V) <= 1e-6
        assert checks.orth_err(U) <= 1e-6 and checks.orth_err(V) <= 1e-6
        assert checks.lower_max(T) == 0.0
