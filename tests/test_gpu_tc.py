"""tcgen05 tensor-core GEMM (C = alpha op(A) op(B) + beta C, TF32 inputs,
FP32 accumulation in tensor memory) against FP64 numpy, for all four
transpose forms (K-major and MN-major shared-memory tiles): exact on
small-integer inputs (every product and partial sum representable), within
the TF32 / 3xTF32 rounding bounds on Gaussian inputs, including ragged tiles
and split K."""
import ctypes
import numpy as np
import pytest
from gpu_util import require_gpu, host

pytestmark = pytest.mark.gpu

FORMS = [(True, False), (False, False), (False, True), (True, True)]


def _r4(x):
    return (x + 3) // 4 * 4


def _store(X):
    """Column-major device storage of X (r, c) with ld = r rounded up to 4."""
    import torch
    r, c = X.shape
    ld = _r4(r)
    st = torch.zeros((c, ld), dtype=torch.float32)
    st[:, :r] = torch.from_numpy(np.ascontiguousarray(X.T))
    return st.cuda(), ld


def run_tc(A, B, C, alpha, beta, passes=1, ta=True, tb=False):
    """op(A) = A.T if ta else A, op(B) = B.T if tb else B (numpy float32);
    returns alpha op(A) op(B) + beta C via randutv_sgemm_tc."""
    import torch
    from paper_1703_00998_gb300 import native
    m = A.shape[1] if ta else A.shape[0]
    k = A.shape[0] if ta else A.shape[1]
    n = B.shape[0] if tb else B.shape[1]
    Ast, lda = _store(A)
    Bst, ldb = _store(B)
    Cst = torch.from_numpy(np.ascontiguousarray(C.T)).cuda()
    lib = native.lib()
    lib.randutv_set_stream(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    st = lib.randutv_sgemm_tc(b"T" if ta else b"N", b"T" if tb else b"N", m, n, k, float(alpha), Ast.data_ptr(),
                              lda, Bst.data_ptr(), ldb, float(beta), Cst.data_ptr(), m, passes)
    assert st == native.OK, native.strerror(st)
    torch.cuda.synchronize()
    return host(Cst).T


def _operands(rng, m, n, k, ta, tb, draw):
    A = draw(rng, (k, m) if ta else (m, k))
    B = draw(rng, (n, k) if tb else (k, n))
    opA = A.astype(np.float64).T if ta else A.astype(np.float64)
    opB = B.astype(np.float64).T if tb else B.astype(np.float64)
    return A, B, opA, opB


def _ints(rng, shape):
    return rng.integers(-4, 5, shape).astype(np.float32)


def _gauss(rng, shape):
    return rng.standard_normal(shape).astype(np.float32)


@pytest.fixture(scope="module")
def ready():
    require_gpu()
    return True


@pytest.mark.parametrize("ta,tb", FORMS)
@pytest.mark.parametrize("passes", [1, 3])
@pytest.mark.parametrize("m,n,k", [(128, 128, 32), (256, 128, 64), (128, 256, 96), (300, 130, 64), (97, 45, 37)])
def test_tc_exact_on_small_integers(ready, m, n, k, passes, ta, tb):
    rng = np.random.default_rng(m + n + k + 2 * ta + tb)
    A, B, opA, opB = _operands(rng, m, n, k, ta, tb, _ints)
    C = np.zeros((m, n), dtype=np.float32)
    out = run_tc(A, B, C, 1.0, 0.0, passes, ta, tb)
    np.testing.assert_array_equal(out, (opA @ opB).astype(np.float32))


@pytest.mark.parametrize("ta,tb", FORMS)
def test_tc_exact_beta_update(ready, ta, tb):
    """C - op(A) op(B) with integer data: the alpha = -1, beta = 1 form of a
    rank-b update, exact."""
    m, n, k = 260, 390, 128
    rng = np.random.default_rng(5 + 2 * ta + tb)
    A, B, opA, opB = _operands(rng, m, n, k, ta, tb, _ints)
    C = rng.integers(-100, 101, (m, n)).astype(np.float32)
    out = run_tc(A, B, C, -1.0, 1.0, 3, ta, tb)
    np.testing.assert_array_equal(out, (C.astype(np.float64) - opA @ opB).astype(np.float32))


@pytest.mark.parametrize("m,n,k", [(1000, 128, 3000), (8000, 128, 8000), (333, 200, 100), (129, 1, 33)])
def test_tc_gaussian_within_tf32_bound(ready, m, n, k):
    rng = np.random.default_rng(7 * m + n + k)
    A, B, opA, opB = _operands(rng, m, n, k, True, False, _gauss)
    C = rng.standard_normal((m, n)).astype(np.float32)
    out = run_tc(A, B, C, 1.5, -0.5).astype(np.float64)
    ref = 1.5 * opA @ opB - 0.5 * C.astype(np.float64)
    # TF32 keeps 10 explicit mantissa bits of each input; FP32 accumulation
    bound = 1.5 * (2.0 ** -9 + k * 2.0 ** -23) * (np.abs(opA) @ np.abs(opB)) + 1e-6
    assert np.all(np.abs(out - ref) <= bound)
    # and it is a real product, not noise: relative Frobenius error near TF32 rounding
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 2e-3


@pytest.mark.parametrize("ta,tb", FORMS)
@pytest.mark.parametrize("m,n,k", [(1000, 128, 3000), (8000, 128, 8000), (333, 200, 100), (2000, 1500, 128)])
def test_tc_3xtf32_at_fp32_level(ready, m, n, k, ta, tb):
    rng = np.random.default_rng(11 * m + n + k + 2 * ta + tb)
    A, B, opA, opB = _operands(rng, m, n, k, ta, tb, _gauss)
    C = rng.standard_normal((m, n)).astype(np.float32)
    out = run_tc(A, B, C, 1.5, -0.5, 3, ta, tb).astype(np.float64)
    ref = 1.5 * opA @ opB - 0.5 * C.astype(np.float64)
    # hi = rna_tf32(x), lo = rna_tf32(x - hi): |x - hi - lo| <= 2^-22 |x|; lo*lo dropped
    # (<= 2^-22 |a||b|); FP32 accumulation of the chunk
    bound = 1.5 * (4 * 2.0 ** -22 + k * 2.0 ** -23) * (np.abs(opA) @ np.abs(opB)) + 1e-6
    assert np.all(np.abs(out - ref) <= bound)
    # the tensor-core FP32 accumulator truncates (about half an ulp of the
    # running sum per K = 8); the kernel restarts it every K = 128 and adds
    # the chunks in FP32 registers, so the error stays near 1e-6 at any K
    # (it grew linearly with K before: 1.9e-5 at K = 8000); plain TF32 ~1e-3
    rel = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert rel < 2e-6
