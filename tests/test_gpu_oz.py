"""Ozaki-scheme FP64 GEMM (BF16 tensor-core slice products, exact group
sums, 64-bit fixed-point accumulation over the K chunks of 128, one FP64
rounding at the end) against FP64 numpy: exact on small-integer inputs for
all four transpose forms and K spanning several chunks (and several CTAs),
within the FP64 dot-product bound on Gaussian inputs, and within the
scheme's max-based bound on rows graded over 16 orders of magnitude."""
import ctypes
import numpy as np
import pytest
from gpu_util import require_gpu, host

pytestmark = pytest.mark.gpu
FORMS = [(False, False), (True, False), (False, True), (True, True)]


def run_oz(A, B, C, alpha, beta, ta=False, tb=False):
    """op(A) = A.T if ta else A, op(B) = B.T if tb else B (numpy float64)."""
    import torch
    from paper_1703_00998_gb300 import native
    m = A.shape[1] if ta else A.shape[0]
    k = A.shape[0] if ta else A.shape[1]
    n = B.shape[0] if tb else B.shape[1]
    # (an empty operand still needs a valid pointer and a leading dimension >= 1)
    Ast = torch.from_numpy(np.ascontiguousarray(A.T)).cuda() if A.size else torch.zeros(1, dtype=torch.float64,
                                                                                        device="cuda")
    Bst = torch.from_numpy(np.ascontiguousarray(B.T)).cuda() if B.size else torch.zeros(1, dtype=torch.float64,
                                                                                        device="cuda")
    Cst = torch.from_numpy(np.ascontiguousarray(C.T)).cuda()
    lib = native.lib()
    lib.randutv_set_stream(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    st = lib.randutv_dgemm_oz(b"T" if ta else b"N", b"T" if tb else b"N", m, n, k, float(alpha), Ast.data_ptr(),
                              max(1, A.shape[0]), Bst.data_ptr(), max(1, B.shape[0]), float(beta), Cst.data_ptr(), m)
    assert st == native.OK, native.strerror(st)
    torch.cuda.synchronize()
    return host(Cst).T


def operands(rng, m, n, k, ta, tb, draw):
    A = draw(rng, (k, m) if ta else (m, k))
    B = draw(rng, (n, k) if tb else (k, n))
    return A, B, (A.T if ta else A), (B.T if tb else B)


@pytest.fixture(scope="module")
def ready():
    require_gpu()
    return True


@pytest.mark.parametrize("ta,tb", FORMS)
# (n < m <= ... runs the transposed-tile path; m <= n or n > 256 the direct one)
@pytest.mark.parametrize("m,n,k", [(128, 64, 128), (300, 130, 64), (97, 45, 300), (256, 200, 1000), (5, 3, 1),
                                   (64, 300, 200), (200, 333, 129), (700, 300, 100)])
def test_oz_exact_on_small_integers(ready, m, n, k, ta, tb):
    rng = np.random.default_rng(m + 7 * n + k + 2 * ta + tb)
    A, B, oA, oB = operands(rng, m, n, k, ta, tb, lambda r, s: r.integers(-100, 101, s).astype(np.float64))
    C = rng.integers(-1000, 1001, (m, n)).astype(np.float64)
    out = run_oz(A, B, C, -1.0, 1.0, ta, tb)
    np.testing.assert_array_equal(out, C - oA @ oB)


@pytest.mark.parametrize("ta,tb", FORMS)
@pytest.mark.parametrize("m,n,k", [(1000, 128, 3000), (333, 200, 100), (2000, 1500, 128), (129, 1, 257)])
def test_oz_gaussian_at_fp64_level(ready, m, n, k, ta, tb):
    rng = np.random.default_rng(3 * m + n + k + 2 * ta + tb)
    A, B, oA, oB = operands(rng, m, n, k, ta, tb, lambda r, s: r.standard_normal(s))
    C = rng.standard_normal((m, n))
    out = run_oz(A, B, C, 1.5, -0.5, ta, tb)
    ref = 1.5 * (oA @ oB) - 0.5 * C
    mag = 1.5 * (np.abs(oA) @ np.abs(oB)) + 0.5 * np.abs(C)
    assert np.all(np.abs(out - ref) <= (k + 64) * 2.0 ** -52 * mag)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-15


def test_oz_graded_rows_within_the_max_bound(ready):
    """Rows of A scaled over 1e-8 .. 1e8 and columns of B over 1e-8 .. 1e8,
    with entries inside a row spread over 1e-6 .. 1: the error is bounded by
    the scheme's per-chunk max-based term (plus FP64 rounding), which is
    what the per-(row, chunk) scales buy."""
    rng = np.random.default_rng(11)
    m, n, k = 300, 150, 700
    A = rng.standard_normal((m, k)) * 10.0 ** rng.uniform(-6, 0, (m, k)) * 10.0 ** rng.uniform(-8, 8, (m, 1))
    B = rng.standard_normal((k, n)) * 10.0 ** rng.uniform(-6, 0, (k, n)) * 10.0 ** rng.uniform(-8, 8, (1, n))
    out = run_oz(A, B, np.zeros((m, n)), 1.0, 0.0)
    ref = A @ B
    bound = np.zeros((m, n))
    for c0 in range(0, k, 128):
        ma = np.abs(A[:, c0:c0 + 128]).max(axis=1)
        mb = np.abs(B[c0:c0 + 128, :]).max(axis=0)
        bound += 2 * 128 * 2.0 ** -55 * np.outer(ma, mb)
    bound += (k // 128 + 2) * 2.0 ** -52 * (np.abs(A) @ np.abs(B))
    assert np.all(np.abs(out - ref) <= bound)


def test_oz_k_zero_scales(ready):
    C = np.arange(12.0).reshape(4, 3)
    out = run_oz(np.zeros((4, 0)), np.zeros((0, 3)), C, 1.0, 2.0)
    np.testing.assert_array_equal(out, 2.0 * C)


def run_oz32(A, B, C, alpha, beta, ta=False, tb=False, entry="randutv_sgemm_oz"):
    """The FP32 form (or, with entry="randutv_sgemm", the CUDA-core FP32 GEMM) on float32 numpy operands."""
    import torch
    from paper_1703_00998_gb300 import native
    m = A.shape[1] if ta else A.shape[0]
    k = A.shape[0] if ta else A.shape[1]
    n = B.shape[0] if tb else B.shape[1]
    Ast = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    Bst = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Cst = torch.from_numpy(np.ascontiguousarray(C.T)).cuda()
    lib = native.lib()
    lib.randutv_set_stream(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    st = getattr(lib, entry)(b"T" if ta else b"N", b"T" if tb else b"N", m, n, k, float(alpha), Ast.data_ptr(),
                             max(1, A.shape[0]), Bst.data_ptr(), max(1, B.shape[0]), float(beta), Cst.data_ptr(), m)
    assert st == native.OK, native.strerror(st)
    torch.cuda.synchronize()
    return host(Cst).T


@pytest.mark.parametrize("ta,tb", FORMS)
@pytest.mark.parametrize("m,n,k", [(128, 64, 128), (300, 130, 64), (97, 45, 300), (64, 300, 200), (5, 3, 1)])
def test_oz32_exact_on_small_integers(ready, m, n, k, ta, tb):
    rng = np.random.default_rng(17 * m + n + k + 2 * ta + tb)
    A, B, oA, oB = operands(rng, m, n, k, ta, tb, lambda r, s: r.integers(-100, 101, s).astype(np.float32))
    C = rng.integers(-1000, 1001, (m, n)).astype(np.float32)
    out = run_oz32(A, B, C, -1.0, 1.0, ta, tb)
    # every exact result is below 2^24 in magnitude: representable in FP32
    np.testing.assert_array_equal(out, (C.astype(np.float64) - oA.astype(np.float64) @ oB.astype(np.float64)))


@pytest.mark.parametrize("ta,tb", FORMS)
@pytest.mark.parametrize("m,n,k", [(1000, 128, 3000), (333, 200, 100), (2000, 1500, 128), (8000, 128, 8000)])
def test_oz32_gaussian_at_fp32_level(ready, m, n, k, ta, tb):
    """Within the FP32 dot-product bound, and no worse than twice the
    CUDA-core FP32 GEMM's own error on the same operands."""
    rng = np.random.default_rng(5 * m + n + k + 2 * ta + tb)
    A, B, oA, oB = operands(rng, m, n, k, ta, tb, lambda r, s: r.standard_normal(s).astype(np.float32))
    C = rng.standard_normal((m, n)).astype(np.float32)
    out = run_oz32(A, B, C, 1.5, -0.5, ta, tb).astype(np.float64)
    ref = 1.5 * (oA.astype(np.float64) @ oB.astype(np.float64)) - 0.5 * C.astype(np.float64)
    mag = 1.5 * (np.abs(oA).astype(np.float64) @ np.abs(oB).astype(np.float64)) + 0.5 * np.abs(C)
    assert np.all(np.abs(out - ref) <= (k // 128 + 4) * 2.0 ** -23 * mag)
    simt = run_oz32(A, B, C, 1.5, -0.5, ta, tb, entry="randutv_sgemm").astype(np.float64)
    e_oz = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    e_simt = np.linalg.norm(simt - ref) / np.linalg.norm(ref)
    assert e_oz <= 2.0 * e_simt + 1e-8, (e_oz, e_simt)


def test_oz32_graded_rows_within_the_max_bound(ready):
    rng = np.random.default_rng(12)
    m, n, k = 300, 150, 700
    A = (rng.standard_normal((m, k)) * 10.0 ** rng.uniform(-3, 0, (m, k)) * 10.0 ** rng.uniform(-4, 4, (m, 1)))
    B = (rng.standard_normal((k, n)) * 10.0 ** rng.uniform(-3, 0, (k, n)) * 10.0 ** rng.uniform(-4, 4, (1, n)))
    A, B = A.astype(np.float32), B.astype(np.float32)
    out = run_oz32(A, B, np.zeros((m, n), np.float32), 1.0, 0.0).astype(np.float64)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = A64 @ B64
    bound = np.zeros((m, n))
    for c0 in range(0, k, 128):
        ma = np.abs(A64[:, c0:c0 + 128]).max(axis=1)
        mb = np.abs(B64[c0:c0 + 128, :]).max(axis=0)
        bound += 2 * 128 * 2.0 ** -27 * np.outer(ma, mb)
    bound += (k // 128 + 2) * 2.0 ** -23 * (np.abs(A64) @ np.abs(B64))
    assert np.all(np.abs(out - ref) <= bound)
