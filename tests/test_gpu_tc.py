"""tcgen05 tensor-core GEMM (C = alpha A^T B + beta C, TF32 inputs, FP32
accumulation in tensor memory) against FP64 numpy: exact on small-integer
inputs (every product and partial sum representable), within the TF32
rounding bound on Gaussian inputs, including ragged tiles and split K."""
import ctypes
import numpy as np
import pytest
from gpu_util import require_gpu, host

pytestmark = pytest.mark.gpu


def _r4(x):
    return (x + 3) // 4 * 4


def run_tc(A, B, C, alpha, beta, passes=1):
    """A (k, m), B (k, n), C (m, n) numpy float32 -> C_out via randutv_sgemm_tc."""
    import torch
    from paper_1703_00998_gb300 import native
    k, m = A.shape
    n = B.shape[1]
    lda, ldb = _r4(k), _r4(k)
    Ast = torch.zeros((m, lda), dtype=torch.float32)
    Ast[:, :k] = torch.from_numpy(A.T.copy())
    Bst = torch.zeros((n, ldb), dtype=torch.float32)
    Bst[:, :k] = torch.from_numpy(B.T.copy())
    Cst = torch.from_numpy(C.T.copy())
    Ast, Bst, Cst = Ast.cuda(), Bst.cuda(), Cst.cuda()
    lib = native.lib()
    lib.randutv_set_stream(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    st = lib.randutv_sgemm_tc(m, n, k, float(alpha), Ast.data_ptr(), lda, Bst.data_ptr(), ldb, float(beta),
                              Cst.data_ptr(), m, passes)
    assert st == native.OK, native.strerror(st)
    torch.cuda.synchronize()
    return host(Cst).T


@pytest.fixture(scope="module")
def ready():
    require_gpu()
    return True


@pytest.mark.parametrize("passes", [1, 3])
@pytest.mark.parametrize("m,n,k", [(128, 128, 32), (256, 128, 64), (128, 256, 96), (300, 130, 64)])
def test_tc_exact_on_small_integers(ready, m, n, k, passes):
    rng = np.random.default_rng(m + n + k)
    A = rng.integers(-4, 5, (k, m)).astype(np.float32)
    B = rng.integers(-4, 5, (k, n)).astype(np.float32)
    C = np.zeros((m, n), dtype=np.float32)
    out = run_tc(A, B, C, 1.0, 0.0, passes)
    np.testing.assert_array_equal(out, (A.astype(np.float64).T @ B.astype(np.float64)).astype(np.float32))


@pytest.mark.parametrize("m,n,k", [(1000, 128, 3000), (8000, 128, 8000), (333, 200, 100), (129, 1, 33)])
def test_tc_gaussian_within_tf32_bound(ready, m, n, k):
    rng = np.random.default_rng(7 * m + n + k)
    A = rng.standard_normal((k, m)).astype(np.float32)
    B = rng.standard_normal((k, n)).astype(np.float32)
    C = rng.standard_normal((m, n)).astype(np.float32)
    out = run_tc(A, B, C, 1.5, -0.5).astype(np.float64)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = 1.5 * A64.T @ B64 - 0.5 * C.astype(np.float64)
    # TF32 keeps 10 explicit mantissa bits of each input; FP32 accumulation
    bound = 1.5 * (2.0 ** -9 + k * 2.0 ** -23) * (np.abs(A64).T @ np.abs(B64)) + 1e-6
    assert np.all(np.abs(out - ref) <= bound)
    # and it is a real product, not noise: relative Frobenius error near TF32 rounding
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 2e-3


@pytest.mark.parametrize("m,n,k", [(1000, 128, 3000), (8000, 128, 8000), (333, 200, 100)])
def test_tc_3xtf32_at_fp32_level(ready, m, n, k):
    rng = np.random.default_rng(11 * m + n + k)
    A = rng.standard_normal((k, m)).astype(np.float32)
    B = rng.standard_normal((k, n)).astype(np.float32)
    C = rng.standard_normal((m, n)).astype(np.float32)
    out = run_tc(A, B, C, 1.5, -0.5, passes=3).astype(np.float64)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = 1.5 * A64.T @ B64 - 0.5 * C.astype(np.float64)
    # hi = rna_tf32(x), lo = rna_tf32(x - hi): |x - hi - lo| <= 2^-22 |x|; lo*lo dropped
    # (<= 2^-22 |a||b|); FP32 accumulation of the chunk
    bound = 1.5 * (4 * 2.0 ** -22 + k * 2.0 ** -23) * (np.abs(A64).T @ np.abs(B64)) + 1e-6
    assert np.all(np.abs(out - ref) <= bound)
    # the tensor-core FP32 accumulator does not round to nearest: its error
    # grows ~ linearly in the chunk length (measured 1.9e-5 at K = 8000,
    # 3 chunks) instead of ~ sqrt; plain TF32 gives ~1e-3
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 4e-5
