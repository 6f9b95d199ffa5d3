"""The mixed-precision form at its large configuration: n = 16000, FP32-stored
A with sigma_j = 1/j and exp(-j/500), b = 256, q = 1.  At full size the
mixed result is checked for residual and orthogonality (FP64, against the
stored FP32 A) and its |diag T| against the FP64 GPU form entry by entry
(max(1e-4 |d_64|, 4 s_j), s_j the FP64 form's sensitivity at the mixed
backward error); on the leading 2000 x 2000 block of the same A (reading:
"n = 2000 slices"), both GPU forms are checked against the oracle on the
same G."""
import numpy as np
import pytest
import synth
import oracle
from oracle import checks
from gpu_util import require_gpu, dev, host
from diag_bound import compare
from parity_util import check_mixed_diag, mixed_residual_orth, oracle_sensitivity

pytestmark = pytest.mark.gpu
SEED = 998
N, B, Q, NS = 16000, 256, 1, 2000


@pytest.fixture(scope="module")
def R():
    require_gpu()
    import paper_1703_00998_gb300 as R
    return R


@pytest.fixture(scope="module", params=["inv", "exp500"])
def A32(request, R):
    import torch
    kind = request.param
    A = synth.make_matrix(kind, N, N, 1703002 + ["exp200", "inv", "gauss", "exp500"].index(kind), device="cuda")
    A = A.to(torch.float32)
    torch.cuda.empty_cache()
    return A


def test_config3_full_size(R, A32):
    import torch
    out = R.factor_mixed(A32, b=B, q=Q, seed=SEED)
    assert out.k_reached == N
    res, ou, ov = mixed_residual_orth(A32, out.U, out.T, out.V)
    print(f"n={N} mixed: residual {res:.3e}, orthogonality {ou:.3e} {ov:.3e}")
    assert res <= 1e-6 and ou <= 1e-6 and ov <= 1e-6, (res, ou, ov)
    assert float(torch.tril(out.T, -1).abs().max()) == 0.0
    T = out.T.clone()
    del out
    torch.cuda.empty_cache()
    r = check_mixed_diag(R, A32, T, res, B, Q, seed=SEED)
    print(f"n={N} mixed |diag T| vs FP64: {r}")
    assert r["ok"]


def test_config3_slice_against_oracle(R, A32):
    As = A32[:NS, :NS].contiguous()
    A64 = host(As).astype(np.float64)
    g = dev(synth.gaussian_stream(SEED, NS, NS, B))
    m = R.factor_mixed(As, b=B, q=Q, g_inject=g)
    res, ou, ov = mixed_residual_orth(As, m.U, m.T, m.V)
    assert res <= 1e-6 and ou <= 1e-6 and ov <= 1e-6, (res, ou, ov)
    f = R.factor(dev(A64), b=B, q=Q, g_inject=g)
    res64, ou64, ov64 = mixed_residual_orth(dev(A64), f.U, f.T, f.V)
    assert res64 <= 1e-13 and ou64 <= 1e-13 and ov64 <= 1e-13, (res64, ou64, ov64)
    gs = lambda i, k, b: synth.step_gaussian(SEED, i, k, b)  # noqa: E731
    Uo, To, Vo, _ = oracle.randutv(A64, B, Q, gs)
    res_o = checks.residual(A64, Uo, To, Vo)
    do = To.diagonal()
    r64 = compare(host(f.T).diagonal(), do, oracle_sensitivity(A64, B, Q, gs, res64 + res_o), 1e-10, 4.0)
    print(f"n={NS} slice, FP64 |diag T| vs oracle: {r64}")
    assert r64["ok"]
    rm = compare(host(m.T).diagonal().astype(np.float64), do, oracle_sensitivity(A64, B, Q, gs, res + res_o), 1e-4,
                 4.0)
    print(f"n={NS} slice, mixed |diag T| vs oracle: {rm}")
    assert rm["ok"]
