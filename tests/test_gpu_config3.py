"""The mixed-precision form at its large configuration: n = 16000, FP32-stored
A with sigma_j = 1/j and exp(-j/500), b = 256, q = 1.  At full size the
mixed result is checked for residual and orthogonality (FP64, against the
stored FP32 A) and its |diag T| against the FP64 GPU form; on the leading
2000 x 2000 block of the same A (reading: "n = 2000 slices"), both GPU forms
are checked against the oracle on the same G."""
import numpy as np
import pytest
import synth
import oracle
from gpu_util import require_gpu, dev, host

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


def _residual_orth(A32, U, T, V):
    """FP64 residual ||A - U T V^T||_F / ||A||_F and max |X^T X - I| of U, V."""
    import torch
    A64 = A32.to(torch.float64)
    U64, V64 = U.to(torch.float64), V.to(torch.float64)
    P = U64 @ T.to(torch.float64)
    P = torch.addmm(A64, P, V64.T, alpha=-1.0)
    res = float(torch.linalg.norm(P) / torch.linalg.norm(A64))
    del P, A64
    eye = torch.eye(U64.shape[1], dtype=torch.float64, device=U64.device)
    ou = float((U64.T @ U64 - eye).abs().max())
    ov = float((V64.T @ V64 - eye).abs().max())
    return res, ou, ov


def _diag_close(d, dref, normA2, rel, unit):
    floor = len(dref) * unit * normA2
    return float(np.max(np.abs(np.abs(d) - np.abs(dref)) / (np.abs(dref) + floor / rel)))


def test_config3_full_size(R, A32):
    import torch
    out = R.factor_mixed(A32, b=B, q=Q, seed=SEED)
    assert out.k_reached == N
    res, ou, ov = _residual_orth(A32, out.U, out.T, out.V)
    print(f"n={N} mixed: residual {res:.3e}, orthogonality {ou:.3e} {ov:.3e}")
    assert res <= 1e-6 and ou <= 1e-6 and ov <= 1e-6, (res, ou, ov)
    Tm = torch.diagonal(out.T).double().cpu().numpy()
    assert float(torch.tril(out.T, -1).abs().max()) == 0.0
    del out
    torch.cuda.empty_cache()
    f = R.factor(A32.to(torch.float64), b=B, q=Q, seed=SEED, form_uv=False)
    d64 = torch.diagonal(f.T).cpu().numpy()
    del f
    torch.cuda.empty_cache()
    # ||A||_2 = sigma_1 = exp(-1/500) or 1 up to the FP32 rounding of A
    dr = _diag_close(Tm, d64, float(np.abs(d64).max()), 1e-4, 2.0 ** -24)
    print(f"n={N} mixed |diag T| vs FP64: {dr:.3e}")
    assert dr <= 1e-4


def test_config3_slice_against_oracle(R, A32):
    import torch
    As = A32[:NS, :NS].contiguous()
    A64 = host(As).astype(np.float64)
    g = dev(synth.gaussian_stream(SEED, NS, NS, B))
    m = R.factor_mixed(As, b=B, q=Q, g_inject=g)
    res, ou, ov = _residual_orth(As, m.U, m.T, m.V)
    assert res <= 1e-6 and ou <= 1e-6 and ov <= 1e-6, (res, ou, ov)
    f = R.factor(dev(A64), b=B, q=Q, g_inject=g)
    res64, ou64, ov64 = _residual_orth(dev(A64), f.U, f.T, f.V)
    assert res64 <= 1e-13 and ou64 <= 1e-13 and ov64 <= 1e-13, (res64, ou64, ov64)
    _, To, _, _ = oracle.randutv(A64, B, Q, lambda i, k, b: synth.step_gaussian(SEED, i, k, b), form_uv=False)
    do = To.diagonal()
    nA = float(np.linalg.norm(A64, 2))
    assert _diag_close(host(f.T).diagonal(), do, nA, 1e-10, 2.0 ** -53) <= 1e-10
    assert _diag_close(host(m.T).diagonal().astype(np.float64), do, nA, 1e-4, 2.0 ** -24) <= 1e-4
