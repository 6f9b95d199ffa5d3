"""Mixed-precision form (FP32 storage and products, FP64 panels and small
SVD): residual and orthogonality at FP32 level, |diag T| against the FP64
path and the oracle on the same Gaussian matrices."""
import numpy as np
import pytest
import synth
import oracle
from gpu_util import require_gpu, dev, host

pytestmark = pytest.mark.gpu
SEED = 998


@pytest.fixture(scope="module")
def R():
    require_gpu()
    import paper_1703_00998_gb300 as R
    return R


def gauss(i, k, b):
    return synth.step_gaussian(SEED, i, k, b)


def metrics(A64, U, T, V):
    import torch
    At, Ut, Tt, Vt = (dev(np.asarray(x, dtype=np.float64)) for x in (A64, U, T, V))
    n = At.shape[1]
    res = float(torch.linalg.norm(At - Ut @ Tt @ Vt.T) / torch.linalg.norm(At))
    ou = float((Ut.T @ Ut - torch.eye(Ut.shape[1], dtype=torch.float64, device="cuda")).abs().max())
    ov = float((Vt.T @ Vt - torch.eye(n, dtype=torch.float64, device="cuda")).abs().max())
    return res, ou, ov


def diag_close(d, dref, normA, rel):
    # relative with an absolute floor at FP32 rounding of the whole matrix
    floor = len(dref) * 2.0 ** -24 * normA
    return float(np.max(np.abs(np.abs(d) - np.abs(dref)) / (np.abs(dref) + floor / rel)))


@pytest.mark.parametrize("tc", [0, 1])
@pytest.mark.parametrize("m,n,b,q", [(500, 500, 32, 1), (300, 200, 32, 1), (200, 300, 32, 1), (257, 257, 64, 0),
                                     (1000, 1000, 128, 1)])
def test_mixed_small_shapes(R, m, n, b, q, tc):
    A = synth.make_matrix("exp50", m, n, 1703001 + m).astype(np.float32)
    A64 = A.astype(np.float64)
    g = dev(synth.gaussian_stream(SEED, m, n, b)) if synth.stream_layout(m, n, b)[1] > 0 else None
    out = R.factor_mixed(dev(A), b=b, q=q, g_inject=g, tensor_cores=tc)
    U, T, V = host(out.U), host(out.T), host(out.V)
    assert out.k_reached == min(m, n)
    res, ou, ov = metrics(A64, U, T, V)
    assert res <= 1e-6 and ou <= 1e-6 and ov <= 1e-6, (res, ou, ov)
    assert np.max(np.abs(np.tril(T, -1))) == 0.0
    f = R.factor(dev(A64), b=b, q=q, g_inject=g)
    d64 = host(f.T).diagonal()
    assert diag_close(T.diagonal(), d64, np.linalg.norm(A64, 2), 1e-4) <= 1e-4
    _, To, _, _ = oracle.randutv(A64, b, q, gauss, form_uv=False)
    assert diag_close(T.diagonal(), To.diagonal(), np.linalg.norm(A64, 2), 1e-4) <= 1e-4


@pytest.mark.parametrize("tc", [0, 1])
@pytest.mark.parametrize("kind", ["exp200", "inv"])
def test_mixed_n4000_against_fp64(R, kind, tc):
    n, b = 4000, 128
    A64 = synth.make_matrix(kind, n, n, 1703002 + ["exp200", "inv"].index(kind))
    A = A64.astype(np.float32)
    A64 = A.astype(np.float64)
    out = R.factor_mixed(dev(A), b=b, q=1, seed=SEED, tensor_cores=tc)
    res, ou, ov = metrics(A64, host(out.U), host(out.T), host(out.V))
    assert res <= 1e-6 and ou <= 1e-6 and ov <= 1e-6, (res, ou, ov)
    f = R.factor(dev(A64), b=b, q=1, seed=SEED)
    nA = np.linalg.norm(A64, 2)
    assert diag_close(host(out.T).diagonal(), host(f.T).diagonal(), nA, 1e-4) <= 1e-4


def test_mixed_t_only_and_tolerance(R):
    A = synth.make_matrix("exp", 400, 400, 8, r=6.0).astype(np.float32)
    out = R.factor_mixed(dev(A), b=32, q=1, tol=1e-4, form_uv=False)
    assert out.U is None and 0 < out.k_reached < 400
    f = R.factor(dev(A.astype(np.float64)), b=32, q=1, tol=1e-4)
    assert out.k_reached == f.k_reached


def test_mixed_overlap_off_matches(R):
    # the U/V stream only reorders independent work: same factors either way
    A = synth.make_matrix("exp50", 600, 600, 31).astype(np.float32)
    g = dev(synth.gaussian_stream(SEED, 600, 600, 64))
    a = R.factor_mixed(dev(A), b=64, q=1, g_inject=g, overlap=True)
    c = R.factor_mixed(dev(A), b=64, q=1, g_inject=g, overlap=False)
    for x, y in ((a.T, c.T), (a.U, c.U), (a.V, c.V)):
        assert float((x - y).abs().max()) <= 1e-5
    res, ou, ov = metrics(A.astype(np.float64), host(a.U), host(a.T), host(a.V))
    assert res <= 1e-6 and ou <= 1e-6 and ov <= 1e-6
