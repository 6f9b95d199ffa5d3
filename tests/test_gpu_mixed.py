"""Mixed-precision form (FP32 storage and products, FP64 panels and small
SVD): residual and orthogonality at FP32 level, and |diag T| against the FP64
path (and, on small cases, the oracle) on the same Gaussian matrices, entry
by entry under max(1e-4 |d_ref|, 4 s_j) with s_j the reference's own measured
sensitivity to a perturbation of the mixed form's backward error."""
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


@pytest.fixture(scope="module")
def R():
    require_gpu()
    import paper_1703_00998_gb300 as R
    return R


def gauss(i, k, b):
    return synth.step_gaussian(SEED, i, k, b)


@pytest.mark.parametrize("sketch", [0, 1])
@pytest.mark.parametrize("m,n,b,q", [(500, 500, 32, 1), (300, 200, 32, 1), (200, 300, 32, 1), (257, 257, 64, 0),
                                     (1000, 1000, 128, 1)])
def test_mixed_small_shapes(R, m, n, b, q, sketch):
    A = synth.make_matrix("exp50", m, n, 1703001 + m).astype(np.float32)
    A64 = A.astype(np.float64)
    g = dev(synth.gaussian_stream(SEED, m, n, b)) if synth.stream_layout(m, n, b)[1] > 0 else None
    out = R.factor_mixed(dev(A), b=b, q=q, g_inject=g, sketch_prec=sketch)
    assert out.k_reached == min(m, n)
    res, ou, ov = mixed_residual_orth(dev(A), out.U, out.T, out.V)
    assert res <= 1e-6 and ou <= 1e-6 and ov <= 1e-6, (res, ou, ov)
    assert float(out.T.tril(-1).abs().max()) == 0.0
    r = check_mixed_diag(R, dev(A), out.T, res, b, q, g_inject=g)
    print(f"mixed {m}x{n} b={b} q={q} sketch={sketch}: residual {res:.2e}; |diag T| vs FP64: {r}")
    assert r["ok"]
    # against the oracle on the same G: the oracle's sensitivity at the two backward errors
    Uo, To, Vo, _ = oracle.randutv(A64, b, q, gauss)
    s = oracle_sensitivity(A64, b, q, gauss, res + checks.residual(A64, Uo, To, Vo))
    ro = compare(host(out.T).diagonal().astype(np.float64), To.diagonal(), s, 1e-4, 4.0)
    print(f"  vs oracle: {ro}")
    assert ro["ok"]


@pytest.mark.parametrize("kind", ["exp200", "inv"])
def test_mixed_n4000_against_fp64(R, kind):
    """n = 4000: the sliced sketch (default) meets max(1e-4 |d|, 4 s) on both spectra."""
    n, b = 4000, 128
    A64 = synth.make_matrix(kind, n, n, 1703002 + ["exp200", "inv"].index(kind))
    A = dev(A64.astype(np.float32))
    out = R.factor_mixed(A, b=b, q=1, seed=SEED)
    res, ou, ov = mixed_residual_orth(A, out.U, out.T, out.V)
    assert res <= 1e-6 and ou <= 1e-6 and ov <= 1e-6, (res, ou, ov)
    r = check_mixed_diag(R, A, out.T, res, b, 1, seed=SEED)
    print(f"mixed n={n} {kind}: residual {res:.2e}, orthogonality {ou:.2e} {ov:.2e}; |diag T| vs FP64: {r}")
    assert r["ok"]


@pytest.mark.parametrize("sketch,tc", [(1, 1), (1, 0), (2, 1)])
def test_mixed_n4000_fp32_level_sketches(R, sketch, tc):
    """The FP32-level sketches (3xTF32 or FP32 CUDA cores; one TF32 product, whose |diag T| is
    only reported) on the fast-decaying spectrum: FP32 residual and orthogonality, |diag T| under
    the same bound as the default.  (On
    sigma_j = 1/j their FP32-level sketch error is amplified by the clustered spectrum and |diag T|
    moves up to 1e-2 relative: the reason the default sketch is sliced.)"""
    n, b = 4000, 128
    A = dev(synth.make_matrix("exp200", n, n, 1703002).astype(np.float32))
    out = R.factor_mixed(A, b=b, q=1, seed=SEED, sketch_prec=sketch, tensor_cores=tc)
    res, ou, ov = mixed_residual_orth(A, out.U, out.T, out.V)
    assert res <= 1e-6 and ou <= 1e-6 and ov <= 1e-6, (res, ou, ov)
    r = check_mixed_diag(R, A, out.T, res, b, 1, seed=SEED)
    print(f"mixed n={n} exp200 sketch={sketch} tc={tc}: residual {res:.2e}; |diag T| vs FP64: {r}")
    if sketch == 1:
        assert r["ok"]


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
    res, ou, ov = mixed_residual_orth(dev(A), a.U, a.T, a.V)
    assert res <= 1e-6 and ou <= 1e-6 and ov <= 1e-6
