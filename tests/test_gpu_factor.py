"""Whole-path parity: the CUDA randUTV through the C ABI against the oracle
(same matrices, same Gaussian matrices), plus the closed-form properties at
the full benchmark size."""
import math
import numpy as np
import pytest
import synth
import oracle
from oracle import checks
from gpu_util import require_gpu, dev, host
from parity_util import check_fp64_diag, oracle_backward_error

pytestmark = pytest.mark.gpu
SEED = 998


@pytest.fixture(scope="module")
def R():
    require_gpu()
    import paper_1703_00998_gb300 as R
    return R


def gauss(i, k, b):
    return synth.step_gaussian(SEED, i, k, b)


def run_gpu(R, A, b, q, inject=True, **kw):
    m, n = A.shape
    g = dev(synth.gaussian_stream(SEED, m, n, b)) if inject and synth.stream_layout(m, n, b)[1] > 0 else None
    out = R.factor(dev(A), b=b, q=q, g_inject=g, seed=SEED, **kw)
    U = host(out.U) if out.U is not None else None
    V = host(out.V) if out.V is not None else None
    return U, host(out.T), V, out.k_reached


def assert_valid_utv(A, U, T, V, b, k=None):
    assert checks.residual(A, U, T, V) <= 1e-13
    assert checks.orth_err(U) <= 1e-13 and checks.orth_err(V) <= 1e-13
    kk = min(A.shape) if k is None else k
    assert checks.lower_max(T[:, :kk]) == 0.0
    assert checks.block_offdiag_max(T, b, kk) == 0.0
    assert np.all(np.diag(T)[:kk] >= 0)


def diag_check(A, U, T, V, b, q, To=None, res_oracle=None, **kw):
    """|diag T| against the oracle's entry by entry under max(1e-10 |d_ref|, 4 s_j), s_j the
    oracle's measured sensitivity to a perturbation of the two sides' backward errors."""
    res = checks.residual(A, U, T, V) if U is not None else 2.0 ** -50
    r = check_fp64_diag(A, T, res, b, q, gauss, To=To, res_oracle=res_oracle, **kw)
    print(f"|diag T| vs oracle: {r}")
    return r


def test_config_500_b32_q1_injected(R):
    A = synth.make_matrix("exp50", 500, 500, 1703001)
    U, T, V, kr = run_gpu(R, A, 32, 1)
    Uo, To, Vo, kro = oracle.randutv(A, 32, 1, gauss)
    assert kr == kro == 500
    assert diag_check(A, U, T, V, 32, 1, To=To, res_oracle=checks.residual(A, Uo, To, Vo))["ok"]
    assert_valid_utv(A, U, T, V, 32)
    # with the same order/sign conventions the factors agree entry by entry
    assert np.max(np.abs(T - To)) <= 1e-9
    assert np.max(np.abs(U - Uo)) <= 1e-9
    assert np.max(np.abs(V - Vo)) <= 1e-9


def test_config_500_philox_stream(R):
    # the device Philox/Box-Muller stream instead of injected G
    A = synth.make_matrix("exp50", 500, 500, 1703001)
    U, T, V, _ = run_gpu(R, A, 32, 1, inject=False)
    assert diag_check(A, U, T, V, 32, 1)["ok"]
    assert_valid_utv(A, U, T, V, 32)


@pytest.mark.parametrize("m,n,b,q", [
    (300, 200, 32, 1), (200, 300, 32, 1), (333, 333, 64, 0), (257, 257, 32, 2), (100, 100, 128, 1),
    (130, 130, 1, 1), (65, 33, 16, 1), (33, 65, 16, 1), (1, 1, 4, 1), (3, 2, 1, 1), (2, 3, 1, 1),
    (129, 129, 64, 1), (64, 64, 64, 1),
])
def test_shapes_against_oracle(R, m, n, b, q):
    A = synth.make_matrix("exp50", m, n, 7 + m + n)
    U, T, V, kr = run_gpu(R, A, b, q)
    Uo, To, Vo, kro = oracle.randutv(A, b, q, gauss)
    assert kr == kro
    assert diag_check(A, U, T, V, b, q, To=To, res_oracle=checks.residual(A, Uo, To, Vo))["ok"]
    assert_valid_utv(A, U, T, V, min(b, m, n))


def test_full_svd_case_matches_spectrum(R):
    A = synth.make_matrix("exp5", 48, 48, 3)
    s = synth.spectrum("exp5", 48)
    U, T, V, _ = run_gpu(R, A, 64, 1)
    np.testing.assert_allclose(np.diag(T), s, rtol=1e-12)
    _, sj, _ = oracle.jacobi_svd(A)
    np.testing.assert_allclose(np.diag(T), sj, rtol=1e-12)


def test_tolerance_stop(R):
    # sigma_j = exp(-j/6): a steep spectrum whose middle diagonal entries move by ~1e3 u ||A||
    # under rounding-level perturbation (measured on the oracle itself)
    A = synth.make_matrix("exp", 400, 400, 8, r=6.0)
    U, T, V, kr = run_gpu(R, A, 32, 1, tol=1e-5)
    Uo, To, Vo, kro = oracle.randutv(A, 32, 1, gauss, tol=1e-5)
    assert kr == kro and 0 < kr < 400
    assert checks.residual(A, U, T, V) <= 1e-13
    r = check_fp64_diag(A, T[:, :kr], checks.residual(A, U, T, V), 32, 1, gauss, To=To[:, :kr],
                        res_oracle=checks.residual(A, Uo, To, Vo), tol=1e-5)
    print(f"|diag T| vs oracle: {r}")
    assert r["ok"] and r["n"] == kr


def test_t_only(R):
    # T-only mode (Table 4) computes the same T; the panel QR adds its
    # cross-CTA partial sums with atomics, so two runs agree to rounding level
    A = synth.make_matrix("inv", 300, 300, 5)
    _, T1, _, _ = run_gpu(R, A, 32, 1)
    U, T2, V, _ = run_gpu(R, A, 32, 1, form_uv=False)
    assert U is None and V is None
    assert np.max(np.abs(T1 - T2)) <= 1e-12 * np.abs(T1).max()


def test_non_finite_input_is_reported(R):
    from paper_1703_00998_gb300 import RandutvError, native
    A = np.ones((40, 40))
    A[3, 5] = np.nan
    with pytest.raises(RandutvError) as e:
        R.factor(dev(A), b=8, q=1)
    assert e.value.status == native.ENAN


def test_zero_matrix(R):
    U, T, V, kr = run_gpu(R, np.zeros((70, 70)), 16, 1)
    assert np.all(T == 0)
    assert checks.orth_err(U) <= 1e-14 and checks.orth_err(V) <= 1e-14


@pytest.mark.parametrize("q", [0, 1, 2])
@pytest.mark.parametrize("kind", ["exp200", "inv", "gauss"])
def test_n4000_b128_against_oracle(R, kind, q):
    """n = 4000, b = 128, q in {0, 1, 2}, the three spectra: every |diag T| entry against the
    oracle's (same Philox G), and the FP64 bounds on residual and orthogonality."""
    import torch
    n = 4000
    A = synth.make_matrix(kind, n, n, 1703002 + ["exp200", "inv", "gauss"].index(kind))
    out = R.factor(dev(A), b=128, q=q, seed=SEED)
    assert out.k_reached == n
    At = dev(A)
    res = float(torch.linalg.norm(At - out.U @ out.T @ out.V.T) / torch.linalg.norm(At))
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    assert res <= 1e-13
    assert float((out.U.T @ out.U - eye).abs().max()) <= 1e-13
    assert float((out.V.T @ out.V - eye).abs().max()) <= 1e-13
    assert float(torch.tril(out.T, -1).abs().max()) == 0.0
    T = host(out.T)
    del out, At
    res_o, To, _ = oracle_backward_error(A, 128, q, gauss)
    r = check_fp64_diag(A, T, res, 128, q, gauss, To=To, res_oracle=res_o)
    print(f"n={n} {kind} q={q}: residual {res:.2e} (oracle {res_o:.2e}); |diag T| vs oracle: {r}")
    assert r["ok"]


@pytest.mark.parametrize("kind", ["exp200", "gauss"])
def test_n8000_b128_q1_full_size(R, kind):
    """The benchmark workload (and an iid Gaussian matrix of the same size):
    properties at full size and the first block against the oracle's first
    step (the diagonal block of step 1 is final)."""
    import torch
    n, b = 8000, 128
    A = synth.make_matrix(kind, n, n, 1703002 + ["exp200", "inv", "gauss"].index(kind), device="cuda")
    Ah = host(A)
    out = R.factor(A, b=b, q=1, seed=SEED)
    U, T, V = out.U, out.T, out.V
    assert out.k_reached == n
    res = float(torch.linalg.norm(A - U @ T @ V.T) / torch.linalg.norm(A))
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    assert res <= 1e-13
    assert float((U.T @ U - eye).abs().max()) <= 1e-13
    assert float((V.T @ V - eye).abs().max()) <= 1e-13
    assert float(torch.tril(T, -1).abs().max()) == 0.0
    d = torch.diagonal(T)
    assert float(d.min()) >= 0
    assert abs(float(torch.linalg.norm(T) / torch.linalg.norm(A)) - 1) <= 1e-13
    _, T1, _, _ = oracle.randutv(Ah, b, 1, gauss, form_uv=False, max_steps=1)
    np.testing.assert_allclose(host(d[:b]), np.diag(T1)[:b], rtol=1e-10)


def test_n8000_closed_forms(R):
    """sigma_j = 1/j at n = 8000: sum_j log t_jj = log|det A| = -log n! and
    ||T||_F^2 = sum_j j^-2 (T triangular, U and V orthogonal)."""
    import torch
    n, b = 8000, 128
    A = synth.make_matrix("inv", n, n, 1703003, device="cuda")
    out = R.factor(A, b=b, q=1, seed=SEED)
    d = torch.diagonal(out.T)
    logdet = float(torch.log(d).sum())
    assert abs(logdet + math.lgamma(n + 1)) <= 1e-10 * n
    s = synth.spectrum("inv", n)
    assert abs(float(torch.linalg.norm(out.T)) / np.linalg.norm(s) - 1) <= 1e-13
    assert float(torch.tril(out.T, -1).abs().max()) == 0.0


def test_fp64_overlap_off_matches(R):
    # the U/V lane only reorders independent work: the same factors either
    # way, up to the run-to-run rounding of the panel QR's atomic sums
    A = synth.make_matrix("exp50", 600, 600, 31)
    g = dev(synth.gaussian_stream(SEED, 600, 600, 64))
    a = R.factor(dev(A), b=64, q=1, g_inject=g, overlap=True)
    c = R.factor(dev(A), b=64, q=1, g_inject=g, overlap=False)
    for x, y in ((a.T, c.T), (a.U, c.U), (a.V, c.V)):
        assert float((x - y).abs().max()) <= 1e-10


def test_fp64_emulation_matches_dfma(R):
    # the Ozaki-scheme products are FP64-accurate: the same factorization as
    # the DFMA GEMM to FP64 rounding (both against the same injected G)
    A = synth.make_matrix("exp50", 700, 700, 41)
    g = dev(synth.gaussian_stream(SEED, 700, 700, 64))
    a = R.factor(dev(A), b=64, q=1, g_inject=g, fp64_emulation=True)
    c = R.factor(dev(A), b=64, q=1, g_inject=g, fp64_emulation=False)
    from diag_bound import compare
    from parity_util import oracle_sensitivity
    ra = checks.residual(A, host(a.U), host(a.T), host(a.V))
    rc = checks.residual(A, host(c.U), host(c.T), host(c.V))
    s = oracle_sensitivity(A, 64, 1, gauss, ra + rc)
    r = compare(host(a.T).diagonal(), host(c.T).diagonal(), s, 1e-10, 4.0)
    print(f"|diag T| Ozaki vs DFMA: {r}")
    assert r["ok"]


@pytest.mark.parametrize("m,n,b,p,q", [(500, 500, 32, 5, 1), (400, 300, 32, 10, 0), (300, 400, 64, 8, 2),
                                       (1000, 1000, 128, 16, 1), (200, 200, 32, 100, 1)])
def test_oversampling_against_oracle(R, m, n, b, p, q):
    """Over-sampling p (Remark "Oversampling") on the same injected G of
    width b + p: |diag T| to the oracle, FP64 residual and orthogonality;
    the last case has b + p above the trailing width of late steps."""
    A = synth.make_matrix("exp50", m, n, 1703005 + m + p)
    g = dev(synth.gaussian_stream(SEED, m, n, b, p)) if synth.stream_layout(m, n, b, p)[1] > 0 else None
    f = R.factor(dev(A), b=b, q=q, g_inject=g, p=p)
    U, T, V = host(f.U), host(f.T), host(f.V)
    assert f.k_reached == min(m, n)
    assert checks.residual(A, U, T, V) <= 1e-13
    assert checks.orth_err(U) <= 1e-13 and checks.orth_err(V) <= 1e-13
    assert checks.lower_max(T) == 0.0
    res_o, To, _ = oracle_backward_error(A, b, q, gauss, p=p)
    r = check_fp64_diag(A, T, checks.residual(A, U, T, V), b, q, gauss, To=To, res_oracle=res_o, p=p)
    print(f"|diag T| vs oracle (p = {p}): {r}")
    assert r["ok"]
