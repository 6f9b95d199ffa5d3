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


def diag_rel(T, To, normA=None):
    """Largest |d_j - d_j^o| / (|d_j^o| + floor), floor = n u ||A||_2 / 1e-10.

    The bar "|diag T| to 1e-10 relative" is read with an absolute floor of
    n u ||A||_2 (u = 2^-53): both sides are backward stable, so an entry near
    the rounding level of the whole factorization is fixed only to about
    u ||A|| in absolute terms, by either implementation."""
    d, do = np.abs(np.diag(T)), np.abs(np.diag(To))
    if normA is None:
        normA = float(np.max(do)) if do.size else 0.0
    floor = len(do) * 2.0 ** -53 * normA / 1e-10
    return float(np.max(np.abs(d - do) / np.maximum(do + floor, 1e-300)))


def test_config_500_b32_q1_injected(R):
    A = synth.make_matrix("exp50", 500, 500, 1703001)
    U, T, V, kr = run_gpu(R, A, 32, 1)
    Uo, To, Vo, kro = oracle.randutv(A, 32, 1, gauss)
    assert kr == kro == 500
    assert diag_rel(T, To) <= 1e-10
    assert_valid_utv(A, U, T, V, 32)
    # with the same order/sign conventions the factors agree entry by entry
    assert np.max(np.abs(T - To)) <= 1e-9
    assert np.max(np.abs(U - Uo)) <= 1e-9
    assert np.max(np.abs(V - Vo)) <= 1e-9


def test_config_500_philox_stream(R):
    # the device Philox/Box-Muller stream instead of injected G
    A = synth.make_matrix("exp50", 500, 500, 1703001)
    U, T, V, _ = run_gpu(R, A, 32, 1, inject=False)
    _, To, _, _ = oracle.randutv(A, 32, 1, gauss)
    assert diag_rel(T, To) <= 1e-10
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
    assert diag_rel(T, To) <= 1e-10
    assert_valid_utv(A, U, T, V, min(b, m, n))


def test_full_svd_case_matches_spectrum(R):
    A = synth.make_matrix("exp5", 48, 48, 3)
    s = synth.spectrum("exp5", 48)
    U, T, V, _ = run_gpu(R, A, 64, 1)
    np.testing.assert_allclose(np.diag(T), s, rtol=1e-12)
    _, sj, _ = oracle.jacobi_svd(A)
    np.testing.assert_allclose(np.diag(T), sj, rtol=1e-12)


def oracle_sensitivity(A, b, q, **kw):
    """max_j |d_j(A) - d_j(A + E)| of the oracle itself for a random E with
    ||E||_2 = u ||A||_2: how far rounding alone moves the diagonal of T."""
    rng = np.random.default_rng(12345)
    E = rng.standard_normal(A.shape)
    E *= 2.0 ** -53 * np.linalg.norm(A, 2) / np.linalg.norm(E, 2)
    _, T1, _, k1 = oracle.randutv(A, b, q, gauss, **kw)
    _, T2, _, k2 = oracle.randutv(A + E, b, q, gauss, **kw)
    k = min(k1, k2)
    return float(np.max(np.abs(np.diag(T1)[:k] - np.diag(T2)[:k])))


def test_tolerance_stop(R):
    # sigma_j = exp(-j/6): a steep spectrum whose middle diagonal entries move
    # by ~1e3 u ||A|| under rounding-level perturbation (measured on the
    # oracle itself); the bar is 1e-10 relative or 10x that sensitivity.
    A = synth.make_matrix("exp", 400, 400, 8, r=6.0)
    U, T, V, kr = run_gpu(R, A, 32, 1, tol=1e-5)
    Uo, To, Vo, kro = oracle.randutv(A, 32, 1, gauss, tol=1e-5)
    assert kr == kro and 0 < kr < 400
    assert checks.residual(A, U, T, V) <= 1e-13
    d, do = np.diag(T)[:kr], np.diag(To)[:kr]
    sens = oracle_sensitivity(A, 32, 1, tol=1e-5)
    assert np.all(np.abs(d - do) <= np.maximum(1e-10 * do, 10 * sens))


def test_t_only(R):
    # T-only mode (Table 4) computes the same T; the panel QR adds its
    # cross-CTA partial sums with atomics, so two runs agree to rounding level
    A = synth.make_matrix("inv", 300, 300, 5)
    _, T1, _, _ = run_gpu(R, A, 32, 1)
    U, T2, V, _ = run_gpu(R, A, 32, 1, form_uv=False)
    assert U is None and V is None
    assert np.max(np.abs(T1 - T2)) <= 1e-12 * np.abs(T1).max()
    assert diag_rel(T2, T1) <= 1e-10


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


@pytest.mark.parametrize("kind", ["exp200", "inv", "gauss"])
def test_n4000_b128_q1_against_oracle(R, kind):
    n = 4000
    A = synth.make_matrix(kind, n, n, 1703002 + ["exp200", "inv", "gauss"].index(kind))
    U, T, V, kr = run_gpu(R, A, 128, 1)
    _, To, _, _ = oracle.randutv(A, 128, 1, gauss, form_uv=False)
    assert kr == n
    assert diag_rel(T, To) <= 1e-10
    import torch
    At, Ut, Tt, Vt = (dev(x) for x in (A, U, T, V))
    res = float(torch.linalg.norm(At - Ut @ Tt @ Vt.T) / torch.linalg.norm(At))
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    assert res <= 1e-13
    assert float((Ut.T @ Ut - eye).abs().max()) <= 1e-13
    assert float((Vt.T @ Vt - eye).abs().max()) <= 1e-13
    assert float(torch.tril(Tt, -1).abs().max()) == 0.0


def test_n8000_b128_q1_full_size(R):
    """The benchmark workload: properties at full size and the first block
    against the oracle's first step (the diagonal block of step 1 is final)."""
    import torch
    n, b = 8000, 128
    A = synth.make_matrix("exp200", n, n, 1703002, device="cuda")
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
    da, dc = host(a.T).diagonal(), host(c.T).diagonal()
    nA = np.linalg.norm(A, 2)
    assert np.max(np.abs(np.abs(da) - np.abs(dc)) / (np.abs(dc) + 700 * 2.0 ** -53 * nA / 1e-10)) <= 1e-10


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
    _, To, _, _ = oracle.randutv(A, b, q, gauss, form_uv=False, p=p)
    assert diag_rel(T, To, float(np.linalg.norm(A, 2))) <= 1e-10
