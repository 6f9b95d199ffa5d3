"""Per-kernel parity of the CUDA building blocks against the oracle and the
shared input generators (same seeded inputs, element by element)."""
import numpy as np
import pytest
import synth
import oracle
from gpu_util import require_gpu, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    require_gpu()
    import paper_1703_00998_gb300 as R
    return R


@pytest.mark.parametrize("step,k,b", [(1, 500, 32), (7, 37, 5), (3, 1, 1), (16, 8000, 128)])
def test_philox_words_bit_exact(R, step, k, b):
    w = host(R.philox_words(998, step, k, b))
    x = synth.gauss.step_words(998, step, k, b)   # each (ceil(k/2), b)
    for t in range(4):
        np.testing.assert_array_equal(w[:, :, t].T, x[t].astype(np.int64))


@pytest.mark.parametrize("seed", [998, 2 ** 40 + 17])
@pytest.mark.parametrize("step,k,b", [(1, 500, 32), (2, 33, 7), (5, 4001, 128)])
def test_gaussian_matches_generator(R, seed, step, k, b):
    g = host(R.gaussian(seed, step, k, b))
    ref = synth.step_gaussian(seed, step, k, b)
    # Same uniforms (bit-exact words); the device takes sincospi(2 u2) and the
    # host cos(fl(2 pi u2)): |dz| <= r |d theta| + |z| few ulps with
    # |d theta| <= 2 pi 2^-52 and r = sqrt(-2 ln u1) <= sqrt(2 ln 2^53) < 8.6.
    np.testing.assert_allclose(g, ref, rtol=1e-14, atol=8.6 * 2 * np.pi * 2.0 ** -52)


SHAPES = [(1, 1, 1), (63, 65, 17), (130, 129, 64), (1000, 128, 3000), (128, 1000, 3000), (257, 300, 5)]


@pytest.mark.parametrize("ta", [False, True])
@pytest.mark.parametrize("tb", [False, True])
@pytest.mark.parametrize("m,n,k", SHAPES)
def test_dgemm(R, ta, tb, m, n, k):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A = rng.standard_normal((k, m) if ta else (m, k))
    B = rng.standard_normal((n, k) if tb else (k, n))
    C = rng.standard_normal((m, n))
    ref = 1.5 * (A.T if ta else A) @ (B.T if tb else B) - 0.5 * C
    out = host(R.dgemm(dev(A), dev(B), ta=ta, tb=tb, alpha=1.5, beta=-0.5, C=dev(C)))
    bound = 4 * k * 2.0 ** -53 * (np.abs(A).max() * np.abs(B).max() * k + 1)
    assert np.max(np.abs(out - ref)) <= bound
    out0 = host(R.dgemm(dev(A), dev(B), ta=ta, tb=tb))
    np.testing.assert_allclose(out0, (A.T if ta else A) @ (B.T if tb else B), atol=bound)


@pytest.mark.parametrize("ta", [False, True])
@pytest.mark.parametrize("tb", [False, True])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (130, 129, 64), (1000, 128, 3000), (128, 1000, 8000), (257, 300, 5)])
def test_sgemm(R, ta, tb, m, n, k):
    import torch
    rng = np.random.default_rng(m + 3 * n + 7 * k)
    A = rng.standard_normal((k, m) if ta else (m, k)).astype(np.float32)
    B = rng.standard_normal((n, k) if tb else (k, n)).astype(np.float32)
    C = rng.standard_normal((m, n)).astype(np.float32)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = 1.5 * (A64.T if ta else A64) @ (B64.T if tb else B64) - 0.5 * C.astype(np.float64)
    out = host(R.sgemm(dev(A), dev(B), ta=ta, tb=tb, alpha=1.5, beta=-0.5, C=dev(C))).astype(np.float64)
    # FP32 accumulation of chunks of <= 1024 products, chunks summed in FP64
    bound = (min(k, 1024) + 2) * 2.0 ** -24 * (np.abs(A64) .max() * np.abs(B64).max() * k * 1.5 + 1)
    assert np.max(np.abs(out - ref)) <= bound


@pytest.mark.parametrize("k,w", [(500, 32), (37, 37), (8000, 128), (300, 1), (1, 1), (4000, 128), (200, 64)])
def test_panel_qr(R, k, w):
    P = np.random.default_rng(k + w).standard_normal((k, w)) * np.logspace(0, -3, w)[None, :]
    Pout, tau, Vexp, S = (host(x) for x in R.panel_qr(dev(P)))
    Vo, to, Ro = oracle.householder_qr(P)
    So = oracle.tfactor(Vo, to)
    Vo[:, to == 0.0] = 0.0   # the explicit vectors of an identity reflector are stored as zero
    np.testing.assert_allclose(tau, to, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(np.triu(Pout[:w]), Ro, rtol=1e-11, atol=1e-13 * np.abs(Ro).max())
    np.testing.assert_allclose(Vexp, Vo, atol=1e-11)
    np.testing.assert_allclose(np.tril(Pout, -1), np.tril(Vo, -1), atol=1e-11)
    np.testing.assert_allclose(S, So, rtol=1e-10, atol=1e-11)
    Q = np.eye(k) - Vexp @ S @ Vexp.T if k <= 600 else None
    if Q is not None:
        assert np.max(np.abs(Q.T @ Q - np.eye(k))) < 1e-13


def test_panel_qr_zero_and_dependent_columns(R):
    P = np.random.default_rng(3).standard_normal((50, 6))
    P[:, 2] = 0.0            # zero column -> tau = 0 there
    P[:, 4] = P[:, 1]        # dependent column: its reflector is built from rounding noise
    Pout, tau, Vexp, S = (host(x) for x in R.panel_qr(dev(P)))
    Vo, to, Ro = oracle.householder_qr(P)
    # determined part: reflectors 0..3 and rows 0..3 of R
    np.testing.assert_allclose(tau[:4], to[:4], atol=1e-13)
    Vo[:, to == 0.0] = 0.0
    np.testing.assert_allclose(Vexp[:, :4], Vo[:, :4], atol=1e-12)
    assert tau[2] == 0.0 and np.all(Vexp[:, 2] == 0.0)
    np.testing.assert_allclose(np.triu(Pout[:4]), np.triu(Ro[:4]), atol=1e-13)
    assert abs(Pout[4, 4]) < 1e-14          # the dependent column leaves a zero pivot
    Q = np.eye(50) - Vexp @ S @ Vexp.T
    assert np.max(np.abs(Q.T @ Q - np.eye(50))) < 1e-14
    np.testing.assert_allclose(Q.T @ P, np.vstack([np.triu(Pout[:6]), np.zeros((44, 6))]), atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 5, 20, 32, 127, 128])
def test_small_svd(R, p):
    A = synth.make_matrix("exp5", p, p, 11 + p)
    M = np.linalg.qr(A)[1] if p > 1 else A   # upper triangular like R11
    Us, d, Vs = (host(x) for x in R.small_svd(dev(M)))
    Uo, do, Vo = oracle.svd_small(M)
    np.testing.assert_allclose(d, do, rtol=1e-12, atol=1e-15 * do[0])
    assert np.all(np.diff(d) <= 0) and np.all(d >= 0)
    assert np.max(np.abs(Us.T @ Us - np.eye(p))) < 1e-13
    assert np.max(np.abs(Vs.T @ Vs - np.eye(p))) < 1e-13
    np.testing.assert_allclose(Us @ np.diag(d) @ Vs.T, M, atol=1e-14 * p)
    # same order and sign convention as the oracle (spectrum exp(-j/5) is well separated)
    np.testing.assert_allclose(Vs, Vo, atol=1e-9)
    np.testing.assert_allclose(Us, Uo, atol=1e-9)


def test_small_svd_zero_and_rank_deficient(R):
    Us, d, Vs = (host(x) for x in R.small_svd(dev(np.zeros((8, 8)))))
    assert np.all(d == 0)
    assert np.max(np.abs(Us.T @ Us - np.eye(8))) < 1e-15
    M = np.outer(np.arange(1.0, 7.0), np.ones(6))
    Us, d, Vs = (host(x) for x in R.small_svd(dev(M)))
    np.testing.assert_allclose(d[0], np.linalg.norm(M, 2), rtol=1e-14)
    assert np.all(d[1:] <= 1e-14 * d[0])
    assert np.max(np.abs(Us.T @ Us - np.eye(6))) < 1e-13
    np.testing.assert_allclose(Us @ np.diag(d) @ Vs.T, M, atol=1e-13)


@pytest.mark.parametrize("scale", [1e-16, 1e-60, 1e40])
def test_small_svd_scale_invariance(R, scale):
    # blocks at the rounding level of a factorization (w_i . w_j far below the
    # FP32 range) converge as fast and as accurately as unit-scale ones
    A = synth.make_matrix("exp50", 64, 64, 77)
    M = np.linalg.qr(A)[1] * scale
    Us, d, Vs = (host(x) for x in R.small_svd(dev(M)))
    Uo, do, Vo = oracle.svd_small(M)
    np.testing.assert_allclose(d, do, rtol=1e-12, atol=1e-15 * do[0])
    assert np.max(np.abs(Us.T @ Us - np.eye(64))) < 1e-13
    assert np.max(np.abs(Vs.T @ Vs - np.eye(64))) < 1e-13
    np.testing.assert_allclose(Us @ np.diag(d) @ Vs.T, M, atol=1e-13 * do[0])


def test_small_svd_sweep_cap_reports_noconv(R):
    from paper_1703_00998_gb300 import RandutvError, native
    M = np.random.default_rng(1).standard_normal((64, 64))
    with pytest.raises(RandutvError) as e:
        R.small_svd(dev(M), max_sweeps=1)
    assert e.value.status == native.ENOCONV
