"""Pins of oracle.householder against LAPACK (scipy) and brute force."""
import numpy as np
import pytest
import scipy.linalg
import scipy.linalg.lapack as lapack
import oracle


@pytest.mark.parametrize("x", [
    [3.0, 4.0, 0.0, -1.0], [-2.0, 1e-3, 5.0], [0.0, 1.0, 1.0], [2.5], [-1.0, 0.0, 0.0], [1e-200, 3e-200],
])
def test_house_matches_dlarfg(x):
    x = np.array(x)
    v, tau, beta = oracle.house(x)
    a, xv, t = lapack.dlarfg(x.size, x[0], x[1:].copy() if x.size > 1 else np.zeros(1))
    assert tau == pytest.approx(t, rel=1e-15, abs=0)
    assert beta == pytest.approx(a, rel=1e-15, abs=0)
    if x.size > 1:
        np.testing.assert_allclose(v[1:], xv[:x.size - 1], rtol=1e-14)
    H = np.eye(x.size) - tau * np.outer(v, v)
    e = np.zeros(x.size)
    e[0] = beta
    np.testing.assert_allclose(H @ x, e, atol=1e-14 * x.size * np.max(np.abs(x)))


@pytest.mark.parametrize("shape", [(40, 8), (33, 33), (100, 17), (5, 1)])
def test_householder_qr_matches_dgeqrf(shape):
    B = np.random.default_rng(1).standard_normal(shape)
    V, tau, R = oracle.householder_qr(B)
    qr, tl, _, info = lapack.dgeqrf(B)
    assert info == 0
    w = shape[1]
    np.testing.assert_allclose(tau, tl, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(R, np.triu(qr[:w, :w]), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(np.tril(V, -1), np.tril(qr, -1), rtol=1e-12, atol=1e-13)
    assert np.all(np.diag(V) == 1.0) and np.all(np.triu(V, 1) == 0.0)


def _explicit_product(V, tau):
    k, w = V.shape
    Q = np.eye(k)
    for j in range(w):
        Q = Q @ (np.eye(k) - tau[j] * np.outer(V[:, j], V[:, j]))
    return Q


@pytest.mark.parametrize("shape", [(30, 6), (64, 16), (17, 17)])
def test_tfactor_equals_reflector_product(shape):
    B = np.random.default_rng(2).standard_normal(shape)
    V, tau, R = oracle.householder_qr(B)
    S = oracle.tfactor(V, tau)
    assert np.all(np.tril(S, -1) == 0)
    Q = np.eye(shape[0]) - V @ S @ V.T
    np.testing.assert_allclose(Q, _explicit_product(V, tau), atol=1e-13)
    # the same Q that LAPACK's dorgqr forms, and Q^T B = [R; 0]
    Qc, Rc = np.linalg.qr(B, mode="complete")
    np.testing.assert_allclose(Q, Qc, atol=1e-13)
    QtB = Q.T @ B
    np.testing.assert_allclose(QtB[:shape[1]], R, atol=1e-13)
    np.testing.assert_allclose(QtB[shape[1]:], 0, atol=1e-13)


def test_wy_apply_right_and_left():
    rng = np.random.default_rng(3)
    V, tau, _ = oracle.householder_qr(rng.standard_normal((25, 7)))
    S = oracle.tfactor(V, tau)
    Q = _explicit_product(V, tau)
    C = rng.standard_normal((11, 25))
    np.testing.assert_allclose(oracle.wy_apply_right(C, V, S), C @ Q, atol=1e-13)
    D = rng.standard_normal((25, 9))
    np.testing.assert_allclose(oracle.wy_apply_left_t(D, V, S), Q.T @ D, atol=1e-13)


def test_zero_panel_gives_identity():
    V, tau, R = oracle.householder_qr(np.zeros((10, 4)))
    assert np.all(tau == 0) and np.all(R == 0)
    S = oracle.tfactor(V, tau)
    np.testing.assert_array_equal(np.eye(10) - V @ S @ V.T, np.eye(10))
