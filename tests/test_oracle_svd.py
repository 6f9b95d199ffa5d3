"""Pins of oracle.small_svd: library SVD, brute-force Jacobi, conventions."""
import numpy as np
import pytest
import oracle
import synth


@pytest.mark.parametrize("n", [1, 2, 7, 32, 48])
def test_jacobi_svd_against_library(n):
    A = np.random.default_rng(n).standard_normal((n + 3, n))
    U, s, V = oracle.jacobi_svd(A)
    ref = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(s, ref, rtol=1e-13)
    np.testing.assert_allclose(U @ np.diag(s) @ V.T, A, atol=1e-13 * ref[0])
    assert np.max(np.abs(U.T @ U - np.eye(n))) < 1e-13
    assert np.max(np.abs(V.T @ V - np.eye(n))) < 1e-13


def test_jacobi_rank_deficient_completes_basis():
    A = np.zeros((6, 4))
    A[:, 0] = 1.0
    U, s, V = oracle.jacobi_svd(A)
    assert s[0] == pytest.approx(np.sqrt(6)) and np.all(s[1:] == 0)
    assert np.max(np.abs(U.T @ U - np.eye(4))) < 1e-15


def test_svd_small_convention():
    A = synth.make_matrix("exp5", 20, 20, 5)
    R = np.linalg.qr(A)[1]
    Us, d, Vs = oracle.svd_small(R)
    assert np.all(np.diff(d) <= 0) and np.all(d >= 0)
    np.testing.assert_allclose(Us @ np.diag(d) @ Vs.T, R, atol=1e-13)
    for j in range(20):
        i = np.argmax(np.abs(Vs[:, j]))
        assert Vs[i, j] > 0
    Uj, sj, Vj = oracle.jacobi_svd(R)
    np.testing.assert_allclose(d, sj, rtol=1e-12, atol=1e-15 * d[0])
    Uj, Vj = oracle.sign_fix(Uj, Vj)
    np.testing.assert_allclose(np.abs(Vs), np.abs(Vj), atol=1e-10)
    np.testing.assert_allclose(Vs, Vj, atol=1e-10)
    np.testing.assert_allclose(Us, Uj, atol=1e-10)
