"""Pins of the Fig. 4 oracle (oracle.randutv)."""
import numpy as np
import pytest
import oracle
import synth
from oracle import checks
import oracle_pins as P


@pytest.mark.parametrize("pin", P.PINS, ids=[p.__name__ for p in P.PINS])
def test_pin(pin):
    assert pin(oracle.randutv)


def test_config_500_b32_q1():
    # 500 x 500, sigma_j = exp(-j/50), b = 32, q = 1: 16 steps, last one 20 x 20
    A = synth.make_matrix("exp50", 500, 500, 1703001)
    s = synth.spectrum("exp50", 500)
    U, T, V, kr = oracle.randutv(A, 32, 1, P.gauss)
    assert kr == 500
    assert checks.residual(A, U, T, V) < 1e-13
    assert checks.orth_err(U) < 1e-13 and checks.orth_err(V) < 1e-13
    assert checks.lower_max(T) == 0.0 and checks.block_offdiag_max(T, 32) == 0.0
    d = np.diag(T)
    assert abs(np.sum(np.log(d)) - np.sum(np.log(s))) < 1e-10
    # the first diagonal block holds the singular values of a b x b section of
    # an orthogonal transform of A, so interlacing bounds them by sigma_1..sigma_b
    assert np.all(d[:32] <= s[:32] * (1 + 1e-12))
    # and with q = 1 they track the spectrum closely (Fig. 9)
    np.testing.assert_allclose(d[:20], s[:20], rtol=0.1)


@pytest.mark.parametrize("m,n,b", [(90, 50, 16), (50, 90, 16), (64, 48, 16), (33, 17, 5), (17, 33, 5), (65, 65, 64), (3, 2, 1), (1, 1, 4)])
def test_rectangular_and_ragged(m, n, b):
    A = synth.make_matrix("exp50", m, n, 21)
    U, T, V, kr = oracle.randutv(A, b, 1, P.gauss)
    assert kr == min(m, n)
    assert checks.residual(A, U, T, V) < 1e-13
    assert checks.orth_err(U) < 1e-13 and checks.orth_err(V) < 1e-13
    assert checks.lower_max(T) == 0.0
    s = np.linalg.svd(A, compute_uv=False)
    assert abs(np.linalg.norm(T) - np.linalg.norm(s)) < 1e-13 * np.linalg.norm(s)
    assert np.all(np.diag(T) >= 0)


def test_tolerance_early_stop():
    n, b = 120, 16
    A = synth.make_matrix("exp", n, n, 8, r=6.0)
    s = synth.spectrum("exp", n, r=6.0)
    tol = 1e-5
    U, T, V, kr = oracle.randutv(A, b, 1, P.gauss, tol=tol)
    assert kr % b == 0 and 0 < kr < n
    # the stop rule: trailing block small at the stop, not small one step before
    assert np.linalg.norm(T[kr:, kr:]) <= tol * np.linalg.norm(A)
    assert checks.residual(A, U, T, V) < 1e-13
    assert checks.lower_max(T[:, :kr]) == 0.0
    # ||T(k+1:, k+1:)|| >= sigma_{k+1} (rank-k error is at least optimal)
    assert np.linalg.norm(T[kr:, kr:], 2) >= s[kr] * (1 - 1e-12)


def test_t_only_mode_matches():
    A = synth.make_matrix("exp50", 70, 70, 4)
    _, T1, _, _ = oracle.randutv(A, 16, 1, P.gauss)
    U, T2, V, _ = oracle.randutv(A, 16, 1, P.gauss, form_uv=False)
    assert U is None and V is None
    np.testing.assert_array_equal(T1, T2)


def test_flop_formula():
    # Section 5.4: (5+2q) m n^2 - (3+2q) n^3/3; with U, V: (24+4q)/3 n^3 square
    assert oracle.flops_randutv(8000, 8000, 128, 1, form_uv=False) == pytest.approx(16 / 3 * 8000 ** 3)
    assert oracle.flops_randutv(8000, 8000, 128, 1) == pytest.approx(28 / 3 * 8000 ** 3)
    assert oracle.flops_randutv(8000, 8000, 128, 1) == pytest.approx(4.779e12, rel=1e-3)
