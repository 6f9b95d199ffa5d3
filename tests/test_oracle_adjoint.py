"""The rank-k map of randUTV and its oracle derivative, on CPU.

Pins: (1) the torch restatement of the steps gives the same A_k as the
numpy oracle; (2) A_k = Q Q^T A with Q an orthonormal basis of A V(:, 1:k)
(the map depends only on span(U(:, 1:k)) = span(A V(:, 1:k)), not on the
small SVDs); (3) the vector-Jacobian product against central differences
(h = 1e-6) for random directions and cotangents, square and rectangular;
(4) a closed form: for A of exact rank k the first k/b steps capture its
column space, A_k = A, and dA_k = dE - (I - P_col) dE (I - P_row) (P_col,
P_row the projectors on the column and row space of A), self-adjoint, for
any G; (5) the loss gradient of ||A - A_k||_F^2 against central
differences; (6) planted mistakes in the torch steps are caught."""
import numpy as np
import pytest
import synth
import oracle
from oracle import randutv_adjoint as RA

torch = pytest.importorskip("torch")
SEED = 998


def _g(step, k, w):
    return synth.step_gaussian(SEED, step, k, w)


def _mat(m, n, r, seed):
    return synth.make_matrix("exp", m, n, seed, r=r)


@pytest.mark.parametrize("m,n,b,k", [(48, 48, 8, 16), (60, 40, 8, 16), (40, 56, 8, 24)])
def test_torch_steps_match_numpy_oracle(m, n, b, k):
    A = _mat(m, n, 10.0, 3)
    Ak = oracle.rank_k_approx(A, b, 1, _g, k)
    Ak2, _ = oracle.rank_k_vjp(A, b, 1, _g, k, np.zeros_like(A))
    np.testing.assert_allclose(Ak2, Ak, atol=1e-13 * np.abs(A).max())


@pytest.mark.parametrize("m,n,b,k", [(48, 48, 8, 16), (60, 40, 8, 16)])
def test_map_is_projection_on_sketched_range(m, n, b, k):
    A = _mat(m, n, 10.0, 4)
    U, T, V, _ = oracle.randutv(A, b, 1, _g, max_steps=k // b)
    Q, _ = np.linalg.qr(A @ V[:, :k])
    np.testing.assert_allclose(oracle.rank_k_approx(A, b, 1, _g, k), Q @ (Q.T @ A), atol=1e-12)


@pytest.mark.parametrize("m,n,b,k,q", [(48, 48, 8, 16, 1), (60, 40, 8, 16, 1), (40, 56, 8, 24, 1), (48, 48, 8, 16, 0),
                                     (50, 30, 6, 18, 2)])
def test_vjp_against_central_differences(m, n, b, k, q):
    A = _mat(m, n, 10.0, 5)
    rng = np.random.default_rng(7)
    C = rng.standard_normal((m, n))
    _, g = oracle.rank_k_vjp(A, b, q, _g, k, C)
    h = 1e-6
    for _ in range(3):
        E = rng.standard_normal((m, n))
        fp = np.sum(C * oracle.rank_k_approx(A + h * E, b, q, _g, k))
        fm = np.sum(C * oracle.rank_k_approx(A - h * E, b, q, _g, k))
        fd = (fp - fm) / (2 * h)
        assert abs(fd - np.sum(g * E)) <= 1e-6 * (abs(fd) + np.linalg.norm(g) * np.linalg.norm(E) * 1e-3), (fd,
                                                                                                          np.sum(g * E))


@pytest.mark.parametrize("m,n,b,k", [(40, 40, 8, 8), (40, 40, 8, 16), (50, 36, 6, 12)])
def test_exact_rank_closed_form(m, n, b, k):
    s = np.concatenate([np.exp(-np.arange(k) / 4.0), np.zeros(min(m, n) - k)])
    q1 = synth.haar_orthogonal(m, 11)
    q2 = synth.haar_orthogonal(n, 12)
    p = min(m, n)
    A = (q1[:, :p] * s[None, :]) @ q2[:, :p].T
    Pc = q1[:, :k] @ q1[:, :k].T
    Pr = q2[:, :k] @ q2[:, :k].T
    rng = np.random.default_rng(13)
    C = rng.standard_normal((m, n))
    Ak, g = oracle.rank_k_vjp(A, b, 1, _g, k, C)
    np.testing.assert_allclose(Ak, A, atol=1e-12)
    ref = C - (np.eye(m) - Pc) @ C @ (np.eye(n) - Pr)
    np.testing.assert_allclose(g, ref, atol=1e-9 * np.abs(C).max())


def test_loss_gradient_against_central_differences():
    m = n = 48
    A = _mat(m, n, 10.0, 6)
    L, gL = oracle.loss_grad(A, 8, 1, _g, 16)
    rng = np.random.default_rng(9)
    h = 1e-6
    for _ in range(3):
        E = rng.standard_normal((m, n))
        lp = np.sum((A + h * E - oracle.rank_k_approx(A + h * E, 8, 1, _g, 16)) ** 2)
        lm = np.sum((A - h * E - oracle.rank_k_approx(A - h * E, 8, 1, _g, 16)) ** 2)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - np.sum(gL * E)) <= 1e-6 * (abs(fd) + 1e-3 * np.linalg.norm(gL) * np.linalg.norm(E))


@pytest.mark.parametrize("mutation", ["tau_sign", "drop_power", "wrong_transpose"])
def test_planted_mistakes_are_caught(mutation, monkeypatch):
    m = n = 40
    A = _mat(m, n, 10.0, 8)
    Ak = oracle.rank_k_approx(A, 8, 1, _g, 16)
    if mutation == "tau_sign":
        orig = RA._house

        def bad(x):
            v, t, beta = orig(x)
            return v, -t, beta
        monkeypatch.setattr(RA, "_house", bad)
    elif mutation == "drop_power":
        monkeypatch.setattr(RA, "_steps", lambda A_, b, q, gauss, ns, f=RA._steps: f(A_, b, 0, gauss, ns))
    else:
        orig = RA._tfactor
        monkeypatch.setattr(RA, "_tfactor", lambda V, tau: orig(V, tau).T)
    Ak2, _ = oracle.rank_k_vjp(A, 8, 1, _g, 16, np.zeros_like(A))
    assert np.max(np.abs(Ak2 - Ak)) > 1e-8
