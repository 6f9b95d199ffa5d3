"""Battery of pins for a randUTV implementation with the oracle's signature.

Each pin compares against something other than the implementation itself:
closed forms for prescribed spectra, Theorem 1 (Section 5.3) recomputed with
independent numpy code, the b >= n special case (a plain SVD), the dense
Section 5.1 formulation, and exact structure.  ``run_battery`` returns the
names of the pins that fail, so a test can plant a mistake in a copy of the
oracle and check that some pin catches it.
"""
import numpy as np
import oracle
import synth
from oracle import checks

GSEED = 998


def gauss(i, k, b):
    return synth.step_gaussian(GSEED, i, k, b)


def _orth(Y):
    return np.linalg.qr(Y)[0]


def pin_structure_and_residual(f, n=96, b=16, q=1):
    A = synth.make_matrix("exp50", n, n, 1703001)
    U, T, V, kr = f(A, b, q, gauss)
    ok = kr == n
    ok &= checks.residual(A, U, T, V) < 1e-13
    ok &= checks.orth_err(U) < 1e-13 and checks.orth_err(V) < 1e-13
    ok &= checks.lower_max(T) == 0.0 and checks.block_offdiag_max(T, b) == 0.0
    d = np.diag(T)
    ok &= bool(np.all(d >= 0))
    for r0 in range(0, n, b):
        ok &= bool(np.all(np.diff(d[r0:r0 + b]) <= 0))
    return bool(ok)


def pin_logdet_and_frobenius(f, n=96, b=16, q=1):
    # sum log|t_jj| = log|det A| = sum log sigma_j; ||T||_F = ||sigma||_2
    A = synth.make_matrix("exp50", n, n, 42)
    s = synth.spectrum("exp50", n)
    _, T, _, _ = f(A, b, q, gauss)
    ok = abs(np.sum(np.log(np.abs(np.diag(T)))) - np.sum(np.log(s))) < 1e-11 * n
    ok &= abs(np.linalg.norm(T) / np.linalg.norm(s) - 1) < 1e-13
    ok &= np.allclose(np.linalg.svd(T, compute_uv=False), s, rtol=1e-11, atol=1e-14)
    return bool(ok)


def pin_full_svd_case(f, n=40):
    # b >= n: one full SVD, |diag T| = sigma(A)
    A = synth.make_matrix("exp5", n, n, 9)
    s = synth.spectrum("exp5", n)
    U, T, V, _ = f(A, n, 1, gauss)
    _, sj, _ = oracle.jacobi_svd(A)
    ok = np.allclose(np.diag(T), s, rtol=1e-12, atol=1e-15)
    ok &= np.allclose(np.diag(T), sj, rtol=1e-12, atol=1e-15)
    ok &= checks.residual(A, U, T, V) < 1e-13
    return bool(ok)


def pin_theorem1(f, n=80, b=8):
    # Theorem 1: after one step, ||[T12; T22]|| = ||A - A Q Q^T|| and
    # ||T22|| = ||A - W W^T A|| (spectral norms), Q = orth(Y), W = orth(A Y).
    ok = True
    for q in (0, 1, 2):
        A = synth.make_matrix("exp50", n, n, 77 + q)
        _, T, _, _ = f(A, b, q, gauss, max_steps=1)
        G = gauss(1, n, b)
        Y = A.T @ G
        for _ in range(q):
            Y = A.T @ (A @ Y)
        Q = _orth(Y)
        W = _orth(A @ Y)
        e1 = np.linalg.norm(A - A @ Q @ Q.T, 2)
        e2 = np.linalg.norm(A - W @ (W.T @ A), 2)
        t1 = np.linalg.norm(T[:, b:], 2)
        t2 = np.linalg.norm(T[b:, b:], 2)
        ok &= abs(t1 - e1) <= 1e-11 * e1 and abs(t2 - e2) <= 1e-11 * e2
    return bool(ok)


def pin_low_rank(f, n=64, b=16, r=10):
    # exact rank r <= b: after step 1 the trailing block vanishes and
    # diag(T)(1:r) = sigma(1:r)
    A = synth.make_matrix("lowrank", n, n, 5, r=r)
    s = synth.spectrum("lowrank", n, r=r)
    _, T, _, _ = f(A, b, 1, gauss, max_steps=1)
    ok = np.linalg.norm(T[b:, b:]) <= 1e-13 * np.linalg.norm(A)
    ok &= np.allclose(np.diag(T)[:r], s[:r], rtol=1e-12)
    return bool(ok)


def pin_dense_equivalence(f, m=72, n=60, b=8, q=1):
    # Section 5.2: the efficient and the dense versions agree (same G, same
    # Householder convention as LAPACK's QR used by the dense version)
    A = synth.make_matrix("exp50", m, n, 3)
    U1, T1, V1, _ = f(A, b, q, gauss)
    U2, T2, V2 = oracle.randutv_dense(A, b, q, gauss)
    return bool(np.max(np.abs(T1 - T2)) < 1e-12 and np.max(np.abs(U1 - U2)) < 1e-11
                and np.max(np.abs(V1 - V2)) < 1e-11)


def pin_oversampling_theorem1(f, n=80, b=8, p=6):
    # Over-sampling (Remark "Oversampling"): after one step the captured space
    # is that of Q = the b dominant left singular vectors of Y = (A^T A)^q A^T G
    # (G with b + p columns), computed here by numpy's SVD; Theorem 1's two
    # identities then hold with Q and W = orth(A Q).
    ok = True
    for q in (0, 1):
        A = synth.make_matrix("exp50", n, n, 91 + q)
        _, T, _, _ = f(A, b, q, gauss, max_steps=1, p=p)
        Y = A.T @ gauss(1, n, b + p)
        for _ in range(q):
            Y = A.T @ (A @ Y)
        Q = np.linalg.svd(Y, full_matrices=False)[0][:, :b]
        W = _orth(A @ Q)
        e1 = np.linalg.norm(A - A @ Q @ Q.T, 2)
        e2 = np.linalg.norm(A - W @ (W.T @ A), 2)
        t1 = np.linalg.norm(T[:, b:], 2)
        t2 = np.linalg.norm(T[b:, b:], 2)
        ok &= abs(t1 - e1) <= 1e-11 * e1 and abs(t2 - e2) <= 1e-11 * e2
    return bool(ok)


def pin_oversampling_invariants(f, n=96, b=16, q=1, p=5):
    # structure, residual and orthogonality, log|det| and ||T||_F with p > 0;
    # and over-sampling never loses the captured space of an exact rank r <= b
    A = synth.make_matrix("exp50", n, n, 1703001)
    s = synth.spectrum("exp50", n)
    U, T, V, kr = f(A, b, q, gauss, p=p)
    ok = kr == n and checks.residual(A, U, T, V) < 1e-13
    ok &= checks.orth_err(U) < 1e-13 and checks.orth_err(V) < 1e-13
    ok &= checks.lower_max(T) == 0.0 and checks.block_offdiag_max(T, b) == 0.0
    ok &= abs(np.sum(np.log(np.abs(np.diag(T)))) - np.sum(np.log(s))) < 1e-11 * n
    Ar = synth.make_matrix("lowrank", 64, 64, 5, r=10)
    sr = synth.spectrum("lowrank", 64, r=10)
    _, Tr, _, _ = f(Ar, 16, 1, gauss, max_steps=1, p=p)
    ok &= np.linalg.norm(Tr[16:, 16:]) <= 1e-13 * np.linalg.norm(Ar)
    ok &= np.allclose(np.diag(Tr)[:10], sr[:10], rtol=1e-12)
    return bool(ok)


PINS = [pin_structure_and_residual, pin_logdet_and_frobenius, pin_full_svd_case,
        pin_theorem1, pin_low_rank, pin_dense_equivalence, pin_oversampling_theorem1,
        pin_oversampling_invariants]


def run_battery(f):
    failed = []
    for p in PINS:
        try:
            if not p(f):
                failed.append(p.__name__)
        except Exception as exc:  # a crash is a caught mistake too
            failed.append(f"{p.__name__}:{type(exc).__name__}")
    return failed
