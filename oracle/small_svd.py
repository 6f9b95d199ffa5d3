"""SVD of the small b x b block R11 (Fig. 4, the ``svd`` of each step and of
the final block).

The paper leaves order and signs of the SVD open.  Convention used here:
singular values descending and non-negative; for each singular pair the
entry of largest magnitude in the column of V_small (lowest index on ties)
is made positive and the matching column of U_small flips with it.

``svd_small`` uses the library SVD (LAPACK through numpy).  ``jacobi_svd`` is
a brute-force one-sided (Hestenes) Jacobi SVD written out with plain loops;
it exists only to pin ``svd_small`` and the b >= n special case on tiny
inputs.
"""
import math
import numpy as np


def sign_fix(Us, Vs):
    """Apply the sign convention in place-free form; returns (Us, Vs)."""
    Us = np.array(Us, dtype=np.float64, copy=True)
    Vs = np.array(Vs, dtype=np.float64, copy=True)
    for j in range(Vs.shape[1]):
        i = int(np.argmax(np.abs(Vs[:, j])))  # first index of the maximum
        if Vs[i, j] < 0:
            Vs[:, j] = -Vs[:, j]
            Us[:, j] = -Us[:, j]
    return Us, Vs


def svd_small(M):
    """Full SVD M = Us diag(d) Vs^T of a p x r block; returns (Us, d, Vs).

    Us is p x p, Vs is r x r, d has min(p, r) entries (descending)."""
    Us, d, Vt = np.linalg.svd(np.asarray(M, dtype=np.float64), full_matrices=True)
    p = min(M.shape)
    Uf, Vf = sign_fix(Us[:, :p], Vt.T[:, :p])
    Us = Us.copy()
    Vs = Vt.T.copy()
    Us[:, :p] = Uf
    Vs[:, :p] = Vf
    return Us, d, Vs


def jacobi_svd(A, tol=None, max_sweeps=60):
    """One-sided cyclic Jacobi SVD of an m x n matrix (m >= n), by brute force.

    Columns i < j are rotated until |c_i . c_j| <= tol * ||c_i|| ||c_j|| for all
    pairs (tol defaults to m * 2^-53).  Returns (U, s, V) with U m x n, s
    descending, V n x n, A = U diag(s) V^T; zero columns get U columns that
    complete an orthonormal set.
    """
    W = np.array(A, dtype=np.float64, copy=True)
    m, n = W.shape
    if m < n:
        raise ValueError("jacobi_svd expects m >= n")
    tol = m * 2.0 ** -53 if tol is None else tol
    V = np.eye(n)
    for _ in range(max_sweeps):
        rotated = False
        for i in range(n - 1):
            for j in range(i + 1, n):
                a = float(W[:, i] @ W[:, i])
                b = float(W[:, j] @ W[:, j])
                g = float(W[:, i] @ W[:, j])
                if g == 0.0 or abs(g) <= tol * math.sqrt(a * b):
                    continue
                rotated = True
                zeta = (b - a) / (2.0 * g)
                t = math.copysign(1.0, zeta) / (abs(zeta) + math.sqrt(1.0 + zeta * zeta))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = c * t
                wi, wj = W[:, i].copy(), W[:, j].copy()
                W[:, i] = c * wi - s * wj
                W[:, j] = s * wi + c * wj
                vi, vj = V[:, i].copy(), V[:, j].copy()
                V[:, i] = c * vi - s * vj
                V[:, j] = s * vi + c * vj
        if not rotated:
            break
    s = np.sqrt(np.sum(W * W, axis=0))
    order = np.argsort(-s, kind="stable")
    s, W, V = s[order], W[:, order], V[:, order]
    U = np.zeros((m, n))
    for j in range(n):
        if s[j] > 0:
            U[:, j] = W[:, j] / s[j]
        else:  # complete with the first unit vector independent of the others
            for e in range(m):
                u = np.zeros(m)
                u[e] = 1.0
                for _ in range(2):
                    u -= U[:, :j] @ (U[:, :j].T @ u)
                nu = np.linalg.norm(u)
                if nu > 0.5:
                    U[:, j] = u / nu
                    break
    return U, s, V
