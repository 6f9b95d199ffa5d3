"""Householder reflectors and the compact WY representation (Section 2.4).

The paper factors a tall-thin matrix B = QR with Q a product of b Householder
reflectors and stores Q in the form Q = I + W Y (eq. WYrepresentation,
refs. Bischof-Van Loan 1987, Schreiber-Van Loan 1989, Joffrain et al. 2006).
Here that form is written Q = H_1 H_2 ... H_b = I - V S V^T, i.e. W = -V S,
Y = V^T, with V unit lower trapezoidal and S upper triangular.

Convention (the paper fixes none; this is LAPACK's dlarfg): for x = [alpha; x2],
  beta = -sign(alpha) * ||x||,  tau = (beta - alpha) / beta,
  v = [1; x2 / (alpha - beta)],  H = I - tau v v^T,  H x = beta e_1,
and tau = 0 (H = I, beta = alpha) when x2 = 0.  sign() follows copysign, so
alpha = +0.0 gives beta < 0.
"""
import math
import numpy as np


def _norm2(x):
    """Euclidean norm with scaling by the largest |entry| (no underflow)."""
    if x.size == 0:
        return 0.0
    s = float(np.max(np.abs(x)))
    if s == 0.0:
        return 0.0
    return s * float(np.sqrt(np.sum((x / s) ** 2)))


def house(x):
    """Householder vector of x: returns (v, tau, beta) with v[0] = 1."""
    x = np.asarray(x, dtype=np.float64)
    alpha = float(x[0])
    xnorm = _norm2(x[1:])
    v = np.zeros_like(x)
    v[0] = 1.0
    if xnorm == 0.0:
        return v, 0.0, alpha
    beta = -math.copysign(math.hypot(alpha, xnorm), alpha)
    tau = (beta - alpha) / beta
    v[1:] = x[1:] / (alpha - beta)
    return v, tau, beta


def householder_qr(B):
    """Unpivoted Householder QR of a k x w matrix B (k >= w), eq. unpivQR.

    Returns (V, tau, R): V is k x w unit lower trapezoidal (column j holds the
    j-th Householder vector), tau has w entries, R is w x w upper triangular,
    and (H_1 ... H_w)^T B = [R; 0].  Reflectors are generated and applied one
    column at a time, left to right.
    """
    A = np.array(B, dtype=np.float64, copy=True)
    k, w = A.shape
    if k < w:
        raise ValueError("householder_qr expects k >= w")
    V = np.zeros((k, w))
    tau = np.zeros(w)
    for j in range(w):
        v, t, beta = house(A[j:, j])
        V[j:, j] = v
        tau[j] = t
        A[j, j] = beta
        A[j + 1:, j] = 0.0
        if j + 1 < w and t != 0.0:
            wrow = v @ A[j:, j + 1:]
            A[j:, j + 1:] -= t * np.outer(v, wrow)
    return V, tau, np.triu(A[:w, :w])


def tfactor(V, tau):
    """Upper triangular S with H_1 ... H_w = I - V S V^T (forward, column-wise).

    Column j: S[j, j] = tau_j and S[:j, j] = -tau_j * S[:j, :j] (V[:, :j]^T v_j);
    this is the accumulation of the product one reflector at a time.
    """
    w = V.shape[1]
    S = np.zeros((w, w))
    for j in range(w):
        S[j, j] = tau[j]
        if j > 0:
            S[:j, j] = -tau[j] * (S[:j, :j] @ (V[:, :j].T @ V[:, j]))
    return S


def wy_apply_right(C, V, S):
    """C Q with Q = I - V S V^T:  C - (C V) S V^T."""
    return C - ((C @ V) @ S) @ V.T


def wy_apply_left_t(C, V, S):
    """Q^T C with Q = I - V S V^T:  C - V S^T (V^T C)."""
    return C - V @ (S.T @ (V.T @ C))
