"""Accuracy measures of a factorization A = U T V^T (all in FP64)."""
import numpy as np


def residual(A, U, T, V):
    """||A - U T V^T||_F / ||A||_F."""
    A = np.asarray(A, dtype=np.float64)
    return float(np.linalg.norm(A - U @ T @ V.T) / np.linalg.norm(A))


def orth_err(Q):
    """max_ij |(Q^T Q - I)_ij|."""
    return float(np.max(np.abs(Q.T @ Q - np.eye(Q.shape[1]))))


def lower_max(T):
    """Largest |T_ij| below the diagonal."""
    return float(np.max(np.abs(np.tril(T, -1)))) if min(T.shape) > 1 else 0.0


def block_offdiag_max(T, b, k=None):
    """Largest off-diagonal |entry| inside the b x b diagonal blocks of T(:k,:k)."""
    k = min(T.shape) if k is None else k
    worst = 0.0
    for r0 in range(0, k, b):
        r1 = min(r0 + b, k)
        blk = T[r0:r1, r0:r1]
        worst = max(worst, float(np.max(np.abs(blk - np.diag(np.diag(blk))))))
    return worst
