"""randUTV with every unitary matrix stored densely (Section 5.1).

Same step sequence as the efficient version, written the simple way of
Sections 4.3-4.5: the full n x n reflector product VV is formed explicitly
(complete QR of the sample matrix Y, LAPACK through numpy), the left factor is
UU diag(Us, I) with UU the explicit complete Q of the panel (Remark 1), and
the step's full transforms Uf, Vf are applied to T, U and V as dense products:
  T([I2,I3],[J2,J3]) <- Uf^T X Vf,  T(I1,[J2,J3]) <- T(I1,[J2,J3]) Vf,
  U(:, [I2,I3]) <- U(:, [I2,I3]) Uf,  V(:, [J2,J3]) <- V(:, [J2,J3]) Vf.
Cost O(n^4); used only for n <= 200 to pin the efficient version, which the
paper states is mathematically equivalent (Section 5.2).  Handles m >= n.
"""
import numpy as np
from .small_svd import svd_small


def _complete_q(B):
    q, _ = np.linalg.qr(B, mode="complete")
    return q


def randutv_dense(A, b, q, gauss):
    T = np.array(A, dtype=np.float64, copy=True)
    m, n = T.shape
    if m < n:
        raise ValueError("dense version written for m >= n")
    U, V = np.eye(m), np.eye(n)
    nsteps = -(-n // b)
    for i in range(1, nsteps + 1):
        r0 = b * (i - 1)
        kr, kc = m - r0, n - r0
        X = T[r0:, r0:].copy()
        if kr > b and kc > b:
            G = np.asarray(gauss(i, kr, b))
            Y = X.T @ G
            for _ in range(q):
                Y = X.T @ (X @ Y)
            VV = _complete_q(Y)                       # kc x kc
            XV = X @ VV
            UU = _complete_q(XV[:, :b])               # kr x kr
            R = (UU.T @ XV[:, :b])[:b, :b]
            Us, d, Vs = svd_small(np.triu(R))
            w = b
        else:
            VV = np.eye(kc)
            if kr > kc:
                UU = _complete_q(X)
                R = (UU.T @ X)[:kc, :kc]
                Us, d, Vs = svd_small(np.triu(R))
            else:
                UU = np.eye(kr)
                Us, d, Vs = svd_small(X)
            w = kc
        Uf = UU.copy()
        Uf[:, :w] = UU[:, :w] @ Us
        Vf = VV.copy()
        Vf[:, :w] = VV[:, :w] @ Vs
        newX = Uf.T @ X @ Vf
        newX[:, :w] = 0.0
        newX[:w, :w] = np.diag(d)
        T[r0:, r0:] = newX
        T[:r0, r0:] = T[:r0, r0:] @ Vf
        U[:, r0:] = U[:, r0:] @ Uf
        V[:, r0:] = V[:, r0:] @ Vf
    return U, T, V
