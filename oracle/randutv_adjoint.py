"""The rank-k approximation of randUTV and its derivative at fixed G.

TEST INFRASTRUCTURE ONLY (see the package header).

A_k = U(:, 1:k) T(1:k, :) V^T (eq. Ak_randUTV), k a multiple of b.  The first
k/b steps of Fig. 4 fix U(:, 1:k) (later steps touch only columns beyond k
of U), and A = U T V^T holds after every step, so T(1:k, :) V^T =
U(:, 1:k)^T A is the same after k/b steps as after all of them: A_k is the
map of the first k/b steps.

``rank_k_approx`` evaluates it with ``randutv`` (numpy, FP64).
``rank_k_vjp`` returns (A_k, (dA_k/dA)^T C) at fixed Gaussian matrices by
reverse-mode differentiation of the same step sequence: the steps of Fig. 4
(sketch, Householder QR of Y and its application to T and V, Householder QR
of the panel and its application to U and T, the small SVD and its five
rotations) written again below with torch CPU operations in FP64 (dlarfg
convention and SVD sign convention as in householder.py and small_svd.py)
and differentiated by torch.autograd.
"""
import numpy as np

from .randutv import randutv


def rank_k_approx(A, b, q, gauss, k):
    """A_k = U(:, :k) T(:k, :) V^T from the first k / b steps (numpy)."""
    if k % b:
        raise ValueError("k must be a multiple of b")
    U, T, V, _ = randutv(A, b, q, gauss, max_steps=k // b)
    return U[:, :k] @ T[:k, :] @ V.T


def _torch():
    import torch
    return torch


def _house(x):
    """dlarfg on a 1-D tensor: (v with v[0] = 1, tau, beta)."""
    torch = _torch()
    alpha, x2 = x[0], x[1:]
    v0 = torch.ones(1, dtype=x.dtype)
    if x2.numel() == 0 or float(torch.max(torch.abs(x2.detach()))) == 0.0:
        return torch.cat([v0, torch.zeros_like(x2)]), torch.zeros((), dtype=x.dtype), alpha
    beta = -torch.copysign(torch.sqrt(alpha * alpha + torch.sum(x2 * x2)), alpha)
    tau = (beta - alpha) / beta
    return torch.cat([v0, x2 / (alpha - beta)]), tau, beta


def _householder_qr(B):
    """(V, tau, R) of B (k x w, k >= w), one reflector at a time."""
    torch = _torch()
    k, w = B.shape
    cols = [B[:, j] for j in range(w)]
    vs, taus, rcols = [], [], []
    for j in range(w):
        v, t, beta = _house(cols[j][j:])
        vs.append(torch.cat([torch.zeros(j, dtype=B.dtype), v]))
        taus.append(t)
        rcols.append(torch.cat([cols[j][:j], beta.reshape(1), torch.zeros(w - j - 1, dtype=B.dtype)]))
        for c in range(j + 1, w):
            seg = cols[c][j:]
            cols[c] = torch.cat([cols[c][:j], seg - t * v * torch.dot(v, seg)])
    return torch.stack(vs, 1), torch.stack(taus), torch.stack(rcols, 1)


def _tfactor(V, tau):
    torch = _torch()
    w = V.shape[1]
    cols = []
    for j in range(w):
        if j == 0:
            cols.append(torch.cat([tau[0].reshape(1), torch.zeros(w - 1, dtype=V.dtype)]))
            continue
        Sj = torch.stack(cols, 1)[:j, :j]
        top = -tau[j] * (Sj @ (V[:, :j].T @ V[:, j]))
        cols.append(torch.cat([top, tau[j].reshape(1), torch.zeros(w - j - 1, dtype=V.dtype)]))
    return torch.stack(cols, 1)


def _svd_small(M):
    """Us, d, Vs with d descending and the largest |entry| of each Vs column positive."""
    torch = _torch()
    Us, d, Vh = torch.linalg.svd(M, full_matrices=False)
    Vs = Vh.T
    idx = torch.argmax(torch.abs(Vs), dim=0)
    sgn = torch.where(Vs[idx, torch.arange(Vs.shape[1])] < 0, -1.0, 1.0).to(M.dtype)
    return Us * sgn[None, :], d, Vs * sgn[None, :]


def _put(X, r0, r1, c0, c1, B):
    """X with the block X[r0:r1, c0:c1] replaced by B (a new tensor)."""
    X = X.clone()
    X[r0:r1, c0:c1] = B
    return X


def _steps(A, b, q, gauss, nsteps):
    """U, T, V after the first nsteps randomized steps of Fig. 4 (torch)."""
    torch = _torch()
    m, n = A.shape
    T = A
    U = torch.eye(m, dtype=A.dtype)
    V = torch.eye(n, dtype=A.dtype)
    for i in range(1, nsteps + 1):
        r0 = b * (i - 1)
        r1, c1 = r0 + b, r0 + b
        if not (r1 < m and c1 < n):
            raise ValueError("the map is defined by randomized steps only (b k/b < min(m, n))")
        X = T[r0:, r0:]
        G = torch.as_tensor(np.asarray(gauss(i, m - r0, b), dtype=np.float64))
        Y = X.T @ G
        for _ in range(q):
            Y = X.T @ (X @ Y)
        Vv, tv, _ = _householder_qr(Y)
        Sv = _tfactor(Vv, tv)
        C = T[:, r0:]
        T = _put(T, 0, m, r0, n, C - ((C @ Vv) @ Sv) @ Vv.T)
        C = V[:, r0:]
        V = _put(V, 0, n, r0, n, C - ((C @ Vv) @ Sv) @ Vv.T)
        Vu, tu, R = _householder_qr(T[r0:, r0:c1])
        Su = _tfactor(Vu, tu)
        C = U[:, r0:]
        U = _put(U, 0, m, r0, m, C - ((C @ Vu) @ Su) @ Vu.T)
        C = T[r0:, c1:]
        T = _put(T, r0, m, c1, n, C - Vu @ (Su.T @ (Vu.T @ C)))
        T = _put(T, r0, m, r0, c1, torch.zeros((m - r0, b), dtype=A.dtype))
        Us, d, Vs = _svd_small(R)
        T = _put(T, r0, r1, r0, c1, torch.diag(d))
        T = _put(T, r0, r1, c1, n, Us.T @ T[r0:r1, c1:])
        T = _put(T, 0, r0, r0, c1, T[:r0, r0:c1] @ Vs)
        U = _put(U, 0, m, r0, r1, U[:, r0:r1] @ Us)
        V = _put(V, 0, n, r0, c1, V[:, r0:c1] @ Vs)
    return U, T, V


def rank_k_vjp(A, b, q, gauss, k, C):
    """(A_k, (dA_k / dA)^T C) at fixed G, both m x n numpy arrays.

    gauss(step, k_rows, b) -> the step's Gaussian matrix (no derivative)."""
    torch = _torch()
    if k % b:
        raise ValueError("k must be a multiple of b")
    At = torch.tensor(np.asarray(A, dtype=np.float64), requires_grad=True)
    U, T, V = _steps(At, b, q, gauss, k // b)
    Ak = U[:, :k] @ T[:k, :] @ V.T
    (g,) = torch.autograd.grad(torch.sum(Ak * torch.as_tensor(np.asarray(C, dtype=np.float64))), At)
    return Ak.detach().numpy(), g.numpy()


def loss_grad(A, b, q, gauss, k):
    """(L, dL/dA) of L = ||A - A_k||_F^2:  dL/dA = 2 (A - A_k) - 2 (dA_k/dA)^T (A - A_k)."""
    Ak = rank_k_approx(A, b, q, gauss, k)
    E = np.asarray(A, dtype=np.float64) - Ak
    _, g = rank_k_vjp(A, b, q, gauss, k, E)
    return float(np.sum(E * E)), 2.0 * E - 2.0 * g
