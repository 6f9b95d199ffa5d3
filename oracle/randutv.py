"""randUTV, the efficient blocked algorithm of Fig. 4 (Section 5.2), in FP64.

Given A (m x n) and block size b, builds A = U T V^T with U (m x m) and V
(n x n) orthogonal and T upper triangular; T overwrites a copy of A and every
transform is applied as soon as it is formed (Section 5.2, first modification).

Step i (1-based) with r0 = b(i-1) works on the index blocks
  I1 = [0, r0), I2 = [r0, min(r0+b, m)), I3 = [r0+b, m)    (rows)
  J1 = [0, r0), J2 = [r0, min(r0+b, n)), J3 = [r0+b, n)    (columns)
and X = T([I2,I3],[J2,J3]).  When I3 and J3 are both non-empty:
  1. G = randn(m - r0, b)                         (Section 4.3 step 1)
  2. Y = X^T G, then q times Y = X^T (X Y)        (Section 4.3 step 2, Section 2.5)
  3. Householder QR of Y gives the reflector product VV (Section 4.3 step 3)
  4. T(:, [J2,J3]) <- T(:, [J2,J3]) VV,  V(:, [J2,J3]) <- V(:, [J2,J3]) VV
  5. Householder QR of T([I2,I3], J2) gives UU and R   (Remark 1)
  6. U(:, [I2,I3]) <- U(:, [I2,I3]) UU,  T([I2,I3], J3) <- UU^T T([I2,I3], J3),
     T(I3, J2) <- 0
  7. R(1:b,1:b) = Us Ds Vs^T;  T(I2,J2) <- Ds;  T(I2,J3) <- Us^T T(I2,J3);
     U(:, I2) <- U(:, I2) Us;  T(I1,J2) <- T(I1,J2) Vs;  V(:, J2) <- V(:, J2) Vs
Otherwise the last block gets a full SVD (Fig. 4, else branch), done
economically through a QR first when the block is tall (Section 5.2, third
modification, with Remark 1) or through a QR of its rows when it is wide
(Remark "The case m < n").

Over-sampling (Remark "Oversampling", Section 4.3 and its appendix): with
p > 0, G has b + p columns, Y = (X^T X)^q X^T G is n_k x (b+p), and the
step's reflectors come from a Householder QR of Z, the b dominant left
singular vectors of Y, instead of Y itself.  Z is formed as Q_Y Us(:, 1:b)
from the Householder QR Y = Q_Y R_Y and the SVD R_Y = Us Ds Vs^T (an SVD of Y
with the small-SVD sign convention; the choice of basis within span(Z)
changes the trailing basis, so it is fixed identically on the GPU).  A step
whose trailing block has fewer than b + p columns uses the first n - r0
columns of G.

Readings where the paper is silent (each is fixed identically on the GPU):
  * tolerance: before step i, stop if ||X||_F <= tol * ||A||_F; then
    k_reached = r0 and the trailing block is left as is (A = U T V^T still
    holds).  tol = 0 never stops early.
  * Householder convention: LAPACK dlarfg (see householder.py).
  * SVD order/signs: see small_svd.py.
  * no re-orthonormalisation between power steps (Fig. 4 has none).
"""
import numpy as np
from .householder import householder_qr, tfactor, wy_apply_right, wy_apply_left_t
from .small_svd import svd_small


def flops_randutv(m, n, b, q, form_uv=True):
    """Flop count used as the throughput numerator (m = n square inputs).

    Section 5.4 gives (5+2q) m n^2 - (3+2q) n^3/3 without U and V (m >= n).
    Forming U and V adds the two block-reflector applications per step to
    U(:, [I2,I3]) (4 m b (m - r0) flops) and V(:, [J2,J3]) (4 n b (n - r0)),
    summed over the n/b steps: 4 m^2 n - 2 m n^2 + 2 n^3.  Square inputs:
    (12+4q)/3 n^3 without and (24+4q)/3 n^3 with U and V."""
    f = (5 + 2 * q) * m * n * n - (3 + 2 * q) * n ** 3 / 3.0
    if form_uv:
        f += 4.0 * m * m * n - 2.0 * m * n * n + 2.0 * n ** 3
    return float(f)


def oversampled_basis(Y, b):
    """Z (k x b): the b dominant left singular vectors of Y (k x (b+p)), as
    Q_Y Us(:, 1:b) with Y = Q_Y R_Y (Householder) and R_Y = Us Ds Vs^T."""
    k, w = Y.shape
    Vq, tq, Rq = householder_qr(Y)
    Sq = tfactor(Vq, tq)
    Us, _, _ = svd_small(Rq[:w, :w])
    E = np.zeros((k, b))
    E[:w, :] = Us[:, :b]
    return E - Vq @ (Sq @ (Vq.T @ E))


def randutv(A, b, q, gauss, tol=0.0, form_uv=True, max_steps=None, p=0):
    """Factor A = U T V^T by Fig. 4 (with over-sampling p, the variant of
    Remark "Oversampling").

    gauss(step, k, w) -> k x w array: the Gaussian matrix of global step
    ``step`` (1-based), w = b + p.  Returns (U, T, V, k_reached); U and V are
    None when form_uv is False.  ``max_steps`` stops after that many steps (a
    partial factorization, used to time a bounded sample)."""
    T = np.array(A, dtype=np.float64, copy=True)
    m, n = T.shape
    U = np.eye(m) if form_uv else None
    V = np.eye(n) if form_uv else None
    normA = np.linalg.norm(T)
    nsteps = min(-(-m // b), -(-n // b))
    k_reached = min(m, n)
    for i in range(1, nsteps + 1):
        if max_steps is not None and i > max_steps:
            k_reached = b * (i - 1)
            break
        r0 = b * (i - 1)
        r1 = min(r0 + b, m)        # end of I2
        c1 = min(r0 + b, n)        # end of J2
        if tol > 0.0 and np.linalg.norm(T[r0:, r0:]) <= tol * normA:
            k_reached = r0
            break
        if r1 < m and c1 < n:      # I3 and J3 both non-empty
            X = T[r0:, r0:]
            # a step whose trailing block has fewer than b + p columns uses the
            # first n - r0 columns of G (a wider sketch adds nothing)
            G = np.asarray(gauss(i, m - r0, b + p), dtype=np.float64)[:, :min(b + p, n - r0)]
            Y = X.T @ G
            for _ in range(q):
                Y = X.T @ (X @ Y)
            if p > 0:
                Y = oversampled_basis(Y, b)
            Vv, tv, _ = householder_qr(Y)
            Sv = tfactor(Vv, tv)
            T[:, r0:] = wy_apply_right(T[:, r0:], Vv, Sv)
            if form_uv:
                V[:, r0:] = wy_apply_right(V[:, r0:], Vv, Sv)
            Vu, tu, R = householder_qr(T[r0:, r0:c1])
            Su = tfactor(Vu, tu)
            if form_uv:
                U[:, r0:] = wy_apply_right(U[:, r0:], Vu, Su)
            T[r0:, c1:] = wy_apply_left_t(T[r0:, c1:], Vu, Su)
            T[r0:, r0:c1] = 0.0
            Us, d, Vs = svd_small(R)
            T[r0:r1, r0:c1] = np.diag(d)
            T[r0:r1, c1:] = Us.T @ T[r0:r1, c1:]
            T[:r0, r0:c1] = T[:r0, r0:c1] @ Vs
            if form_uv:
                U[:, r0:r1] = U[:, r0:r1] @ Us
                V[:, r0:c1] = V[:, r0:c1] @ Vs
        else:
            _final_block(T, U, V, r0, form_uv)
    return U, T, V, k_reached


def _final_block(T, U, V, r0, form_uv):
    """Full SVD of the last block T([I2,I3],[J2,J3]) and its updates."""
    m, n = T.shape
    kr, kc = m - r0, n - r0
    p = min(kr, kc)
    X = T[r0:, r0:]
    if kr > kc:      # tall: QR of the columns, then SVD of R (Remark 1)
        Vq, tq, R = householder_qr(X)
        Sq = tfactor(Vq, tq)
        if form_uv:
            U[:, r0:] = wy_apply_right(U[:, r0:], Vq, Sq)
        core = R
    elif kr < kc:    # wide: QR of the rows, then SVD of L = R^T
        Vq, tq, R = householder_qr(X.T)
        Sq = tfactor(Vq, tq)
        T[:, r0:] = wy_apply_right(T[:, r0:], Vq, Sq)
        if form_uv:
            V[:, r0:] = wy_apply_right(V[:, r0:], Vq, Sq)
        core = R.T
    else:
        core = X.copy()
    Us, d, Vs = svd_small(core)
    T[r0:, r0:] = 0.0
    T[r0:r0 + p, r0:r0 + p] = np.diag(d)
    T[:r0, r0:r0 + p] = T[:r0, r0:r0 + p] @ Vs
    if form_uv:
        U[:, r0:r0 + p] = U[:, r0:r0 + p] @ Us
        V[:, r0:r0 + p] = V[:, r0:r0 + p] @ Vs
