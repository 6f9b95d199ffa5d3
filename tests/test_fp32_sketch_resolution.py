"""The FP32 sketch-resolution reading used by the batched parity tests, on
CPU.  Fig. 4's steps are run in FP64 with only the sketch Y = (X^T X)^q X^T G
formed in FP32 (the one place where the batched form's precision changes
which subspace a step captures): over the leading entries the resolution
criterion keeps (2^-24 (d_{r0} / d_j)^(2q+1) <= 1e-3 within each block),
|diag T| agrees with the FP64 oracle to 1e-4 relative, entry by entry; on a block whose singular
values span ~180 the entries beyond the prefix move by more than 1e-3."""
import numpy as np
import pytest
import synth
import oracle
from oracle.householder import householder_qr, tfactor, wy_apply_right, wy_apply_left_t
from test_gpu_batched import _resolved_prefix


def _diag_fp32_sketch(A, b, q, gauss):
    T = A.copy()
    m, n = T.shape
    for i in range(1, min(-(-m // b), -(-n // b)) + 1):
        r0 = b * (i - 1)
        r1, c1 = min(r0 + b, m), min(r0 + b, n)
        if not (r1 < m and c1 < n):
            s = np.linalg.svd(T[r0:, r0:], compute_uv=False)
            T[r0:, r0:] = 0.0
            T[r0:r0 + len(s), r0:r0 + len(s)] = np.diag(s)
            break
        X32 = T[r0:, r0:].astype(np.float32)
        Y = X32.T @ gauss(i, m - r0, b).astype(np.float32)
        for _ in range(q):
            Y = X32.T @ (X32 @ Y)
        Vv, tv, _ = householder_qr(Y.astype(np.float64))
        T[:, r0:] = wy_apply_right(T[:, r0:], Vv, tfactor(Vv, tv))
        Vu, tu, R = householder_qr(T[r0:, r0:c1])
        T[r0:, c1:] = wy_apply_left_t(T[r0:, c1:], Vu, tfactor(Vu, tu))
        T[r0:, r0:c1] = 0.0
        Us, d, Vs = np.linalg.svd(R)
        T[r0:r1, r0:c1] = np.diag(d)
        T[r0:r1, c1:] = Us.T @ T[r0:r1, c1:]
        T[:r0, r0:c1] = T[:r0, r0:c1] @ Vs.T
    return np.abs(np.diag(T))


def _g(i, k, w):
    return synth.step_gaussian_f32(998, i, k, w, index=0).astype(np.float64)


@pytest.mark.parametrize("m,n,r,b", [(64, 64, 6.0, 32), (64, 64, 6.0, 16), (96, 80, 12.0, 32), (100, 90, 8.0, 32)])
def test_resolved_entries_agree(m, n, r, b):
    A = synth.make_matrix("exp", m, n, 3, r=r)
    _, To, _, _ = oracle.randutv(A, b, 1, _g, form_uv=False)
    do = np.abs(np.diag(To))
    d32 = _diag_fp32_sketch(A, b, 1, _g)
    kk = _resolved_prefix(do, b)
    dr = np.abs(d32 - do) / do
    assert kk > 0
    assert dr[:kk].max() <= 1e-4, (kk, dr[:kk].max())


def test_unresolved_entries_move():
    A = synth.make_matrix("exp", 64, 64, 3, r=6.0)
    _, To, _, _ = oracle.randutv(A, 32, 1, _g, form_uv=False)
    do = np.abs(np.diag(To))
    d32 = _diag_fp32_sketch(A, 32, 1, _g)
    kk = _resolved_prefix(do, 32)
    assert kk < 32
    assert (np.abs(d32 - do) / do)[kk:32].max() > 1e-3
