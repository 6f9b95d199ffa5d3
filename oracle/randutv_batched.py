"""randUTV of a batch of independent matrices (the batched form), FP64.

TEST INFRASTRUCTURE ONLY (see the package header).

A batch is a list of independent problems: matrix i is factored by Fig. 4
(``randutv``) with its own block size b_i, its own Gaussian matrices and the
early stop of Section 1.1 (ii) (before each step, stop once the trailing
block has ||T(I2 I3, J2 J3)||_F <= tol ||A_i||_F).  Tall and wide matrices
end with the economic final blocks of Section 5.2 and of the Remark on
m < n, which ``randutv`` implements.
"""
from .randutv import randutv


def randutv_batched(As, bs, q, gauss, tol=0.0, form_uv=True):
    """[(U_i, T_i, V_i, k_i)] for the matrices As with block sizes bs.

    gauss(i, step, k, w) -> k x w array: the Gaussian matrix of matrix i at
    global step ``step``.  Each matrix runs ``randutv`` in FP64 on its own."""
    out = []
    for i, (A, b) in enumerate(zip(As, bs)):
        out.append(randutv(A, int(b), q, lambda s, k, w, i=i: gauss(i, s, k, w), tol=tol, form_uv=form_uv))
    return out
