"""Plain, slow, FP64 CPU oracle of randUTV (Martinsson, Quintana-Orti, Heavner,
"randUTV: A blocked randomized algorithm for computing a rank-revealing UTV
factorization", arXiv 1703.00998).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this package.  The CUDA product path
shares no code with it and never calls it.

Contents
  householder   Householder vectors (LAPACK dlarfg convention), unpivoted
                Householder QR, the compact-WY factor S, WY application
                (Section 2.4, eqs. unpivQR and WYrepresentation).
  small_svd     SVD of a small block with a fixed order/sign convention
                (library SVD) and a brute-force one-sided Jacobi SVD used only
                to pin it.
  randutv       the efficient blocked algorithm of Fig. 4 (Section 5.2).
  randutv_dense the simplistic dense version of Section 5.1 (all unitary
                matrices stored densely), used to pin the efficient one.
  randutv_batched  a batch of independent problems, each by Fig. 4 with the
                early stop of Section 1.1 (ii).
  randutv_adjoint  the rank-k approximation A_k = U(:,1:k) T(1:k,:) V^T
                (eq. Ak_randUTV) and its vector-Jacobian product at fixed G
                (reverse mode of the same steps, torch.autograd on CPU).
  checks        residual / orthogonality / structure measures.

Parity status: every function is pinned by tests/test_oracle_*.py against
library routines, closed forms, Theorem 1 or brute force; nothing here is
"parity unpinned".
"""
from .householder import house, householder_qr, tfactor, wy_apply_right, wy_apply_left_t
from .small_svd import svd_small, jacobi_svd, sign_fix
from .randutv import randutv, flops_randutv
from .randutv_dense import randutv_dense
from .randutv_batched import randutv_batched
from .randutv_adjoint import rank_k_approx, rank_k_vjp, loss_grad
from . import checks

__all__ = ["house", "householder_qr", "tfactor", "wy_apply_right", "wy_apply_left_t",
           "svd_small", "jacobi_svd", "sign_fix", "randutv", "flops_randutv",
           "randutv_dense", "randutv_batched", "rank_k_approx", "rank_k_vjp", "loss_grad", "checks"]
