"""The rank-k approximation A_k = U(:, 1:k) T(1:k, :) V^T of randUTV (eq.
Ak_randUTV) as a differentiable torch function on the GPU.

Argument marshalling only: the forward (the first k/b randomized steps of
Fig. 4 in FP64) and the hand-written reverse pass run in librandutv's
kernels (randutv_rank_k, randutv_rank_k_vjp).  The Gaussian matrices are
fixed by ``seed`` (or ``g_inject``), so the map is a function of A alone.

    Ak = rank_k(A, b=32, q=1, k=64)          # A: (m, n) float64 CUDA tensor
    loss = ((A - Ak) ** 2).sum(); loss.backward()
"""
import ctypes

from . import native


def _torch():
    import torch
    return torch


class _State:
    """Device state kept by the forward for the reverse pass."""

    def __init__(self, handle, m, n):
        self.h, self.m, self.n = handle, m, n

    def __del__(self):
        try:
            if self.h:
                native.lib().randutv_rank_k_free(self.h)
        except Exception:
            pass


def _bind_stream():
    torch = _torch()
    native.lib().randutv_set_stream(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _forward(A, b, q, k, seed, g_inject, keep):
    torch = _torch()
    if not (isinstance(A, torch.Tensor) and A.dim() == 2 and A.dtype == torch.float64 and A.is_cuda):
        raise TypeError("A must be a 2-D float64 CUDA tensor")
    m, n = A.shape
    Ast = A.detach().t().contiguous()
    Fst = torch.empty((n, m), dtype=torch.float64, device=A.device)
    o = native.default_opts()
    o.seed = int(seed)
    o.g_inject = ctypes.c_void_p(g_inject.data_ptr()) if g_inject is not None else None
    h = ctypes.c_void_p()
    _bind_stream()
    st = native.lib().randutv_rank_k(m, n, Ast.data_ptr(), m, int(b), int(q), int(k), Fst.data_ptr(), m,
                                     ctypes.byref(o), ctypes.byref(h) if keep else None)
    native.check(st, "randutv_rank_k")
    return Fst.t(), (_State(h, m, n) if keep else None)


def vjp(state, Fbar):
    """(dA_k/dA)^T Fbar for the state of a forward call (torch layout)."""
    torch = _torch()
    Fb = Fbar.detach().to(torch.float64).t().contiguous()
    Ab = torch.empty_like(Fb)
    _bind_stream()
    st = native.lib().randutv_rank_k_vjp(state.h, Fb.data_ptr(), state.m, Ab.data_ptr(), state.m)
    native.check(st, "randutv_rank_k_vjp")
    return Ab.t()


class RankK(_torch().autograd.Function):
    """A -> A_k with the library's hand-written reverse pass."""

    @staticmethod
    def forward(ctx, A, b, q, k, seed, g_inject):
        F, state = _forward(A, b, q, k, seed, g_inject, True)
        ctx.state = state
        return F

    @staticmethod
    def backward(ctx, Fbar):
        return vjp(ctx.state, Fbar), None, None, None, None, None


def rank_k(A, b=32, q=1, k=64, seed=998, g_inject=None):
    """A_k = U(:, 1:k) T(1:k, :) V^T of randUTV at fixed G (differentiable)."""
    return RankK.apply(A, b, q, k, seed, g_inject)


def rank_k_forward(A, b=32, q=1, k=64, seed=998, g_inject=None, keep=False):
    """(A_k, state) without autograd; state (keep=True) serves ``vjp``."""
    return _forward(A, b, q, k, seed, g_inject, keep)
