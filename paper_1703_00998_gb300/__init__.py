"""GB300-native randUTV (Martinsson, Quintana-Orti, Heavner, arXiv 1703.00998).

Python face of librandutv.so: torch supplies device memory and the stream;
every step of the factorization runs in the library's CUDA kernels.  All
functions here take and return torch tensors in the usual (row-major) torch
layout and convert to the library's column-major layout at the boundary.

    U, T, V, k = paper_1703_00998_gb300.factor(A, b=128, q=1)   # A = U T V^T
"""
import ctypes
from collections import namedtuple

from . import native
from .native import RandutvError
from .batched import BatchedPlan, BatchedUTV, batched_gaussian
from .adjoint import rank_k, rank_k_forward, vjp as rank_k_vjp

__all__ = ["factor", "factor_mixed", "factor_host", "gaussian", "philox_words", "dgemm", "sgemm", "panel_qr", "small_svd",
           "RandutvError", "UTV", "BatchedPlan", "BatchedUTV", "batched_gaussian",
           "rank_k", "rank_k_forward", "rank_k_vjp"]

UTV = namedtuple("UTV", ["U", "T", "V", "k_reached"])


def _torch():
    import torch
    return torch


def _check_cuda64(x, name):
    torch = _torch()
    if not isinstance(x, torch.Tensor) or x.dim() != 2 or x.dtype != torch.float64 or not x.is_cuda:
        raise TypeError(f"{name} must be a 2-D float64 CUDA tensor")


def _colmajor(x):
    """Column-major storage of a 2-D tensor: a contiguous (cols, rows) tensor."""
    return x.t().contiguous()


def _bind_stream():
    torch = _torch()
    native.lib().randutv_set_stream(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _opts(seed, form_uv, max_sweeps, g_inject, overlap=True, fp64_emulation=True, p=0, g_capture=None):
    o = native.default_opts()
    if g_capture is not None:
        torch = _torch()
        if g_capture.dtype != torch.float64 or not g_capture.is_cuda or not g_capture.is_contiguous():
            raise TypeError("g_capture must be a contiguous float64 CUDA tensor")
        o.g_capture = ctypes.c_void_p(g_capture.data_ptr())
    o.p = int(p)
    o.overlap = 1 if overlap else 0
    o.fp64_emulation = 1 if fp64_emulation else 0
    o.seed = int(seed)
    o.form_uv = 1 if form_uv else 0
    o.max_sweeps = int(max_sweeps)
    o.g_inject = ctypes.c_void_p(g_inject.data_ptr()) if g_inject is not None else None
    return o


def factor(A, b=128, q=1, tol=0.0, seed=998, g_inject=None, form_uv=True, max_sweeps=30, overlap=True,
           fp64_emulation=True, p=0, g_capture=None):
    """A = U T V^T by randUTV (Fig. 4) on A's CUDA device, FP64.

    A: (m, n) float64 CUDA tensor.  g_inject: optional 1-D float64 CUDA tensor
    with every randomized step's Gaussian G concatenated (column-major per
    step, the layout of ``synth.stream_layout``) used instead of the Philox
    stream.  Returns UTV(U, T, V, k_reached) as (m, m), (m, n), (n, n) views
    (U, V are None when form_uv is False).  ENOCONV raises too.
    fp64_emulation: the large products through the Ozaki-scheme tensor-core
    GEMM (FP64-accurate) instead of the FP64 DFMA GEMM.  p: over-sampling
    (each step sketches b + p columns; g_inject then holds (k, b + p) per step).
    g_capture: optional 1-D float64 CUDA tensor of the g_inject layout that
    receives every randomized step's G."""
    torch = _torch()
    _check_cuda64(A, "A")
    m, n = A.shape
    with torch.cuda.device(A.device):
        Tst = _colmajor(A)                     # in place: T overwrites this copy of A
        Ust = torch.empty((m, m), dtype=torch.float64, device=A.device) if form_uv else None
        Vst = torch.empty((n, n), dtype=torch.float64, device=A.device) if form_uv else None
        if g_inject is not None:
            if g_inject.dtype != torch.float64 or not g_inject.is_cuda or not g_inject.is_contiguous():
                raise TypeError("g_inject must be a contiguous float64 CUDA tensor")
        o = _opts(seed, form_uv, max_sweeps, g_inject, overlap, fp64_emulation, p, g_capture)
        kr = ctypes.c_int64(0)
        _bind_stream()
        st = native.lib().randutv_factor_ex(
            m, n, Tst.data_ptr(), m, int(b), int(q), float(tol),
            Ust.data_ptr() if form_uv else None, m, Tst.data_ptr(), m,
            Vst.data_ptr() if form_uv else None, n, ctypes.byref(kr), ctypes.byref(o))
        native.check(st, "randutv_factor_ex")
    return UTV(Ust.t() if form_uv else None, Tst.t(), Vst.t() if form_uv else None, kr.value)


def factor_mixed(A, b=128, q=1, tol=0.0, seed=998, g_inject=None, form_uv=True, max_sweeps=30, overlap=True,
                 tensor_cores=1, sketch_prec=0, g_capture=None):
    """Mixed-precision randUTV: A is an (m, n) float32 CUDA tensor; U, T, V
    come back float32.  Panel QRs and small SVDs run in FP64 inside.
    sketch_prec: 0 forms the sketch products from BF16 slices on the tensor
    cores (the FP32 block exactly, G / Y / Z to 35 bits); 1 as 3xTF32 and 2
    as one TF32 product on the tcgen05 tensor cores (tensor_cores = 1) or
    the FP32 CUDA cores (tensor_cores = 0)."""
    torch = _torch()
    if not isinstance(A, torch.Tensor) or A.dim() != 2 or A.dtype != torch.float32 or not A.is_cuda:
        raise TypeError("A must be a 2-D float32 CUDA tensor")
    m, n = A.shape
    with torch.cuda.device(A.device):
        Tst = _colmajor(A)
        Ust = torch.empty((m, m), dtype=torch.float32, device=A.device) if form_uv else None
        Vst = torch.empty((n, n), dtype=torch.float32, device=A.device) if form_uv else None
        if g_inject is not None:
            if g_inject.dtype != torch.float64 or not g_inject.is_cuda or not g_inject.is_contiguous():
                raise TypeError("g_inject must be a contiguous float64 CUDA tensor")
        o = _opts(seed, form_uv, max_sweeps, g_inject, overlap, g_capture=g_capture)
        o.tensor_cores = int(tensor_cores)
        o.sketch_prec = int(sketch_prec)
        kr = ctypes.c_int64(0)
        _bind_stream()
        st = native.lib().randutv_factor_mixed(
            m, n, Tst.data_ptr(), m, int(b), int(q), float(tol),
            Ust.data_ptr() if form_uv else None, m, Tst.data_ptr(), m,
            Vst.data_ptr() if form_uv else None, n, ctypes.byref(kr), ctypes.byref(o))
        native.check(st, "randutv_factor_mixed")
    return UTV(Ust.t() if form_uv else None, Tst.t(), Vst.t() if form_uv else None, kr.value)


def factor_host(A, b=128, q=1, tol=0.0, seed=998, form_uv=True, max_sweeps=30, out=None):
    """randUTV of a HOST matrix through randutv_factor_host (copies inside).

    A: (m, n) float64 CPU tensor; for speed pass page-locked column-major
    storage, i.e. ``A = S.t()`` with S a pinned contiguous (n, m) tensor.
    ``out`` may hold preallocated pinned (U, T, V) column-major views."""
    torch = _torch()
    if A.dim() != 2 or A.dtype != torch.float64 or A.is_cuda:
        raise TypeError("A must be a 2-D float64 CPU tensor")
    m, n = A.shape
    Ast = A.t() if A.t().is_contiguous() else _colmajor(A)
    if out is None:
        pin = torch.cuda.is_available()
        Ust = torch.empty((m, m), dtype=torch.float64, pin_memory=pin) if form_uv else None
        Tst = torch.empty((n, m), dtype=torch.float64, pin_memory=pin)
        Vst = torch.empty((n, n), dtype=torch.float64, pin_memory=pin) if form_uv else None
    else:
        Ust, Tst, Vst = (x.t() if x is not None else None for x in out)
    o = _opts(seed, form_uv, max_sweeps, None)
    kr = ctypes.c_int64(0)
    _bind_stream()
    st = native.lib().randutv_factor_host(
        m, n, Ast.data_ptr(), m, int(b), int(q), float(tol),
        Ust.data_ptr() if form_uv else None, m, Tst.data_ptr(), m,
        Vst.data_ptr() if form_uv else None, n, ctypes.byref(kr), ctypes.byref(o))
    native.check(st, "randutv_factor_host")
    return UTV(Ust.t() if form_uv else None, Tst.t(), Vst.t() if form_uv else None, kr.value)


def gaussian(seed, step, k, b, device="cuda"):
    """(k, b) float64 CUDA tensor: the Gaussian G of global step ``step``."""
    torch = _torch()
    st_ = torch.empty((b, k), dtype=torch.float64, device=device)
    _bind_stream()
    native.check(native.lib().randutv_gaussian(int(seed), int(step), int(k), int(b), st_.data_ptr(), max(1, k)),
                 "randutv_gaussian")
    return st_.t()


def philox_words(seed, step, k, b, device="cuda"):
    """Raw Philox words, int64 tensor of shape (b, ceil(k/2), 4) (uint32 values)."""
    torch = _torch()
    npairs = (k + 1) // 2
    w = torch.empty((b, npairs, 4), dtype=torch.int32, device=device)
    _bind_stream()
    native.check(native.lib().randutv_philox_words(int(seed), int(step), int(k), int(b), w.data_ptr()),
                 "randutv_philox_words")
    return w.to(torch.int64) & 0xFFFFFFFF


def dgemm(A, B, ta=False, tb=False, alpha=1.0, beta=0.0, C=None):
    """alpha op(A) op(B) + beta C with the library's FP64 GEMM (torch layout)."""
    torch = _torch()
    _check_cuda64(A, "A")
    _check_cuda64(B, "B")
    Ac, Bc = _colmajor(A), _colmajor(B)
    m = A.shape[1] if ta else A.shape[0]
    k = A.shape[0] if ta else A.shape[1]
    n = B.shape[0] if tb else B.shape[1]
    if (B.shape[1] if tb else B.shape[0]) != k:
        raise ValueError("inner dimensions differ")
    Cst = _colmajor(C) if C is not None else torch.empty((n, m), dtype=torch.float64, device=A.device)
    _bind_stream()
    st = native.lib().randutv_dgemm(b"T" if ta else b"N", b"T" if tb else b"N", m, n, k, float(alpha),
                                    Ac.data_ptr(), A.shape[0], Bc.data_ptr(), B.shape[0], float(beta),
                                    Cst.data_ptr(), m)
    native.check(st, "randutv_dgemm")
    return Cst.t()


def sgemm(A, B, ta=False, tb=False, alpha=1.0, beta=0.0, C=None):
    """alpha op(A) op(B) + beta C with the library's FP32 GEMM (torch layout)."""
    torch = _torch()
    for x, nm in ((A, "A"), (B, "B")):
        if not isinstance(x, torch.Tensor) or x.dim() != 2 or x.dtype != torch.float32 or not x.is_cuda:
            raise TypeError(f"{nm} must be a 2-D float32 CUDA tensor")
    Ac, Bc = _colmajor(A), _colmajor(B)
    m = A.shape[1] if ta else A.shape[0]
    k = A.shape[0] if ta else A.shape[1]
    n = B.shape[0] if tb else B.shape[1]
    if (B.shape[1] if tb else B.shape[0]) != k:
        raise ValueError("inner dimensions differ")
    Cst = _colmajor(C) if C is not None else torch.empty((n, m), dtype=torch.float32, device=A.device)
    _bind_stream()
    st = native.lib().randutv_sgemm(b"T" if ta else b"N", b"T" if tb else b"N", m, n, k, float(alpha),
                                    Ac.data_ptr(), A.shape[0], Bc.data_ptr(), B.shape[0], float(beta),
                                    Cst.data_ptr(), m)
    native.check(st, "randutv_sgemm")
    return Cst.t()


def panel_qr(P):
    """Householder QR of a (k, w) panel: returns (P_out, tau, Vexp, S) with
    P_out holding R above and the vectors below the diagonal."""
    torch = _torch()
    _check_cuda64(P, "P")
    k, w = P.shape
    Pst = _colmajor(P)
    tau = torch.empty(w, dtype=torch.float64, device=P.device)
    Vst = torch.empty((w, k), dtype=torch.float64, device=P.device)
    Sst = torch.empty((w, w), dtype=torch.float64, device=P.device)
    _bind_stream()
    native.check(native.lib().randutv_panel_qr(k, w, Pst.data_ptr(), k, tau.data_ptr(), Vst.data_ptr(),
                                               Sst.data_ptr()), "randutv_panel_qr")
    return Pst.t(), tau, Vst.t(), Sst.t()


def small_svd(M, max_sweeps=30):
    """Jacobi SVD of a (p, p) block: (Us, d, Vs) with M = Us diag(d) Vs^T."""
    torch = _torch()
    _check_cuda64(M, "M")
    p = M.shape[0]
    if M.shape[1] != p:
        raise ValueError("M must be square")
    Mst = _colmajor(M)
    Us = torch.empty((p, p), dtype=torch.float64, device=M.device)
    Vs = torch.empty((p, p), dtype=torch.float64, device=M.device)
    d = torch.empty(p, dtype=torch.float64, device=M.device)
    _bind_stream()
    native.check(native.lib().randutv_small_svd(p, Mst.data_ptr(), p, Us.data_ptr(), d.data_ptr(),
                                                Vs.data_ptr(), int(max_sweeps)), "randutv_small_svd")
    return Us.t(), d, Vs.t()
