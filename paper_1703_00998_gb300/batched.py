"""Batched randUTV of many small FP32 matrices (librandutv's batched form).

Argument marshalling only: the factorization runs in the library's
persistent CUDA kernel.  Matrices travel packed: one 1-D float32 CUDA
tensor holding every matrix column-major, back to back (offsets from the
plan).  ``BatchedPlan.matrix(buf, i)`` views matrix i in torch layout.

    plan = BatchedPlan(ms, ns)             # b = 0: per size class
    plan.autotune(A, q=1, tol=1e-5)        # b in {16, 32} per class, timed
    out = plan.factor(A, q=1, tol=1e-5)    # out.T, out.U, out.V packed; out.k
"""
import ctypes
from collections import namedtuple

import numpy as np

from . import native

BatchedUTV = namedtuple("BatchedUTV", ["U", "T", "V", "k_reached", "info"])


def _torch():
    import torch
    return torch


def _bind_stream():
    torch = _torch()
    native.lib().randutv_set_stream(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _ptr(x):
    return ctypes.c_void_p(x.data_ptr()) if x is not None else None


class BatchedPlan:
    """Sizes, block sizes and the device work table of one batch."""

    def __init__(self, ms, ns, b=0):
        self.m = np.ascontiguousarray(ms, dtype=np.int32)
        self.n = np.ascontiguousarray(ns, dtype=np.int32)
        if self.m.shape != self.n.shape or self.m.ndim != 1:
            raise ValueError("ms and ns must be 1-D of equal length")
        self.count = int(self.m.size)
        h = ctypes.c_void_p()
        native.check(native.lib().randutv_batched_plan_create(
            self.count, self.m.ctypes.data_as(ctypes.c_void_p), self.n.ctypes.data_as(ctypes.c_void_p), int(b),
            ctypes.byref(h)), "randutv_batched_plan_create")
        self._h = h
        self._read_layout()

    def _read_layout(self):
        c = max(self.count, 1)
        self.off_a = np.zeros(c, dtype=np.int64)
        self.off_u = np.zeros(c, dtype=np.int64)
        self.off_v = np.zeros(c, dtype=np.int64)
        self.off_g = np.zeros(c, dtype=np.int64)
        self.b = np.zeros(c, dtype=np.int32)
        tot = np.zeros(4, dtype=np.int64)
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        native.check(native.lib().randutv_batched_layout(self._h, vp(self.off_a), vp(self.off_u), vp(self.off_v),
                                                         vp(self.off_g), vp(self.b), vp(tot)),
                     "randutv_batched_layout")
        self.off_a, self.off_u, self.off_v = self.off_a[:self.count], self.off_u[:self.count], self.off_v[:self.count]
        self.off_g, self.b = self.off_g[:self.count], self.b[:self.count]
        self.total_a, self.total_u, self.total_v, self.total_g = (int(t) for t in tot)

    def close(self):
        if getattr(self, "_h", None):
            native.lib().randutv_batched_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _opts(self, form_uv, seed, max_sweeps, g_inject, graph):
        o = native.default_batched_opts()
        o.form_uv = 1 if form_uv else 0
        o.seed = int(seed)
        o.max_sweeps = int(max_sweeps)
        o.g_inject = _ptr(g_inject)
        o.graph = 1 if graph else 0
        return o

    def set_classes(self, b_per_class):
        arr = np.ascontiguousarray(b_per_class, dtype=np.int32)
        if arr.shape != (8,):
            raise ValueError("eight size classes")
        native.check(native.lib().randutv_batched_set_classes(self._h, arr.ctypes.data_as(ctypes.c_void_p)),
                     "randutv_batched_set_classes")
        self._read_layout()

    def autotune(self, A, q=1, tol=1e-5, form_uv=True, seed=998, max_sweeps=30):
        """Pick b in {16, 32} per size class by timing the batch with each."""
        _bind_stream()
        o = self._opts(form_uv, seed, max_sweeps, None, False)
        choice = np.zeros(8, dtype=np.int32)
        native.check(native.lib().randutv_batched_autotune(self._h, _ptr(A), int(q), float(tol), ctypes.byref(o),
                                                           choice.ctypes.data_as(ctypes.c_void_p)),
                     "randutv_batched_autotune")
        self._read_layout()
        return choice

    def factor(self, A, q=1, tol=1e-5, form_uv=True, seed=998, g_inject=None, graph=False, max_sweeps=30,
               out=None, check=True):
        """Factor every matrix: A packed float32 CUDA tensor (not modified).
        Returns BatchedUTV of packed T, U, V and int32 k_reached, info.  With
        check=False a per-matrix status (info: no convergence, non-finite
        input) does not raise."""
        torch = _torch()
        if not (isinstance(A, torch.Tensor) and A.is_cuda and A.dtype == torch.float32 and A.dim() == 1
                and A.is_contiguous() and A.numel() == self.total_a):
            raise TypeError(f"A must be a contiguous 1-D float32 CUDA tensor of {self.total_a} elements")
        dev = A.device
        if out is None:
            T = torch.empty(self.total_a, dtype=torch.float32, device=dev)
            U = torch.empty(self.total_u, dtype=torch.float32, device=dev) if form_uv else None
            V = torch.empty(self.total_v, dtype=torch.float32, device=dev) if form_uv else None
            k = torch.empty(max(self.count, 1), dtype=torch.int32, device=dev)
            info = torch.empty(max(self.count, 1), dtype=torch.int32, device=dev)
        else:
            U, T, V, k, info = out
        if g_inject is not None and (g_inject.dtype != torch.float32 or not g_inject.is_cuda
                                     or g_inject.numel() < self.total_g):
            raise TypeError("g_inject must be a float32 CUDA tensor holding every matrix's Gaussian stream")
        _bind_stream()
        o = self._opts(form_uv, seed, max_sweeps, g_inject, graph)
        st = native.lib().randutv_factor_batched(self._h, _ptr(A), _ptr(T), _ptr(U), _ptr(V), int(q), float(tol),
                                                 _ptr(k), _ptr(info), ctypes.byref(o))
        if check or st not in (native.OK, native.ENOCONV, native.ENAN):
            native.check(st, "randutv_factor_batched")
        return BatchedUTV(U, T, V, k[:self.count], info[:self.count])

    def matrix(self, buf, i, which="a"):
        """Matrix i of a packed buffer, torch layout (rows, cols): which is
        'a' (A or T), 'u' or 'v'."""
        m, n = int(self.m[i]), int(self.n[i])
        off, r, c = {"a": (self.off_a, m, n), "u": (self.off_u, m, m), "v": (self.off_v, n, n)}[which]
        o = int(off[i])
        return buf[o:o + r * c].view(c, r).t()


def batched_gaussian(seed, index, step, k, w, device="cuda"):
    """(k, w) float32 CUDA tensor: the G the batched kernel draws for matrix
    ``index`` at step ``step``."""
    torch = _torch()
    st_ = torch.empty((w, k), dtype=torch.float32, device=device)
    _bind_stream()
    native.check(native.lib().randutv_batched_gaussian(int(seed), int(index), int(step), int(k), int(w),
                                                       st_.data_ptr(), max(1, k)), "randutv_batched_gaussian")
    return st_.t()
