"""Helpers for the GPU parity tests: build once, move arrays, run the oracle."""
import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def host(x):
    return x.detach().cpu().numpy()


_CUDART = None


def cudart():
    """The CUDA runtime torch loaded (ctypes), for raw copies of device
    pointers the library returns (it shares the process's device context)."""
    global _CUDART
    if _CUDART is None:
        import ctypes
        import torch
        torch.cuda.init()
        path = None
        for line in open("/proc/self/maps"):
            parts = line.split()
            if len(parts) >= 6 and "libcudart.so" in parts[-1]:
                path = parts[-1]
                break
        _CUDART = ctypes.CDLL(path or "libcudart.so.13")
    return _CUDART


def device_to_host(ptr, shape_colmajor):
    """Copy a column-major FP64 device matrix (m, n) at a raw pointer to numpy (m, n)."""
    import ctypes
    m, n = shape_colmajor
    out = np.empty((n, m), dtype=np.float64)
    rt = cudart()
    rt.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    st = rt.cudaMemcpy(out.ctypes.data, ptr, out.nbytes, 2)   # cudaMemcpyDeviceToHost
    assert st == 0, f"cudaMemcpy returned {st}"
    return out.T
