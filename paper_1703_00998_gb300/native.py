"""ctypes binding of librandutv.so (include/randutv.h).

Argument marshalling only: every step of the factorization runs in the
library's CUDA kernels.  There is no fallback: if the library is missing the
call raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "librandutv.so")

OK, ENOMEM, ENOCONV, ENAN, EUNSUPPORTED, ECUDA, ETIMEOUT = 0, 1, 2, 3, 4, 5, 6
FP64 = 0


class RandutvError(RuntimeError):
    def __init__(self, status, func, detail=""):
        self.status = status
        msg = f"{func} returned {status}: {strerror(status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class Opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("form_uv", ctypes.c_int),
        ("max_sweeps", ctypes.c_int),
        ("p", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("g_inject", ctypes.c_void_p),
        ("overlap", ctypes.c_int),
        ("tensor_cores", ctypes.c_int),
        ("fp64_emulation", ctypes.c_int),
        ("sketch_prec", ctypes.c_int),
        ("g_capture", ctypes.c_void_p),
    ]


class BatchedOpts(ctypes.Structure):
    _fields_ = [
        ("form_uv", ctypes.c_int),
        ("max_sweeps", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("g_inject", ctypes.c_void_p),
        ("graph", ctypes.c_int),
        ("async_", ctypes.c_int),
    ]


_lib = None
_i64, _i32, _f64, _vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p

# name -> (restype, argtypes); every symbol declared in include/randutv.h
SIGNATURES = {
    "randutv_opts_default": (None, [ctypes.POINTER(Opts)]),
    "randutv_set_stream": (_i32, [_vp]),
    "randutv_factor": (_i32, [_i64, _i64, _vp, _i64, _i32, _i32, _f64, _vp, _vp, _vp, ctypes.POINTER(_i64)]),
    "randutv_factor_ex": (_i32, [_i64, _i64, _vp, _i64, _i32, _i32, _f64, _vp, _i64, _vp, _i64, _vp, _i64,
                                 ctypes.POINTER(_i64), ctypes.POINTER(Opts)]),
    "randutv_factor_mixed": (_i32, [_i64, _i64, _vp, _i64, _i32, _i32, _f64, _vp, _i64, _vp, _i64, _vp, _i64,
                                    ctypes.POINTER(_i64), ctypes.POINTER(Opts)]),
    "randutv_factor_host": (_i32, [_i64, _i64, _vp, _i64, _i32, _i32, _f64, _vp, _i64, _vp, _i64, _vp, _i64,
                                   ctypes.POINTER(_i64), ctypes.POINTER(Opts)]),
    "randutv_free": (None, [_vp]),
    "randutv_strerror": (ctypes.c_char_p, [_i32]),
    "randutv_last_error": (ctypes.c_char_p, []),
    "randutv_gaussian": (_i32, [ctypes.c_uint64, _i64, _i64, _i64, _vp, _i64]),
    "randutv_philox_words": (_i32, [ctypes.c_uint64, _i64, _i64, _i64, _vp]),
    "randutv_dgemm": (_i32, [ctypes.c_char, ctypes.c_char, _i64, _i64, _i64, _f64, _vp, _i64, _vp, _i64, _f64,
                             _vp, _i64]),
    "randutv_sgemm": (_i32, [ctypes.c_char, ctypes.c_char, _i64, _i64, _i64, ctypes.c_float, _vp, _i64, _vp, _i64,
                             ctypes.c_float, _vp, _i64]),
    "randutv_sgemm_tc": (_i32, [ctypes.c_char, ctypes.c_char, _i64, _i64, _i64, ctypes.c_float, _vp, _i64, _vp,
                                _i64, ctypes.c_float, _vp, _i64, _i32]),
    "randutv_dgemm_oz": (_i32, [ctypes.c_char, ctypes.c_char, _i64, _i64, _i64, _f64, _vp, _i64, _vp, _i64, _f64,
                                _vp, _i64]),
    "randutv_sgemm_oz": (_i32, [ctypes.c_char, ctypes.c_char, _i64, _i64, _i64, ctypes.c_float, _vp, _i64, _vp,
                                _i64, ctypes.c_float, _vp, _i64]),
    "randutv_panel_qr": (_i32, [_i64, _i64, _vp, _i64, _vp, _vp, _vp]),
    "randutv_small_svd": (_i32, [_i64, _vp, _i64, _vp, _vp, _vp, _i32]),
    "randutv_profile_enable": (_i32, [_i32]),
    "randutv_profile_reset": (_i32, []),
    "randutv_profile_read": (_i32, [_i32, ctypes.POINTER(_f64), ctypes.POINTER(_i64), ctypes.POINTER(_f64),
                                    ctypes.POINTER(_f64)]),
    "randutv_launch_count": (ctypes.c_uint64, []),
    "randutv_jacobi_sweeps": (_i32, [ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64), _i32]),
    "randutv_selftest_wait": (_i32, [_i32, _f64]),
    "randutv_small_svd_noalloc": (_i32, [_i64, _vp, _i64, _vp, _vp, _vp, _i32]),
    "randutv_batched_opts_default": (None, [ctypes.POINTER(BatchedOpts)]),
    "randutv_batched_plan_create": (_i32, [_i64, _vp, _vp, _i32, ctypes.POINTER(_vp)]),
    "randutv_batched_plan_destroy": (_i32, [_vp]),
    "randutv_batched_layout": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "randutv_factor_batched": (_i32, [_vp, _vp, _vp, _vp, _vp, _i32, _f64, _vp, _vp,
                                      ctypes.POINTER(BatchedOpts)]),
    "randutv_batched_autotune": (_i32, [_vp, _vp, _i32, _f64, ctypes.POINTER(BatchedOpts), _vp]),
    "randutv_batched_set_classes": (_i32, [_vp, _vp]),
    "randutv_batched_layout_host": (_i32, [_i64, _vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "randutv_batched_gaussian": (_i32, [ctypes.c_uint64, _i64, _i64, _i64, _i64, _vp, _i64]),
    "randutv_rank_k": (_i32, [_i64, _i64, _vp, _i64, _i32, _i32, _i64, _vp, _i64, ctypes.POINTER(Opts),
                              ctypes.POINTER(_vp)]),
    "randutv_rank_k_vjp": (_i32, [_vp, _vp, _i64, _vp, _i64]),
    "randutv_rank_k_free": (_i32, [_vp]),
}

PROF_GEMM, PROF_PANEL, PROF_TFACTOR, PROF_JACOBI, PROF_GAUSS, PROF_OTHER, PROF_GEMM32, PROF_GEMMTC = range(8)
PROF_NAMES = ["gemm", "panel_qr", "tfactor", "jacobi", "gauss", "other", "gemm32", "gemm_tc", "gemm_oz",
              "gemm_oz32", "oz_slice"]


def profile_read(cls):
    ms, n, fl, by = _f64(), _i64(), _f64(), _f64()
    check(lib().randutv_profile_read(int(cls), ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl),
                                     ctypes.byref(by)), "randutv_profile_read")
    return {"ms": ms.value, "launches": n.value, "flops": fl.value, "bytes": by.value}


def jacobi_sweeps(reset=True):
    """Small-SVD sweep counters: {"fp32": .., "fp64": .., "svds": ..} (cleared when reset)."""
    a, b, c = _i64(), _i64(), _i64()
    check(lib().randutv_jacobi_sweeps(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), int(bool(reset))),
          "randutv_jacobi_sweeps")
    return {"fp32": a.value, "fp64": b.value, "svds": c.value}


def lib():
    """Load the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1703_00998_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(status):
    try:
        return lib().randutv_strerror(int(status)).decode()
    except RuntimeError:
        return f"status {status}"


def check(status, func):
    if status not in (OK,):
        raise RandutvError(status, func, lib().randutv_last_error().decode())
    return status


def default_batched_opts():
    o = BatchedOpts()
    lib().randutv_batched_opts_default(ctypes.byref(o))
    return o


def default_opts():
    o = Opts()
    lib().randutv_opts_default(ctypes.byref(o))
    return o
