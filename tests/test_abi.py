"""The C ABI library loads, exports every symbol include/randutv.h declares,
and rejects invalid arguments before touching the GPU (no GPU needed)."""
import ctypes
import os
import re
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "randutv.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(randutv_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1703_00998_gb300 import native
    return native.lib()


def test_header_lists_entry_points():
    names = declared_functions()
    for must in ("randutv_factor", "randutv_factor_ex", "randutv_set_stream", "randutv_free",
                 "randutv_strerror", "randutv_factor_host"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1703_00998_gb300 import native
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in native.SIGNATURES, f"binding misses {name}"


def test_strerror_and_defaults(lib):
    from paper_1703_00998_gb300 import native
    assert lib.randutv_strerror(0) == b"success"
    assert b"max_sweeps" in lib.randutv_strerror(2)
    o = native.default_opts()
    assert (o.precision, o.form_uv, o.max_sweeps, o.p, o.seed, o.overlap, o.tensor_cores, o.fp64_emulation) == (
        0, 1, 30, 0, 998, 1, 1, 1)
    assert o.g_inject is None
    assert o.sketch_prec == 0 and o.g_capture is None


def test_sketch_prec_validation(lib):
    # the FP64 form has one sketch precision; the mixed form takes the two tensor-core forms
    from paper_1703_00998_gb300 import native
    k = ctypes.c_int64(0)
    dummy = ctypes.c_void_p(16)
    o = native.default_opts()
    o.sketch_prec = 1
    assert lib.randutv_factor_ex(4, 4, dummy, 4, 2, 1, 0.0, dummy, 4, dummy, 4, dummy, 4, ctypes.byref(k),
                                 ctypes.byref(o)) == -15
    o.sketch_prec = 3
    assert lib.randutv_factor_mixed(4, 4, dummy, 4, 2, 1, 0.0, dummy, 4, dummy, 4, dummy, 4, ctypes.byref(k),
                                    ctypes.byref(o)) == -15


def test_argument_validation(lib):
    k = ctypes.c_int64(0)
    dummy = ctypes.c_void_p(16)
    f = lib.randutv_factor_ex
    assert f(0, 4, dummy, 4, 2, 1, 0.0, dummy, 4, dummy, 4, dummy, 4, ctypes.byref(k), None) == -1
    assert f(4, 0, dummy, 4, 2, 1, 0.0, dummy, 4, dummy, 4, dummy, 4, ctypes.byref(k), None) == -2
    assert f(4, 4, None, 4, 2, 1, 0.0, dummy, 4, dummy, 4, dummy, 4, ctypes.byref(k), None) == -3
    assert f(4, 4, dummy, 3, 2, 1, 0.0, dummy, 4, dummy, 4, dummy, 4, ctypes.byref(k), None) == -4
    assert f(4, 4, dummy, 4, 0, 1, 0.0, dummy, 4, dummy, 4, dummy, 4, ctypes.byref(k), None) == -5
    assert f(4, 4, dummy, 4, 2, -1, 0.0, dummy, 4, dummy, 4, dummy, 4, ctypes.byref(k), None) == -6
    assert f(4, 4, dummy, 4, 2, 1, -1.0, dummy, 4, dummy, 4, dummy, 4, ctypes.byref(k), None) == -7
    assert f(4, 4, dummy, 4, 2, 1, float("nan"), dummy, 4, dummy, 4, dummy, 4, ctypes.byref(k), None) == -7
    assert f(4, 4, dummy, 4, 2, 1, 0.0, None, 4, dummy, 4, dummy, 4, ctypes.byref(k), None) == -8
    assert f(4, 4, dummy, 4, 2, 1, 0.0, dummy, 4, dummy, 3, dummy, 4, ctypes.byref(k), None) == -11
    assert f(4, 4, dummy, 4, 2, 1, 0.0, dummy, 4, dummy, 4, dummy, 4, None, None) == -14
    assert lib.randutv_factor(4, 4, dummy, 4, 2, 1, 0.0, None, None, None, ctypes.byref(k)) == -8
    assert lib.randutv_dgemm(b"X", b"N", 1, 1, 1, 1.0, dummy, 1, dummy, 1, 0.0, dummy, 1) == -1
    assert lib.randutv_panel_qr(4, 5, dummy, 4, dummy, dummy, dummy) == -2
    assert lib.randutv_small_svd(0, dummy, 1, dummy, dummy, dummy, 30) == -1
    assert lib.randutv_gaussian(1, 0, 4, 4, dummy, 4) == -2


def test_opts_validation(lib):
    from paper_1703_00998_gb300 import native
    k = ctypes.c_int64(0)
    dummy = ctypes.c_void_p(16)
    o = native.default_opts()
    o.p = -1                      # over-sampling must be >= 0
    assert lib.randutv_factor_ex(4, 4, dummy, 4, 2, 1, 0.0, dummy, 4, dummy, 4, dummy, 4, ctypes.byref(k),
                                 ctypes.byref(o)) == -15
    o.p = 300                     # b + p above 256: refused before any device work
    assert lib.randutv_factor_ex(4, 4, dummy, 4, 2, 1, 0.0, dummy, 4, dummy, 4, dummy, 4, ctypes.byref(k),
                                 ctypes.byref(o)) == native.EUNSUPPORTED
    o.p = 5                       # the mixed form has no over-sampling
    assert lib.randutv_factor_mixed(4, 4, dummy, 4, 2, 1, 0.0, dummy, 4, dummy, 4, dummy, 4, ctypes.byref(k),
                                    ctypes.byref(o)) == -15


def test_batched_argument_validation(lib):
    import numpy as np
    h = ctypes.c_void_p()
    m = np.array([64, 80], dtype=np.int32)
    n = np.array([70, 64], dtype=np.int32)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    f = lib.randutv_batched_plan_create
    assert f(-1, vp(m), vp(n), 0, ctypes.byref(h)) == -1
    assert f(2, None, vp(n), 0, ctypes.byref(h)) == -2
    assert f(2, vp(m), None, 0, ctypes.byref(h)) == -3
    assert f(2, vp(m), vp(n), 33, ctypes.byref(h)) == -4
    assert f(2, vp(m), vp(n), -1, ctypes.byref(h)) == -4
    assert f(2, vp(m), vp(n), 0, None) == -5
    bad = np.array([64, 0], dtype=np.int32)
    assert f(2, vp(bad), vp(n), 0, ctypes.byref(h)) == -2
    assert f(2, vp(m), vp(bad), 0, ctypes.byref(h)) == -3
    big = np.array([64, 513], dtype=np.int32)
    from paper_1703_00998_gb300 import native
    assert f(2, vp(big), vp(n), 0, ctypes.byref(h)) == native.EUNSUPPORTED
    assert b"512" in lib.randutv_last_error()
    dummy = ctypes.c_void_p(16)
    o = native.default_batched_opts()
    assert (o.form_uv, o.max_sweeps, o.seed, o.graph, o.async_) == (1, 30, 998, 0, 0)
    assert lib.randutv_factor_batched(None, dummy, dummy, dummy, dummy, 1, 1e-5, dummy, None, ctypes.byref(o)) == -1
    assert lib.randutv_batched_layout(None, None, None, None, None, None, None) == -1
    assert lib.randutv_batched_autotune(None, dummy, 1, 1e-5, None, None) == -1
    assert lib.randutv_batched_set_classes(None, None) == -1
    assert lib.randutv_batched_plan_destroy(None) == -1
    g = lib.randutv_batched_gaussian
    assert g(1, -1, 1, 4, 4, dummy, 4) == -2
    assert g(1, 0, 0, 4, 4, dummy, 4) == -3
    assert g(1, 0, 1, -1, 4, dummy, 4) == -4
    assert g(1, 0, 1, 4, -1, dummy, 4) == -5
    assert g(1, 0, 1, 4, 4, None, 4) == -6
    assert g(1, 0, 1, 4, 4, dummy, 3) == -7


def test_rank_k_argument_validation(lib):
    dummy = ctypes.c_void_p(16)
    from paper_1703_00998_gb300 import native
    f = lib.randutv_rank_k
    h = ctypes.c_void_p()
    assert f(0, 8, dummy, 8, 2, 1, 4, dummy, 8, None, ctypes.byref(h)) == -1
    assert f(8, 0, dummy, 8, 2, 1, 4, dummy, 8, None, ctypes.byref(h)) == -2
    assert f(8, 8, None, 8, 2, 1, 4, dummy, 8, None, ctypes.byref(h)) == -3
    assert f(8, 8, dummy, 7, 2, 1, 4, dummy, 8, None, ctypes.byref(h)) == -4
    assert f(8, 8, dummy, 8, 0, 1, 4, dummy, 8, None, ctypes.byref(h)) == -5
    assert f(8, 8, dummy, 8, 2, -1, 4, dummy, 8, None, ctypes.byref(h)) == -6
    assert f(8, 8, dummy, 8, 2, 1, 3, dummy, 8, None, ctypes.byref(h)) == -7      # k not a multiple of b
    assert f(8, 8, dummy, 8, 2, 1, 4, None, 8, None, ctypes.byref(h)) == -8
    assert f(8, 8, dummy, 8, 2, 1, 4, dummy, 7, None, ctypes.byref(h)) == -9
    assert f(80, 80, dummy, 80, 40, 1, 40, dummy, 80, None, ctypes.byref(h)) == native.EUNSUPPORTED   # b > 32
    assert f(8, 8, dummy, 8, 2, 1, 8, dummy, 8, None, ctypes.byref(h)) == native.EUNSUPPORTED        # k = min(m, n)
    o = native.default_opts()
    o.p = 3
    assert f(8, 8, dummy, 8, 2, 1, 4, dummy, 8, ctypes.byref(o), ctypes.byref(h)) == -10
    assert lib.randutv_rank_k_vjp(None, dummy, 8, dummy, 8) == -1
    assert lib.randutv_rank_k_free(None) == -1


def test_selftest_wait_argument_validation(lib):
    # rejected before any CUDA call: unknown kind, limits outside (0, 2] s
    assert lib.randutv_selftest_wait(2, 0.1) == -1
    assert lib.randutv_selftest_wait(-1, 0.1) == -1
    assert lib.randutv_selftest_wait(0, 0.0) == -2
    assert lib.randutv_selftest_wait(1, 2.5) == -2
    assert lib.randutv_selftest_wait(0, float("nan")) == -2
