"""The C-ABI library builds, loads and exports every symbol include/flr.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(flr_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1306_1970_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("flr_create", "flr_solve", "flr_solve_batch", "flr_destroy", "flr_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    import paper_1306_1970_gb300 as flr
    assert sorted(flr.EXPORTS) == declared_functions()


def test_strerror_without_gpu(lib):
    lib.flr_strerror.restype = ctypes.c_char_p
    lib.flr_strerror.argtypes = [ctypes.c_int32]
    assert lib.flr_strerror(0).startswith(b"FLR_OK")
    assert lib.flr_strerror(1).startswith(b"FLR_EINVAL")
    assert lib.flr_strerror(99) == b"unknown flr_status"


def test_invalid_arguments_rejected_before_any_device_work(lib):
    import paper_1306_1970_gb300 as flr
    flr.load()
    out = ctypes.c_void_p()
    g = flr.FlrGraph()
    g.kind = flr.FLR_E_CHAIN
    # null X / n < 1 / ldx < p are refused without touching the GPU
    assert lib.flr_create(None, 1, 10, 5, 5, None, ctypes.byref(g), 0, None, ctypes.byref(out)) == 1
    buf = (ctypes.c_double * 50)()
    assert lib.flr_create(buf, 1, 0, 5, 5, buf, ctypes.byref(g), 1, None, ctypes.byref(out)) == 1
    assert lib.flr_create(buf, 1, 10, 5, 4, buf, ctypes.byref(g), 1, None, ctypes.byref(out)) == 1
    assert lib.flr_create(buf, 9, 10, 5, 5, buf, ctypes.byref(g), 1, None, ctypes.byref(out)) == 1
    g.kind, g.q1, g.q2 = flr.FLR_E_LATTICE, 2, 3
    assert lib.flr_create(buf, 1, 10, 5, 5, buf, ctypes.byref(g), 1, None, ctypes.byref(out)) == 1


def test_footprint_estimate_is_monotone_and_validates(lib):
    lib.flr_footprint.restype = ctypes.c_int64
    lib.flr_footprint.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                  ctypes.c_int32]
    f = lib.flr_footprint
    base = f(1000, 10000, 19800, 1, 0)
    assert base >= 1000 * 10000 * 4          # at least the column-major copy of X
    assert f(1000, 10000, 19800, 1, 1) > base  # host inputs add a staging copy
    assert f(2000, 10000, 19800, 1, 0) > base
    assert f(1000, 20000, 19800, 1, 0) > base
    assert f(1000, 10000, 19800, 2, 0) < base  # 16-bit X
    assert f(0, 10, 9, 1, 0) < 0 and f(10, 10, 9, 7, 0) < 0
