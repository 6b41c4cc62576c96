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


def _c_layout():
    """sizeof/offsetof of the header's structs and its enum values, from a C program
    compiled against include/flr.h (gcc; no CUDA needed)."""
    import shutil
    import subprocess
    import tempfile
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    fields = {
        "flr_graph": ["kind", "q1", "q2", "edges", "m"],
        "flr_opts": ["max_mm", "max_cg", "min_cg", "precond", "tol_cg", "grid", "inject_stall",
                     "wait_cycles", "max_refine", "x_smem", "tol_cg_rel"],
        "flr_stats": ["mm_iters", "f", "ms", "refine_steps", "est_err"],
        "flr_server_opts": [],
        "flr_request": ["opts", "use_opts", "data_id"],
        "flr_result": ["stats", "t_submit", "footprint", "dev_t0_ns", "dev_t1_ns", "reused"],
    }
    enums = ["FLR_OK", "FLR_EINVAL", "FLR_ENOMEM", "FLR_ECUDA", "FLR_ENOTCONV", "FLR_EBREAKDOWN",
             "FLR_ENONFINITE", "FLR_ETIMEOUT", "FLR_ENOTIMPL", "FLR_ESCRATCH", "FLR_F64", "FLR_F32",
             "FLR_BF16", "FLR_F16", "FLR_IDENTITY", "FLR_MEM_DEVICE", "FLR_MEM_HOST", "FLR_E_CHAIN", "FLR_E_LATTICE",
             "FLR_E_EDGES", "FLR_PC_AUTO", "FLR_PC_JACOBI", "FLR_PC_TRIDIAG", "FLR_PC_PAPER",
             "FLR_PC_TWOLEVEL"]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "flr.h"', "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'  printf("size {st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'  printf("off {st}.{f} %zu\\n", offsetof({st}, {f}));')
    for e in enums:
        lines.append(f'  printf("enum {e} %d\\n", (int){e});')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as fh:
            fh.write("\n".join(lines))
        subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                       check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    res = {}
    for ln in out.splitlines():
        kind, key, val = ln.split()
        res[(kind, key)] = int(val)
    return res


def test_binding_structs_and_enums_match_the_header():
    """The ctypes mirrors in the binding have the header's sizes, field offsets
    and enum values, so no call marshals a shifted field."""
    import paper_1306_1970_gb300 as flr
    c = _c_layout()
    mirrors = {"flr_graph": flr.FlrGraph, "flr_opts": flr.FlrOpts, "flr_stats": flr.FlrStats,
               "flr_server_opts": flr.FlrServerOpts, "flr_request": flr.FlrRequest,
               "flr_result": flr.FlrResult}
    for name, cls in mirrors.items():
        assert ctypes.sizeof(cls) == c[("size", name)], name
    for (kind, key), val in c.items():
        if kind == "off":
            st, f = key.split(".")
            assert getattr(mirrors[st], f).offset == val, key
    for (kind, key), val in c.items():
        if kind != "enum":
            continue
        if key.startswith("FLR_PC_"):
            assert flr.PRECOND[key[len("FLR_PC_"):].lower()] == val, key
        else:
            assert getattr(flr, key) == val, key
