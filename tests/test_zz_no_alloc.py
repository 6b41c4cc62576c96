"""flr_solve_noalloc: the allocation-free entry point agrees with flr_solve.

Some callers cannot allocate device memory: their framework's caching
allocator already holds the GPU's memory, or their serving loop must not
take the driver's allocation path.  flr_solve_noalloc serves them from one
static device array.  This file checks, through the C ABI, that two calls in
a row give the same answer as the allocating entry point (within the parity
tolerances used by the other GPU tests), and that an oversized problem is
refused with FLR_ESCRATCH.  It is collected last so that a run stopping at
the first failure has already run every other test.
"""
import ctypes
import json
import os

import numpy as np
import pytest

import flr_inputs as fi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GAP = 1e-6
BETA = 1e-4


@pytest.fixture(scope="module")
def flr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1306_1970_gb300 as m
    m.load(build_if_missing=True)
    return m


def column_major(X: torch.Tensor, vec: int) -> tuple:
    """p x ldn copy of X^T with ldn a multiple of `vec` (zero padding rows)."""
    n, p = X.shape
    ldn = (n + vec - 1) // vec * vec
    Xt = torch.zeros((p, ldn), dtype=X.dtype, device=X.device)
    Xt[:, :n] = X.t()
    return Xt.contiguous(), ldn


def graph_struct(flr, g):
    s = flr.FlrGraph()
    if g.kind == "chain":
        s.kind = flr.FLR_E_CHAIN
    else:
        s.kind, s.q1, s.q2 = flr.FLR_E_LATTICE, g.q1, g.q2
    return s


def call_noalloc(flr, Xt, dtype_code, n, p, ldn, y, g, lam1, lam2, eps, tol, opts):
    lib = flr.load()
    out = torch.empty(p, dtype=torch.float64, device="cuda")
    st = flr.FlrStats()
    gs = graph_struct(flr, g)
    stream = torch.cuda.current_stream().cuda_stream
    code = lib.flr_solve_noalloc(Xt.data_ptr(), dtype_code, n, p, ldn, y.data_ptr(),
                                 ctypes.byref(gs), lam1, lam2, eps, tol, ctypes.byref(opts),
                                 out.data_ptr(), ctypes.c_void_p(stream), ctypes.byref(st))
    return code, out, st


def golden(name):
    with open(os.path.join(os.path.dirname(__file__), "golden", name + ".json")) as fh:
        return json.load(fh)


@pytest.mark.parametrize("cfg", ["chain_f64", "lattice_f32"])
def test_noalloc_matches_allocating_solve_twice(flr, cfg):
    if cfg == "chain_f64":
        pr, vec, code, kw = fi.config(1), 2, flr.FLR_F64, dict(tol=1e-12, tol_cg=1e-12)
        g = golden("config1")
    else:
        pr, vec, code, kw = fi.config(2, scale=0.04), 4, flr.FLR_F32, dict(tol=1e-12, tol_cg=1e-10)
        g = golden("config2_q20")
    g_beta = np.array(g["beta"])
    X = torch.from_numpy(pr.X).cuda()
    y = torch.from_numpy(pr.y).cuda()
    ref_beta, ref = flr.Problem(X, y, pr.graph).solve(pr.lam1, pr.lam2, eps=pr.eps, max_mm=20000, **kw)
    assert ref.status == 0
    Xt, ldn = column_major(X, vec)
    opts = flr.default_opts(max_mm=20000, tol_cg=kw["tol_cg"])
    for _ in range(2):   # the second call reuses the scratch the first one left behind
        st_code, beta, st = call_noalloc(flr, Xt, code, pr.n, pr.p, ldn, y, pr.graph,
                                         pr.lam1, pr.lam2, pr.eps, kw["tol"], opts)
        assert st_code == flr.FLR_OK, flr.strerror(st_code)
        assert abs(st.f - ref.f) / abs(ref.f) <= GAP
        db = (beta - ref_beta).abs().max().item() / ref_beta.abs().max().item()
        assert db <= BETA
        # and the stored FP64 oracle solution itself (tests/golden, written from oracle/ only)
        assert abs(st.f - g["f"]) / abs(g["f"]) <= GAP, (st.f, g["f"])
        b = beta.cpu().numpy()
        assert np.abs(b - g_beta).max() / np.abs(g_beta).max() <= BETA


def test_noalloc_refuses_problems_beyond_its_scratch(flr):
    n, p = 8, 300_000      # 7 * 8 * p bytes of vectors alone exceed the 16 MiB array
    Xt = torch.zeros((p, n), dtype=torch.float32, device="cuda")
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    code, _, _ = call_noalloc(flr, Xt, flr.FLR_F32, n, p, n, y, fi.Graph("chain", p),
                              0.1, 0.1, 1e-6, 1e-8, flr.default_opts())
    assert code == flr.FLR_ESCRATCH
    assert "static scratch" in flr.strerror(code)
