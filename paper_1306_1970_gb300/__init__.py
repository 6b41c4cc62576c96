"""Python binding of the GB300 fused lasso regression solver (libflr.so).

Argument marshalling only: every step of the solve runs in the CUDA library
whose C ABI is declared in include/flr.h.  PyTorch supplies device memory
and streams.  There is no CPU fallback: without the built library every
entry point raises.

    from paper_1306_1970_gb300 import Problem
    prob = Problem(X, y, graph)            # X: n x p tensor (cuda or host)
    beta, st = prob.solve(lam1, lam2, eps=1e-6, tol=1e-9)
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional

from . import _build

FLR_OK, FLR_EINVAL, FLR_ENOMEM, FLR_ECUDA, FLR_ENOTCONV = 0, 1, 2, 3, 4
FLR_EBREAKDOWN, FLR_ENONFINITE, FLR_ETIMEOUT, FLR_ENOTIMPL, FLR_ESCRATCH = 5, 6, 7, 8, 9
FLR_F64, FLR_F32, FLR_BF16, FLR_F16, FLR_IDENTITY = 0, 1, 2, 3, 4
FLR_MEM_DEVICE, FLR_MEM_HOST = 0, 1
FLR_E_CHAIN, FLR_E_LATTICE, FLR_E_EDGES = 0, 1, 2
PRECOND = {"auto": 0, "jacobi": 1, "tridiag": 2, "paper": 3, "twolevel": 4}
DTYPE_CODES = {"f64": FLR_F64, "f32": FLR_F32, "bf16": FLR_BF16, "f16": FLR_F16,
               "identity": FLR_IDENTITY}

# every symbol declared in include/flr.h
EXPORTS = ("flr_default_opts", "flr_strerror", "flr_create", "flr_solve", "flr_solve_batch",
           "flr_destroy", "flr_get_info", "flr_solve_noalloc", "flr_server_create",
           "flr_server_submit", "flr_server_poll", "flr_server_wait", "flr_server_destroy",
           "flr_footprint", "flr_solve_dense")


class FlrGraph(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("q1", ctypes.c_int64),
                ("q2", ctypes.c_int64), ("edges", ctypes.c_void_p), ("m", ctypes.c_int64)]


class FlrOpts(ctypes.Structure):
    _fields_ = [("max_mm", ctypes.c_int32), ("max_cg", ctypes.c_int32), ("min_cg", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("tol_cg", ctypes.c_double), ("grid", ctypes.c_int32),
                ("inject_stall", ctypes.c_int32), ("wait_cycles", ctypes.c_int64),
                ("max_refine", ctypes.c_int32), ("x_smem", ctypes.c_int32),
                ("tol_cg_rel", ctypes.c_double)]


class FlrStats(ctypes.Structure):
    _fields_ = [("mm_iters", ctypes.c_int32), ("cg_iters", ctypes.c_int32),
                ("status", ctypes.c_int32), ("grid", ctypes.c_int32), ("f", ctypes.c_double),
                ("f_eps", ctypes.c_double), ("rel_change", ctypes.c_double),
                ("cg_relres", ctypes.c_double), ("ms", ctypes.c_double),
                ("refine_steps", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("est_err", ctypes.c_double)]


class FlrServerOpts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("grid_per_slot", ctypes.c_int32),
                ("hbm_budget", ctypes.c_int64), ("reserved", ctypes.c_int32 * 8)]


class FlrRequest(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("mem", ctypes.c_int32),
                ("n", ctypes.c_int64), ("p", ctypes.c_int64), ("ldx", ctypes.c_int64),
                ("y", ctypes.c_void_p), ("E", FlrGraph), ("lambda1", ctypes.c_double),
                ("lambda2", ctypes.c_double), ("eps", ctypes.c_double), ("tol", ctypes.c_double),
                ("opts", FlrOpts), ("use_opts", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("data_id", ctypes.c_uint64)]


class FlrResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("slot", ctypes.c_int32), ("stats", FlrStats),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_end", ctypes.c_double), ("footprint", ctypes.c_int64),
                ("dev_t0_ns", ctypes.c_uint64), ("dev_t1_ns", ctypes.c_uint64),
                ("reused", ctypes.c_int32), ("reserved2", ctypes.c_int32)]


class FlrError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)}")


_LIB = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libflr.so (optionally building it first); raises if it is absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_missing and _build.stale():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libflr.so is not built; run __graft_entry__.build() "
                           "(paper_1306_1970_gb300._build.build()) first")
    lib = ctypes.CDLL(_build.LIB)
    c = ctypes
    lib.flr_default_opts.argtypes = [c.POINTER(FlrOpts)]
    lib.flr_default_opts.restype = None
    lib.flr_strerror.argtypes = [c.c_int32]
    lib.flr_strerror.restype = c.c_char_p
    lib.flr_create.argtypes = [c.c_void_p, c.c_int32, c.c_int64, c.c_int64, c.c_int64, c.c_void_p,
                               c.POINTER(FlrGraph), c.c_int32, c.c_void_p, c.POINTER(c.c_void_p)]
    lib.flr_create.restype = c.c_int32
    lib.flr_solve.argtypes = [c.c_void_p, c.c_double, c.c_double, c.c_double, c.c_double,
                              c.POINTER(FlrOpts), c.c_void_p, c.c_void_p, c.c_int32,
                              c.POINTER(FlrStats)]
    lib.flr_solve.restype = c.c_int32
    lib.flr_solve_batch.argtypes = [c.c_void_p, c.c_int32, c.c_void_p, c.c_void_p, c.c_double,
                                    c.c_double, c.POINTER(FlrOpts), c.c_void_p, c.c_int32,
                                    c.c_void_p, c.POINTER(FlrStats)]
    lib.flr_solve_batch.restype = c.c_int32
    lib.flr_destroy.argtypes = [c.c_void_p]
    lib.flr_destroy.restype = None
    lib.flr_get_info.argtypes = [c.c_void_p] + [c.c_void_p] * 4
    lib.flr_get_info.restype = c.c_int32
    lib.flr_solve_noalloc.argtypes = [c.c_void_p, c.c_int32, c.c_int64, c.c_int64, c.c_int64,
                                      c.c_void_p, c.POINTER(FlrGraph), c.c_double, c.c_double,
                                      c.c_double, c.c_double, c.POINTER(FlrOpts), c.c_void_p,
                                      c.c_void_p, c.POINTER(FlrStats)]
    lib.flr_solve_noalloc.restype = c.c_int32
    lib.flr_server_create.argtypes = [c.POINTER(FlrServerOpts), c.POINTER(c.c_void_p)]
    lib.flr_server_create.restype = c.c_int32
    lib.flr_server_submit.argtypes = [c.c_void_p, c.POINTER(FlrRequest), c.POINTER(c.c_uint64)]
    lib.flr_server_submit.restype = c.c_int32
    lib.flr_server_poll.argtypes = [c.c_void_p, c.c_uint64, c.POINTER(c.c_int32)]
    lib.flr_server_poll.restype = c.c_int32
    lib.flr_server_wait.argtypes = [c.c_void_p, c.c_uint64, c.c_void_p, c.POINTER(FlrResult)]
    lib.flr_server_wait.restype = c.c_int32
    lib.flr_server_destroy.argtypes = [c.c_void_p]
    lib.flr_server_destroy.restype = c.c_int32
    lib.flr_footprint.argtypes = [c.c_int64, c.c_int64, c.c_int64, c.c_int32, c.c_int32]
    lib.flr_footprint.restype = c.c_int64
    lib.flr_solve_dense.argtypes = [c.c_void_p, c.c_double, c.c_double, c.c_double, c.c_double,
                                    c.c_int32, c.c_void_p, c.c_void_p, c.c_int32, c.POINTER(FlrStats)]
    lib.flr_solve_dense.restype = c.c_int32
    _LIB = lib
    return lib


def strerror(status: int) -> str:
    try:
        return load().flr_strerror(int(status)).decode()
    except RuntimeError:
        return f"flr_status {status}"


def default_opts(**kw) -> FlrOpts:
    o = FlrOpts()
    load().flr_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precond" and isinstance(v, str):
            v = PRECOND[v]
        setattr(o, k, v)
    return o


@dataclasses.dataclass
class Stats:
    mm_iters: int
    cg_iters: int
    status: int
    grid: int
    f: float
    f_eps: float
    rel_change: float
    cg_relres: float
    ms: float
    refine_steps: int = 0
    est_err: float = float("nan")

    @classmethod
    def from_c(cls, s: FlrStats) -> "Stats":
        return cls(s.mm_iters, s.cg_iters, s.status, s.grid, s.f, s.f_eps, s.rel_change,
                   s.cg_relres, s.ms, s.refine_steps, s.est_err)


def _torch():
    import torch
    return torch


def _dtype_code(X, dtype: Optional[str]) -> int:
    if dtype is not None:
        return DTYPE_CODES[dtype]
    torch = _torch()
    m = {torch.float64: FLR_F64, torch.float32: FLR_F32, torch.bfloat16: FLR_BF16,
         torch.float16: FLR_F16}
    if X.dtype not in m:
        raise TypeError(f"unsupported X dtype {X.dtype}; give dtype= for raw 16-bit patterns")
    return m[X.dtype]


def _graph(graph, p: int, keep: list) -> FlrGraph:
    """Accept an object with .kind in {'chain','lattice','edges'} (+ q1, q2, edges)."""
    g = FlrGraph()
    kind = graph.kind if not isinstance(graph, dict) else graph["kind"]
    get = (lambda k, d=None: graph.get(k, d)) if isinstance(graph, dict) else \
        (lambda k, d=None: getattr(graph, k, d))
    if kind == "chain":
        g.kind = FLR_E_CHAIN
    elif kind == "lattice":
        g.kind, g.q1, g.q2 = FLR_E_LATTICE, int(get("q1")), int(get("q2"))
    elif kind == "edges":
        torch = _torch()
        e = torch.as_tensor(get("edges")).to(torch.int64).contiguous().reshape(-1, 2)
        keep.append(e)
        g.kind, g.m = FLR_E_EDGES, int(e.shape[0])
        g.edges = e.data_ptr() if e.numel() else None
    else:
        raise ValueError(f"unknown graph kind {kind!r}")
    return g


class Problem:
    """An FLR problem bound to the current CUDA device and a stream.

    X (n x p, row-major) and y (n) are torch tensors on the GPU or on the
    host (pinned for asynchronous copies); both are copied by the library.
    For BF16/FP16 X pass a torch.bfloat16/float16 tensor, or raw 16-bit
    patterns (int16/uint16) with dtype="bf16"/"f16".  X = None with
    dtype="identity" is the FLSA (X = I, n = p = len(y)).
    """

    def __init__(self, X, y, graph, dtype: Optional[str] = None, stream=None):
        torch = _torch()
        lib = load()
        if X is None:
            if dtype != "identity":
                raise ValueError('X = None needs dtype="identity"')
            self.n = self.p = int(y.shape[0])
            self.dtype = FLR_IDENTITY
            on_dev = y.is_cuda
            dev = y.device
            y = y.to(dtype=torch.float64).contiguous()
            xptr, ldx = None, 0
        else:
            if X.dim() != 2:
                raise ValueError("X must be 2-D (n x p)")
            if X.stride(1) != 1:
                X = X.contiguous()
            self.n, self.p = int(X.shape[0]), int(X.shape[1])
            self.dtype = _dtype_code(X, dtype)
            on_dev = X.is_cuda
            dev = X.device
            y = y.to(device=X.device, dtype=torch.float64).contiguous()
            xptr, ldx = X.data_ptr(), X.stride(0)
        keep = [X, y]
        g = _graph(graph, self.p, keep)
        if g.kind == FLR_E_EDGES and on_dev and g.m:
            keep[-1] = keep[-1].to(dev)
            g.edges = keep[-1].data_ptr()
        self.device = dev if on_dev else torch.device("cuda", torch.cuda.current_device())
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        h = ctypes.c_void_p()
        st = lib.flr_create(xptr, self.dtype, self.n, self.p, ldx, y.data_ptr(),
                            ctypes.byref(g), FLR_MEM_DEVICE if on_dev else FLR_MEM_HOST,
                            ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if st != FLR_OK:
            raise FlrError(st, "flr_create")
        self._h = h
        self._lib = lib

    def solve(self, lam1: float, lam2: float, eps: float = 1e-6, tol: float = 1e-9,
              beta_init=None, out=None, opts: Optional[FlrOpts] = None, check: bool = True,
              **opt_kw):
        """Run the MM solve; returns (beta, Stats).  `out` may be a CUDA or host float64 tensor."""
        torch = _torch()
        if opts is None:
            opts = default_opts(**opt_kw)
        if out is None:
            out = torch.empty(self.p, dtype=torch.float64, device=self.device)
        mem = FLR_MEM_DEVICE if out.is_cuda else FLR_MEM_HOST
        bi = None
        if beta_init is not None:
            bi = beta_init.to(dtype=torch.float64, device=out.device).contiguous()
        s = FlrStats()
        st = self._lib.flr_solve(self._h, float(lam1), float(lam2), float(eps), float(tol),
                                 ctypes.byref(opts), bi.data_ptr() if bi is not None else None,
                                 out.data_ptr(), mem, ctypes.byref(s))
        stats = Stats.from_c(s)
        stats.status = st
        if check and st not in (FLR_OK, FLR_ENOTCONV):
            raise FlrError(st, "flr_solve")
        return out, stats

    def solve_dense(self, lam1: float, lam2: float, eps: float = 1e-6, tol: float = 1e-9,
                    max_mm: int = 10000, beta_init=None, out=None, check: bool = True):
        """Algorithm 1 with a dense FP64 Cholesky per MM iteration (flr_solve_dense)."""
        torch = _torch()
        if out is None:
            out = torch.empty(self.p, dtype=torch.float64, device=self.device)
        mem = FLR_MEM_DEVICE if out.is_cuda else FLR_MEM_HOST
        bi = None
        if beta_init is not None:
            bi = beta_init.to(dtype=torch.float64, device=out.device).contiguous()
        s = FlrStats()
        st = self._lib.flr_solve_dense(self._h, float(lam1), float(lam2), float(eps), float(tol),
                                       int(max_mm), bi.data_ptr() if bi is not None else None,
                                       out.data_ptr(), mem, ctypes.byref(s))
        stats = Stats.from_c(s)
        stats.status = st
        if check and st not in (FLR_OK, FLR_ENOTCONV):
            raise FlrError(st, "flr_solve_dense")
        return out, stats

    def solve_batch(self, lam1s, lam2s, eps: float = 1e-6, tol: float = 1e-9,
                    opts: Optional[FlrOpts] = None, check: bool = True, **opt_kw):
        """Solve a list of (lam1, lam2) pairs; returns (betas p x K, objectives, [Stats])."""
        torch = _torch()
        import numpy as np
        l1 = np.ascontiguousarray(lam1s, dtype=np.float64)
        l2 = np.ascontiguousarray(lam2s, dtype=np.float64)
        K = int(l1.shape[0])
        if opts is None:
            opts = default_opts(**opt_kw)
        betas = torch.empty((K, self.p), dtype=torch.float64, device=self.device)
        objs = np.zeros(K)
        sts = (FlrStats * max(K, 1))()
        st = self._lib.flr_solve_batch(self._h, K, l1.ctypes.data, l2.ctypes.data, float(eps),
                                       float(tol), ctypes.byref(opts), betas.data_ptr(),
                                       FLR_MEM_DEVICE, objs.ctypes.data, sts)
        if check and st not in (FLR_OK, FLR_ENOTCONV):
            raise FlrError(st, "flr_solve_batch")
        return betas.T, objs, [Stats.from_c(sts[k]) for k in range(K)]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.flr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request loop over the solver: `slots` concurrent solves, admission by device
    memory footprint (flr_server_* in include/flr.h).  Inputs are borrowed until
    wait() returns for the request; this object keeps references to them."""

    def __init__(self, slots: int = 4, grid_per_slot: int = 0, hbm_budget: int = 0):
        self._lib = load()
        o = FlrServerOpts()
        o.slots, o.grid_per_slot, o.hbm_budget = slots, grid_per_slot, hbm_budget
        h = ctypes.c_void_p()
        st = self._lib.flr_server_create(ctypes.byref(o), ctypes.byref(h))
        if st != FLR_OK:
            raise FlrError(st, "flr_server_create")
        self._h = h
        self._keep = {}

    def submit(self, X, y, graph, lam1, lam2, eps=1e-6, tol=1e-9, dtype=None, opts=None,
               data_id=0, **opt_kw):
        torch = _torch()
        if X.stride(1) != 1:
            X = X.contiguous()
        on_dev = X.is_cuda
        y = y.to(device=X.device, dtype=torch.float64).contiguous()
        keep = [X, y]
        r = FlrRequest()
        r.X, r.dtype, r.mem = X.data_ptr(), _dtype_code(X, dtype), FLR_MEM_DEVICE if on_dev else FLR_MEM_HOST
        r.n, r.p, r.ldx = int(X.shape[0]), int(X.shape[1]), X.stride(0)
        r.y = y.data_ptr()
        r.E = _graph(graph, r.p, keep)
        if r.E.kind == FLR_E_EDGES and on_dev and r.E.m:
            keep[-1] = keep[-1].to(X.device)
            r.E.edges = keep[-1].data_ptr()
        r.lambda1, r.lambda2, r.eps, r.tol = float(lam1), float(lam2), float(eps), float(tol)
        r.data_id = int(data_id)
        if opts is not None or opt_kw:
            r.opts = opts if opts is not None else default_opts(**opt_kw)
            r.use_opts = 1
        rid = ctypes.c_uint64()
        st = self._lib.flr_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid))
        if st != FLR_OK:
            raise FlrError(st, "flr_server_submit")
        self._keep[rid.value] = (keep, r.p)
        return rid.value

    def poll(self, rid: int) -> bool:
        d = ctypes.c_int32()
        st = self._lib.flr_server_poll(self._h, rid, ctypes.byref(d))
        if st != FLR_OK:
            raise FlrError(st, "flr_server_poll")
        return bool(d.value)

    def wait(self, rid: int):
        """(beta as numpy float64, FlrResult) for a submitted request."""
        import numpy as np
        _, p = self._keep[rid]
        beta = np.zeros(p)
        res = FlrResult()
        self._lib.flr_server_wait(self._h, rid, beta.ctypes.data, ctypes.byref(res))
        del self._keep[rid]
        return beta, res

    def footprint(self, n, p, m, dtype, host=True) -> int:
        return int(self._lib.flr_footprint(n, p, m, DTYPE_CODES.get(dtype, dtype),
                                           FLR_MEM_HOST if host else FLR_MEM_DEVICE))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.flr_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
