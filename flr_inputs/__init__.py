"""Seeded synthetic inputs for fused lasso regression (FLR) problems.

This module produces problem data only: design matrices X (quantised to a
storage dtype), responses y, true coefficient patterns and edge sets E.  It
holds none of the method's arithmetic (no weights, no surrogate systems, no
objective), so both the CPU oracle and the GPU path may import it.

Workload shapes follow the paper's numerical studies (Section 5):
  * standard (chain) FLR, y = X beta + noise with X rows iid N(0, I_p)
    (Section 5.1, Eq. gener); true-coefficient scenarios C1-C3;
  * two-dimensional FLR on a q1 x q2 lattice with block patterns (Section 5.2,
    scenario C4);
plus the five benchmark configurations of this library (chain FP64, lattice
FP32, batched chain BF16, large lattice FP16, a served mixed stream).

All randomness comes from numpy.random.default_rng(seed).  Storage
quantisation (FP32 / BF16 / FP16) is applied on the host, and the exact
float64 widening of the stored values is what every solver sees as X.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

DTYPES = ("f64", "f32", "bf16", "f16")


# ----------------------------------------------------------------------------
# storage dtypes
# ----------------------------------------------------------------------------
def f32_to_bf16_bits(x32: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even).

    Returns the 16-bit patterns as uint16.  NaN/Inf are not expected in
    generated data and are not special-cased beyond keeping them NaN/Inf.
    """
    u = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32)
    lsb = (u >> np.uint32(16)) & np.uint32(1)
    rounded = (u + np.uint32(0x7FFF) + lsb) >> np.uint32(16)
    return rounded.astype(np.uint16)


def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    """Exact widening of bfloat16 bit patterns to float64."""
    u = bits.astype(np.uint32) << np.uint32(16)
    return u.view(np.float32).astype(np.float64)


def quantize(x: np.ndarray, dtype: str):
    """Quantise float64 data to a storage dtype.

    Returns (stored, widened): `stored` is the array whose bytes are handed
    to a solver (float64 / float32 / uint16 bf16 patterns / float16) and
    `widened` is its exact float64 value.
    """
    if dtype == "f64":
        s = np.ascontiguousarray(x, dtype=np.float64)
        return s, s
    if dtype == "f32":
        s = np.ascontiguousarray(x, dtype=np.float32)
        return s, s.astype(np.float64)
    if dtype == "bf16":
        s = f32_to_bf16_bits(np.asarray(x, dtype=np.float32))
        return s, bf16_bits_to_f64(s)
    if dtype == "f16":
        s = np.ascontiguousarray(x, dtype=np.float16)
        return s, s.astype(np.float64)
    raise ValueError(f"unknown dtype {dtype!r}")


def widen(stored: np.ndarray, dtype: str) -> np.ndarray:
    """Exact float64 value of stored X bytes."""
    if dtype == "bf16":
        return bf16_bits_to_f64(stored)
    return np.asarray(stored).astype(np.float64)


# ----------------------------------------------------------------------------
# edge sets (Section 1: chain for the standard FLR, lattice for 2D FLR)
# ----------------------------------------------------------------------------
def chain_edges(p: int) -> np.ndarray:
    """E = {(j-1, j)}: the standard FLR chain, 0-based, shape (p-1, 2)."""
    j = np.arange(1, p, dtype=np.int64)
    return np.stack([j - 1, j], axis=1) if p > 1 else np.zeros((0, 2), np.int64)


def lattice_edges(q1: int, q2: int) -> np.ndarray:
    """Horizontal + vertical neighbours on a q1 x q2 lattice.

    Coefficient (i, j) has index i*q2 + j (row-major).  Horizontal edges come
    first (row by row), then vertical edges.  m = q1(q2-1) + (q1-1)q2.
    """
    idx = np.arange(q1 * q2, dtype=np.int64).reshape(q1, q2)
    h = np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()], axis=1)
    v = np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()], axis=1)
    return np.concatenate([h, v], axis=0)


def knn_edges(points: np.ndarray, k: int) -> np.ndarray:
    """Symmetrised k-nearest-neighbour graph (union), as sorted unique pairs j<k.

    Neighbours by Euclidean distance; equal distances are ordered by the
    lower index (a stable argsort over a full distance row).
    """
    pts = np.asarray(points, dtype=np.float64)
    p = pts.shape[0]
    if p <= 1 or k <= 0:
        return np.zeros((0, 2), np.int64)
    kk = min(k, p - 1)
    pairs = []
    block = 2048
    for s in range(0, p, block):
        e = min(p, s + block)
        d2 = ((pts[s:e, None, :] - pts[None, :, :]) ** 2).sum(-1)
        d2[np.arange(e - s), np.arange(s, e)] = np.inf
        nb = np.argsort(d2, axis=1, kind="stable")[:, :kk]
        rows = np.repeat(np.arange(s, e, dtype=np.int64), kk)
        pairs.append(np.stack([rows, nb.ravel().astype(np.int64)], axis=1))
    pr = np.concatenate(pairs, axis=0)
    lo = np.minimum(pr[:, 0], pr[:, 1])
    hi = np.maximum(pr[:, 0], pr[:, 1])
    key = np.unique(lo * p + hi)
    return np.stack([key // p, key % p], axis=1).astype(np.int64)


@dataclasses.dataclass
class Graph:
    """An edge set E in one of three forms.

    kind: "chain" (E = {(j-1,j)}), "lattice" (q1 x q2, row-major index) or
    "edges" (explicit list).  `edges` always holds the explicit (m, 2) list.
    """
    kind: str
    p: int
    q1: int = 1
    q2: int = 0
    edges: Optional[np.ndarray] = None

    def __post_init__(self):
        if self.edges is None:
            if self.kind == "chain":
                self.edges = chain_edges(self.p)
                self.q1, self.q2 = 1, self.p
            elif self.kind == "lattice":
                assert self.q1 * self.q2 == self.p
                self.edges = lattice_edges(self.q1, self.q2)
            else:
                raise ValueError("explicit edge list required")

    @property
    def m(self) -> int:
        return int(self.edges.shape[0])


# ----------------------------------------------------------------------------
# true-coefficient patterns
# ----------------------------------------------------------------------------
def beta_c1(p: int) -> np.ndarray:
    """Scenario C1 (sparse, 41 non-zeros; Section 5.1).  1-based j in the paper."""
    b = np.zeros(p)
    for j in list(range(1, 21)) + list(range(121, 126)):
        if j <= p:
            b[j - 1] = 2.0
    if 41 <= p:
        b[40] = 3.0
    for j in range(71, 86):
        if j <= p:
            b[j - 1] = 1.0
    return b


def beta_c2(p: int) -> np.ndarray:
    """Scenario C2 (30 % non-zero; Section 5.1): 1 on (p/10, 2p/10], 2 on (2p/10, 4p/10]."""
    b = np.zeros(p)
    b[p // 10: 2 * p // 10] = 1.0
    b[2 * p // 10: 4 * p // 10] = 2.0
    return b


def beta_c3(p: int) -> np.ndarray:
    """Scenario C3 (dense; Section 5.1): +1 on the first half, -1 on the second."""
    b = -np.ones(p)
    b[: 5 * p // 10] = 1.0
    return b


def beta_c4(q1: int, q2: int) -> np.ndarray:
    """Scenario C4 (Section 5.2): +2 on the diagonal blocks, -2 on the anti-diagonal.

    Blocks are floor(q1/4) x floor(q2/4); returned row-major (index i*q2+j).
    """
    B = np.zeros((q1, q2))
    b1, b2 = q1 // 4, q2 // 4
    for k in range(4):
        B[k * b1:(k + 1) * b1, k * b2:(k + 1) * b2] = 2.0
        B[k * b1:(k + 1) * b1, (3 - k) * b2:(4 - k) * b2] = -2.0
    return B.ravel()


def beta_blocks10(p: int = 200) -> np.ndarray:
    """Chain benchmark pattern: blocks of 10 at 20-29=+1, 60-69=-2, 100-109=+2, 150-159=-1."""
    b = np.zeros(p)
    for s, v in ((20, 1.0), (60, -2.0), (100, 2.0), (150, -1.0)):
        b[s:s + 10] = v
    return b


def beta_rectangles(q: int = 100) -> np.ndarray:
    """Lattice benchmark image: three constant rectangles (values 1, 2, 3) on 0."""
    B = np.zeros((q, q))
    s = q / 100.0
    def r(a, b):
        return slice(int(round(a * s)), int(round(b * s)))
    B[r(10, 40), r(10, 40)] = 1.0
    B[r(50, 90), r(15, 45)] = 2.0
    B[r(20, 70), r(60, 90)] = 3.0
    return B.ravel()


# ----------------------------------------------------------------------------
# problems
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Problem:
    """One FLR instance: min 1/2||y - X b||^2 + lam1 ||b||_1 + lam2 sum_E |b_j - b_k|."""
    name: str
    X: np.ndarray            # stored bytes, row-major n x p (dtype per `dtype`)
    dtype: str               # "f64" | "f32" | "bf16" | "f16"
    y: np.ndarray            # float64, length n
    graph: Graph
    lam1: float
    lam2: float
    eps: float
    beta_true: np.ndarray
    lam_grid: Optional[np.ndarray] = None   # (K, 2) for batched workloads

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def p(self) -> int:
        return int(self.X.shape[1])

    def X64(self) -> np.ndarray:
        """Exact float64 value of the stored X."""
        return widen(self.X, self.dtype)


def gaussian_design(rng, n: int, p: int, ar_rho: float = 0.0) -> np.ndarray:
    """n x p design, rows iid N(0, Sigma).

    ar_rho = 0: Sigma = I (Section 5.1).  ar_rho > 0: each row is an AR(1)
    sequence along the column index, x_1 = z_1, x_j = rho x_{j-1} +
    sqrt(1-rho^2) z_j, so Sigma_jk = rho^|j-k|.
    """
    Z = rng.standard_normal((n, p))
    if ar_rho == 0.0:
        return Z
    from scipy.signal import lfilter
    Z[:, 1:] *= math.sqrt(1.0 - ar_rho * ar_rho)
    return lfilter([1.0], [1.0, -ar_rho], Z, axis=1)


def make_problem(name: str, n: int, p: int, dtype: str, graph: Graph,
                 beta_true: np.ndarray, lam1: float, lam2: float, eps: float,
                 noise_sd: float, seed: int, ar_rho: float = 0.0) -> Problem:
    """y = X beta + noise (Eq. gener), with X quantised to `dtype` first."""
    rng = np.random.default_rng(seed)
    Xd = gaussian_design(rng, n, p, ar_rho)
    Xs, Xw = quantize(Xd, dtype)
    del Xd
    noise = rng.standard_normal(n) * noise_sd
    y = Xw @ beta_true + noise
    return Problem(name, Xs, dtype, y, graph, lam1, lam2, eps, beta_true)


def config(k: int, s: int = 0, scale: float = 1.0) -> Problem:
    """Benchmark configuration k (1..4), dataset s, seed 1000*k + s.

    `scale` < 1 shrinks n and p (lattice side lengths by sqrt) with the same
    recipe, for tests that need the shape of a workload at a size a CPU
    solver finishes quickly.
    """
    seed = 1000 * k + s
    if k == 1:
        p = max(20, int(round(200 * scale)))
        n = max(10, int(round(100 * scale)))
        b = beta_blocks10(200)[:p] if p <= 200 else np.resize(beta_blocks10(200), p)
        return make_problem("chain-f64-n100-p200", n, p, "f64", Graph("chain", p), b,
                            0.1, 0.5, 1e-6, 1.0, seed)
    if k == 2:
        q = max(8, int(round(100 * math.sqrt(scale))))
        n = max(20, int(round(1000 * scale)))
        return make_problem(f"lattice-f32-q{q}-n{n}", n, q * q, "f32",
                            Graph("lattice", q * q, q, q), beta_rectangles(q),
                            0.05, 0.2, 1e-6, 0.5, seed)
    if k == 3:
        p = max(40, int(round(20000 * scale)))
        n = max(20, int(round(2000 * scale)))
        pr = make_problem(f"chain-bf16-n{n}-p{p}-grid64", n, p, "bf16", Graph("chain", p),
                          beta_c2(p), 0.0, 0.0, 1e-6, 1.0, seed)
        g = 10.0 ** (-3.0 + 3.0 * np.arange(8) / 7.0)
        L1, L2 = np.meshgrid(g, g, indexing="ij")
        pr.lam_grid = np.stack([L1.ravel(), L2.ravel()], axis=1)
        pr.lam1, pr.lam2 = float(pr.lam_grid[0, 0]), float(pr.lam_grid[0, 1])
        return pr
    if k == 4:
        q1 = max(8, int(round(250 * math.sqrt(scale))))
        q2 = max(8, int(round(400 * math.sqrt(scale))))
        n = max(20, int(round(5000 * scale)))
        return make_problem(f"lattice-f16-{q1}x{q2}-n{n}", n, q1 * q2, "f16",
                            Graph("lattice", q1 * q2, q1, q2), beta_c4(q1, q2),
                            0.01, 0.1, 1e-6, 1.0, seed, ar_rho=0.5)
    raise ValueError(f"no configuration {k}")


def paper_scenario(c: int, p: int, n: int = 1000, lam1: float = 0.1, lam2: float = 0.1,
                   s: int = 0, dtype: str = "f64", eps: float = 1e-8) -> Problem:
    """The paper's scenarios C1-C3 (chain) and C4 (q x q lattice, p = q^2)."""
    seed = 100000 + 1000 * c + s
    if c in (1, 2, 3):
        b = {1: beta_c1, 2: beta_c2, 3: beta_c3}[c](p)
        return make_problem(f"paper-C{c}-p{p}", n, p, dtype, Graph("chain", p), b,
                            lam1, lam2, eps, 1.0, seed)
    if c == 4:
        q = int(round(math.sqrt(p)))
        return make_problem(f"paper-C4-q{q}", n, q * q, dtype, Graph("lattice", q * q, q, q),
                            beta_c4(q, q), lam1, lam2, eps, 1.0, seed)
    raise ValueError(c)


# ----------------------------------------------------------------------------
# served mixed stream
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Request:
    rid: int
    arrival: float           # seconds, relative to the stream start (rate 1)
    p: int
    n: int
    dtype: str
    kind: str                # "chain" | "lattice" | "knn"
    q1: int
    q2: int
    lam1: float
    lam2: float
    seed: int


@dataclasses.dataclass
class DenoiseProblem:
    """An FLSA instance (X = I, n = p): a noisy image y on a q1 x q2 lattice."""
    name: str
    y: np.ndarray
    image: np.ndarray          # the noise-free image, row-major (q1 * q2,)
    graph: Graph
    lam1: float
    lam2: float
    eps: float

    @property
    def p(self) -> int:
        return int(self.y.shape[0])


def image_pattern(q1: int, q2: int) -> np.ndarray:
    """A piecewise-constant test image with values in [0, 1], row-major: background
    0.2, a disc of 0.9, a square of 0.5 and a bar of 1.0, placed at fixed fractions
    of the frame (our choice; the image the paper denoises is not available)."""
    r = (np.arange(q1)[:, None] + 0.5) / q1
    c = (np.arange(q2)[None, :] + 0.5) / q2
    img = np.full((q1, q2), 0.2)
    img[(r - 0.3) ** 2 + (c - 0.35) ** 2 <= 0.2 ** 2] = 0.9
    img[(r >= 0.6) & (r < 0.85) & (c >= 0.1) & (c < 0.4)] = 0.5
    img[(r >= 0.15) & (r < 0.9) & (c >= 0.65) & (c < 0.8)] = 1.0
    return img.reshape(-1)


def denoise(q1: int = 256, q2: int = 256, s: int = 0, noise_sd: float = 0.3,
            lam1: float = 0.0, lam2: float = 0.1, eps: float = 1e-6) -> DenoiseProblem:
    """Image denoising as the two-dimensional FLSA (X = I; Section 5.2's image study
    with its lambda = (0, 0.1) and (0, 1)): y = image + N(0, noise_sd^2), seed
    1000 * 6 + s."""
    img = image_pattern(q1, q2)
    rng = np.random.default_rng(6000 + s)
    y = img + noise_sd * rng.standard_normal(img.shape[0])
    return DenoiseProblem(f"denoise-{q1}x{q2}-s{s}", y, img, Graph("lattice", q1 * q2, q1, q2),
                          lam1, lam2, eps)


def served_stream(count: int, seed: int = 5000, p_lo: int = 500, p_hi: int = 50000):
    """Request descriptors of the served mixed stream (Poisson arrivals at rate 1).

    p log-uniform in [p_lo, p_hi] (lattice: q1 = floor(sqrt p), q2 = ceil(p/q1),
    p := q1 q2), n = floor(p/4), dtype FP32 or BF16 with equal probability,
    E uniform over {chain, lattice, 5-NN}, lam1 and lam2 log-uniform in
    [1e-3, 1].  Scale `arrival` by 1/rate for another arrival rate.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(count):
        t += rng.exponential(1.0)
        p = int(round(math.exp(rng.uniform(math.log(p_lo), math.log(p_hi)))))
        kind = ("chain", "lattice", "knn")[int(rng.integers(3))]
        q1, q2 = 1, p
        if kind == "lattice":
            q1 = int(math.isqrt(p))
            q2 = -(-p // q1)
            p = q1 * q2
        dtype = ("f32", "bf16")[int(rng.integers(2))]
        lam1 = 10.0 ** rng.uniform(-3, 0)
        lam2 = 10.0 ** rng.uniform(-3, 0)
        out.append(Request(r, t, p, max(1, p // 4), dtype, kind, q1, q2, lam1, lam2,
                           int(rng.integers(2**31))))
    return out


def request_graph_and_pattern(req: Request):
    """E and the true coefficients of a served request (host; the k-NN graph by a
    k-d tree for large p, the recipe's Euclidean neighbours)."""
    rng = np.random.default_rng(req.seed)
    p = req.p
    if req.kind == "chain":
        return Graph("chain", p), beta_c2(p), rng
    if req.kind == "lattice":
        B = np.zeros((req.q1, req.q2))
        B[req.q1 // 4: req.q1 // 2, req.q2 // 4: 3 * req.q2 // 4] = 1.0
        return Graph("lattice", p, req.q1, req.q2), B.ravel(), rng
    pts = rng.uniform(0.0, 1.0, (p, 2))
    if p <= 4096:
        e = knn_edges(pts, 5)
    else:
        from scipy.spatial import cKDTree
        _, nb = cKDTree(pts).query(pts, k=6)
        rows = np.repeat(np.arange(p, dtype=np.int64), 5)
        cols = nb[:, 1:].reshape(-1).astype(np.int64)
        lo, hi = np.minimum(rows, cols), np.maximum(rows, cols)
        key = np.unique(lo * p + hi)
        e = np.stack([key // p, key % p], axis=1).astype(np.int64)
    b = np.where(pts[:, 0] < 0.3, 1.0, np.where(pts[:, 0] > 0.7, -1.0, 0.0))
    return Graph("edges", p, edges=e), b, rng


def request_problem_device(req: Request, device):
    """A served request generated on the GPU (for the large requests of the stream):
    X iid N(0,1) from torch's seeded counter-based generator on `device`, stored in
    the request's dtype; y = X beta + N(0,1) in FP64 from the stored X.  Returns
    (X stored, y, graph, beta_true) as device tensors."""
    import torch
    g, b, _ = request_graph_and_pattern(req)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(req.seed))
    X = torch.randn((req.n, req.p), generator=gen, device=device, dtype=torch.float32)
    if req.dtype == "bf16":
        X = X.to(torch.bfloat16)
    bt = torch.from_numpy(b).to(device)
    y = X.to(torch.float64) @ bt
    y += torch.randn(req.n, generator=gen, device=device, dtype=torch.float64)
    return X, y, g, b


def request_problem(req: Request) -> Problem:
    """Materialise one served request: X, y, E and the true pattern."""
    rng = np.random.default_rng(req.seed)
    p, n = req.p, req.n
    if req.kind == "chain":
        g = Graph("chain", p)
        b = beta_c2(p)
    elif req.kind == "lattice":
        g = Graph("lattice", p, req.q1, req.q2)
        B = np.zeros((req.q1, req.q2))
        B[req.q1 // 4: req.q1 // 2, req.q2 // 4: 3 * req.q2 // 4] = 1.0
        b = B.ravel()
    else:
        pts = rng.uniform(0.0, 1.0, (p, 2))
        g = Graph("edges", p, edges=knn_edges(pts, 5))
        b = np.where(pts[:, 0] < 0.3, 1.0, np.where(pts[:, 0] > 0.7, -1.0, 0.0))
    return make_problem(f"req{req.rid}", n, p, req.dtype, g, b, req.lam1, req.lam2, 1e-6,
                        1.0, int(rng.integers(2**31)))
