"""Exact (non-MM) solvers for special cases of fused lasso regression.

TEST INFRASTRUCTURE ONLY (same rule as oracle/mm.py).  These pin the MM
oracle to results fixed by mathematics rather than by the oracle itself:

  soft_threshold     X = I, lam2 = 0: beta = S(y, lam1) (the separable lasso,
                     the lam2 = 0 case of the Hunter-Li MM of Section 3.1)
  least_squares      lam1 = lam2 = 0, full column rank: normal equations
  flsa_chain         X = I on a chain (the standard FLSA of Section 2.1):
                     exact 1D total-variation denoising by the dynamic
                     programme of N. Johnson (2013), followed by the
                     soft-threshold relation of Eq. soft for lam1 > 0
  brute_force        any small problem with n >= p: enumerate every face
                     (sign / zero / fusion pattern) of the piecewise
                     quadratic f, minimise the face quadratic on its affine
                     hull and keep the best true f
  kkt_residual       subgradient optimality of Eq. obj checked by a small LP
"""
from __future__ import annotations

import itertools

import numpy as np


def soft_threshold(y, lam):
    """sign(y) max(|y| - lam, 0), elementwise (Eq. soft)."""
    y = np.asarray(y, dtype=np.float64)
    return np.sign(y) * np.maximum(np.abs(y) - lam, 0.0)


def least_squares(X, y):
    """argmin ||y - X beta||^2 for full column rank X."""
    return np.linalg.lstsq(np.asarray(X, np.float64), np.asarray(y, np.float64), rcond=None)[0]


# ----------------------------------------------------------------------------
# 1D fused lasso signal approximator
# ----------------------------------------------------------------------------
class _PWL:
    """Increasing piecewise-linear function given by breakpoints xs (sorted),
    values vs at the breakpoints and slopes sl / sr beyond the ends."""

    def __init__(self, xs, vs, sl, sr):
        self.xs, self.vs, self.sl, self.sr = xs, vs, sl, sr

    def inverse(self, c: float) -> float:
        xs, vs = self.xs, self.vs
        if c <= vs[0]:
            return xs[0] + (c - vs[0]) / self.sl
        if c >= vs[-1]:
            return xs[-1] + (c - vs[-1]) / self.sr
        i = int(np.searchsorted(vs, c, side="right")) - 1
        i = min(max(i, 0), len(xs) - 2)
        x0, x1, v0, v1 = xs[i], xs[i + 1], vs[i], vs[i + 1]
        if v1 == v0:
            return x0
        return x0 + (c - v0) * (x1 - x0) / (v1 - v0)

    def value(self, x: np.ndarray) -> np.ndarray:
        return np.interp(x, self.xs, self.vs)


def tv_denoise_chain(y, lam):
    """argmin_b 1/2 sum (y_i - b_i)^2 + lam sum |b_i - b_{i-1}| (exact).

    Dynamic programme (Johnson 2013): with F_k(b) the optimal cost of the
    first k terms given b_k = b, F_k' = (b - y_k) + clip(F_{k-1}', -lam, lam).
    The clip points b-_k, b+_k (where F_{k-1}' = -lam, +lam) give the
    back-pointers b_{k-1} = clip(b_k, b-_k, b+_k); b_n solves F_n'(b) = 0.
    The derivative is kept as an explicit breakpoint list (O(n^2) worst case),
    which is plenty for test sizes.
    """
    y = np.asarray(y, dtype=np.float64)
    n = y.shape[0]
    if n == 0:
        return y.copy()
    if lam <= 0:
        return y.copy()
    lo = np.zeros(n)
    hi = np.zeros(n)
    f = _PWL(np.array([y[0]]), np.array([0.0]), 1.0, 1.0)
    for k in range(1, n):
        bm = f.inverse(-lam)
        bp = f.inverse(lam)
        lo[k], hi[k] = bm, bp
        inner = (f.xs > bm) & (f.xs < bp)
        xs = np.concatenate([[bm], f.xs[inner], [bp]])
        vs = np.concatenate([[-lam], f.vs[inner], [lam]])
        # add (b - y_k): slope +1 everywhere
        f = _PWL(xs, vs + (xs - y[k]), 1.0, 1.0)
    b = np.zeros(n)
    b[-1] = f.inverse(0.0)
    for k in range(n - 1, 0, -1):
        b[k - 1] = min(max(b[k], lo[k]), hi[k])
    return b


def flsa_chain(y, lam1, lam2):
    """Standard FLSA (X = I, chain E): TV denoising, then Eq. soft by lam1."""
    return soft_threshold(tv_denoise_chain(y, lam2), lam1)


# ----------------------------------------------------------------------------
# brute force over faces
# ----------------------------------------------------------------------------
def _objective(X, y, beta, lam1, lam2, edges):
    r = y - X @ beta
    d = beta[edges[:, 0]] - beta[edges[:, 1]] if edges.shape[0] else np.zeros(0)
    return 0.5 * float(r @ r) + lam1 * float(np.abs(beta).sum()) + lam2 * float(np.abs(d).sum())


def brute_force(X, y, lam1, lam2, edges, max_faces: int = 2_000_000):
    """Global minimiser of Eq. obj for tiny p (needs X of full column rank).

    A face fixes sign(beta_j) in {-1, 0, +1} for every j and sign(beta_j -
    beta_k) for every edge.  On its affine hull (zeros and fusions imposed)
    the objective with those signs is a quadratic that lies below f, and it
    equals f near any point of the face; the minimiser of f therefore
    minimises the quadratic of its own face.  Evaluating the true f at each
    face's minimiser and keeping the smallest gives the exact optimum.
    Returns (beta, f).
    """
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    edges = np.asarray(edges, np.int64).reshape(-1, 2)
    n, p = X.shape
    m = edges.shape[0]
    if 3 ** (p + m) > max_faces:
        raise ValueError("too many faces for brute force")
    G = X.T @ X
    c = X.T @ y
    D = np.zeros((m, p))
    for e in range(m):
        D[e, edges[e, 0]] = 1.0
        D[e, edges[e, 1]] = -1.0
    best_f, best_b = np.inf, None
    seen = set()
    for sb in itertools.product((-1, 0, 1), repeat=p):
        s = np.array(sb, np.float64)
        zero = [j for j in range(p) if sb[j] == 0]
        for se in itertools.product((-1, 0, 1), repeat=m):
            t = np.array(se, np.float64)
            fused = [e for e in range(m) if se[e] == 0]
            key = (sb, se)
            if key in seen:
                continue
            seen.add(key)
            rows = [np.eye(p)[j] for j in zero] + [D[e] for e in fused]
            if rows:
                C = np.array(rows)
                _, sv, vt = np.linalg.svd(C)
                rank = int((sv > 1e-12).sum())
                N = vt[rank:].T
            else:
                N = np.eye(p)
            if N.shape[1] == 0:
                b = np.zeros(p)
            else:
                H = N.T @ G @ N
                g = N.T @ (c - lam1 * s - lam2 * (D.T @ t if m else 0.0))
                theta = np.linalg.lstsq(H, g, rcond=None)[0]
                b = N @ theta
            fb = _objective(X, y, b, lam1, lam2, edges)
            if fb < best_f:
                best_f, best_b = fb, b
    return best_b, best_f


# ----------------------------------------------------------------------------
# KKT check
# ----------------------------------------------------------------------------
def kkt_residual(X, y, beta, lam1, lam2, edges, zero_tol=1e-9):
    """Smallest ||X^T(X b - y) + lam1 s + lam2 D^T t||_inf over subgradients.

    s_j = sign(b_j) where |b_j| > zero_tol, else s_j in [-1, 1]; t_e likewise
    for the edge differences.  Solved as an LP (scipy.optimize.linprog).
    A minimiser of Eq. obj has residual 0.
    """
    from scipy.optimize import linprog
    X = np.asarray(X, np.float64)
    edges = np.asarray(edges, np.int64).reshape(-1, 2)
    p = X.shape[1]
    m = edges.shape[0]
    g = X.T @ (X @ beta - y)
    d = beta[edges[:, 0]] - beta[edges[:, 1]] if m else np.zeros(0)
    D = np.zeros((m, p))
    for e in range(m):
        D[e, edges[e, 0]] = 1.0
        D[e, edges[e, 1]] = -1.0
    # variables: s (p), t (m), r (1); minimise r s.t. -r <= g + lam1 s + lam2 D^T t <= r
    nv = p + m + 1
    cost = np.zeros(nv)
    cost[-1] = 1.0
    Amat = np.zeros((p, nv))
    Amat[:, :p] = lam1 * np.eye(p)
    if m:
        Amat[:, p:p + m] = lam2 * D.T
    A_ub = np.vstack([np.hstack([Amat[:, :-1], -np.ones((p, 1))]),
                      np.hstack([-Amat[:, :-1], -np.ones((p, 1))])])
    b_ub = np.concatenate([-g, g])
    bounds = []
    for j in range(p):
        if abs(beta[j]) > zero_tol:
            v = float(np.sign(beta[j]))
            bounds.append((v, v))
        else:
            bounds.append((-1.0, 1.0))
    for e in range(m):
        if abs(d[e]) > zero_tol:
            v = float(np.sign(d[e]))
            bounds.append((v, v))
        else:
            bounds.append((-1.0, 1.0))
    bounds.append((0.0, None))
    res = linprog(cost, A_ub=A_ub, b_ub=b_ub, bounds=bounds, method="highs")
    if not res.success:
        raise RuntimeError(res.message)
    return float(res.x[-1])
