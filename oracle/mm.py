"""FP64 CPU oracle for the MM method of fused lasso regression.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import this module.  It shares
no code with the CUDA path and is deliberately plain and slow: every formula
is written out as the paper states it, with library primitives (matrix
products, Cholesky) used as single steps.

Paper: Yu, Won, Lee, Lim, Yoon, "High-dimensional fused lasso regression
using majorization-minimization and parallel processing".

  objective        f(beta)                        Section 1, Eq. obj
  objective_eps    f_eps(beta)                    Section 3.1, Eq. pert
  majorizer        g_eps(beta | beta0)            Section 3.1, Eq. major
  mm_weights       A^(r) diagonal, B^(r) weights  Section 3.1, Eq. lin-sys
  surrogate_matrix X^T X + lam1 A + lam2 B         Section 3.1, Eq. lin-sys
  init_beta        beta_j = X_j^T y / X_j^T X_j   Algorithm 1 (initialisation)
  mm_dense         Algorithm 1 with a dense Cholesky solve per iteration
  mm_woodbury      Algorithm 1, surrogate solved by the Woodbury identity
                   with a banded/sparse factor of lam1 A + lam2 B (same
                   iterates as mm_dense up to rounding; for large p)
  mm_identity      Algorithm 1 for X = I (the FLSA): the surrogate
                   I + lam1 A + lam2 B is sparse and factored by a sparse LU

Readings where the paper is silent:
  * a zero column (X_j^T X_j = 0) initialises beta_j = 0;
  * the outer stop uses the true objective f (Algorithm 1, RE in Section 5);
  * the "dpotri" inverse of Algorithm 1 is read as a Cholesky solve with
    the same result.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.linalg as sla


# ----------------------------------------------------------------------------
# objective, perturbed objective and majorizer
# ----------------------------------------------------------------------------
def _diffs(beta: np.ndarray, edges: np.ndarray) -> np.ndarray:
    """beta_j - beta_k for every (j, k) in E."""
    if edges.shape[0] == 0:
        return np.zeros(0)
    return beta[edges[:, 0]] - beta[edges[:, 1]]


def objective(X, y, beta, lam1, lam2, edges) -> float:
    """f(beta) = 1/2 ||y - X beta||^2 + lam1 sum|beta_j| + lam2 sum_E |beta_j - beta_k| (Eq. obj)."""
    r = y - X @ beta
    return float(0.5 * (r @ r) + lam1 * np.abs(beta).sum()
                 + lam2 * np.abs(_diffs(beta, edges)).sum())


def _p_eps(x, eps):
    """|x| - eps log(1 + |x|/eps): the perturbed absolute value of Eq. pert."""
    ax = np.abs(x)
    return ax - eps * np.log1p(ax / eps)


def objective_eps(X, y, beta, lam1, lam2, edges, eps) -> float:
    """f_eps(beta) of Eq. pert."""
    r = y - X @ beta
    return float(0.5 * (r @ r) + lam1 * _p_eps(beta, eps).sum()
                 + lam2 * _p_eps(_diffs(beta, edges), eps).sum())


def majorizer(X, y, beta, beta0, lam1, lam2, edges, eps) -> float:
    """g_eps(beta | beta0) of Eq. major: each penalty term is replaced by
    p_eps(x0) + (x^2 - x0^2) / (2 (|x0| + eps))."""
    r = y - X @ beta
    d = _diffs(beta, edges)
    d0 = _diffs(beta0, edges)
    t1 = _p_eps(beta0, eps) + (beta ** 2 - beta0 ** 2) / (2.0 * (np.abs(beta0) + eps))
    t2 = _p_eps(d0, eps) + (d ** 2 - d0 ** 2) / (2.0 * (np.abs(d0) + eps))
    return float(0.5 * (r @ r) + lam1 * t1.sum() + lam2 * t2.sum())


def eps_gap(beta, lam1, lam2, edges, eps) -> float:
    """f(beta) - f_eps(beta) = lam1 sum eps log(1+|b_j|/eps) + lam2 sum_E eps log(1+|d|/eps).

    The bound of Proposition 1(ii) (Appendix A.1) used as the exact-vs-
    perturbed optimality certificate.
    """
    return float(lam1 * (eps * np.log1p(np.abs(beta) / eps)).sum()
                 + lam2 * (eps * np.log1p(np.abs(_diffs(beta, edges)) / eps)).sum())


# ----------------------------------------------------------------------------
# the surrogate linear system
# ----------------------------------------------------------------------------
def mm_weights(beta, edges, eps):
    """a_j = 1/(|beta_j| + eps) and w_jk = 1/(|beta_j - beta_k| + eps) (Eq. lin-sys)."""
    a = 1.0 / (np.abs(beta) + eps)
    w = 1.0 / (np.abs(_diffs(beta, edges)) + eps)
    return a, w


def laplacian_dense(w, edges, p) -> np.ndarray:
    """B with b_jj = sum_{k:(j,k) in E} w_jk and b_jk = b_kj = -w_jk (Eq. lin-sys)."""
    B = np.zeros((p, p))
    for e in range(edges.shape[0]):
        j, k = int(edges[e, 0]), int(edges[e, 1])
        B[j, j] += w[e]
        B[k, k] += w[e]
        B[j, k] -= w[e]
        B[k, j] -= w[e]
    return B


def laplacian_sparse(w, edges, p):
    """The same B as laplacian_dense, as a scipy CSR matrix."""
    import scipy.sparse as sp
    j, k = edges[:, 0], edges[:, 1]
    rows = np.concatenate([j, k, j, k])
    cols = np.concatenate([j, k, k, j])
    vals = np.concatenate([w, w, -w, -w])
    return sp.csr_matrix((vals, (rows, cols)), shape=(p, p))


def surrogate_matrix(XtX, a, w, edges, lam1, lam2) -> np.ndarray:
    """X^T X + lam1 A + lam2 B, dense (Eq. lin-sys; Algorithm 1's M^(r))."""
    p = XtX.shape[0]
    return XtX + lam1 * np.diag(a) + lam2 * laplacian_dense(w, edges, p)


def init_beta(X, y) -> np.ndarray:
    """beta_j^(0) = X_j^T y / X_j^T X_j (Algorithm 1); zero column -> 0."""
    c = X.T @ y
    d = np.einsum("ij,ij->j", X, X)
    out = np.zeros_like(c)
    nz = d != 0
    out[nz] = c[nz] / d[nz]
    return out


# ----------------------------------------------------------------------------
# Algorithm 1
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class MMResult:
    beta: np.ndarray
    f: float                    # f(beta) at the returned iterate
    f_eps: float                # f_eps(beta)
    iters: int                  # MM iterations performed
    rel_change: float           # last RE
    f_trace: List[float]        # f(beta^(r)), r = 0..iters
    feps_trace: List[float]     # f_eps(beta^(r))
    converged: bool


def _mm_loop(X, y, edges, lam1, lam2, eps, tol, max_iter, solve, beta0=None,
             stall_stop: bool = False) -> MMResult:
    beta = init_beta(X, y) if beta0 is None else np.array(beta0, dtype=np.float64)
    f_prev = objective(X, y, beta, lam1, lam2, edges)
    ftr = [f_prev]
    fetr = [objective_eps(X, y, beta, lam1, lam2, edges, eps)]
    re = np.inf
    best_re = np.inf
    stall = 0
    converged = False
    it = 0
    while it < max_iter:
        a, w = mm_weights(beta, edges, eps)
        beta = solve(a, w)
        it += 1
        f_new = objective(X, y, beta, lam1, lam2, edges)
        ftr.append(f_new)
        fetr.append(objective_eps(X, y, beta, lam1, lam2, edges, eps))
        re = abs(f_new - f_prev) / abs(f_prev) if f_prev != 0 else abs(f_new - f_prev)
        f_prev = f_new
        if re <= tol:
            converged = True
            break
        if stall_stop:
            # RE at rounding level stops decreasing: the iterate is as exact as FP64 allows.
            if re < best_re:
                best_re, stall = re, 0
            else:
                stall += 1
                if stall >= 20 and re < 1e-13:
                    converged = True
                    break
    return MMResult(beta, ftr[-1], fetr[-1], it, re, ftr, fetr, converged)


def mm_dense(X, y, edges, lam1, lam2, eps, tol=1e-12, max_iter=10000, beta0=None,
             stall_stop: bool = True) -> MMResult:
    """Algorithm 1: form X^T X + lam1 A + lam2 B, Cholesky-solve against X^T y, repeat
    until |f(b_new) - f(b_old)| / |f(b_old)| <= tol."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    XtX = X.T @ X
    c = X.T @ y

    def solve(a, w):
        Q = surrogate_matrix(XtX, a, w, edges, lam1, lam2)
        fac = sla.cho_factor(Q, lower=True, check_finite=False)
        return sla.cho_solve(fac, c, check_finite=False)

    return _mm_loop(X, y, edges, lam1, lam2, eps, tol, max_iter, solve, beta0, stall_stop)


def _banded_lower(S_sparse, bw):
    """Lower band storage (LAPACK 'L' layout) of a symmetric sparse matrix."""
    p = S_sparse.shape[0]
    ab = np.zeros((bw + 1, p))
    S = S_sparse.tocoo()
    keep = (S.row >= S.col) & (S.row - S.col <= bw)
    r, c, v = S.row[keep], S.col[keep], S.data[keep]
    np.add.at(ab, (r - c, c), v)
    return ab


def mm_woodbury(X, y, edges, lam1, lam2, eps, tol=1e-12, max_iter=10000, beta0=None,
                bandwidth: Optional[int] = None, stall_stop: bool = True) -> MMResult:
    """Algorithm 1 with the surrogate system solved through the Woodbury identity.

    With S = lam1 A + lam2 B (SPD for lam1 > 0) and Q = X^T X + S:
        Q^-1 c = S^-1 c - S^-1 X^T (I_n + X S^-1 X^T)^-1 X S^-1 c.
    S is factored banded (bandwidth = max |j - k| over E, the chain has 1, a
    q1 x q2 row-major lattice q2) when `bandwidth` is small, else by a sparse
    LU.  The n x n system uses a dense Cholesky.  Requires lam1 > 0.
    """
    if not lam1 > 0:
        raise ValueError("mm_woodbury needs lam1 > 0 (S must be nonsingular)")
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    n, p = X.shape
    c = X.T @ y
    if bandwidth is None:
        bandwidth = int(np.abs(edges[:, 0] - edges[:, 1]).max()) if edges.shape[0] else 0
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    def solve(a, w):
        S = (sp.diags(lam1 * a) + lam2 * laplacian_sparse(w, edges, p)).tocsr()
        rhs = np.concatenate([c[:, None], X.T], axis=1)          # p x (n+1)
        if bandwidth <= 512:
            ab = _banded_lower(S, bandwidth)
            cb = sla.cholesky_banded(ab, lower=True, check_finite=False)
            sol = sla.cho_solve_banded((cb, True), rhs, check_finite=False)
        else:
            lu = spla.splu(S.tocsc())
            sol = lu.solve(rhs)
        Sc, SXt = sol[:, 0], sol[:, 1:]
        K = np.eye(n) + X @ SXt
        fac = sla.cho_factor(K, lower=True, check_finite=False)
        return Sc - SXt @ sla.cho_solve(fac, X @ Sc, check_finite=False)

    return _mm_loop(X, y, edges, lam1, lam2, eps, tol, max_iter, solve, beta0, stall_stop)


def mm_identity(y, edges, lam1, lam2, eps, tol=1e-12, max_iter=10000, beta0=None,
                stall_stop: bool = True) -> MMResult:
    """Algorithm 1 for X = I (the FLSA of Section 1; image denoising in Section 5.2):
    X^T X = I and X^T y = y, so each surrogate is the sparse system
        (I + lam1 A + lam2 B) beta = y,
    factored by a sparse LU (one library step) instead of a dense Cholesky.
    beta^(0)_j = y_j (X_j^T y / X_j^T X_j with X = I).  lam1 = 0 is allowed:
    I + lam2 B stays positive definite."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    y = np.asarray(y, dtype=np.float64)
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    p = y.shape[0]
    eye = sp.identity(p, format="csr")

    def solve(a, w):
        Q = (eye + sp.diags(lam1 * a) + lam2 * laplacian_sparse(w, edges, p)).tocsc()
        return spla.splu(Q).solve(y)

    if beta0 is None:
        beta0 = y.copy()
    # X = I as a sparse identity: f and f_eps evaluate y - X beta without a dense p x p matrix
    return _mm_loop(eye, y, edges, lam1, lam2, eps, tol, max_iter, solve, beta0, stall_stop)


def surrogate_gradient(X, y, beta, lam1, lam2, edges, eps) -> np.ndarray:
    """grad f_eps(beta) = X^T(X beta - y) + lam1 A(beta) beta + lam2 B(beta) beta.

    Equals Q(beta) beta - X^T y with Q of Eq. lin-sys evaluated at beta itself,
    so a fixed point of the MM map has zero gradient (Lemma 2).
    """
    a, w = mm_weights(beta, edges, eps)
    g = X.T @ (X @ beta - y) + lam1 * a * beta
    if edges.shape[0]:
        d = w * _diffs(beta, edges)
        np.add.at(g, edges[:, 0], lam2 * d)
        np.add.at(g, edges[:, 1], -lam2 * d)
    return g
