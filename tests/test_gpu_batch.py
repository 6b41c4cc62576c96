"""GPU parity of the batched lambda-grid solve (tensor-core multi-RHS path).

flr_solve_batch on BF16 X with a chain or lattice runs all (lambda1, lambda2)
pairs in one persistent launch whose X contractions use tcgen05 MMAs.  Each
result must match the FP64 oracle (relative objective gap <= 1e-6, max
|beta diff| <= 1e-4 max|beta|) and the single-problem solve.
"""
import numpy as np
import pytest

import flr_inputs as fi
from oracle import mm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def flr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1306_1970_gb300 as m
    m.load(build_if_missing=True)
    return m


def bf16_problem(flr, pr):
    X = torch.from_numpy(np.ascontiguousarray(pr.X)).view(torch.int16).cuda()
    return flr.Problem(X, torch.from_numpy(pr.y).cuda(), pr.graph, dtype="bf16")


@pytest.mark.parametrize("K", [3])
def test_batch_chain_bf16_matches_oracle(flr, K):
    pr = fi.config(3, scale=0.01)          # n=20, p=200, BF16 X, chain
    grid = pr.lam_grid[np.linspace(0, 63, K).astype(int)]
    prob = bf16_problem(flr, pr)
    betas, objs, sts = prob.solve_batch(grid[:, 0], grid[:, 1], eps=pr.eps, tol=1e-12,
                                        tol_cg=1e-10, max_mm=20000)
    X64 = pr.X64()
    for k, (l1, l2) in enumerate(grid):
        ref = mm.mm_dense(X64, pr.y, pr.graph.edges, l1, l2, pr.eps, tol=1e-13)
        assert sts[k].status == 0, sts[k]
        gap = abs(sts[k].f - ref.f) / abs(ref.f)
        assert gap <= 1e-6, (k, l1, l2, gap, sts[k])
        b = betas[:, k].cpu().numpy()
        db = np.abs(b - ref.beta).max() / max(np.abs(ref.beta).max(), 1e-300)
        assert db <= 1e-4, (k, l1, l2, db)
        fe = mm.objective_eps(X64, pr.y, b, l1, l2, pr.graph.edges, pr.eps)
        assert abs(sts[k].f_eps - fe) <= 1e-9 * abs(fe)


def test_batch_lattice_bf16_matches_single_solves(flr):
    pr = fi.config(2, scale=0.04)          # 20x20 lattice, n=40 (quantised to BF16 here)
    Xs, Xw = fi.quantize(pr.X64(), "bf16")
    y = Xw @ pr.beta_true + 0.5 * np.random.default_rng(7).standard_normal(pr.n)
    g = pr.graph
    X = torch.from_numpy(Xs).view(torch.int16).cuda()
    prob = flr.Problem(X, torch.from_numpy(y).cuda(), g, dtype="bf16")
    l1 = np.array([0.05, 0.1, 0.02, 0.3, 0.05])
    l2 = np.array([0.2, 0.1, 0.5, 0.05, 0.02])
    betas, objs, sts = prob.solve_batch(l1, l2, eps=1e-6, tol=1e-10, tol_cg=1e-9, max_mm=20000)
    for k in range(len(l1)):
        ref = mm.mm_dense(Xw, y, g.edges, l1[k], l2[k], 1e-6, tol=1e-13)
        assert sts[k].status == 0
        assert abs(sts[k].f - ref.f) / ref.f <= 1e-6, (k, sts[k], ref.f)
    b1, s1 = prob.solve(l1[0], l2[0], eps=1e-6, tol=1e-10, tol_cg=1e-9, max_mm=20000)
    assert abs(sts[0].f - s1.f) / s1.f <= 1e-6


def test_batch_more_than_32_rhs(flr):
    """40 problems: one launch with the 64-wide MMA and 24 padded right-hand sides."""
    pr = fi.config(3, scale=0.01)
    grid = pr.lam_grid[24:64]
    prob = bf16_problem(flr, pr)
    betas, objs, sts = prob.solve_batch(grid[:, 0], grid[:, 1], eps=pr.eps, tol=1e-10,
                                        tol_cg=1e-9, max_mm=20000)
    X64 = pr.X64()
    for k in (0, 17, 39):
        l1, l2 = grid[k]
        ref = mm.mm_dense(X64, pr.y, pr.graph.edges, l1, l2, pr.eps, tol=1e-13)
        assert abs(sts[k].f - ref.f) / abs(ref.f) <= 1e-6, (k, sts[k], ref.f)
