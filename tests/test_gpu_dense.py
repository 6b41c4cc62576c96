"""GPU parity of flr_solve_dense: Algorithm 1 with a dense FP64 Cholesky per MM
iteration on the GPU (the paper's route for a general edge set), against the
oracle's Algorithm 1 (oracle.mm.mm_dense, the same iteration with a LAPACK
Cholesky).  Both compute the same FP64 iterates, so they are compared after a
fixed number of MM iterations as well as at convergence."""
import json
import os

import numpy as np
import pytest

import flr_inputs as fi
from oracle import mm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def flr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1306_1970_gb300 as m
    m.load(build_if_missing=True)
    return m


def rel_beta(b, ref):
    b = b.cpu().numpy() if hasattr(b, "cpu") else b
    return np.abs(b - ref).max() / np.abs(ref).max()


def test_dense_config1_matches_golden(flr):
    """Standard FLR (chain, FP64 X, n = 100, p = 200) to the oracle's converged solve."""
    with open(os.path.join(GOLD, "config1.json")) as fh:
        g = json.load(fh)
    pr = fi.config(1)
    prob = flr.Problem(torch.from_numpy(pr.X).cuda(), torch.from_numpy(pr.y).cuda(), pr.graph)
    beta, st = prob.solve_dense(pr.lam1, pr.lam2, eps=pr.eps, tol=1e-12, max_mm=20000)
    assert st.status == 0, st
    assert abs(st.f - g["f"]) / g["f"] <= 1e-6
    assert rel_beta(beta, np.array(g["beta"])) <= 1e-4


@pytest.mark.parametrize("case", ["knn_f32", "lattice_f32", "chain_bf16", "lattice_f16"])
def test_dense_iterates_match_oracle(flr, case):
    """Same FP64 iteration on both sides: beta after 40 MM iterations agrees to 1e-8 of
    max |beta| on a general k-NN graph, a lattice and a chain, for 32- and 16-bit X
    (p = 150 to 400, ragged last 64 x 64 tile)."""
    rng = np.random.default_rng(51)
    if case == "knn_f32":
        p, n = 150, 60
        pts = rng.uniform(size=(p, 2))
        E = fi.knn_edges(pts, 5)
        graph = {"kind": "edges", "edges": E}
        Xs, Xw = fi.quantize(rng.standard_normal((n, p)), "f32")
        lam1, lam2 = 0.1, 0.3
    elif case == "lattice_f32":
        pr = fi.config(2, scale=0.04)
        Xs, Xw, E, graph, lam1, lam2 = pr.X, pr.X64(), pr.graph.edges, pr.graph, pr.lam1, pr.lam2
        n, p = Xs.shape
    elif case == "chain_bf16":
        pr = fi.config(3, scale=0.02)
        Xs, Xw, E, graph, lam1, lam2 = pr.X, pr.X64(), pr.graph.edges, pr.graph, 0.05, 0.2
        n, p = Xs.shape
    else:
        pr = fi.config(4, scale=0.004)
        Xs, Xw, E, graph, lam1, lam2 = pr.X, pr.X64(), pr.graph.edges, pr.graph, pr.lam1, pr.lam2
        n, p = Xs.shape
    y = Xw @ np.sin(np.arange(p) / 7.0) + rng.standard_normal(n)
    X = torch.from_numpy(np.ascontiguousarray(Xs))
    dt = None
    if case == "chain_bf16":
        X, dt = X.view(torch.int16), "bf16"
    prob = flr.Problem(X.cuda(), torch.from_numpy(y).cuda(), graph, dtype=dt)
    beta, st = prob.solve_dense(lam1, lam2, eps=1e-6, tol=1e-300, max_mm=40)
    assert st.status == flr.FLR_ENOTCONV and st.mm_iters == 40, st
    ref = mm.mm_dense(Xw, y, E, lam1, lam2, 1e-6, tol=0.0, max_iter=40, stall_stop=False)
    assert rel_beta(beta, ref.beta) <= 1e-8
    assert abs(st.f - ref.f) <= 1e-10 * abs(ref.f)
    fe = mm.objective_eps(Xw, y, beta.cpu().numpy(), lam1, lam2, E, 1e-6)
    assert abs(st.f_eps - fe) <= 1e-10 * abs(fe)


def test_dense_equals_cg_solve_at_convergence(flr):
    """The dense and the CG routes reach the same MM limit (q = 20 lattice)."""
    pr = fi.config(2, scale=0.04)
    prob = flr.Problem(torch.from_numpy(pr.X).cuda(), torch.from_numpy(pr.y).cuda(), pr.graph)
    b1, s1 = prob.solve_dense(pr.lam1, pr.lam2, eps=pr.eps, tol=1e-13, max_mm=20000)
    b2, s2 = prob.solve(pr.lam1, pr.lam2, eps=pr.eps, tol=1e-13, tol_cg=1e-12, max_refine=20,
                        max_mm=20000)
    assert s1.status == 0 and s2.status == 0
    assert abs(s1.f - s2.f) <= 1e-9 * abs(s1.f)
    assert rel_beta(b1, b2.cpu().numpy()) <= 1e-4


def test_dense_breakdown_when_not_positive_definite(flr):
    """lam1 = lam2 = 0 with p > n: X^T X is singular, a pivot is not positive."""
    rng = np.random.default_rng(52)
    X = torch.from_numpy(rng.standard_normal((10, 30))).cuda()
    y = torch.from_numpy(rng.standard_normal(10)).cuda()
    prob = flr.Problem(X, y, {"kind": "chain"})
    _, st = prob.solve_dense(0.0, 0.0, eps=1e-6, tol=1e-9, max_mm=5, check=False)
    assert st.status == flr.FLR_EBREAKDOWN
