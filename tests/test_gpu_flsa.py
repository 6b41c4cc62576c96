"""GPU parity of the FLSA path (X = I, dtype FLR_IDENTITY): no matrix is stored or
read, so every CG iteration is the Laplacian product and vector work only.

The oracle is Algorithm 1 for X = I (oracle.mm.mm_identity: each surrogate
I + lam1 A + lam2 B factored by a sparse LU), pinned on the CPU against the
dense oracle, the exact chain FLSA and soft-thresholding.  X = I makes f_eps
strongly convex (modulus >= 1), so beta is checked at convergence as well as
on fixed-iteration iterates.  The image is a synthetic piecewise-constant
256 x 256 picture plus Gaussian noise (flr_inputs.denoise), standing in for
the image the paper denoises in Section 5.2, with its lambda = (0, 0.1), (0, 1).
"""
import json
import os

import numpy as np
import pytest

import flr_inputs as fi
from oracle import exact, mm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
GAP = 1e-6
BETA = 1e-4
EXACT = dict(tol_cg=1e-12, max_refine=20, max_cg=20000)


@pytest.fixture(scope="module")
def flr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1306_1970_gb300 as m
    m.load(build_if_missing=True)
    return m


def golden(name):
    path = os.path.join(GOLD, name + ".json")
    if not os.path.exists(path):
        pytest.skip(f"golden {name} not generated")
    with open(path) as fh:
        return json.load(fh)


def flsa(flr, y, graph):
    return flr.Problem(None, torch.from_numpy(np.asarray(y, np.float64)).cuda(), graph,
                       dtype="identity")


def rel_beta(b, ref):
    b = b.cpu().numpy() if hasattr(b, "cpu") else b
    return np.abs(b - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("lam1,lam2", [(0.0, 0.5), (0.3, 0.8)])
def test_flsa_chain_is_exact_flsa(flr, lam1, lam2):
    """Chain: the exact 1D FLSA (Johnson's dynamic programme, then Eq. soft) within
    the eps certificate of Prop. 1(ii), and the oracle's MM limit at 1e-4."""
    rng = np.random.default_rng(31)
    p = 300
    y = np.repeat(rng.standard_normal(10) * 2, 30) + 0.3 * rng.standard_normal(p)
    E = fi.chain_edges(p)
    eps = 1e-7
    prob = flsa(flr, y, {"kind": "chain"})
    beta, st = prob.solve(lam1, lam2, eps=eps, tol=1e-14, max_mm=50000, **EXACT)
    assert st.status == 0, st
    b = beta.cpu().numpy()
    b_star = exact.flsa_chain(y, lam1, lam2)
    f_star = mm.objective(np.eye(p), y, b_star, lam1, lam2, E)
    assert f_star - 1e-9 <= st.f <= f_star + mm.eps_gap(b, lam1, lam2, E, eps) + 1e-8 * f_star
    ref = mm.mm_identity(y, E, lam1, lam2, eps, tol=1e-14, max_iter=50000)
    assert abs(st.f - ref.f) / ref.f <= GAP
    assert rel_beta(b, ref.beta) <= BETA


@pytest.mark.parametrize("lam2", [0.1, 1.0])
def test_flsa_lattice_64_matches_oracle(flr, lam2):
    """A 64 x 64 instance of the denoising image: the converged objective and every
    pixel of the converged beta against the oracle."""
    d = fi.denoise(64, 64, lam2=lam2)
    prob = flsa(flr, d.y, d.graph)
    beta, st = prob.solve(d.lam1, d.lam2, eps=d.eps, tol=1e-13, max_mm=20000, **EXACT)
    assert st.status == 0, st
    ref = mm.mm_identity(d.y, d.graph.edges, d.lam1, d.lam2, d.eps, tol=1e-13, max_iter=20000)
    assert abs(st.f - ref.f) / ref.f <= GAP, (st.f, ref.f)
    assert rel_beta(beta, ref.beta) <= BETA


@pytest.mark.parametrize("name", ["denoise256_r30", "denoise256_l1_r30"])
def test_flsa_image_256_iterates(flr, name):
    """Full 256 x 256 image (p = 65536): the MM iterate after 30 iterations equals the
    oracle's (beta at 1e-4 of max |beta|, f at 1e-6)."""
    g = golden(name)
    d = fi.denoise(256, 256, lam2=g["lam2"])
    np.testing.assert_allclose(d.y[:4], g["fingerprint"]["y_head"], rtol=1e-12)
    prob = flsa(flr, d.y, d.graph)
    R = g["fixed_iterations"]
    beta, st = prob.solve(d.lam1, d.lam2, eps=d.eps, tol=1e-300, max_mm=R, **EXACT)
    assert st.status == flr.FLR_ENOTCONV and st.mm_iters == R, st
    db = rel_beta(beta, np.array(g["beta"]))
    assert db <= BETA, db
    assert abs(st.f - g["f"]) / g["f"] <= GAP, (st.f, g["f"])
    print(f"{name}: max|dbeta|/|beta|inf = {db:.2e}, df/f = {abs(st.f - g['f']) / g['f']:.2e}")


def test_flsa_image_256_converged(flr):
    """Full image, lambda = (0, 0.1): the objective at the solver's own stop settings
    and, solved to the oracle's accuracy, every pixel at 1e-4."""
    g = golden("denoise256")
    d = fi.denoise(256, 256, lam2=g["lam2"])
    prob = flsa(flr, d.y, d.graph)
    _, st = prob.solve(d.lam1, d.lam2, eps=d.eps, tol=1e-9, tol_cg=1e-9, max_mm=20000)
    assert st.status == 0 and abs(st.f - g["f"]) / g["f"] <= GAP, (st, g["f"])
    beta, st = prob.solve(d.lam1, d.lam2, eps=d.eps, tol=1e-13, max_mm=20000, **EXACT)
    assert st.status == 0, st
    assert abs(st.f - g["f"]) / g["f"] <= GAP
    assert rel_beta(beta, np.array(g["beta"])) <= BETA


def test_flsa_edge_list_matches_stencil(flr):
    """The same lattice as an explicit edge list (CSR path) and as a stencil."""
    d = fi.denoise(24, 32, lam2=0.3)
    a = flsa(flr, d.y, d.graph)
    b = flsa(flr, d.y, {"kind": "edges", "edges": d.graph.edges})
    kw = dict(eps=d.eps, tol=1e-12, max_mm=20000, **EXACT)
    ba, sa = a.solve(0.05, d.lam2, **kw)
    bb, sb = b.solve(0.05, d.lam2, **kw)
    assert sa.status == 0 and sb.status == 0
    assert abs(sa.f - sb.f) <= 1e-9 * sa.f
    assert (ba - bb).abs().max().item() <= 1e-6 * ba.abs().max().item()


def test_flsa_rejects_a_matrix_or_mismatched_sizes(flr):
    import ctypes
    lib = flr.load()
    y = torch.zeros(10, dtype=torch.float64).cuda()
    g = flr.FlrGraph()
    g.kind = flr.FLR_E_CHAIN
    h = ctypes.c_void_p()
    X = torch.zeros(10, 10, dtype=torch.float64).cuda()
    assert lib.flr_create(X.data_ptr(), flr.FLR_IDENTITY, 10, 10, 10, y.data_ptr(), ctypes.byref(g),
                          flr.FLR_MEM_DEVICE, None, ctypes.byref(h)) == flr.FLR_EINVAL
    assert lib.flr_create(None, flr.FLR_IDENTITY, 10, 12, 0, y.data_ptr(), ctypes.byref(g),
                          flr.FLR_MEM_DEVICE, None, ctypes.byref(h)) == flr.FLR_EINVAL
