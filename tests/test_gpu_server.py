"""Serving loop: mixed requests run concurrently and give the same answers as alone.

Requests of mixed p, n, dtype and edge set (chain, lattice, 5-NN graph; the
served-stream recipe at reduced p) go through a 4-slot server.  Each result
must equal the same problem solved alone through flr_solve with the same
block count (objective to 1e-8, beta to 1e-4 of max |beta|), the solve
kernels of at least two requests must have overlapped on the GPU (device
global-timer spans), and the server must refuse what cannot fit or is
malformed.  Every surrogate is solved to FP64 accuracy (max_refine), so a
request follows the exact MM map whatever else shares the GPU.
"""
import numpy as np
import pytest

import flr_inputs as fi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def flr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1306_1970_gb300 as m
    m.load(build_if_missing=True)
    return m


def host_X(pr):
    X = torch.from_numpy(np.ascontiguousarray(pr.X))
    if pr.dtype == "bf16":
        X = X.view(torch.int16)
    return X.pin_memory(), torch.from_numpy(pr.y).pin_memory()


def test_mixed_stream_equals_alone(flr):
    reqs = fi.served_stream(8, seed=77, p_lo=300, p_hi=3000)
    probs = [fi.request_problem(r) for r in reqs]
    slots, gps = 4, 16
    srv = flr.Server(slots=slots, grid_per_slot=gps)
    ids = []
    kw = dict(tol_cg=1e-12, max_refine=20, max_mm=30000)
    for r, pr in zip(reqs, probs):
        X, y = host_X(pr)
        ids.append(srv.submit(X, y, pr.graph, r.lam1, r.lam2, eps=pr.eps, tol=1e-11,
                              dtype="bf16" if pr.dtype == "bf16" else None, **kw))
    out = [srv.wait(i) for i in ids]
    srv.close()
    spans = []
    for (beta, res), r, pr in zip(out, reqs, probs):
        assert res.status == 0, (r, res.status)
        assert 0 < res.dev_t0_ns < res.dev_t1_ns, (res.dev_t0_ns, res.dev_t1_ns)
        spans.append((res.dev_t0_ns, res.dev_t1_ns))
        X, y = host_X(pr)
        alone = flr.Problem(X.cuda(), y.cuda(), pr.graph,
                            dtype="bf16" if pr.dtype == "bf16" else None)
        g = min(gps, max(1, -(-pr.n * pr.p // 65536)))
        b1, s1 = alone.solve(r.lam1, r.lam2, eps=pr.eps, tol=1e-11, grid=g, **kw)
        assert abs(res.stats.f - s1.f) <= 1e-8 * abs(s1.f), (r, res.stats.f, s1.f)
        db = np.abs(beta - b1.cpu().numpy()).max() / max(np.abs(beta).max(), 1e-300)
        assert db <= 1e-4, (r, db)
    # the solve kernels of at least two requests ran on the GPU at the same time
    spans.sort()
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1)), spans


def test_refuses_oversized_and_malformed(flr):
    pr = fi.config(1, scale=0.5)
    X, y = host_X(pr)
    srv = flr.Server(slots=2, grid_per_slot=4, hbm_budget=1 << 20)   # 1 MiB budget
    big = torch.zeros((4000, 2000), dtype=torch.float32)
    with pytest.raises(flr.FlrError) as ei:
        srv.submit(big, torch.zeros(4000, dtype=torch.float64), {"kind": "chain"}, 0.1, 0.1)
    assert ei.value.status == flr.FLR_ENOMEM
    with pytest.raises(flr.FlrError) as ei:
        srv.submit(X, y, pr.graph, -1.0, 0.1)
    assert ei.value.status == flr.FLR_EINVAL
    rid = srv.submit(X, y, pr.graph, pr.lam1, pr.lam2, eps=pr.eps, tol=1e-10)
    beta, res = srv.wait(rid)
    assert res.status == 0 and res.footprint <= 1 << 20
    srv.close()


def test_resident_handle_serves_a_lambda_path(flr):
    """Requests that share X, y and E under one data_id run on the slot's resident
    handle (no new copy of X), and each result equals the same problem solved alone."""
    pr = fi.config(2, scale=0.04)
    X, y = host_X(pr)
    srv = flr.Server(slots=1, grid_per_slot=16)
    lams = [(0.05, 0.2), (0.1, 0.1), (0.02, 0.4)]
    kw = dict(tol_cg=1e-12, max_refine=20, max_mm=30000)
    ids = [srv.submit(X, y, pr.graph, l1, l2, eps=pr.eps, tol=1e-11, data_id=7, **kw) for l1, l2 in lams]
    other = srv.submit(X, y, pr.graph, 0.05, 0.2, eps=pr.eps, tol=1e-11, **kw)   # no data_id
    out = [srv.wait(i) for i in ids]
    bo, ro = srv.wait(other)
    srv.close()
    assert [r.reused for _, r in out] == [0, 1, 1]
    assert ro.reused == 0 and ro.status == 0
    alone = flr.Problem(X.cuda(), y.cuda(), pr.graph)
    for (beta, res), (l1, l2) in zip(out, lams):
        assert res.status == 0
        b1, s1 = alone.solve(l1, l2, eps=pr.eps, tol=1e-11, grid=res.stats.grid, **kw)
        assert abs(res.stats.f - s1.f) <= 1e-8 * abs(s1.f)
        assert np.abs(beta - b1.cpu().numpy()).max() <= 1e-4 * np.abs(beta).max()
    assert abs(ro.stats.f - out[0][1].stats.f) <= 1e-8 * abs(ro.stats.f)
