"""Write the oracle's reference solutions used by the parity tests and bench.py.

Calls only oracle/ and flr_inputs/.  Each case is written to
tests/golden/<name>.json:  the converged MM objective f and f_eps, the
iteration count, the final relative change, input fingerprints (so a changed
generator is caught before a parity comparison) and beta (all of it for
p <= 100000, otherwise 512 sampled indices plus max |beta|; none for the
config2_s<seed> cases, which only the objective gap uses).

Cases whose name ends in _r<R> hold the MM iterate after exactly R
iterations of Algorithm 1 from its initialisation (no stop test), beta(R)
and f(beta(R)): the MM map is deterministic, so a solver that solves every
surrogate system exactly reproduces these values whatever the conditioning
of f_eps along its flattest directions.

usage: python tests/golden/make_golden.py [case ...]     (default: the quick cases)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import flr_inputs as fi  # noqa: E402
from oracle import mm  # noqa: E402


def fingerprint(pr):
    if isinstance(pr, fi.DenoiseProblem):
        return {"y_head": [float(v) for v in pr.y[:4]], "y_sum": float(pr.y.sum())}
    X = pr.X64()
    return {"x_sum": float(X.sum()), "x_sq": float((X * X).sum()),
            "y_head": [float(v) for v in pr.y[:4]], "y_sum": float(pr.y.sum())}


def cases():
    """name -> (builder, solver, lam pairs or None)."""
    return {
        "config1": (lambda: fi.config(1), "dense", None),
        "config2_q20": (lambda: fi.config(2, scale=0.04), "dense", None),
        "config2_q40": (lambda: fi.config(2, scale=0.16), "woodbury", None),
        "config4_small": (lambda: fi.config(4, scale=0.004), "dense", None),
        "config4_q50x80": (lambda: fi.config(4, scale=0.04), "woodbury", None),
        "config3_small": (lambda: fi.config(3, scale=0.02), "dense", "grid"),
        "paper_c1_p200": (lambda: fi.paper_scenario(1, 200, eps=1e-6), "dense", None),
        "config2": (lambda: fi.config(2), "woodbury", None),
        # fixed-iteration MM iterates
        "config2_r200": (lambda: fi.config(2), "woodbury", None),
        "config2_q40_r300": (lambda: fi.config(2, scale=0.16), "woodbury", None),
        "config4_q50x80_r300": (lambda: fi.config(4, scale=0.04), "woodbury", None),
        # batched chain, n = 512, p = 5120, BF16 X: 8 points of the lambda grid
        # (the four corners and four interior points), 40 MM iterations each
        "config3_mid_r40": (lambda: fi.config(3, scale=0.256), "woodbury", "grid8"),
        # FLSA (X = I): the 256 x 256 denoising image, lambda = (0, 0.1) and (0, 1)
        "denoise256": (lambda: fi.denoise(lam2=0.1), "identity", None),
        "denoise256_r30": (lambda: fi.denoise(lam2=0.1), "identity", None),
        "denoise256_l1_r30": (lambda: fi.denoise(lam2=1.0), "identity", None),
        # the bench workload's other dataset seeds (objective only, no beta)
        **{f"config2_s{s}": ((lambda s=s: fi.config(2, s=s)), "woodbury", "nobeta") for s in range(1, 10)},
    }


GRID8 = [0, 7, 56, 63, 18, 27, 36, 45]   # indices into the 8 x 8 lambda grid


QUICK = ["config1", "config2_q20", "config4_small", "config3_small", "paper_c1_p200",
         "config2_q40"]


def fixed_iterations(name):
    """R of a case named ..._r<R>, else None."""
    tail = name.rsplit("_", 1)[-1]
    return int(tail[1:]) if tail.startswith("r") and tail[1:].isdigit() else None


def solve(pr, solver, lam1, lam2, log=None, fixed=None, keep_beta=True):
    E = pr.graph.edges
    t = time.time()
    if solver == "identity":
        def f(X, y, E, l1, l2, eps, **kw):
            return mm.mm_identity(y, E, l1, l2, eps, **kw)
        X = None
    else:
        X = pr.X64()
        f = mm.mm_dense if solver == "dense" else mm.mm_woodbury
    if fixed is None:
        r = f(X, pr.y, E, lam1, lam2, pr.eps, tol=1e-13, max_iter=12000)
    else:
        r = f(X, pr.y, E, lam1, lam2, pr.eps, tol=0.0, max_iter=fixed, stall_stop=False)
    out = {"lam1": lam1, "lam2": lam2, "f": r.f, "f_eps": r.f_eps, "iters": r.iters,
           "rel_change": r.rel_change, "seconds": time.time() - t,
           "f_trace_head": [float(v) for v in r.f_trace[:3]]}
    if fixed is None:
        # first MM iteration whose objective is within 1e-6 of the converged one
        gaps = np.abs(np.asarray(r.f_trace) - r.f) / abs(r.f)
        out["iters_to_gap_1e-6"] = int(np.argmax(gaps <= 1e-6))
    else:
        out["fixed_iterations"] = fixed
    b = r.beta
    out["beta_absmax"] = float(np.abs(b).max())
    if not keep_beta:
        pass
    elif b.shape[0] <= 100000:
        out["beta"] = [float(v) for v in b]
    else:
        idx = np.sort(np.random.default_rng(0).choice(b.shape[0], 512, replace=False))
        out["beta_idx"] = [int(i) for i in idx]
        out["beta_sample"] = [float(b[i]) for i in idx]
    if log:
        print(f"  lam=({lam1:g},{lam2:g}) iters={r.iters} f={r.f:.15g} {out['seconds']:.1f}s",
              file=log, flush=True)
    return out


def make(name):
    build, solver, lam = cases()[name]
    pr = build()
    n_ = pr.p if isinstance(pr, fi.DenoiseProblem) else pr.n
    dt_ = "identity" if isinstance(pr, fi.DenoiseProblem) else pr.dtype
    rec = {"name": name, "problem": pr.name, "n": n_, "p": pr.p, "dtype": dt_,
           "graph": pr.graph.kind, "q1": pr.graph.q1, "q2": pr.graph.q2, "eps": pr.eps,
           "solver": solver, "fingerprint": fingerprint(pr)}
    print(name, pr.name, flush=True)
    R = fixed_iterations(name)
    if lam == "grid":
        rec["solutions"] = [solve(pr, solver, float(l1), float(l2), sys.stdout, R)
                            for l1, l2 in pr.lam_grid]
    elif lam == "grid8":
        rec["grid_index"] = GRID8
        rec["solutions"] = [solve(pr, solver, float(pr.lam_grid[i, 0]), float(pr.lam_grid[i, 1]),
                                  sys.stdout, R) for i in GRID8]
    else:
        rec.update(solve(pr, solver, pr.lam1, pr.lam2, sys.stdout, R, keep_beta=lam != "nobeta"))
    with open(os.path.join(HERE, name + ".json"), "w") as fh:
        # large vectors on one line each
        json.dump(rec, fh, indent=None if pr.p > 4096 else 1)


if __name__ == "__main__":
    for nm in (sys.argv[1:] or QUICK):
        make(nm)
