"""Writes the oracle's whole-pipeline results (toolbox built by the FP64 oracle walks, then the
oracle's solve) that the GPU pipeline tests compare with.  Calls only ``oracle/`` (and the
seeded input generators of ``workloads.py``); nothing here comes from the CUDA path.

    python tests/golden/make_pipeline_golden.py [square4096|ball8000|star23 ...]

Cases (the same seeds and sizes the GPU tests build with):
  square4096    unit square, 4096 nodes, 512 boundary nodes, 10^4 walks/node, eps 1e-4, seed 0;
                exact cell weights 1/n; the linear problem of the square workload, LU of the
                Tikhonov-shifted system (Sec. 3.1, eq. linear_q).
  ball8000      unit ball, 8000 nodes, 2000 boundary nodes, 1000 walks/node (a tenth of the
                workload's 10^4, to keep the FP64 brute-force walks to minutes), eps 1e-4, seed 0;
                Monte Carlo cell weights (10^7 samples, seed 0); -Laplace u + u^3 = f by Newton
                on R(s) + alpha s = 0 (Sec. 3.2, eq. gradJ).
  star23        instance 23 of the 32 star polygons (1022 nodes, 127 boundary nodes, 2000
                walks/node, eps 1e-4, Philox instance 23); Monte Carlo cell weights (10^7
                samples); -div((1 + u^2) grad u) = f by Picard.
Each file holds u (the oracle's solution at the nodes), its lambda-weighted L2 error against
the manufactured u*, the shift alpha, the iteration count, and a JSON header with the command.
The solves use LAPACK's LU (oracle.solve.LU_BACKEND = "lapack") at these sizes.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle                                     # noqa: E402
from oracle import solve as S                     # noqa: E402
from paper_2608_07017_b300 import workloads as W  # noqa: E402

CELL_SAMPLES = 10_000_000
BALL_WALKS = 1000
STAR_INDEX = 23


def _toolbox(w, walks, instance=0):
    d = w.domain.dim
    r = oracle.walk_rows(d, w.domain.kind, w.domain.params, w.x, w.z, walks, w.eps, w.seed, instance=instance)
    return dict(G=r["G"], gradG=r["gradG"], H=r["Hc"] / float(walks), gradH=r["gradH"]), r["steps"]


def _lam(w, instance=0):
    if w.lam is not None:
        return w.lam
    cnt = oracle.cell_counts(w.domain.dim, w.domain.kind, w.domain.params, w.x, CELL_SAMPLES, seed=w.seed,
                             instance=instance)
    return cnt / cnt.sum()


def case(name):
    t0 = time.time()
    if name == "square4096":
        w = W.square4096()
        walks, inst = w.walks, 0
    elif name == "ball8000":
        w = W.ball8000()
        walks, inst = BALL_WALKS, 0
    elif name == "star23":
        w = W.stars()[STAR_INDEX]
        walks, inst = w.walks, STAR_INDEX
    else:
        raise SystemExit(f"unknown case {name}")
    pb = w.problem
    tb, steps = _toolbox(w, walks, inst)
    t_walk = time.time() - t0
    lam = _lam(w, inst)
    if pb.kind == "linear":
        sol = S.solve_linear(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g)
        iters = 1
    elif pb.kind == "semilinear":
        sol = S.newton(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g, pb.nl)
        iters = sol["iters"]
        assert sol["converged"]
    else:
        sol = S.picard(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g, pb.kappa)
        iters = sol["iters"]
        assert sol["converged"]
    e = S.errors(sol["u"], pb.u_star, lam)
    meta = dict(case=name, n=int(w.x.shape[0]), p=int(w.z.shape[0]), walks=int(walks), eps=w.eps, seed=w.seed,
                instance=inst, cell_samples=None if w.lam is not None else CELL_SAMPLES, kind=pb.kind,
                wos_steps=int(steps), seconds_walks=round(t_walk, 1), seconds_total=round(time.time() - t0, 1),
                l2_error=e["l2"], linf_error=e["linf"], iters=int(iters),
                alpha=float(sol.get("alpha", np.nan)) if "alpha" in sol else None,
                command="python tests/golden/make_pipeline_golden.py " + name,
                lu="LAPACK getrf/getrs through scipy.linalg (oracle.solve.LU_BACKEND)")
    out = os.path.join(HERE, f"pipeline_{name}.npz")
    np.savez_compressed(out, u=sol["u"], lam=lam, meta=np.array(json.dumps(meta)))
    print(json.dumps(meta), flush=True)


def main():
    S.LU_BACKEND = "lapack"
    oracle.build()
    names = sys.argv[1:] or ["star23", "square4096", "ball8000"]
    for nm in names:
        case(nm)


if __name__ == "__main__":
    main()
