"""Whole pipeline against the oracle's: the GPU builds the toolbox (FP32 walks) and solves, the
stored oracle result built its own toolbox with the FP64 walks on the same Philox stream and
solved with the FP64 textbook algorithms (tests/golden/make_pipeline_golden.py, which calls only
oracle/).  Bar (solutions): the lambda-weighted L2 error against the manufactured solution
agrees with the oracle's, |e_GPU - e_oracle| <= 1e-3 max(1e-3, e_oracle), in both solve modes
(Sec. 3.1, eq. linear_q; Sec. 3.2, eq. gradJ; Picard for the quasilinear case).
"""
import json
import os

import numpy as np
import pytest

from paper_2608_07017_b300 import ewos
from paper_2608_07017_b300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2608_07017_b300 import build
    build.build()


def _golden(name):
    g = np.load(os.path.join(GOLDEN, f"pipeline_{name}.npz"))
    return g["u"], g["lam"], json.loads(str(g["meta"]))


def _workload(name, walks):
    if name == "square4096":
        return W.square4096(walks=walks), 0
    if name == "ball8000":
        return W.ball8000(walks=walks), 0
    k = int(name[4:])
    w = W.stars()[k]
    w.walks = walks
    return w, k


@pytest.mark.parametrize("name", ["star23", "square4096", "ball8000"])
def test_pipeline_matches_oracle_pipeline(name):
    u_orc, lam_orc, meta = _golden(name)
    w, inst = _workload(name, meta["walks"])
    pb = w.problem
    kw = dict(instance=inst)
    if meta["cell_samples"]:
        kw["cell_samples"] = meta["cell_samples"]
    tb = ewos.build_workload(w, **kw)
    assert tb.status == ewos.OK
    lam = tb.get("lambda")
    # Monte Carlo cell weights: the same samples, binned in FP32 against FP64
    assert np.max(np.abs(lam - lam_orc)) <= 4.0 / (meta["cell_samples"] or 1e12) + 1e-15
    e_orc = meta["l2_error"]
    tol = 1e-3 * max(1e-3, e_orc)
    kind = {"linear": "linear", "semilinear": "semilinear", "quasilinear": "quasilinear"}[meta["kind"]]
    coef = pb.nl if kind == "semilinear" else (pb.kappa if kind == "quasilinear" else None)
    for mode in ("mixed", "fp64"):
        u, _, rep = tb.solve(pb.A, pb.f, pb.g, b=pb.b, c=pb.c, kind=kind, coef=coef, mode=mode)
        assert rep["converged"], (name, mode, rep)
        e = float(np.sqrt(np.sum(lam * (u - pb.u_star) ** 2)))
        du = float(np.sqrt(np.sum(lam * (u - u_orc) ** 2)))
        assert abs(e - e_orc) <= tol, (name, mode, e, e_orc, tol, du)
    tb.close()
