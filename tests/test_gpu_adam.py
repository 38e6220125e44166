"""The Euler-Lagrange route on the GPU against the oracle (Sec. 3.2, eq. gradJ; the appendix Adam
algorithm).

* grad J(s) = R(s): the same FP64 toolbox on both sides (the oracle's matrices loaded into the
  library), linear and semilinear; FP64 on both sides, only the order of rounding differs, so
  1e-11 relative to the largest component.
* A GPU-built FP32 toolbox: the gradient against the oracle's residual on the downloaded
  matrices (the library multiplies the stored FP32 entries by a two-float split of the FP64
  operand and accumulates the pairs, the refinement's residual): 1e-10; and a 30-step Adam
  trajectory against the oracle's on those matrices.
* Adam: the GPU trajectory against the oracle's for the same start, steps and hyper-parameters.
  Adam divides m_j by sqrt(v_j), so a rounding difference in a component of the gradient moves
  that component by at most alpha_j |delta m_j| / sqrt(v_j); after tens of steps on this
  conditioning the two trajectories stay within 1e-8 of max|s| of each other.
* The early stop: grad_norm is the lambda-weighted norm of R at the returned s.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import solve as S
from paper_2608_07017_b300 import ewos
from paper_2608_07017_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def disk():
    from paper_2608_07017_b300 import build
    build.build()
    w = W.disk400()
    r = oracle.walk_rows(2, "ball", w.domain.params, w.x, w.z, 1000, 1e-3, 0)
    counts = oracle.cell_counts(2, "ball", w.domain.params, w.x, 1_000_000, seed=1)
    lam = counts / counts.sum()
    tb = dict(G=r["G"], gradG=r["gradG"], H=r["Hc"] / 1000.0, gradH=r["gradH"])
    gtb = ewos.toolbox_from_host(2, w.x, w.z, tb["G"], tb["gradG"], tb["H"], tb["gradH"], lam, precision=64)
    yield w, tb, lam, gtb
    gtb.close()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_gradient_matches_oracle_residual(disk):
    w, tb, lam, gtb = disk
    pb = w.problem
    rng = np.random.default_rng(5)
    for s in (np.zeros(gtb.m), rng.normal(size=gtb.m), 30.0 * rng.normal(size=gtb.m)):
        ref = S.residual(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g, s)
        got = gtb.gradient(s, pb.A, pb.f, pb.g)
        assert _rel(got, ref) < 1e-11
    # with first- and zeroth-order terms and a semilinear N(u) = u + 2 u^3
    b = np.stack([np.sin(3 * w.x[:, 0]), np.cos(2 * w.x[:, 1])], axis=1)
    c = 1.0 + w.x[:, 0] ** 2
    coef = [0.0, 1.0, 0.0, 2.0]
    s = rng.normal(size=gtb.m)
    ref = S.residual(tb, lam, pb.A, b, c, pb.f, pb.g, s, coef)
    got = gtb.gradient(s, pb.A, pb.f, pb.g, b=b, c=c, kind="semilinear", coef=coef)
    assert _rel(got, ref) < 1e-11
    assert got.shape == (gtb.m,)


def test_gradient_and_adam_fp32_built_toolbox():
    # FP32 toolbox: the gradient is the refinement's FP32-pair residual
    w = W.disk400()
    pb = w.problem
    gtb = ewos.build_workload(w, cell_samples=200_000)
    tb = gtb.matrices()
    lam = gtb.get("lambda")
    rng = np.random.default_rng(6)
    s = rng.normal(size=gtb.m)
    got = gtb.gradient(s, pb.A, pb.f, pb.g)
    coef = [0.0, 0.0, 0.0, 1.0]
    got3 = gtb.gradient(s, pb.A, pb.f, pb.g, kind="semilinear", coef=coef)
    s0 = rng.normal(size=gtb.m)
    sa, _, rep = gtb.minimize_adam(pb.A, pb.f, pb.g, s0=s0, alpha=0.1, max_iter=30)
    gtb.close()
    assert _rel(got, S.residual(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g, s)) < 1e-10
    assert _rel(got3, S.residual(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g, s, coef)) < 1e-10
    assert _rel(sa, S.adam(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g, s0, 0.1, iters=30)) < 1e-8


@pytest.mark.parametrize("alpha,iters", [(0.1, 1), (0.1, 40), (0.5, 25)])
def test_adam_trajectory_matches_oracle(disk, alpha, iters):
    w, tb, lam, gtb = disk
    pb = w.problem
    s0 = np.random.default_rng(7).normal(size=gtb.m)
    s, u, rep = gtb.minimize_adam(pb.A, pb.f, pb.g, s0=s0, alpha=alpha, max_iter=iters)
    ref = S.adam(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g, s0, alpha, iters=iters)
    assert rep["iters"] == iters and not rep["converged"]
    assert _rel(s, ref) < 1e-8
    assert _rel(u, S.reconstruct(tb, ref, pb.g)[0]) < 1e-8
    R = S.residual(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g, ref)
    assert abs(rep["grad_norm"] - math.sqrt(np.sum(lam * R * R))) <= 1e-8 * rep["grad_norm"]


def test_adam_semilinear_matches_oracle(disk):
    w, tb, lam, gtb = disk
    pb = w.problem
    coef = [0.0, 0.0, 0.0, 1.0]
    f3 = pb.f + pb.u_star ** 3
    s, u, rep = gtb.minimize_adam(pb.A, f3, pb.g, kind="semilinear", coef=coef, alpha=0.1, max_iter=30)
    ref = S.adam(tb, lam, pb.A, pb.b, pb.c, f3, pb.g, np.zeros(gtb.m), 0.1, iters=30, nl=coef)
    assert _rel(s, ref) < 1e-8


def test_adam_early_stop(disk):
    w, tb, lam, gtb = disk
    pb = w.problem
    R0 = S.residual(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g, np.zeros(gtb.m))
    tol = 0.3 * math.sqrt(np.sum(lam * R0 * R0))
    s, u, rep = gtb.minimize_adam(pb.A, pb.f, pb.g, alpha=0.1, max_iter=5000, tol=tol, check_every=5)
    assert rep["converged"] and rep["grad_norm"] <= tol
    assert 0 < rep["iters"] < 5000 and rep["iters"] % 5 == 0
    R = S.residual(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g, s)
    assert abs(rep["grad_norm"] - math.sqrt(np.sum(lam * R * R))) <= 1e-9 * tol
    ref = S.adam(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g, np.zeros(gtb.m), 0.1, iters=rep["iters"])
    assert _rel(s, ref) < 1e-8
    # the check before the last block of steps had not yet met the tolerance
    prev = S.adam(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g, np.zeros(gtb.m), 0.1, iters=rep["iters"] - 5)
    Rp = S.residual(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g, prev)
    assert math.sqrt(np.sum(lam * Rp * Rp)) > tol
    # zero steps return the start and its gradient norm
    s0, _, rep0 = gtb.minimize_adam(pb.A, pb.f, pb.g, max_iter=0)
    assert rep0["iters"] == 0 and np.all(s0 == 0.0)


def test_invalid_arguments(disk):
    w, tb, lam, gtb = disk
    pb = w.problem
    with pytest.raises(ewos.EwosError) as e:
        gtb.gradient(np.zeros(gtb.m), pb.A, pb.f, pb.g, kind="quasilinear", coef=[1.0])
    assert e.value.status == ewos.EINVAL
    for kw in (dict(alpha=0.0), dict(beta1=1.0), dict(beta2=-0.1), dict(eps=0.0), dict(max_iter=-1)):
        with pytest.raises(ewos.EwosError) as e:
            gtb.minimize_adam(pb.A, pb.f, pb.g, **kw)
        assert e.value.status == ewos.EINVAL
