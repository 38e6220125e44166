"""GPU solves against the oracle's solves (Sec. 3; eq. linear_q with the Tikhonov shift,
Newton, Picard).

* Same toolbox on both sides (the oracle's FP64 matrices loaded into the library): the FP64
  path must agree with the oracle to 1e-9 relative (both solve the same FP64 system, only the
  order of rounding differs; kappa(Lambda + alpha I) <= ~1e3).
* Whole pipeline (GPU build + GPU solve vs oracle build + oracle solve): the error against the
  manufactured solution must agree within 1e-3 * max(1e-3, e_oracle) (the stated bar).
* Full size: the FP64 residual of the GPU solution of the square workload, evaluated with
  numpy from the downloaded toolbox, is at rounding level.
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


@pytest.mark.parametrize("rcond", [3e-2, 1e-3])
def test_linear_fp64_matches_oracle_same_toolbox(disk, rcond):
    w, tb, lam, gtb = disk
    pb = w.problem
    ref = S.solve_linear(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g, rcond=rcond)
    u, s, rep = gtb.solve(pb.A, pb.f, pb.g, b=pb.b, c=pb.c, rcond=rcond, want_s=True)
    assert _rel(u, ref["u"]) < 1e-9
    assert _rel(s, ref["s"]) < 1e-8
    assert abs(rep["alpha"] - ref["alpha"]) <= 1e-12 * ref["alpha"]
    assert rep["residual"] < 1e-10 * np.linalg.norm(ref["rhs"])


def test_linear_with_first_and_zeroth_order_terms(disk):
    w, tb, lam, gtb = disk
    pb = w.problem
    rng = np.random.default_rng(2)
    b = rng.uniform(-1, 1, (w.x.shape[0], 2))
    c = rng.uniform(0, 2, w.x.shape[0])
    ref = S.solve_linear(tb, lam, pb.A, b, c, pb.f, pb.g)
    u, _, _ = gtb.solve(pb.A, pb.f, pb.g, b=b, c=c)
    assert _rel(u, ref["u"]) < 1e-9


def test_multiple_rhs_equal_single_solves(disk):
    w, tb, lam, gtb = disk
    pb = w.problem
    rng = np.random.default_rng(3)
    F = np.stack([pb.f, pb.f * 0.5 + 1.0, rng.normal(size=pb.f.shape)])
    Gb = np.stack([pb.g, pb.g * 2.0, rng.normal(size=pb.g.shape)])
    U, _, _ = gtb.solve(pb.A, F, Gb)
    for r in range(3):
        ref = S.solve_linear(tb, lam, pb.A, None, None, F[r], Gb[r])
        assert _rel(U[r], ref["u"]) < 1e-9


def test_newton_matches_oracle(disk):
    w, tb, lam, gtb = disk
    pb = w.problem
    f3 = pb.f + pb.u_star ** 3
    ref = S.newton(tb, lam, pb.A, None, None, f3, pb.g, [0, 0, 0, 1])
    u, _, rep = gtb.solve(pb.A, f3, pb.g, kind="semilinear", coef=[0, 0, 0, 1])
    assert rep["converged"] and rep["iters"] == ref["iters"]
    assert _rel(u, ref["u"]) < 1e-9


def test_picard_matches_oracle(disk):
    w, tb, lam, gtb = disk
    st = W.make_problem("star", w.x, w.z)
    ref = S.picard(tb, lam, st.A, None, None, st.f, st.g, st.kappa)
    u, _, rep = gtb.solve(st.A, st.f, st.g, kind="quasilinear", coef=st.kappa)
    assert rep["converged"] and abs(rep["iters"] - ref["iters"]) <= 1
    assert _rel(u, ref["u"]) < 1e-8


def test_ragged_sizes_lu():
    # m not a multiple of the 64-wide panels (m = 130, 67, 1), FP32 toolbox
    for k, per in ((11, 3), (8, 2), (1, 1)):
        x = W.square_nodes(k)
        x = x[: max(1, x.shape[0] - (3 if k > 1 else 0))]
        z = W.square_boundary_nodes(per * 2)
        r = oracle.walk_rows(2, "box", [0, 0, 1, 1], x, z, 400, 1e-4, 7)
        lam = np.full(x.shape[0], 1.0 / x.shape[0])
        tb = dict(G=r["G"], gradG=r["gradG"], H=r["Hc"] / 400.0, gradH=r["gradH"])
        pb = W.make_problem("square", x, z)
        ref = S.solve_linear(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g)
        gtb = ewos.toolbox_from_host(2, x, z, tb["G"], tb["gradG"], tb["H"], tb["gradH"], lam, precision=64)
        u, _, _ = gtb.solve(pb.A, pb.f, pb.g, b=pb.b)
        gtb.close()
        assert _rel(u, ref["u"]) < 1e-9, x.shape


def test_whole_pipeline_disk400_fp64():
    w = W.disk400()
    pb = w.problem
    gtb = ewos.build_workload(w, cell_samples=1_000_000)
    lam_g = gtb.get("lambda")
    u, _, _ = gtb.solve(pb.A, pb.f, pb.g)
    gtb.close()
    r = oracle.walk_rows(2, "ball", w.domain.params, w.x, w.z, 1000, 1e-3, 0)
    counts = oracle.cell_counts(2, "ball", w.domain.params, w.x, 1_000_000, seed=0)
    lam = counts / counts.sum()
    tb = dict(G=r["G"], gradG=r["gradG"], H=r["Hc"] / 1000.0, gradH=r["gradH"])
    ref = S.solve_linear(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g)
    e_g = S.errors(u, pb.u_star, lam)["l2"]
    e_o = S.errors(ref["u"], pb.u_star, lam)["l2"]
    assert abs(e_g - e_o) <= 1e-3 * max(1e-3, e_o)
    assert np.max(np.abs(lam_g - lam)) < 1e-5


def test_square4096_full_size_fp64_residual():
    w = W.square4096()
    pb = w.problem
    gtb = ewos.build_workload(w)
    u, s, rep = gtb.solve(pb.A, pb.f, pb.g, b=pb.b, want_s=True)
    mats = gtb.matrices()
    lam = gtb.get("lambda")
    gtb.close()
    Lam = S.assemble(mats["G"], mats["gradG"], lam, pb.A, pb.b, None)
    r = S.rhs(mats["G"], mats["gradG"], mats["H"], mats["gradH"], lam, pb.A, pb.b, None, pb.f, pb.g)
    alpha = S.shift(Lam, 3e-2)
    res = (Lam + alpha * np.eye(Lam.shape[0])) @ s - r
    assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(r)
    u_ref = mats["G"] @ s + mats["H"] @ pb.g
    assert _rel(u, u_ref) < 1e-10
    ref_norm = math.sqrt(np.sum(lam * pb.u_star ** 2))
    assert S.errors(u, pb.u_star, lam)["l2"] < 0.2 * ref_norm


# ------------------------------------------------------------------ mixed precision
# The mixed path assembles Lambda in 32-bit, factors Lambda + alpha I in FP32 and refines with the
# FP64 matrix-free residual to 1e-12.  Its shift alpha comes from its own 32-bit Lambda, so it is
# compared with the oracle run with that alpha (1e-9), and with the FP64 GPU path by the R16
# solution bar.

@pytest.mark.parametrize("assembly", ["fp16", "tf32"])
def test_mixed_linear_matches_oracle(disk, assembly):
    # Lambda assembled on the tensor cores from scaled FP16 halves (the default) or TF32 parts:
    # either way the refined solution is the oracle's for the same shift alpha
    w, tb, lam, gtb = disk
    pb = w.problem
    u, s, rep = gtb.solve(pb.A, pb.f, pb.g, b=pb.b, c=pb.c, mode="mixed", want_s=True, assembly=assembly)
    assert rep["converged"] and rep["refine_iters"] >= 1
    ref = S.solve_linear(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g, alpha=rep["alpha"])
    assert _rel(u, ref["u"]) < 1e-9
    ref_alpha = S.shift(ref["Lam"], 3e-2)
    assert abs(rep["alpha"] - ref_alpha) <= 1e-5 * ref_alpha
    u64, _, _ = gtb.solve(pb.A, pb.f, pb.g, b=pb.b, c=pb.c, mode="fp64")
    e_m = S.errors(u, pb.u_star, lam)["l2"]
    e_d = S.errors(u64, pb.u_star, lam)["l2"]
    assert abs(e_m - e_d) <= 1e-3 * max(1e-3, e_d)


def test_mixed_newton_matches_oracle(disk):
    w, tb, lam, gtb = disk
    pb = w.problem
    f3 = pb.f + pb.u_star ** 3
    u, _, rep = gtb.solve(pb.A, f3, pb.g, kind="semilinear", coef=[0, 0, 0, 1], mode="mixed")
    assert rep["converged"]
    ref = S.newton(tb, lam, pb.A, None, None, f3, pb.g, [0, 0, 0, 1], alpha=rep["alpha"])
    assert _rel(u, ref["u"]) < 1e-8


def test_mixed_picard_equal_accuracy(disk):
    w, tb, lam, gtb = disk
    st = W.make_problem("star", w.x, w.z)
    um, _, rm = gtb.solve(st.A, st.f, st.g, kind="quasilinear", coef=st.kappa, mode="mixed")
    ud, _, rd = gtb.solve(st.A, st.f, st.g, kind="quasilinear", coef=st.kappa, mode="fp64")
    assert rm["converged"] and rd["converged"]
    e_m = S.errors(um, st.u_star, lam)["l2"]
    e_d = S.errors(ud, st.u_star, lam)["l2"]
    assert abs(e_m - e_d) <= 1e-3 * max(1e-3, e_d)
    assert _rel(um, ud) < 1e-4


def test_mixed_square4096_full_size():
    w = W.square4096()
    pb = w.problem
    gtb = ewos.build_workload(w)
    u, s, rep = gtb.solve(pb.A, pb.f, pb.g, b=pb.b, want_s=True, mode="mixed")
    # the two tensor-core assemblies reach the same refined solution, in as many sweeps; the shift
    # alpha = rcond ||Lambda_32||_F comes from each assembly's own FP32 matrix (within a few 1e-6
    # of the exact norm: the tensor cores truncate, the chunked accumulation bounds that)
    ut, _, rept = gtb.solve(pb.A, pb.f, pb.g, b=pb.b, mode="mixed", assembly="tf32")
    assert rept["converged"] and abs(rept["refine_iters"] - rep["refine_iters"]) <= 1
    assert abs(rept["alpha"] - rep["alpha"]) <= 1e-5 * rep["alpha"]
    assert _rel(u, ut) < 1e-5
    u64, s64, rep64 = gtb.solve(pb.A, pb.f, pb.g, b=pb.b, want_s=True, mode="fp64")
    mats = gtb.matrices()
    lam = gtb.get("lambda")
    gtb.close()
    assert rep["converged"]
    Lam = S.assemble(mats["G"], mats["gradG"], lam, pb.A, pb.b, None)
    r = S.rhs(mats["G"], mats["gradG"], mats["H"], mats["gradH"], lam, pb.A, pb.b, None, pb.f, pb.g)
    res = (Lam + rep["alpha"] * np.eye(Lam.shape[0])) @ s - r
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(r)
    e_m = S.errors(u, pb.u_star, lam)["l2"]
    e_d = S.errors(u64, pb.u_star, lam)["l2"]
    assert abs(e_m - e_d) <= 1e-3 * max(1e-3, e_d)


# ------------------------------------------------------------------ mixed-mode LU variants
# The mixed mode factors with the diagonal pivots and keeps that factorisation only when every
# multiplier has |l| <= 1 (it is then the partial-pivoting one); otherwise it refactors with
# row interchanges.  Both must give the oracle's solution after refinement.

def test_mixed_unpivoted_accepted_and_equal_to_pivoted(disk):
    w, tb, lam, gtb = disk
    pb = w.problem
    u0, _, r0 = gtb.solve(pb.A, pb.f, pb.g, b=pb.b, c=pb.c, mode="mixed")
    u1, _, r1 = gtb.solve(pb.A, pb.f, pb.g, b=pb.b, c=pb.c, mode="mixed", pivoting=1)
    assert r0["factorizations"] == 1 and r0["pivoted_factorizations"] == 0
    assert r1["factorizations"] == 1 and r1["pivoted_factorizations"] == 1
    assert _rel(u0, u1) < 1e-9


def _random_toolbox(seed, n_drop=0):
    # G ~ N(0, 1), grad G ~ N(0, 1e-4) and a strong drift: Lambda is dominated by its
    # non-symmetric b . grad G^T G part and needs row interchanges (max |l| ~ 80 without)
    rng = np.random.default_rng(seed)
    x = W.disk_nodes(0.15, 0.9)
    x = x[: x.shape[0] - n_drop]
    n = m = x.shape[0]
    z = W.circle_nodes(24)
    G = rng.normal(size=(n, m))
    gradG = rng.normal(size=(2, n, m)) * 0.01
    H = rng.uniform(0, 1, (n, z.shape[0]))
    H /= H.sum(1, keepdims=True)
    gradH = rng.normal(size=(2, n, z.shape[0])) * 0.01
    lam = np.full(n, 1.0 / n)
    A = np.tile(np.eye(2), (n, 1, 1))
    b = rng.normal(size=(n, 2)) * 50
    f = rng.normal(size=n)
    g = rng.normal(size=z.shape[0])
    tb = dict(G=G, gradG=gradG, H=H, gradH=gradH)
    return x, z, tb, lam, A, b, f, g


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_falls_back_to_interchanges(mode):
    x, z, tb, lam, A, b, f, g = _random_toolbox(5)
    gtb = ewos.toolbox_from_host(2, x, z, tb["G"], tb["gradG"], tb["H"], tb["gradH"], lam, precision=64)
    u, s, rep = gtb.solve(A, f, g, b=b, mode=mode, want_s=True)
    gtb.close()
    assert rep["converged"]
    assert rep["factorizations"] == 1 and rep["pivoted_factorizations"] == 1
    ref = S.solve_linear(tb, lam, A, b, None, f, g, alpha=rep["alpha"] if mode == "mixed" else None)
    assert _rel(u, ref["u"]) < 1e-9


def test_fp64_unpivoted_accepted(disk):
    w, tb, lam, gtb = disk
    pb = w.problem
    u0, _, r0 = gtb.solve(pb.A, pb.f, pb.g, b=pb.b, c=pb.c)
    u1, _, r1 = gtb.solve(pb.A, pb.f, pb.g, b=pb.b, c=pb.c, pivoting=1)
    assert r0["pivoted_factorizations"] == 0 and r1["pivoted_factorizations"] == 1
    assert _rel(u0, u1) < 1e-11


@pytest.mark.parametrize("k,per", [(11, 3), (8, 2), (1, 1)])
def test_mixed_ragged_sizes(k, per):
    # m = 118, 61, 1 (not multiples of the 64-wide panels), unpivoted FP32 LU
    x = W.square_nodes(k)
    x = x[: max(1, x.shape[0] - (3 if k > 1 else 0))]
    z = W.square_boundary_nodes(per * 2)
    r = oracle.walk_rows(2, "box", [0, 0, 1, 1], x, z, 400, 1e-4, 7)
    lam = np.full(x.shape[0], 1.0 / x.shape[0])
    tb = dict(G=r["G"], gradG=r["gradG"], H=r["Hc"] / 400.0, gradH=r["gradH"])
    pb = W.make_problem("square", x, z)
    gtb = ewos.toolbox_from_host(2, x, z, tb["G"], tb["gradG"], tb["H"], tb["gradH"], lam, precision=64)
    u, _, rep = gtb.solve(pb.A, pb.f, pb.g, b=pb.b, mode="mixed")
    gtb.close()
    assert rep["converged"]
    ref = S.solve_linear(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g, alpha=rep["alpha"])
    assert _rel(u, ref["u"]) < 1e-9, x.shape


@pytest.mark.parametrize("drop", [11, 8])
def test_mixed_tensor_core_updates_ragged(drop):
    # m = 389 (rows of the LU not 16-byte aligned: the update's C tile is read from global memory)
    # and m = 392 (aligned, C staged in shared memory, last tiles ragged): trailing updates of at
    # least 256 rows run on the tensor cores; K = 3 n is padded to a multiple of 32 in the
    # one-pass operand preparation of the assembly
    x = W.square_nodes(20)[:-drop]
    z = W.square_boundary_nodes(6)
    r = oracle.walk_rows(2, "box", [0, 0, 1, 1], x, z, 300, 1e-4, 5)
    lam = np.full(x.shape[0], 1.0 / x.shape[0])
    tb = dict(G=r["G"], gradG=r["gradG"], H=r["Hc"] / 300.0, gradH=r["gradH"])
    pb = W.make_problem("square", x, z)
    gtb = ewos.toolbox_from_host(2, x, z, tb["G"], tb["gradG"], tb["H"], tb["gradH"], lam, precision=32)
    u, _, rep = gtb.solve(pb.A, pb.f, pb.g, b=pb.b, mode="mixed")
    gtb.close()
    assert rep["converged"] and rep["factorizations"] == 1
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    ref = S.solve_linear({k: f32(v) for k, v in tb.items()}, lam, pb.A, pb.b, pb.c, pb.f, pb.g, alpha=rep["alpha"])
    assert _rel(u, ref["u"]) < 1e-9, x.shape


def test_ball8000_full_size_newton_mixed_and_fp64():
    # -Laplace u + u^3 = f on the unit ball, 8000 unknowns: Newton with the tensor-core
    # assembly, FP32 LU and FP64 refinement against the plain FP64 path (R16 bar)
    w = W.ball8000()
    pb = w.problem
    gtb = ewos.build_workload(w)
    um, _, rm = gtb.solve(pb.A, pb.f, pb.g, kind="semilinear", coef=pb.nl, mode="mixed")
    ud, _, rd = gtb.solve(pb.A, pb.f, pb.g, kind="semilinear", coef=pb.nl, mode="fp64")
    lam = gtb.get("lambda")
    gtb.close()
    assert rm["converged"] and rd["converged"]
    assert rm["iters"] == rd["iters"]
    e_m = S.errors(um, pb.u_star, lam)["l2"]
    e_d = S.errors(ud, pb.u_star, lam)["l2"]
    assert abs(e_m - e_d) <= 1e-3 * max(1e-3, e_d)
    assert e_m < 0.2 * math.sqrt(np.sum(lam * pb.u_star ** 2))


def test_mixed_lu_with_rank512_fp16_update():
    # m = 1100: the unpivoted FP32 LU's first super panel (512 columns) ends with the rank-512
    # update of the trailing 588 x 588 matrix, on the FP16 tensor-core path (rows and columns
    # scaled by powers of two); the refined solution is the oracle's, in few sweeps
    rng = np.random.default_rng(11)
    n = 1100
    x = rng.uniform(0.05, 0.95, size=(n, 2))
    z = W.square_boundary_nodes(8)
    sc = 2.0 ** rng.uniform(-1, 1, size=n)
    G = (rng.normal(size=(n, n)) * 0.05 + np.eye(n)) * sc
    gradG = (rng.normal(size=(2, n, n)) * 0.05 + 2.0 * np.eye(n)[None]) * sc
    H = rng.uniform(0, 1, (n, z.shape[0]))
    H /= H.sum(1, keepdims=True)
    gradH = rng.normal(size=(2, n, z.shape[0])) * 0.01
    lam = np.full(n, 1.0 / n)
    A = np.tile(np.eye(2), (n, 1, 1))
    c = np.ones(n)
    f = rng.normal(size=n)
    g = rng.normal(size=z.shape[0])
    gtb = ewos.toolbox_from_host(2, x, z, G, gradG, H, gradH, lam, precision=32)
    u, _, rep = gtb.solve(A, f, g, c=c, mode="mixed")
    gtb.close()
    assert rep["converged"] and rep["factorizations"] == 1 and rep["pivoted_factorizations"] == 0
    assert rep["refine_iters"] <= 4
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    tb = dict(G=f32(G), gradG=f32(gradG), H=f32(H), gradH=f32(gradH))
    ref = S.solve_linear(tb, lam, A, None, c, f, g, alpha=rep["alpha"])
    assert _rel(u, ref["u"]) < 1e-9
