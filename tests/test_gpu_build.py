"""GPU toolbox build against the oracle (same Philox stream, element by element).

Bars (stated tolerances): exit cells equal on >= 99.9 % of walks; matrix entries within 1e-4
relative after the divergent-walk bound of tests/parity.py; H row sums exactly N; Philox bit
exact; the d = 2 Green radius within 1e-13 (FP64) / 4e-6 (FP32) relative of the oracle's.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2608_07017_b300 import ewos
from paper_2608_07017_b300 import workloads as W
from parity import compare_rows, gpu_arrays

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2608_07017_b300 import build
    build.build()
    oracle.build()


def _r0(dim, kind, params, x):
    return np.array([oracle.sdf(dim, kind, params, xi) for xi in x])


def test_philox_bit_exact():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(1 << 20, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:8] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1],
               [0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [7, 7, 7, 7]]
    for key in ([0, 0], [0xa4093822, 0x299f31d0], [0xFFFFFFFF, 1]):
        assert np.array_equal(ewos.debug_philox(ctr, key), oracle.philox_batch(ctr, key))


def test_green_radius_matches_oracle():
    u = np.concatenate([[2.0 ** -24, 1 - 2.0 ** -24, 0.5, 1e-6, 1 - 1e-6],
                        (np.arange(1 << 16) + 0.5) / (1 << 16)])
    ref = np.array([oracle.green_radius_2d(v) for v in u])
    r64 = ewos.debug_green_radius(u, 64)
    assert np.max(np.abs(r64 - ref) / ref) < 1e-13
    u32 = u.astype(np.float32)
    ref32 = np.array([oracle.green_radius_2d(float(v)) for v in u32])
    r32 = ewos.debug_green_radius(u32, 32).astype(np.float64)
    assert np.max(np.abs(r32 - ref32) / ref32) < 4e-6


def _parity(w, rows, N, precision, max_steps=10000, min_exit=0.999, walk_kernel=0):
    tb = ewos.build_toolbox(w.domain.kind, w.domain.dim, w.domain.params, w.x, w.z, N, w.eps, seed=w.seed,
                            precision=precision, record_walks=True, cell_samples=100000, max_steps=max_steps,
                            walk_kernel=walk_kernel)
    if walk_kernel:
        assert tb.report()["walk_kernel"] == walk_kernel
    g = gpu_arrays(tb, N)
    orc = oracle.walk_rows(w.domain.dim, w.domain.kind, w.domain.params, w.x, w.z, N, w.eps, w.seed, rows=rows,
                           records=True, max_steps=max_steps)
    r0 = _r0(w.domain.dim, w.domain.kind, w.domain.params, w.x[rows])
    rep = compare_rows(g, orc, rows, N, w.domain.dim, r0, fp32=precision == 32)
    assert rep["exit_equal"] >= min_exit, rep
    assert np.all(g["Hc"].sum(1) == N)
    br = tb.report()
    assert br["walks"] == w.x.shape[0] * N
    tb.close()
    return rep, g, br


def test_disk400_fp64_full_parity():
    w = W.disk400(problem=False)
    rows = np.arange(400)
    rep, g, br = _parity(w, rows, 1000, 64)
    assert rep["exit_equal"] >= 0.9999
    orc_steps = oracle.walk_rows(2, "ball", w.domain.params, w.x, w.z, 1000, 1e-3, 0, rows=[0, 1])["steps"]
    assert br["steps"] > 0 and orc_steps > 0
    # closed form on the GPU output: G 1 = (1 - |x|^2)/4 within 4 SE + eps/2
    se = g["walk_mass"].std(1) / math.sqrt(1000)
    ex = (1 - (w.x ** 2).sum(1)) / 4
    assert np.all(np.abs(g["G"].sum(1) - ex) <= 4 * se + 1e-3 / 2)


def test_square_fp32_parity_small():
    w = W.square(16, 16, walks=2000, eps=1e-4, problem=False)
    rep, _, _ = _parity(w, np.arange(w.x.shape[0]), 2000, 32)
    assert rep["exit_equal"] >= 0.999


def test_ball3d_fp32_parity_small():
    x, _ = W.ball_nodes(500, seed=1)
    w = W.Workload("ball500", W.Domain(3, "ball", np.array([0.0, 0, 0, 1])), x, W.fibonacci_sphere(200), 1000,
                   1e-4, 32, 3)
    _parity(w, np.arange(0, 500, 3), 1000, 32)


def test_star_polygon_fp32_parity_small():
    V = W.star_polygon(5)
    rng = np.random.default_rng(4)
    x = W.star_nodes(V, 300, rng)
    w = W.Workload("star300", W.Domain(2, "polygon", V.ravel().copy()), x, W.polygon_boundary_nodes(V, 40), 500,
                   1e-4, 32, 1)
    _parity(w, np.arange(300), 500, 32)


def test_disk_fp32_parity_and_ragged_sizes():
    # n, p not multiples of any tile; a node close to the boundary; p = 1
    x = np.concatenate([W.disk_nodes(0.3, 0.9), [[0.0, 0.9995], [0.3, -0.2]]])
    w = W.Workload("ragged", W.Domain(2, "ball", np.array([0.0, 0, 1])), x, W.circle_nodes(37), 777, 1e-3, 32, 11)
    _parity(w, np.arange(x.shape[0]), 777, 32)
    w1 = W.Workload("p1", W.Domain(2, "ball", np.array([0.0, 0, 1])), x[:5], W.circle_nodes(1), 300, 1e-3, 32, 2)
    rep, g, _ = _parity(w1, np.arange(5), 300, 32)
    assert np.all(g["Hc"][:, 0] == 300)


def test_single_walk_single_node_and_shell_start():
    # N = 1 and n = 1; r0 < eps (the node sits inside the stopping shell)
    for x, eps in (([[0.2, 0.1]], 1e-3), ([[0.0, 0.99995]], 1e-4)):
        w = W.Workload("one", W.Domain(2, "ball", np.array([0.0, 0, 1])), np.array(x), W.circle_nodes(16), 1, eps,
                       64, 9)
        _parity(w, np.array([0]), 1, 64, min_exit=1.0)


def test_step_cap_reported_and_matches_oracle():
    w = W.Workload("cap", W.Domain(2, "ball", np.array([0.0, 0, 1])), W.disk_nodes(0.4, 0.9), W.circle_nodes(16),
                   200, 1e-12, 64, 5)
    tb = ewos.build_toolbox("ball", 2, w.domain.params, w.x, w.z, 200, 1e-12, seed=5, precision=64, max_steps=4,
                            cell_samples=10000)
    assert tb.status == ewos.ESTEPCAP
    orc = oracle.walk_rows(2, "ball", w.domain.params, w.x, w.z, 200, 1e-12, 5, max_steps=4)
    assert tb.report()["capped"] == orc["capped"] == w.x.shape[0] * 200
    assert np.array_equal(tb.get("Hc").astype(np.int64), orc["Hc"])
    tb.close()


def test_cell_weights_match_oracle_counts():
    w = W.disk400(problem=False)
    K = 2_000_000
    tb = ewos.build_toolbox("ball", 2, w.domain.params, w.x, w.z, 4, 1e-3, seed=3, precision=64, cell_samples=K)
    lam = tb.get("lambda")
    cnt = oracle.cell_counts(2, "ball", w.domain.params, w.x, K, seed=3)
    assert np.max(np.abs(lam * cnt.sum() - cnt)) <= 2.0
    assert abs(lam.sum() - 1) < 1e-12
    tb.close()


def _full_size_rows(w, rows, N, ctas_per_sm=0):
    """Matrices from the timed launch configuration (no records), records from a second launch
    (the trajectories do not depend on the record switch), oracle on the sampled rows."""
    tb = ewos.build_workload(w, ctas_per_sm=ctas_per_sm)
    g = gpu_arrays(tb, N, records=False)
    br = tb.report()
    tb.close()
    tbr = ewos.build_workload(w, record_walks=True, ctas_per_sm=ctas_per_sm)
    import torch
    n, d = w.x.shape
    rt = torch.as_tensor(rows, device="cuda")
    specs = {"walk_exit": ((n, N), torch.int32, np.int32), "walk_steps": ((n, N), torch.int32, np.int32),
             "walk_vhash": ((n, N), torch.int32, np.uint32), "walk_mass": ((n, N), torch.float64, np.float64),
             "walk_xexit": ((n, N, d), torch.float64, np.float64)}
    for k, (shape, tdt, ndt) in specs.items():
        buf = torch.empty(shape, dtype=tdt, device="cuda")
        tbr.get_device(k, buf)
        full = np.zeros((n,) + shape[1:], dtype=ndt)
        full[rows] = buf.index_select(0, rt).cpu().numpy().view(ndt)
        g[k] = full
        del buf
    tbr.close()
    orc = oracle.walk_rows(w.domain.dim, w.domain.kind, w.domain.params, w.x, w.z, N, w.eps, w.seed, rows=rows,
                           records=True)
    r0 = _r0(w.domain.dim, w.domain.kind, w.domain.params, w.x[rows])
    rep = compare_rows(g, orc, rows, N, w.domain.dim, r0, fp32=True)
    assert rep["exit_equal"] >= 0.999, rep
    assert np.all(g["Hc"].sum(1) == N)
    # grad H 1 = 0 on every row (E U_0 = 0): 4 SE of the per-walk terms (d/r0^2) w_c
    d = w.domain.dim
    per = (d / r0 ** 2)[:, None, None] * orc["records"]["w"]
    se = per.std(1) / np.sqrt(N)
    gh1 = np.stack([g["gradH"][c][rows].sum(1) for c in range(d)], axis=1)
    assert np.all(np.abs(gh1) <= 4 * se + 1e-6), (gh1, se)
    return rep, g, br, orc, r0


def test_square4096_full_size_sampled_rows():
    w = W.square4096(problem=False)
    rows = np.array([0, 63, 2080, 2047, 4032, 4095])
    rep, g, br, orc, _ = _full_size_rows(w, rows, w.walks)
    assert br["capped"] == 0
    # G 1 = the torsion function of the square (its Fourier series), 4 SE + the eps-shell bias
    from test_oracle_walks import _square_torsion
    ex = np.array([_square_torsion(*p) for p in w.x[rows]])
    se = orc["records"]["gmass"].std(1) / np.sqrt(w.walks)
    assert np.all(np.abs(g["G"][rows].sum(1) - ex) <= 4 * se + 1e-4)


def test_ball8000_full_size_sampled_rows():
    w = W.ball8000(problem=False)
    rows = np.array([0, 3999, 7999])
    rep, g, br, orc, r0 = _full_size_rows(w, rows, w.walks)
    x = w.x[rows]
    # G 1 = (1 - |x|^2)/6 on the sampled rows, 4 SE (per-walk masses) + the eps-shell bias
    se = np.sqrt(g["walk_mass"][rows].var(1) / w.walks)
    assert np.all(np.abs(g["G"][rows].sum(1) - (1 - (x ** 2).sum(1)) / 6) <= 4 * se + 1e-4 / 3)
    # grad G 1 = -x/3, 4 SE of the per-walk gradient masses + the eps-shell bias
    gse = orc["records"]["gradmass"].std(1) / np.sqrt(w.walks)
    gg1 = np.stack([g["gradG"][c][rows].sum(1) for c in range(3)], axis=1)
    assert np.all(np.abs(gg1 + x / 3) <= 4 * gse + (1e-4 / (3 * r0))[:, None])


def test_separate_v_partition_fp64_parity_and_solve():
    # V-centres y (the source partition of Sec. 2.3) different from the nodes x: m != n
    x = W.disk_nodes(0.12, 0.9)
    y = W.disk_nodes(0.17, 0.88) * 0.97
    z = W.circle_nodes(40)
    prm = np.array([0.0, 0, 1])
    N = 500
    tb = ewos.build_toolbox("ball", 2, prm, x, z, N, 1e-3, seed=4, precision=64, record_walks=True,
                            cell_samples=200000, y=y)
    assert tb.n == x.shape[0] and tb.m == y.shape[0] != x.shape[0]
    g = gpu_arrays(tb, N)
    assert g["G"].shape == (x.shape[0], y.shape[0])
    rows = np.arange(0, x.shape[0], 3)
    orc = oracle.walk_rows(2, "ball", prm, x, z, N, 1e-3, 4, rows=rows, y=y, records=True)
    rep = compare_rows(g, orc, rows, N, 2, _r0(2, "ball", prm, x[rows]), fp32=False)
    assert rep["exit_equal"] >= 0.9999, rep
    # cell weights are those of the nodes' own cells
    cnt = oracle.cell_counts(2, "ball", prm, x, 200000, seed=4)
    lam = tb.get("lambda")
    assert lam.shape == (x.shape[0],) and np.max(np.abs(lam * cnt.sum() - cnt)) <= 2.0
    # the solve on the m-column toolbox agrees with the oracle's solve of the same matrices
    from oracle import solve as S
    pb = W.make_problem("disk", x, z)
    mats = dict(G=g["G"], gradG=g["gradG"], H=g["H"], gradH=g["gradH"])
    for mode in ("fp64", "mixed"):
        u, s, r = tb.solve(pb.A, pb.f, pb.g, mode=mode, want_s=True)
        ref = S.solve_linear(mats, lam, pb.A, None, None, pb.f, pb.g, alpha=r["alpha"])
        assert s.shape == (y.shape[0],)
        assert np.max(np.abs(u - ref["u"])) <= 1e-9 * np.max(np.abs(ref["u"])), mode
    tb.close()


@pytest.mark.parametrize("walk_kernel", [1, 2])
def test_both_walk_kernels_parity(walk_kernel):
    """The row kernel with its G / grad G accumulators in global memory (1: one 16-byte L2
    reduction per walk point) and in shared memory (2: one FP32 atomic per value; the build
    without allocation uses it): both meet the same bars against the oracle, on small square,
    ball and star cases and ragged shapes (N = 1 and 3, fewer rows than CTAs, p = 1, FP64)."""
    w = W.square(16, 16, walks=2000, eps=1e-4, problem=False)
    _parity(w, np.arange(0, w.x.shape[0], 2), 2000, 32, walk_kernel=walk_kernel)
    x, _ = W.ball_nodes(500, seed=1)
    wb = W.Workload("ball500", W.Domain(3, "ball", np.array([0.0, 0, 0, 1])), x, W.fibonacci_sphere(200), 1000,
                    1e-4, 32, 3)
    _parity(wb, np.arange(0, 500, 5), 1000, 32, walk_kernel=walk_kernel)
    V = W.star_polygon(5)
    xs = W.star_nodes(V, 300, np.random.default_rng(4))
    ws = W.Workload("star300", W.Domain(2, "polygon", V.ravel().copy()), xs, W.polygon_boundary_nodes(V, 40), 500,
                    1e-4, 32, 1)
    _parity(ws, np.arange(0, 300, 3), 500, 32, walk_kernel=walk_kernel)
    # N = 1 and N = 3 (a row's walks run out at once), fewer rows than CTAs, p = 1, FP64
    xr = np.concatenate([W.disk_nodes(0.3, 0.9), [[0.0, 0.9995], [0.3, -0.2]]])
    for N, prec, pz in ((1, 64, 16), (3, 64, 1), (777, 32, 37)):
        wr = W.Workload("ragged", W.Domain(2, "ball", np.array([0.0, 0, 1])), xr, W.circle_nodes(pz), N, 1e-3, prec, 11)
        _parity(wr, np.arange(xr.shape[0]), N, prec, walk_kernel=walk_kernel, min_exit=0.99 if N < 10 else 0.999)
    # the disk workload in FP64 at full size
    wd = W.disk400(problem=False)
    rep, g, _ = _parity(wd, np.arange(0, 400, 7), 1000, 64, walk_kernel=walk_kernel)
    assert rep["exit_equal"] >= 0.9999
