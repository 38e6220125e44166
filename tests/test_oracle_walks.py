"""Pins of the oracle's toolbox estimator (Algorithm 5, eqs. Estimator_A/B/H/K) against closed
forms of potential theory, none of which the oracle computes itself:

* G 1 = (1 - |x|^2)/(2d) on the unit ball (E tau, Prop. 2.2 (i) with f = 1), and the Fourier
  series of the torsion function on the unit square;
* gradG 1 = -x/d on the unit ball (Prop. 2.2 (ii));
* H reproduces harmonic polynomials and gradH reproduces gradients of linear functions
  (Prop. 2.4), with every H row summing to N exactly;
* exit-cell frequencies follow the Poisson kernel of the disk (harmonic measure, proof of
  Prop. 2.4) -- chi-square test;
* entries of G and gradG equal the integrals of the disk's Dirichlet Green function (and its
  x-gradient) over the Voronoi cells, computed by independent Monte Carlo quadrature.

Tolerances: 4 standard errors plus the deterministic eps-shell and binning bounds stated at
each test.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats
from scipy.spatial import cKDTree

from paper_2608_07017_b300 import workloads as W

DISK = dict(dim=2, kind="ball", params=[0.0, 0.0, 1.0])


@pytest.fixture(scope="module")
def disk_run(oracle_lib):
    w = W.disk400(problem=False)
    rows = np.arange(0, 400, 9)
    r = oracle_lib.walk_rows(2, "ball", w.domain.params, w.x, w.z, 4000, 1e-3, seed=5, rows=rows,
                             records=True)
    return w, r


def test_h_rows_sum_to_walk_count(disk_run):
    _, r = disk_run
    assert np.all(r["Hc"].sum(1) == 4000)
    assert r["capped"] == 0


def test_g_times_one_is_expected_exit_time(disk_run):
    w, r = disk_run
    x = w.x[r["rows"]]
    est = r["G"].sum(1)
    ex = (1 - (x ** 2).sum(1)) / 4
    se = r["records"]["gmass"].std(1) / math.sqrt(4000)
    eps_bias = 1e-3 / 2                       # E(1-|X|^2)/(2d) from the eps-shell
    assert np.all(np.abs(est - ex) <= 4 * se + eps_bias)
    # G 1 must not be A 1 = 2 G 1 (reading: G = A/2)
    assert np.all(np.abs(est - 2 * ex) > 4 * se + eps_bias)


def test_gradg_times_one(disk_run):
    w, r = disk_run
    x = w.x[r["rows"]]
    r0 = 1 - np.hypot(x[:, 0], x[:, 1])
    est = r["gradG"].sum(2).T
    se = r["records"]["gradmass"].std(1) / math.sqrt(4000)
    bias = 1e-3 / (2 * r0)
    assert np.all(np.abs(est - (-x / 2)) <= 4 * se + bias[:, None])


@pytest.mark.parametrize("name,g,lip", [
    ("x", lambda p: p[:, 0], 1.0),
    ("x2-y2", lambda p: p[:, 0] ** 2 - p[:, 1] ** 2, 2.0),
    ("xy", lambda p: p[:, 0] * p[:, 1], 1.0),
    ("re z^3", lambda p: p[:, 0] ** 3 - 3 * p[:, 0] * p[:, 1] ** 2, 3.0),
])
def test_h_reproduces_harmonic_polynomials(disk_run, name, g, lip):
    w, r = disk_run
    x = w.x[r["rows"]]
    H = r["Hc"] / 4000.0
    est = H @ g(w.z)
    per_walk = g(w.z)[r["records"]["exit"]]
    se = per_walk.std(1) / math.sqrt(4000)
    bind = lip * (1e-3 + math.pi / w.z.shape[0])    # |z_cell - X_exit| <= eps + half arc
    assert np.all(np.abs(est - g(x)) <= 4 * se + bind), name


def test_gradh_reproduces_linear_gradients(disk_run):
    w, r = disk_run
    x = w.x[r["rows"]]
    r0 = 1 - np.hypot(x[:, 0], x[:, 1])
    rec = r["records"]
    for a in (np.array([1.0, 0.0]), np.array([0.3, -0.7])):
        gz = w.z @ a
        est = np.stack([r["gradH"][k] @ gz for k in range(2)], 1)
        per_walk = (2 / r0[:, None, None] ** 2) * gz[rec["exit"]][:, :, None] * rec["w"]
        se = per_walk.std(1) / math.sqrt(4000)
        bind = 2 / r0 * np.linalg.norm(a) * (1e-3 + math.pi / w.z.shape[0])
        assert np.all(np.abs(est - a[None, :]) <= 4 * se + bind[:, None])
    # grad H 1 = 0 exactly in expectation (no binning error for a constant)
    est0 = r["gradH"].sum(2).T
    per0 = (2 / r0[:, None, None] ** 2) * rec["w"]
    se0 = per0.std(1) / math.sqrt(4000)
    assert np.all(np.abs(est0) <= 4 * se0 + 1e-12)


def _poisson_arc(x, a, b):
    rr, ph = np.hypot(*x), math.atan2(x[1], x[0])
    f = lambda t: (1 - rr * rr) / (2 * math.pi * (1 - 2 * rr * math.cos(t - ph) + rr * rr))
    return integrate.quad(f, a, b, limit=200)[0]


def test_exit_cells_follow_the_poisson_kernel(oracle_lib):
    p = 32
    z = W.circle_nodes(p)
    x = np.array([[0.0, 0.0], [0.5, 0.2], [-0.3, -0.6], [0.85, 0.0]])
    N = 20000
    r = oracle_lib.walk_rows(2, "ball", [0, 0, 1], x, z, N, 1e-4, seed=9)
    for i in range(x.shape[0]):
        probs = np.array([_poisson_arc(x[i], 2 * math.pi * (j - 0.5) / p, 2 * math.pi * (j + 0.5) / p)
                          for j in range(p)])
        assert abs(probs.sum() - 1) < 1e-9
        obs = r["Hc"][i]
        chi2 = np.sum((obs - N * probs) ** 2 / (N * probs))
        assert stats.chi2.sf(chi2, p - 1) > 1e-4


def _green_disk(x, Y):
    d1 = np.linalg.norm(Y - x, axis=1)
    ny = np.linalg.norm(Y, axis=1)
    ys = Y / (ny ** 2)[:, None]
    d2 = np.linalg.norm(x - ys, axis=1)
    return (1 / (2 * math.pi)) * (-np.log(d1) + np.log(ny) + np.log(d2))


def _green_disk_grad(x, Y):
    ny2 = (Y ** 2).sum(1)
    ys = Y / ny2[:, None]
    a = x - Y
    b = x - ys
    return (1 / (2 * math.pi)) * (-a / (a ** 2).sum(1)[:, None] + b / (b ** 2).sum(1)[:, None])


def test_g_and_gradg_entries_match_green_function_quadrature(oracle_lib):
    y = W.disk_nodes(0.2, 0.9)                       # coarse V centres: many hits per cell
    z = W.circle_nodes(64)
    rows = np.array([0, len(y) // 3, len(y) // 2, len(y) - 5])
    B, N = 24, 2500
    Gs, GGs = [], []
    for bt in range(B):
        r = oracle_lib.walk_rows(2, "ball", [0, 0, 1], y, z, N, 1e-4, seed=100 + bt, rows=rows)
        Gs.append(r["G"]); GGs.append(r["gradG"])
    Gs, GGs = np.array(Gs), np.array(GGs)
    Gm, Gse = Gs.mean(0), Gs.std(0, ddof=1) / math.sqrt(B)
    GGm, GGse = GGs.mean(0), GGs.std(0, ddof=1) / math.sqrt(B)
    # independent quadrature: uniform points in the disk, Green function weight, nearest centre
    rng = np.random.default_rng(77)
    K = 3_000_000
    rad = np.sqrt(rng.random(K)); th = 2 * math.pi * rng.random(K)
    Y = np.stack([rad * np.cos(th), rad * np.sin(th)], 1)
    cell = cKDTree(y).query(Y)[1]
    m = y.shape[0]
    zs, zmax = [], 0.0
    for t, i in enumerate(rows):
        gv = math.pi * _green_disk(y[i], Y)
        Q = np.bincount(cell, weights=gv, minlength=m) / K
        Q2 = np.bincount(cell, weights=gv * gv, minlength=m) / K
        Qse = np.sqrt(np.maximum(Q2 - Q * Q, 0) / K)
        zz = (Gm[t] - Q) / np.sqrt(Gse[t] ** 2 + Qse ** 2 + 1e-30)
        zs.append(zz)
        # gradient entries away from the node's own neighbourhood (finite quadrature variance)
        gg = math.pi * _green_disk_grad(y[i], Y)
        far = np.linalg.norm(y - y[i], axis=1) > 0.45
        for k in range(2):
            Qk = np.bincount(cell, weights=gg[:, k], minlength=m) / K
            Qk2 = np.bincount(cell, weights=gg[:, k] ** 2, minlength=m) / K
            Qkse = np.sqrt(np.maximum(Qk2 - Qk * Qk, 0) / K)
            zk = (GGm[k, t] - Qk) / np.sqrt(GGse[k, t] ** 2 + Qkse ** 2 + 1e-30)
            zs.append(zk[far])
    allz = np.concatenate(zs)
    assert np.mean(allz ** 2) < 1.6
    assert np.max(np.abs(allz)) < 7.0


def _square_torsion(x, y, terms=199):
    out = 0.0
    for mm in range(1, terms + 1, 2):
        for nn in range(1, terms + 1, 2):
            out += 16 / (math.pi ** 4 * mm * nn * (mm * mm + nn * nn)) * math.sin(mm * math.pi * x) * math.sin(nn * math.pi * y)
    return out


def test_square_g_times_one_is_torsion_series(oracle_lib):
    x = np.array([[0.5, 0.5], [0.2, 0.7], [0.1, 0.1], [0.9, 0.4]])
    z = W.square_boundary_nodes(16)
    N = 8000
    r = oracle_lib.walk_rows(2, "box", [0, 0, 1, 1], x, z, N, 1e-4, seed=3, records=True)
    est = r["G"].sum(1)
    se = r["records"]["gmass"].std(1) / math.sqrt(N)
    ex = np.array([_square_torsion(*p) for p in x])
    assert np.all(np.abs(est - ex) <= 4 * se + 1e-4)


def test_ball3d_closed_forms(oracle_lib):
    y = W.ball_nodes(300, seed=4)[0]
    z = W.fibonacci_sphere(200)
    rows = np.arange(0, 300, 25)
    N = 3000
    r = oracle_lib.walk_rows(3, "ball", [0, 0, 0, 1], y, z, N, 1e-4, seed=8, rows=rows, records=True)
    x = y[rows]
    r0 = 1 - np.linalg.norm(x, axis=1)
    rec = r["records"]
    assert np.all(r["Hc"].sum(1) == N)
    est = r["G"].sum(1)
    se = rec["gmass"].std(1) / math.sqrt(N)
    assert np.all(np.abs(est - (1 - (x ** 2).sum(1)) / 6) <= 4 * se + 1e-4 / 3)
    gest = r["gradG"].sum(2).T
    gse = rec["gradmass"].std(1) / math.sqrt(N)
    assert np.all(np.abs(gest + x / 3) <= 4 * gse + (1e-4 / (3 * r0))[:, None])
    # binning radius of the Fibonacci cells, measured on the sphere
    rng = np.random.default_rng(0)
    S = rng.normal(size=(200000, 3)); S /= np.linalg.norm(S, axis=1)[:, None]
    cell_rad = cKDTree(z).query(S)[0].max()
    for g, lip in ((lambda p: p[:, 0] * p[:, 1], 1.0), (lambda p: p[:, 0] ** 2 - p[:, 2] ** 2, 2.0)):
        H = r["Hc"] / N
        per = g(z)[rec["exit"]]
        se = per.std(1) / math.sqrt(N)
        assert np.all(np.abs(H @ g(z) - g(x)) <= 4 * se + lip * (1e-4 + cell_rad))


def test_rows_are_independent_and_seeded(oracle_lib):
    w = W.disk400(problem=False)
    a = oracle_lib.walk_rows(2, "ball", w.domain.params, w.x, w.z, 200, 1e-3, seed=1, rows=[5, 17, 230])
    b = oracle_lib.walk_rows(2, "ball", w.domain.params, w.x, w.z, 200, 1e-3, seed=1, rows=[230, 5])
    assert np.array_equal(a["G"][2], b["G"][0]) and np.array_equal(a["G"][0], b["G"][1])
    assert np.array_equal(a["Hc"][2], b["Hc"][0])
    c = oracle_lib.walk_rows(2, "ball", w.domain.params, w.x, w.z, 200, 1e-3, seed=2, rows=[5])
    assert not np.array_equal(a["G"][0], c["G"][0])


def test_step_cap_is_reported(oracle_lib):
    w = W.disk400(problem=False)
    r = oracle_lib.walk_rows(2, "ball", w.domain.params, w.x, w.z, 100, 1e-12, seed=1, rows=[0],
                             max_steps=3, records=True)
    assert r["capped"] == 100
    assert np.all(r["records"]["steps"] == 3)
    assert np.all(r["Hc"].sum(1) == 100)
