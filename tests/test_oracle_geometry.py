"""Pins of the oracle's geometry: distance functions (eq. r), nearest-centre lookup (Voronoi
cells, Sec. 2.3) and Monte Carlo cell weights lambda_i (Sec. 3.1)."""
import math

import numpy as np
from scipy.spatial import cKDTree

from paper_2608_07017_b300 import workloads as W


def test_ball_and_box_distance(oracle_lib):
    rng = np.random.default_rng(0)
    for _ in range(50):
        x = rng.uniform(-0.7, 0.7, 2)
        assert abs(oracle_lib.sdf(2, "ball", [0, 0, 1], x) - (1 - np.hypot(*x))) < 1e-15
        x3 = rng.uniform(-0.5, 0.5, 3)
        assert abs(oracle_lib.sdf(3, "ball", [0.1, 0, 0, 1.5], x3)
                   - (1.5 - np.linalg.norm(x3 - [0.1, 0, 0]))) < 1e-15
        y = rng.uniform(0, 1, 2)
        assert abs(oracle_lib.sdf(2, "box", [0, 0, 1, 1], y) - min(y[0], y[1], 1 - y[0], 1 - y[1])) < 1e-15


def test_polygon_distance_matches_box_and_sign(oracle_lib):
    sq = np.array([0, 0, 1, 0, 1, 1, 0, 1], dtype=float)
    rng = np.random.default_rng(1)
    for _ in range(100):
        y = rng.uniform(0.001, 0.999, 2)
        assert abs(oracle_lib.sdf(2, "polygon", sq, y) - min(y[0], y[1], 1 - y[0], 1 - y[1])) < 1e-14
    assert oracle_lib.sdf(2, "polygon", sq, [1.5, 0.5]) < 0
    assert abs(oracle_lib.sdf(2, "polygon", sq, [1.5, 0.5]) + 0.5) < 1e-15
    # a regular 64-gon inscribed in the unit circle: distance = apothem - |x| on the bisectors
    V = W.star_polygon(3, 64, amp=0.0)
    apo = math.cos(math.pi / 64)
    th = 2 * math.pi * (0.5) / 64
    for rr in (0.0, 0.3, 0.9):
        x = rr * np.array([math.cos(th), math.sin(th)])
        assert abs(oracle_lib.sdf(2, "polygon", V.ravel(), x) - (apo - rr)) < 1e-12


def test_nearest_matches_kdtree_and_breaks_ties_low(oracle_lib):
    rng = np.random.default_rng(2)
    pts = rng.uniform(-1, 1, (300, 2))
    tree = cKDTree(pts)
    q = rng.uniform(-1, 1, (500, 2))
    _, idx = tree.query(q)
    for k in range(q.shape[0]):
        assert oracle_lib.nearest(q[k], pts) == idx[k]
    dup = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 0.0]])
    assert oracle_lib.nearest([0.2, 0.0], dup) == 0
    assert oracle_lib.nearest([0.5, 0.0], dup) == 0          # exact tie between 0 and 1
    pts3 = rng.uniform(-1, 1, (200, 3))
    q3 = rng.uniform(-1, 1, (200, 3))
    _, idx3 = cKDTree(pts3).query(q3)
    assert all(oracle_lib.nearest(q3[k], pts3) == idx3[k] for k in range(200))


def test_cell_weights_box_grid_and_disk_area(oracle_lib):
    x = W.square_nodes(4)
    K = 400000
    c = oracle_lib.cell_counts(2, "box", [0, 0, 1, 1], x, K, seed=3)
    assert c.sum() == K                                      # every box sample is inside
    p = 1.0 / 16
    chi2 = np.sum((c - K * p) ** 2 / (K * p))
    assert chi2 < 16 + 6 * math.sqrt(2 * 15)
    # disk: fraction of the bounding-box samples that are inside = pi/4
    y = W.disk_nodes(0.25, 0.95)
    cd = oracle_lib.cell_counts(2, "ball", [0, 0, 1], y, K, seed=4)
    frac = cd.sum() / K
    assert abs(frac - math.pi / 4) < 4 * math.sqrt(frac * (1 - frac) / K)
    # polygon domain of a star: inside fraction equals the shoelace area / bbox area
    V = W.star_polygon(5)
    cp = oracle_lib.cell_counts(2, "polygon", V.ravel(), V * 0.5, K, seed=5)
    area = 0.5 * abs(np.sum(V[:, 0] * np.roll(V[:, 1], -1) - np.roll(V[:, 0], -1) * V[:, 1]))
    lo, hi = V.min(0), V.max(0)
    q = area / np.prod(hi - lo)
    assert abs(cp.sum() / K - q) < 4 * math.sqrt(q * (1 - q) / K)
