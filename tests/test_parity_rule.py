"""The comparison rule of tests/parity.py checked on the CPU: the oracle's own rows pass it with
no divergent walk, and doctored copies of them (the kinds of mistake a GPU toolbox could make)
fail it -- a 1e-4 scale on every r^2 weight (every walk drifts), a scale on the matrices alone,
and exit cells moved for more than 0.1 % of the walks.  A few moved walks within the cap, with
the matrices moved consistently, still pass."""
import numpy as np
import pytest

from paper_2608_07017_b300 import workloads as W
from parity import compare_rows

N = 500


@pytest.fixture(scope="module")
def rows(oracle_lib):
    x = W.disk_nodes(0.3, 0.9)
    z = W.circle_nodes(24)
    prm = [0.0, 0.0, 1.0]
    orc = oracle_lib.walk_rows(2, "ball", prm, x, z, N, 1e-3, seed=6, records=True)
    r0 = 1.0 - np.linalg.norm(x, axis=1)
    return x, orc, r0


def _as_gpu(orc):
    rec = orc["records"]
    return dict(G=orc["G"].copy(), gradG=orc["gradG"].copy(), Hc=orc["Hc"].astype(np.uint32),
                gradH=orc["gradH"].copy(), walk_exit=rec["exit"].copy(), walk_steps=rec["steps"].copy(),
                walk_vhash=rec["vhash"].copy(), walk_mass=rec["gmass"].copy(), walk_xexit=rec["xexit"].copy())


def _compare(g, orc, x, r0, fp32=False):
    return compare_rows(g, orc, np.arange(x.shape[0]), N, 2, r0, fp32=fp32)


def test_identical_rows_pass_with_no_divergent_walk(rows):
    x, orc, r0 = rows
    rep = _compare(_as_gpu(orc), orc, x, r0)
    assert rep["ndiv"] == 0 and rep["exit_equal"] == 1.0 and rep["walks"] == x.shape[0] * N


def test_scaled_r2_weight_fails(rows):
    # a kernel that weights every source contribution r^2 by (1 + 1e-4): no binning changes, but
    # every walk's G mass drifts, and the drift class is capped like the others
    x, orc, r0 = rows
    g = _as_gpu(orc)
    g["walk_mass"] *= 1 + 1e-4
    g["G"] *= 1 + 1e-4
    g["gradG"] *= 1 + 1e-4
    with pytest.raises(AssertionError, match="walks diverge"):
        _compare(g, orc, x, r0)


def test_scaled_r2_weight_under_fp32_drift_fails(rows):
    # the same scale error while every stopping point is off by 2e-5 (FP32-like drift that makes
    # the per-walk and per-entry rounding bounds loose): the row sums still expose it
    x, orc, r0 = rows
    g = _as_gpu(orc)
    rng = np.random.default_rng(1)
    g["walk_xexit"] = g["walk_xexit"] + rng.choice([-2e-5, 2e-5], size=g["walk_xexit"].shape)
    rep = _compare(g, orc, x, r0, fp32=True)
    assert rep["ndiv"] == 0
    g["walk_mass"] *= 1 + 1e-4
    g["G"] *= 1 + 1e-4
    g["gradG"] *= 1 + 1e-4
    with pytest.raises(AssertionError, match="walks diverge|row sums"):
        _compare(g, orc, x, r0, fp32=True)


def test_scaled_matrix_fails(rows):
    # the records agree but the accumulated G is off by 3e-4 relative
    x, orc, r0 = rows
    g = _as_gpu(orc)
    g["G"] *= 1 + 3e-4
    with pytest.raises(AssertionError, match="G: "):
        _compare(g, orc, x, r0)


def _move_exits(orc, r0, count, rng):
    """Moves the exit cell of ``count`` walks to the neighbouring boundary cell, with Hc and
    gradH moved along (a consistent toolbox whose walks disagree with the oracle's)."""
    g = _as_gpu(orc)
    rec = orc["records"]
    nr, p = g["Hc"].shape
    flat = rng.choice(nr * N, size=count, replace=False)
    for f in flat:
        i, l = divmod(int(f), N)
        old = int(g["walk_exit"][i, l])
        new = (old + 1) % p
        g["walk_exit"][i, l] = new
        g["Hc"][i, old] -= 1
        g["Hc"][i, new] += 1
        for c in range(2):
            dH = 2.0 / r0[i] ** 2 * rec["w"][i, l, c] / N
            g["gradH"][c][i, old] -= dH
            g["gradH"][c][i, new] += dH
    return g


def test_moved_exit_cells_within_and_beyond_the_cap(rows):
    x, orc, r0 = rows
    walks = x.shape[0] * N
    rng = np.random.default_rng(0)
    few = max(1, int(0.0005 * walks))
    rep = _compare(_move_exits(orc, r0, few, rng), orc, x, r0)
    assert rep["n_exit"] == few and rep["ndiv"] == few
    many = int(0.002 * walks) + 1
    with pytest.raises(AssertionError, match="walks diverge"):
        _compare(_move_exits(orc, r0, many, rng), orc, x, r0)
