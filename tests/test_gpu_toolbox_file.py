"""Toolbox files on the GPU: a toolbox written with ewos_toolbox_save and read back with
ewos_toolbox_load is bit-identical (every array, the shape and the build report) and solves to the
same result, for a built FP32 toolbox with exit counts, a toolbox made from FP64 matrices (no
counts) and a toolbox with a separate V-partition (m != n)."""
import numpy as np
import pytest

from paper_2608_07017_b300 import ewos
from paper_2608_07017_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2608_07017_b300 import build
    build.build()


def _same_arrays(a, b, names):
    for name in names:
        x, y = a.get(name), b.get(name)
        assert x.dtype == y.dtype and x.shape == y.shape, name
        assert np.array_equal(x, y), name


def _round_trip(tb, path):
    tb.save(path)
    return ewos.load_toolbox(path)


def test_built_fp32_toolbox_round_trip(tmp_path):
    x = W.square_nodes(12)
    z = W.square_boundary_nodes(8)
    tb = ewos.build_toolbox("box", 2, [0, 0, 1, 1], x, z, 300, 1e-4, seed=3, precision=32, cell_samples=100000)
    tb2 = _round_trip(tb, tmp_path / "square.ewtb")
    _same_arrays(tb, tb2, ("G", "gradG", "H", "gradH", "Hc", "lambda"))
    r1, r2 = tb.report(), tb2.report()
    assert r1["walks"] == r2["walks"] and r1["steps"] == r2["steps"] and r1["capped"] == r2["capped"]
    pb = W.make_problem("square", x, z)
    u1, _, _ = tb.solve(pb.A, pb.f, pb.g, b=pb.b, mode="mixed")
    u2, _, _ = tb2.solve(pb.A, pb.f, pb.g, b=pb.b, mode="mixed")
    # (the refinement's FP64 reductions add their partial sums by atomics in no fixed order, so
    # two solves agree to rounding, well inside the refinement tolerance)
    assert np.linalg.norm(u1 - u2) <= 1e-9 * np.linalg.norm(u1)
    tb.close()
    tb2.close()


def test_fp64_matrix_toolbox_round_trip(tmp_path):
    rng = np.random.default_rng(4)
    x = W.square_nodes(9)
    z = W.square_boundary_nodes(5)
    n, p = x.shape[0], z.shape[0]
    G = rng.normal(size=(n, n))
    gradG = rng.normal(size=(2, n, n))
    H = rng.uniform(size=(n, p))
    gradH = rng.normal(size=(2, n, p))
    lam = np.full(n, 1.0 / n)
    tb = ewos.toolbox_from_host(2, x, z, G, gradG, H, gradH, lam, precision=64)
    tb2 = _round_trip(tb, tmp_path / "matrices.ewtb")
    _same_arrays(tb, tb2, ("G", "gradG", "H", "gradH", "lambda"))
    assert np.array_equal(tb2.get("G"), G)
    tb.close()
    tb2.close()


def test_v_partition_toolbox_round_trip(tmp_path):
    x = W.disk_nodes(0.15, 0.9)
    y = W.disk_nodes(0.22, 0.9)
    z = W.circle_nodes(24)
    tb = ewos.build_toolbox("ball", 2, [0, 0, 1], x, z, 200, 1e-3, seed=2, precision=32, cell_samples=100000, y=y)
    tb2 = _round_trip(tb, tmp_path / "vpart.ewtb")
    assert tb2.get("G").shape == (x.shape[0], y.shape[0])
    _same_arrays(tb, tb2, ("G", "gradG", "H", "gradH", "Hc", "lambda"))
    tb.close()
    tb2.close()
