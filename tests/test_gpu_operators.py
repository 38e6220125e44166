"""Operator estimates on the GPU (Sec. 3.1, after eq. linear_inversion) against the oracle's.

Same FP64 toolbox on both sides (the oracle's matrices loaded into the library); the estimates
are the solve map of the shifted linear system, so the bar is the linear solve's: 1e-9 relative
to the largest entry (FP64 on both sides, only the order of rounding differs; the mixed path is
refined to FP64 and compared with the oracle run at the mixed path's own shift).
"""
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


def _coefs(w):
    b = np.stack([np.sin(3 * w.x[:, 0]), np.cos(2 * w.x[:, 1])], axis=1)
    c = 1.0 + w.x[:, 0] ** 2
    return b, c


@pytest.mark.parametrize("lower", [False, True])
def test_operators_fp64_match_oracle(disk, lower):
    w, tb, lam, gtb = disk
    b, c = _coefs(w) if lower else (None, None)
    GL, HL, rep = gtb.operators(w.problem.A, b, c)
    ref = S.operators(tb, lam, w.problem.A, b, c)
    assert abs(rep["alpha"] - ref["alpha"]) <= 1e-12 * ref["alpha"]
    assert _rel(GL, ref["GL"]) < 1e-9
    assert _rel(HL, ref["HL"]) < 1e-9


def test_operators_mixed_match_oracle(disk):
    w, tb, lam, gtb = disk
    b, c = _coefs(w)
    GL, HL, rep = gtb.operators(w.problem.A, b, c, mode="mixed")
    ref = S.operators(tb, lam, w.problem.A, b, c, alpha=rep["alpha"])
    assert _rel(GL, ref["GL"]) < 1e-9
    assert _rel(HL, ref["HL"]) < 1e-9


def test_operators_are_the_solve_map(disk):
    w, tb, lam, gtb = disk
    b, c = _coefs(w)
    GL, HL, _ = gtb.operators(w.problem.A, b, c)
    rng = np.random.default_rng(3)
    f = rng.normal(size=(3, gtb.n))
    g = rng.normal(size=(3, gtb.p))
    u, _, _ = gtb.solve(w.problem.A, f, g, b=b, c=c)
    assert _rel((GL @ f.T + HL @ g.T).T, u) < 1e-9
    # one output only (the FP64 path sums with atomics, so equal up to rounding, not bitwise)
    GL1, HL1, _ = gtb.operators(w.problem.A, b, c, want=("HL",))
    assert GL1 is None and _rel(HL1, HL) < 1e-12


def test_operators_ragged_sizes():
    from paper_2608_07017_b300 import build
    build.build()
    rng = np.random.default_rng(4)
    for n, p in ((1, 3), (70, 1), (197, 41)):
        x = rng.uniform(-0.6, 0.6, size=(n, 2))
        z = rng.normal(size=(p, 2))
        z /= np.linalg.norm(z, axis=1, keepdims=True)
        tb = dict(G=rng.random((n, n)) * 0.01 + np.eye(n) * 0.05, gradG=rng.normal(size=(2, n, n)) * 0.1,
                  H=rng.random((n, p)) / p, gradH=rng.normal(size=(2, n, p)))
        lam = rng.random(n) + 0.5
        lam /= lam.sum()
        A = np.tile(np.eye(2), (n, 1, 1))
        gtb = ewos.toolbox_from_host(2, x, z, tb["G"], tb["gradG"], tb["H"], tb["gradH"], lam, precision=64)
        GL, HL, _ = gtb.operators(A)
        gtb.close()
        ref = S.operators(tb, lam, A)
        assert GL.shape == (n, n) and HL.shape == (n, p)
        assert _rel(GL, ref["GL"]) < 1e-9 and _rel(HL, ref["HL"]) < 1e-9


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_operators_in_chunks_match_oracle(mode):
    """m = 1400: the columns go in several chunks (1024 in mixed mode, 32 in FP64 mode), the
    chunks after the first on the first chunk's factors."""
    from paper_2608_07017_b300 import build
    build.build()
    rng = np.random.default_rng(9)
    n, p = 1400, 100
    x = rng.uniform(-0.6, 0.6, size=(n, 2))
    z = rng.normal(size=(p, 2))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    tb = dict(G=rng.random((n, n)) * 1e-3, gradG=rng.normal(size=(2, n, n)) * 0.05,
              H=rng.random((n, p)) / p, gradH=rng.normal(size=(2, n, p)) * 0.1)
    lam = rng.random(n) + 0.5
    lam /= lam.sum()
    A = np.tile(np.array([[1.2, 0.1], [0.1, 0.9]]), (n, 1, 1))
    gtb = ewos.toolbox_from_host(2, x, z, tb["G"], tb["gradG"], tb["H"], tb["gradH"], lam, precision=64)
    GL, HL, rep = gtb.operators(A, mode=mode)
    gtb.close()
    ref = S.operators(tb, lam, A, alpha=rep["alpha"])
    assert _rel(GL, ref["GL"]) < 1e-9 and _rel(HL, ref["HL"]) < 1e-9


def test_operators_reject_nonlinear(disk):
    w, tb, lam, gtb = disk
    pb = ewos._Problem(w.problem.A.ctypes.data, None, None, None, None, 0, ewos.NL["semilinear"], None, 0, 0,
                       -1.0, 0.0, 0, 0, None, 0, 0)
    out = np.zeros((gtb.n, gtb.n))
    import ctypes
    assert ewos.lib().ewos_operators(gtb._h, ctypes.byref(pb), out.ctypes.data, None, 0, None) == ewos.EINVAL
