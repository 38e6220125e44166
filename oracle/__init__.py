"""Plain FP64 CPU oracle of the extended Walk-on-Spheres toolbox (test infrastructure only).

Nothing in the product path may import this package: only ``tests/``, the smoke check of
``__graft_entry__`` and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA library under ``paper_2608_07017_b300/``.

* ``wos_oracle.c`` -- Philox4x32-10, the samplers of Prop. 2.6, the distance functions, brute
  force Voronoi lookup, and the fused walk estimator of Algorithm 5 (eqs. Estimator_A/B/H/K),
  OpenMP over rows.  Loaded here through ctypes.
* ``solve.py`` -- the finite-dimensional systems of Sec. 3 (linear system eq. linear_q,
  Newton on the Euler-Lagrange residual of Sec. 3.2, Picard for the quasilinear case) with a
  textbook LU.

Parity status of each function is listed in ``solve.py`` and in the header of the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wos_oracle.c")
_LIB = os.path.join(_HERE, "liborcwos.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP) next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", _LIB, _SRC, "-lm"])
    return _LIB


class _Spec(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("sdf_kind", ctypes.c_int),
        ("sdf_params", ctypes.c_void_p), ("n_sdf_params", ctypes.c_int64),
        ("x", ctypes.c_void_p), ("n", ctypes.c_int64),
        ("y", ctypes.c_void_p), ("m", ctypes.c_int64),
        ("z", ctypes.c_void_p), ("p", ctypes.c_int64),
        ("walks", ctypes.c_int64), ("eps", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("max_steps", ctypes.c_int64),
        ("instance", ctypes.c_uint32),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        L.oracle_philox4x32_10.argtypes = [P, P, P]
        L.oracle_u01.argtypes = [ctypes.c_uint32]
        L.oracle_u01.restype = ctypes.c_double
        L.oracle_green_radius_2d.argtypes = [ctypes.c_double]
        L.oracle_green_radius_2d.restype = ctypes.c_double
        L.oracle_sdf.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int64, P]
        L.oracle_sdf.restype = ctypes.c_double
        L.oracle_nearest.argtypes = [ctypes.c_int, P, P, ctypes.c_int64]
        L.oracle_nearest.restype = ctypes.c_int64
        L.oracle_walk_rows.argtypes = [ctypes.POINTER(_Spec), P, ctypes.c_int64] + [P] * 14
        L.oracle_philox_batch.argtypes = [P, P, P, ctypes.c_int64]
        L.oracle_walk_rows.restype = ctypes.c_int
        L.oracle_cell_counts.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int64, P,
                                         ctypes.c_int64, P, P, ctypes.c_int64, ctypes.c_uint64,
                                         ctypes.c_uint32, P]
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


SDF_KINDS = {"ball": 0, "box": 1, "polygon": 2}


def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11): 4 counter words, 2 key words -> 4 words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox_batch(ctr, key):
    """Philox4x32-10 for many counters: ctr [count][4] -> out [count][4]."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros_like(c)
    lib().oracle_philox_batch(_ptr(c), _ptr(k), _ptr(out), c.shape[0])
    return out


def u01(x: int) -> float:
    return lib().oracle_u01(int(x) & 0xFFFFFFFF)


def green_radius_2d(u: float) -> float:
    """Inverse of F(t) = t^2 - t^2 ln t^2 (Prop. 2.6 (i.1))."""
    return lib().oracle_green_radius_2d(float(u))


def sdf(dim, kind, params, x) -> float:
    prm = np.ascontiguousarray(params, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    return lib().oracle_sdf(dim, SDF_KINDS[kind], _ptr(prm), prm.size, _ptr(xx))


def nearest(q, pts) -> int:
    qq = np.ascontiguousarray(q, dtype=np.float64)
    pp = np.ascontiguousarray(pts, dtype=np.float64)
    return lib().oracle_nearest(pp.shape[1], _ptr(qq), _ptr(pp), pp.shape[0])


def num_threads() -> int:
    return lib().oracle_num_threads()


def walk_rows(dim, kind, params, x, z, walks, eps, seed, rows=None, y=None, max_steps=10000,
              instance=0, records=False):
    """Toolbox rows for the node indices ``rows`` (default: all), Algorithm 5 with the
    readings listed in ``wos_oracle.c``.  Returns a dict with G [r][m], gradG [d][r][m],
    Hc [r][p] (int64 exit counts), gradH [d][r][p], steps, capped and, when ``records``,
    per-walk arrays (exit, steps, capped, gmass, gradmass, w, vhash, xexit) of shape [r][N](...)
    and Grsum (sum of r/(2dN) over the binnings of G, a rounding-bound diagnostic)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    y = x if y is None else np.ascontiguousarray(y, dtype=np.float64)
    prm = np.ascontiguousarray(params, dtype=np.float64)
    rows = np.arange(x.shape[0], dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nr, m, p, N = rows.size, y.shape[0], z.shape[0], int(walks)
    spec = _Spec(dim, SDF_KINDS[kind], _ptr(prm), prm.size, _ptr(x), x.shape[0], _ptr(y), m,
                 _ptr(z), p, N, float(eps), int(seed), int(max_steps), int(instance))
    G = np.zeros((nr, m)); gG = np.zeros((dim, nr, m))
    Hc = np.zeros((nr, p), dtype=np.int64); gH = np.zeros((dim, nr, p))
    stats = np.zeros(2, dtype=np.int64)
    Grs = np.zeros((nr, m)) if records else None
    rec = {}
    if records:
        rec = dict(exit=np.zeros((nr, N), np.int32), steps=np.zeros((nr, N), np.int32),
                   capped=np.zeros((nr, N), np.int8), gmass=np.zeros((nr, N)),
                   gradmass=np.zeros((nr, N, dim)), w=np.zeros((nr, N, dim)),
                   vhash=np.zeros((nr, N), np.uint32), xexit=np.zeros((nr, N, dim)))
    rc = lib().oracle_walk_rows(ctypes.byref(spec), _ptr(rows), nr, _ptr(G), _ptr(gG), _ptr(Hc), _ptr(gH),
                                _ptr(rec.get("exit")), _ptr(rec.get("steps")), _ptr(rec.get("capped")),
                                _ptr(rec.get("gmass")), _ptr(rec.get("gradmass")), _ptr(rec.get("w")),
                                _ptr(rec.get("vhash")), _ptr(rec.get("xexit")), _ptr(Grs), _ptr(stats))
    if rc != 0:
        raise ValueError("oracle_walk_rows: invalid input (a node outside the domain or bad dim)")
    out = dict(G=G, gradG=gG, Hc=Hc, gradH=gH, steps=int(stats[0]), capped=int(stats[1]), rows=rows)
    if records:
        out["records"] = rec
        out["Grsum"] = Grs
    return out


def domain_bbox(dim, kind, params):
    prm = np.asarray(params, dtype=np.float64)
    if kind == "ball":
        c, R = prm[:dim], prm[dim]
        return c - R, c + R
    if kind == "box":
        return prm[:dim].copy(), prm[dim:2 * dim].copy()
    v = prm.reshape(-1, 2)
    return v.min(axis=0), v.max(axis=0)


def cell_counts(dim, kind, params, y, nsamples, seed, instance=0):
    """Monte Carlo cell volumes: counts of uniform bounding-box samples inside D per nearest
    centre (lambda_i = counts_i / sum counts, Sec. 3.1)."""
    prm = np.ascontiguousarray(params, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    lo, hi = domain_bbox(dim, kind, prm)
    lo = np.ascontiguousarray(lo); hi = np.ascontiguousarray(hi)
    counts = np.zeros(y.shape[0], dtype=np.int64)
    lib().oracle_cell_counts(dim, SDF_KINDS[kind], _ptr(prm), prm.size, _ptr(y), y.shape[0],
                             _ptr(lo), _ptr(hi), int(nsamples), int(seed), int(instance), _ptr(counts))
    return counts
