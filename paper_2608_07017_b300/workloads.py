"""Seeded synthetic workloads: node sets, domains and manufactured problems.

This module holds input generators only (no step of the method): it is shared by the tests,
the benchmark and the oracle calls.  Node layouts follow the shapes of the paper's toolboxes
(Sec. 3.3, eqs. unit disk points / unit square points: cell-centred grids, equispaced boundary
centres) at the sizes of the workloads below; all randomness comes from numpy's PCG64 seeded
explicitly.

Workloads (names used by the tests and the benchmark):
  disk400      2D unit disk, 400 interior nodes (half-offset grid, spacing 0.0835, |x| < 0.95),
               128 equispaced boundary nodes, 1000 walks/node, eps 1e-3, FP64 walks.
  square4096   2D unit square, 64 x 64 cell-centred interior nodes, 4 x 128 cell-centred
               boundary nodes, 10^4 walks/node, eps 1e-4, FP32 walks.
  ball8000     3D unit ball, 8000 interior nodes (jittered cubic lattice), 2000 boundary nodes
               (Fibonacci sphere), 10^4 walks/node, eps 1e-4, FP32 walks.
  stars32      32 star-shaped polygons (64 edges, radius 1 + 0.2 cos(k theta), k in 3..7),
               n log-uniform in [256, 4096], p = n/8, 2000 walks/node, eps 1e-4, FP32 walks.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Domain:
    dim: int
    kind: str                      # "ball" | "box" | "polygon"
    params: np.ndarray             # ball: centre, radius; box: lo, hi; polygon: x0,y0,x1,y1,...

    def bbox(self):
        p = self.params
        if self.kind == "ball":
            return p[: self.dim] - p[self.dim], p[: self.dim] + p[self.dim]
        if self.kind == "box":
            return p[: self.dim].copy(), p[self.dim: 2 * self.dim].copy()
        v = p.reshape(-1, 2)
        return v.min(axis=0), v.max(axis=0)


@dataclass
class Problem:
    """-div(A grad u) + b.grad u + c u + N(u) = f, u = g on the boundary; N(u) = sum nl[k] u^k,
    or A(u) = (sum kappa[k] u^k) A for the quasilinear case."""
    A: np.ndarray                  # [n][d][d]
    b: np.ndarray | None           # [n][d]
    c: np.ndarray | None           # [n]
    f: np.ndarray                  # [n]
    g: np.ndarray                  # [p]
    u_star: np.ndarray             # [n] manufactured solution at the nodes
    nl: list | None = None         # semilinear polynomial coefficients
    kappa: list | None = None      # quasilinear polynomial coefficients
    kind: str = "linear"           # "linear" | "semilinear" | "quasilinear"


@dataclass
class Workload:
    name: str
    domain: Domain
    x: np.ndarray                  # [n][d] interior nodes (W and V centres)
    z: np.ndarray                  # [p][d] boundary nodes (Gamma centres)
    walks: int
    eps: float
    precision: int                 # 32 | 64
    seed: int = 0
    problem: Problem | None = None
    lam: np.ndarray | None = None  # exact cell weights when known (cell-centred box grids)
    meta: dict = field(default_factory=dict)


# ------------------------------------------------------------------ node sets

def disk_nodes(h=0.0835, rmax=0.95):
    k = int(math.ceil(rmax / h)) + 1
    t = (np.arange(-k, k) + 0.5) * h
    X, Y = np.meshgrid(t, t, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel()], axis=1)
    keep = np.hypot(P[:, 0], P[:, 1]) < rmax
    return P[keep]


def circle_nodes(p, R=1.0):
    th = 2.0 * np.pi * np.arange(p) / p
    return np.stack([R * np.cos(th), R * np.sin(th)], axis=1)


def square_nodes(k):
    t = (np.arange(k) + 0.5) / k
    X, Y = np.meshgrid(t, t, indexing="ij")
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def square_boundary_nodes(per_side):
    t = (np.arange(per_side) + 0.5) / per_side
    zeros, ones = np.zeros_like(t), np.ones_like(t)
    return np.concatenate([
        np.stack([t, zeros], 1), np.stack([ones, t], 1),
        np.stack([t[::-1], ones], 1), np.stack([zeros, t[::-1]], 1)])


def ball_nodes(n, seed=1):
    """Jittered cubic lattice in the unit ball: spacing h chosen by bisection so that at least
    n lattice points with jitter U(-h/4, h/4)^3 lie at distance > h/4 from the sphere; the
    surplus is dropped uniformly at random."""
    rng = np.random.default_rng(seed)

    def gen(h):
        k = int(math.ceil(1.0 / h)) + 1
        t = np.arange(-k, k + 1) * h
        X, Y, Z = np.meshgrid(t, t, t, indexing="ij")
        P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
        return P

    lo, hi = 0.02, 0.5
    for _ in range(60):
        h = 0.5 * (lo + hi)
        P = gen(h)
        cnt = np.count_nonzero(np.linalg.norm(P, axis=1) < 1.0 - h / 2)
        if cnt >= n:
            lo = h
        else:
            hi = h
    h = lo
    P = gen(h)
    P = P + rng.uniform(-h / 4, h / 4, size=P.shape)
    P = P[np.linalg.norm(P, axis=1) < 1.0 - h / 4]
    if P.shape[0] > n:
        P = P[np.sort(rng.choice(P.shape[0], n, replace=False))]
    return P, h


def fibonacci_sphere(p):
    k = np.arange(p)
    zc = 1.0 - (2.0 * k + 1.0) / p
    ph = k * np.pi * (3.0 - math.sqrt(5.0))
    rho = np.sqrt(1.0 - zc * zc)
    return np.stack([rho * np.cos(ph), rho * np.sin(ph), zc], 1)


def star_polygon(kfold, nv=64, amp=0.2):
    th = 2.0 * np.pi * np.arange(nv) / nv
    rad = 1.0 + amp * np.cos(kfold * th)
    return np.stack([rad * np.cos(th), rad * np.sin(th)], 1)


def _inside_polygon(P, V):
    inside = np.zeros(P.shape[0], dtype=bool)
    nv = V.shape[0]
    for e in range(nv):
        a, b = V[e], V[(e + 1) % nv]
        cond = (a[1] > P[:, 1]) != (b[1] > P[:, 1])
        with np.errstate(divide="ignore", invalid="ignore"):
            xc = a[0] + (P[:, 1] - a[1]) / (b[1] - a[1]) * (b[0] - a[0])
        inside ^= cond & (P[:, 0] < xc)
    return inside


def _dist_polygon(P, V):
    best = np.full(P.shape[0], np.inf)
    nv = V.shape[0]
    for e in range(nv):
        a, b = V[e], V[(e + 1) % nv]
        ab = b - a
        t = np.clip(((P - a) @ ab) / (ab @ ab), 0.0, 1.0)
        d = np.linalg.norm(P - a - t[:, None] * ab, axis=1)
        best = np.minimum(best, d)
    return best


def star_nodes(V, n, rng):
    """Jittered grid inside the polygon (spacing from the area), surplus dropped at random."""
    area = 0.5 * abs(np.sum(V[:, 0] * np.roll(V[:, 1], -1) - np.roll(V[:, 0], -1) * V[:, 1]))
    h = math.sqrt(area / (n * 1.15))
    for _ in range(20):
        lo, hi = V.min(0) - h, V.max(0) + h
        tx = np.arange(lo[0], hi[0], h)
        ty = np.arange(lo[1], hi[1], h)
        X, Y = np.meshgrid(tx, ty, indexing="ij")
        P = np.stack([X.ravel(), Y.ravel()], 1) + rng.uniform(-h / 4, h / 4, size=(X.size, 2))
        keep = _inside_polygon(P, V)
        keep[keep] = _dist_polygon(P[keep], V) > h / 4
        P = P[keep]
        if P.shape[0] >= n:
            return P[np.sort(rng.choice(P.shape[0], n, replace=False))]
        h *= 0.95
    raise RuntimeError("star_nodes: could not place nodes")


def polygon_boundary_nodes(V, p):
    seg = np.roll(V, -1, axis=0) - V
    L = np.linalg.norm(seg, axis=1)
    cum = np.concatenate([[0.0], np.cumsum(L)])
    s = (np.arange(p) + 0.5) * cum[-1] / p
    e = np.searchsorted(cum, s, side="right") - 1
    t = (s - cum[e]) / L[e]
    return V[e] + t[:, None] * seg[e]


# ------------------------------------------------------------------ manufactured problems

def _manufactured(dim, u_expr, A_expr, b_expr=None, c_expr=None, nl=None, kappa=None):
    """Symbolic f = -div(kappa(u) A grad u) + b.grad u + c u + N(u) for a manufactured u."""
    import sympy as sp
    xs = sp.symbols("x0:%d" % dim)
    u = u_expr(*xs)
    A = sp.Matrix(A_expr(*xs))
    kap = 1 if kappa is None else sum(a * u ** k for k, a in enumerate(kappa))
    grad = sp.Matrix([sp.diff(u, v) for v in xs])
    flux = kap * (A * grad)
    f = -sum(sp.diff(flux[i], xs[i]) for i in range(dim))
    if b_expr is not None:
        bb = b_expr(*xs)
        f += sum(bb[i] * grad[i] for i in range(dim))
    if c_expr is not None:
        f += c_expr(*xs) * u
    if nl is not None:
        f += sum(a * u ** k for k, a in enumerate(nl))
    lam = lambda e: sp.lambdify(xs, e, "numpy")
    fu, ff = lam(u), lam(f)
    fA = [[lam(A[i, j]) for j in range(dim)] for i in range(dim)]
    fb = None if b_expr is None else [[lam(e)] for e in b_expr(*xs)]
    fc = None if c_expr is None else lam(c_expr(*xs))
    return fu, ff, fA, fb, fc


def _eval(fn, P, shape=None):
    cols = [P[:, k] for k in range(P.shape[1])]
    if shape is None:
        return np.broadcast_to(np.asarray(fn(*cols), dtype=np.float64), (P.shape[0],)).copy()
    arr = np.empty((P.shape[0],) + shape)
    for idx in np.ndindex(*shape):
        e = fn[idx[0]][idx[1]]
        arr[(slice(None),) + idx] = np.broadcast_to(np.asarray(e(*cols), dtype=np.float64), (P.shape[0],))
    return arr


def make_problem(kind_name, x, z):
    """Problems of the workloads (see module docstring), evaluated at the nodes."""
    import sympy as sp
    dim = x.shape[1]
    nl = kappa = None
    b_expr = c_expr = None
    kind = "linear"
    if kind_name == "disk":
        u_expr = lambda a, b: sp.sin(sp.pi * a) * sp.cos(sp.pi * b) + a ** 2 * b
        A_expr = lambda a, b: [[1 + sp.Rational(1, 2) * sp.sin(sp.pi * a), 0], [0, 1]]
    elif kind_name == "square":
        u_expr = lambda a, b: sp.exp(a) * sp.sin(2 * b)
        A_expr = lambda a, b: [[1 + a ** 2, sp.Rational(3, 10)], [sp.Rational(3, 10), 1 + b ** 2]]
        b_expr = lambda a, b: [1, -sp.Rational(1, 2)]
    elif kind_name == "ball":
        u_expr = lambda a, b, c: a ** 2 - b ** 2 + sp.Rational(1, 2) * c * sp.sin(sp.pi * a)
        A_expr = lambda a, b, c: [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
        nl = [0, 0, 0, 1]
        kind = "semilinear"
    elif kind_name == "star":
        u_expr = lambda a, b: a * b + sp.Rational(3, 10) * sp.sin(sp.pi * a)
        A_expr = lambda a, b: [[1, 0], [0, 1]]
        kappa = [1, 0, 1]
        kind = "quasilinear"
    elif kind_name == "poisson":
        u_expr = (lambda a, b: sp.sin(sp.pi * a) * sp.sin(sp.pi * b)) if dim == 2 else \
                 (lambda a, b, c: sp.sin(sp.pi * a) * sp.sin(sp.pi * b) * sp.sin(sp.pi * c))
        A_expr = (lambda *v: sp.eye(dim).tolist())
    else:
        raise ValueError(kind_name)
    fu, ff, fA, fb, fc = _manufactured(dim, u_expr, A_expr, b_expr, c_expr, nl, kappa)
    A = _eval(fA, x, (dim, dim))
    b = None if fb is None else _eval(fb, x, (dim, 1))[:, :, 0]
    c = None if fc is None else _eval(fc, x)
    return Problem(A=A, b=b, c=c, f=_eval(ff, x), g=_eval(fu, z), u_star=_eval(fu, x),
                   nl=nl, kappa=kappa, kind=kind)


# ------------------------------------------------------------------ workloads

def disk400(walks=1000, eps=1e-3, seed=0, problem=True):
    x = disk_nodes()
    z = circle_nodes(128)
    w = Workload("disk400", Domain(2, "ball", np.array([0.0, 0.0, 1.0])), x, z, walks, eps, 64, seed)
    if problem:
        w.problem = make_problem("disk", x, z)
    w.meta["grid_spacing"] = 0.0835
    return w


def square(k=64, per_side=128, walks=10_000, eps=1e-4, seed=0, precision=32, problem=True):
    x = square_nodes(k)
    z = square_boundary_nodes(per_side)
    w = Workload(f"square{k * k}", Domain(2, "box", np.array([0.0, 0.0, 1.0, 1.0])), x, z, walks, eps,
                 precision, seed)
    w.lam = np.full(x.shape[0], 1.0 / x.shape[0])
    if problem:
        w.problem = make_problem("square", x, z)
    return w


def square4096(**kw):
    return square(64, 128, **kw)


def ball(n=8000, p=2000, walks=10_000, eps=1e-4, seed=0, node_seed=1, problem=True):
    x, h = ball_nodes(n, node_seed)
    z = fibonacci_sphere(p)
    w = Workload(f"ball{n}", Domain(3, "ball", np.array([0.0, 0.0, 0.0, 1.0])), x, z, walks, eps, 32, seed)
    w.meta["lattice_spacing"] = h
    if problem:
        w.problem = make_problem("ball", x, z)
    return w


def ball8000(**kw):
    return ball(8000, 2000, **kw)


def stars(count=32, nmin=256, nmax=4096, walks=2000, eps=1e-4, seed=2, problem=True):
    rng = np.random.default_rng(seed)
    out = []
    for t in range(count):
        kfold = int(rng.integers(3, 8))
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        p = max(8, n // 8)
        V = star_polygon(kfold)
        x = star_nodes(V, n, rng)
        z = polygon_boundary_nodes(V, p)
        w = Workload(f"star{t}", Domain(2, "polygon", V.ravel().copy()), x, z, walks, eps, 32, 0)
        w.meta["kfold"] = kfold
        if problem:
            w.problem = make_problem("star", x, z)
        out.append(w)
    return out


WORKLOADS = {"disk400": disk400, "square4096": square4096, "ball8000": ball8000}


# ------------------------------------------------------------------ serving requests
# Random coefficient fields and manufactured solutions for the request server (no counterpart in
# the paper's experiments).  A = I + S(x), S symmetric, each of its d(d+1)/2 entries a sum of 8
# modes a_k cos(w_k . x) or a_k sin(w_k . x) with a_k ~ U(-0.3, 0.3)/8 and w_k ~ U(-pi, pi)^d,
# redrawn until the smallest eigenvalue of A at every node is at least 0.2; b ~ U(-1, 1)^d
# (constant); each right-hand side is a manufactured u* = sum_j c_j phi_j over a fixed basis
# (1, x_i, x_i x_j, sin(pi x_0), cos(pi x_1), exp(x_0 / 2)) with c_j ~ U(-1, 1)/sqrt(#basis);
# f = -div(A grad u*) + b . grad u* (+ u*^3 for semilinear requests), g = u* on the boundary.

_BASIS_CACHE = {}


def _basis(dim):
    if dim in _BASIS_CACHE:
        return _BASIS_CACHE[dim]
    import sympy as sp
    xs = sp.symbols("x0:%d" % dim)
    exprs = [sp.Integer(1)] + list(xs) + [xs[i] * xs[j] for i in range(dim) for j in range(i, dim)]
    exprs += [sp.sin(sp.pi * xs[0]), sp.cos(sp.pi * xs[1]), sp.exp(xs[0] / 2)]
    fns = []
    for e in exprs:
        grad = [sp.diff(e, v) for v in xs]
        hess = [[sp.diff(e, a, b) for b in xs] for a in xs]
        lam = lambda q: sp.lambdify(xs, q, "numpy")
        fns.append((lam(e), [lam(g) for g in grad], [[lam(h) for h in row] for row in hess]))
    _BASIS_CACHE[dim] = fns
    return fns


def _ev(fn, P):
    return np.broadcast_to(np.asarray(fn(*[P[:, k] for k in range(P.shape[1])]), dtype=np.float64),
                           (P.shape[0],)).astype(np.float64)


def random_field(x, rng, modes=8, return_spec=False):
    """(A [n][d][d], dA [n][d][d][d] with dA[:, l, i, j] = d_l A_ij) of one random field (and the
    modes (i, j, a, w, kind) when return_spec)."""
    n, dim = x.shape
    while True:
        A = np.tile(np.eye(dim), (n, 1, 1))
        dA = np.zeros((n, dim, dim, dim))
        spec = []
        for i in range(dim):
            for j in range(i, dim):
                a = rng.uniform(-0.3, 0.3, modes) / modes
                w = rng.uniform(-np.pi, np.pi, (modes, dim))
                kind = rng.integers(0, 2, modes)
                spec.append((i, j, a, w, kind))
                ph = x @ w.T                                    # [n][modes]
                val = np.where(kind == 0, np.cos(ph), np.sin(ph)) @ a
                der = np.where(kind == 0, -np.sin(ph), np.cos(ph))   # d/d(phase)
                A[:, i, j] += val
                if i != j:
                    A[:, j, i] += val
                for l in range(dim):
                    dl = der @ (a * w[:, l])
                    dA[:, l, i, j] += dl
                    if i != j:
                        dA[:, l, j, i] += dl
        if np.linalg.eigvalsh(A).min() >= 0.2:
            return (A, dA, spec) if return_spec else (A, dA)


def serving_requests(x, z, count, seed=3, nrhs_max=64, p_semilinear=0.5, nrhs=None):
    """count requests: dicts with A, b, f [R][n], g [R][p], u_star [R][n], kind, coef."""
    n, dim = x.shape
    rng = np.random.default_rng(seed)
    B = _basis(dim)
    nb = len(B)
    phi_x = np.stack([_ev(f, x) for f, _, _ in B])                                  # [nb][n]
    phi_z = np.stack([_ev(f, z) for f, _, _ in B])                                  # [nb][p]
    grad = np.stack([np.stack([_ev(g, x) for g in gr], 1) for _, gr, _ in B])        # [nb][n][d]
    hess = np.stack([np.stack([np.stack([_ev(h, x) for h in row], 1) for row in he], 1) for _, _, he in B])
    out = []
    for _ in range(count):
        A, dA = random_field(x, rng)
        b = np.tile(rng.uniform(-1, 1, dim), (n, 1))
        # L phi_j = -(sum_ij d_i A_ij d_j phi + A_ij d_ij phi) + b . grad phi
        divA = np.einsum("niij->nj", dA)                                            # sum_i d_i A_ij
        Lphi = -(np.einsum("nj,bnj->bn", divA, grad) + np.einsum("nij,bnij->bn", A, hess)) \
            + np.einsum("nj,bnj->bn", b, grad)
        R = int(nrhs) if nrhs is not None else int(np.exp(rng.uniform(0, np.log(nrhs_max + 1))))
        R = max(1, min(nrhs_max, R))
        C = rng.uniform(-1, 1, (R, nb)) / np.sqrt(nb)
        us = C @ phi_x
        semi = rng.uniform() < p_semilinear
        f = C @ Lphi + (us ** 3 if semi else 0.0)
        out.append(dict(A=A, b=b, f=f, g=C @ phi_z, u_star=us, kind="semilinear" if semi else "linear",
                        coef=[0.0, 0.0, 0.0, 1.0] if semi else None))
    return out
