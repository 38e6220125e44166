"""The serving-request generator (random coefficient fields, manufactured right-hand sides)
against a symbolic derivation of the same problem (sympy), and its ellipticity guard."""
import numpy as np
import sympy as sp

from paper_2608_07017_b300 import workloads as W


def _symbolic_f(spec, dim, bvec, coeffs, x):
    xs = sp.symbols("x0:%d" % dim)
    A = sp.eye(dim)
    for i, j, a, w, kind in spec:
        e = 0
        for ak, wk, kk in zip(a, w, kind):
            ph = sum(float(wk[l]) * xs[l] for l in range(dim))
            e += float(ak) * (sp.cos(ph) if kk == 0 else sp.sin(ph))
        A[i, j] += e
        if i != j:
            A[j, i] += e
    basis = [sp.Integer(1)] + list(xs) + [xs[i] * xs[j] for i in range(dim) for j in range(i, dim)]
    basis += [sp.sin(sp.pi * xs[0]), sp.cos(sp.pi * xs[1]), sp.exp(xs[0] / 2)]
    u = sum(float(c) * p for c, p in zip(coeffs, basis))
    grad = sp.Matrix([sp.diff(u, v) for v in xs])
    flux = A * grad
    f = -sum(sp.diff(flux[i], xs[i]) for i in range(dim)) + sum(float(bvec[i]) * grad[i] for i in range(dim))
    fn = sp.lambdify(xs, f, "numpy")
    return np.asarray(fn(*[x[:, k] for k in range(dim)]), dtype=np.float64)


def test_random_field_operator_matches_sympy():
    rng = np.random.default_rng(11)
    x = np.random.default_rng(1).uniform(-0.7, 0.7, (40, 2))
    A, dA, spec = W.random_field(x, rng, return_spec=True)
    assert np.linalg.eigvalsh(A).min() >= 0.2
    # same draws as serving_requests: rebuild one request's f with the generator's pieces
    B = W._basis(2)
    nb = len(B)
    coeffs = np.random.default_rng(5).uniform(-1, 1, nb) / np.sqrt(nb)
    bvec = np.array([0.3, -0.7])
    grad = np.stack([np.stack([W._ev(g, x) for g in gr], 1) for _, gr, _ in B])
    hess = np.stack([np.stack([np.stack([W._ev(h, x) for h in row], 1) for row in he], 1) for _, _, he in B])
    divA = np.einsum("niij->nj", dA)
    Lphi = -(np.einsum("nj,bnj->bn", divA, grad) + np.einsum("nij,bnij->bn", A, hess)) \
        + np.einsum("nj,bnj->bn", np.tile(bvec, (40, 1)), grad)
    f = coeffs @ Lphi
    ref = _symbolic_f(spec, 2, bvec, coeffs, x)
    assert np.max(np.abs(f - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_serving_requests_shapes_and_mix():
    x = W.disk_nodes(0.2, 0.9)
    z = W.circle_nodes(16)
    rq = W.serving_requests(x, z, 12, seed=3, nrhs_max=64)
    kinds = {r["kind"] for r in rq}
    assert kinds == {"linear", "semilinear"}
    for r in rq:
        R = r["f"].shape[0]
        assert 1 <= R <= 64 and r["g"].shape == (R, z.shape[0]) and r["A"].shape == (x.shape[0], 2, 2)
        if r["kind"] == "semilinear":
            assert r["coef"] == [0.0, 0.0, 0.0, 1.0]
