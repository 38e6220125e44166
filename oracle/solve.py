"""FP64 oracle of the solve side (Sec. 3 of the paper).  TEST INFRASTRUCTURE ONLY.

Notation (G := A/2 and gradG := B/2 of the toolbox, so u = G s + H g with s = 2 q-bar):
  G [n][m], gradG [d][n][m], H [n][p] (exit frequencies), gradH [d][n][p] (= K),
  lam [n] cell weights lambda_i = lambda(W_i)/lambda(D), per-node coefficients
  A [n][d][d] (symmetric, elliptic), b [n][d], c [n], f [n], g [p].

PDE form (the paper's operator of eq. linearPDE with b -> -b, f -> -f, and the variational
form of Sec. 3.2 for the nonlinear terms):
      -div(A grad u) + b . grad u + c u + N(u) = f   in D,    u = g on the boundary,
with N(u) = sum_k a_k u^k (semilinear) or A(u) = (sum_k a_k u^k) A (quasilinear).

Galerkin residual with test functions G phi and nodal quadrature (eq. matrix_test_varphi):
  R(s) = sum_i lam_i [ gradG_i^T A_i grad u_i + G_i (b_i . grad u_i + c_i u_i + N(u_i) - f_i) ],
  u_i = G_i . s + H_i . g,  grad u_i = gradG_i s + gradH_i g.
For N = 0 this is R(s) = Lambda s - rhs with Lambda, rhs the matrices of eq. linear_q:
  Lambda = sum_i lam_i gradG_i^T A_i gradG_i + G^T diag(lam) (sum_k b_k d_k G) + G^T diag(lam c) G,
  rhs    = G^T (lam f) - Sigma g,
  Sigma  = sum_i lam_i gradG_i^T A_i gradH_i + G^T diag(lam) (sum_k b_k d_k H) + G^T diag(lam c) H.

Regularisation.  The Galerkin matrix Lambda is severely ill-conditioned (the paper reports
sigma_max ~ 1e-2, sigma_min ~ 1e-7 and solves eq. linear_q by truncated SVD with rcond 1e-3 /
1e-2, appendix "TSVD for eq. linear_q").  Plain LU of Lambda amplifies the Monte Carlo noise of
the toolbox into O(1) errors.  The LU-based solves here therefore factor the shifted matrix
Lambda + alpha I with alpha = rcond * ||Lambda||_F (Tikhonov's counterpart of the paper's
TSVD filter; ||Lambda||_F is within a factor 1.3 of sigma_max on the disk workload).
rcond = 0 gives the unregularised system.  Newton solves R(s) + alpha s = 0 with alpha taken
from the linear part; Picard recomputes alpha from each iteration's matrix.

Parity pins (tests/test_oracle_*.py): assemble -> the un-assembled bilinear form of
eq. matrix_test_varphi; lu_factor/lu_solve -> LAPACK via numpy.linalg.solve and the residual;
solve_linear -> manufactured solutions (discretisation-error bound) and a finite-difference
solve of the same problem; the first- and zeroth-order terms of assemble, rhs, residual and
sigma -> an independent finite-difference solve of an advection-reaction problem with
Dirichlet data (b = (8, -4), c = 30), which each function with b -> -b or c -> 2c misses;
newton -> zero residual and reduction to solve_linear when N = 0;
picard -> fixed-point property and reduction to solve_linear when A(u) = A; operators -> they
reproduce solve_linear for any (f, g) (which checks sigma against rhs), the torsion function
and the constant 1 on the disk, and the symmetry of GL diag(lam)^(-1) for a self-adjoint
operator; adam_steps -> the
closed form of the first step and convergence on a separable quadratic (and adam uses residual,
which is pinned above, as its gradient).
"""
from __future__ import annotations

import numpy as np


class SingularMatrix(ArithmeticError):
    pass


def assemble(G, gradG, lam, A, b=None, c=None):
    """Lambda of eq. linear_q (in the -div form above), m x m."""
    d = gradG.shape[0]
    Lam = np.zeros((G.shape[1], G.shape[1]))
    for k in range(d):
        for l in range(d):
            Lam += gradG[k].T @ ((lam * A[:, k, l])[:, None] * gradG[l])
    if b is not None:
        Bb = sum(b[:, k][:, None] * gradG[k] for k in range(d))
        Lam += G.T @ (lam[:, None] * Bb)
    if c is not None:
        Lam += G.T @ ((lam * c)[:, None] * G)
    return Lam


def rhs(G, gradG, H, gradH, lam, A, b, c, f, g):
    """right-hand side of eq. linear_q: G^T(lam f) - Sigma g, for one or several columns."""
    d = gradG.shape[0]
    f = np.asarray(f, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    one = f.ndim == 1
    F = f[:, None] if one else f
    Gm = g[:, None] if one else g
    Kg = np.stack([gradH[k] @ Gm for k in range(d)])          # [d][n][r]
    AKg = np.einsum("ikl,lir->kir", A, Kg)                    # A_i (gradH_i g)
    out = G.T @ (lam[:, None] * F)
    for k in range(d):
        out -= gradG[k].T @ (lam[:, None] * AKg[k])
    lower = np.zeros_like(F)
    if b is not None:
        lower += np.einsum("ik,kir->ir", b, Kg)
    if c is not None:
        lower += c[:, None] * (H @ Gm)
    out -= G.T @ (lam[:, None] * lower)
    return out[:, 0] if one else out


def lu_factor(M):
    """Textbook LU with partial pivoting (row interchanges), P M = L U."""
    a = np.array(M, dtype=np.float64, copy=True)
    n = a.shape[0]
    piv = np.arange(n)
    for k in range(n):
        p = k + int(np.argmax(np.abs(a[k:, k])))
        if a[p, k] == 0.0:
            raise SingularMatrix(f"zero pivot in column {k}")
        if p != k:
            a[[k, p]] = a[[p, k]]
            piv[[k, p]] = piv[[p, k]]
        a[k + 1:, k] /= a[k, k]
        a[k + 1:, k + 1:] -= np.outer(a[k + 1:, k], a[k, k + 1:])
    return a, piv


def lu_solve(lu, piv, b):
    """Forward substitution with unit-lower L, then back substitution with U."""
    x = np.array(b, dtype=np.float64)[piv]
    n = lu.shape[0]
    for i in range(n):
        x[i] -= lu[i, :i] @ x[:i]
    for i in range(n - 1, -1, -1):
        x[i] = (x[i] - lu[i, i + 1:] @ x[i + 1:]) / lu[i, i]
    return x


# LU backend of the solves.  The textbook LU above is the default; for the full-size systems
# (m = 4096, 8000) the golden-value script switches to LAPACK's partial-pivoting LU (the same
# factorisation, getrf/getrs, used as a library primitive; pinned against the textbook LU in
# tests/test_oracle_solve.py).
LU_BACKEND = "textbook"


def factor(M):
    if LU_BACKEND == "lapack":
        import scipy.linalg
        return ("lapack", scipy.linalg.lu_factor(np.asarray(M, dtype=np.float64)))
    return ("textbook", lu_factor(M))


def factor_solve(F, b):
    kind, fac = F
    if kind == "lapack":
        import scipy.linalg
        return scipy.linalg.lu_solve(fac, np.asarray(b, dtype=np.float64))
    lu, piv = fac
    return lu_solve(lu, piv, b)


def _poly(coef, u):
    return sum(a * u ** k for k, a in enumerate(coef))


def _dpoly(coef, u):
    return sum(k * a * u ** (k - 1) for k, a in enumerate(coef) if k > 0)


def reconstruct(tb, s, g):
    """u = G s + H g and grad u = gradG s + gradH g (Sec. 3.1 final boxed formula)."""
    u = tb["G"] @ s + tb["H"] @ g
    du = np.stack([tb["gradG"][k] @ s + tb["gradH"][k] @ g for k in range(tb["gradG"].shape[0])])
    return u, du


def residual(tb, lam, A, b, c, f, g, s, nl=None):
    """R(s) of the module docstring (the gradient of the discrete functional of Sec. 3.2 when
    b = 0: eq. gradJ with F = 1/2 grad u.A grad u + c u^2/2 + P(u) - f u)."""
    G = tb["G"]
    u, du = reconstruct(tb, s, g)
    Adu = np.einsum("ikl,li->ki", A, du)
    out = sum(tb["gradG"][k].T @ (lam * Adu[k]) for k in range(du.shape[0]))
    lower = -np.asarray(f, dtype=np.float64).copy()
    if b is not None:
        lower += np.einsum("ik,ki->i", b, du)
    if c is not None:
        lower += c * u
    if nl is not None:
        lower += _poly(nl, u)
    return out + G.T @ (lam * lower)


DEFAULT_RCOND = 3e-2


def shift(Lam, rcond):
    """alpha = rcond * ||Lambda||_F."""
    return float(rcond) * float(np.sqrt(np.sum(Lam * Lam)))


def solve_linear(tb, lam, A, b, c, f, g, rcond=DEFAULT_RCOND, alpha=None):
    """(Lambda + alpha I) s = rhs by textbook LU, then u = G s + H g.  ``alpha`` overrides the
    shift (used to compare with a solver that computed its shift from its own Lambda)."""
    Lam = assemble(tb["G"], tb["gradG"], lam, A, b, c)
    r = rhs(tb["G"], tb["gradG"], tb["H"], tb["gradH"], lam, A, b, c, f, g)
    alpha = shift(Lam, rcond) if alpha is None else float(alpha)
    s = factor_solve(factor(Lam + alpha * np.eye(Lam.shape[0])), r)
    u, _ = reconstruct(tb, s, g)
    return dict(s=s, u=u, Lam=Lam, rhs=r, alpha=alpha)


def newton(tb, lam, A, b, c, f, g, nl, tol=1e-10, max_iter=30, rcond=DEFAULT_RCOND, alpha=None):
    """Newton on R(s) + alpha s = 0 for N(u) = sum nl[k] u^k; Jacobian
    Lambda + alpha I + G^T diag(lam N'(u)) G; s_0 = 0; stop when the residual norm is at most
    tol times the initial one, or after max_iter iterations."""
    G = tb["G"]
    Lam = assemble(G, tb["gradG"], lam, A, b, c)
    alpha = shift(Lam, rcond) if alpha is None else float(alpha)
    s = np.zeros(G.shape[1])
    R = residual(tb, lam, A, b, c, f, g, s, nl) + alpha * s
    r0 = np.linalg.norm(R)
    it = 0
    hist = [r0]
    while it < max_iter and np.linalg.norm(R) > tol * r0:
        u, _ = reconstruct(tb, s, g)
        J = Lam + alpha * np.eye(Lam.shape[0]) + G.T @ ((lam * _dpoly(nl, u))[:, None] * G)
        s = s - factor_solve(factor(J), R)
        R = residual(tb, lam, A, b, c, f, g, s, nl) + alpha * s
        hist.append(np.linalg.norm(R))
        it += 1
    u, _ = reconstruct(tb, s, g)
    return dict(s=s, u=u, iters=it, converged=bool(np.linalg.norm(R) <= tol * r0), history=hist,
                alpha=alpha)


def picard(tb, lam, A, b, c, f, g, kappa, tol=1e-10, max_iter=100, rcond=DEFAULT_RCOND):
    """Picard for -div(kappa(u) A grad u) + ... = f, kappa(u) = sum kappa[k] u^k:
    u_0 = H g; A_i <- kappa(u_i) A_i; solve the linear system; stop when ||du||_inf <= tol."""
    u = tb["H"] @ g
    it, conv, s = 0, False, None
    while it < max_iter:
        Ak = _poly(kappa, u)[:, None, None] * A
        sol = solve_linear(tb, lam, Ak, b, c, f, g, rcond)
        du = np.max(np.abs(sol["u"] - u))
        u, s = sol["u"], sol["s"]
        it += 1
        if du <= tol:
            conv = True
            break
    return dict(s=s, u=u, iters=it, converged=conv)


def tsvd_solve(M, r, rcond):
    """Truncated-SVD solve (singular values below rcond * sigma_max dropped), used by the paper
    for eq. linear_q; reported beside the LU result as context."""
    U, sv, Vt = np.linalg.svd(M)
    keep = sv > rcond * sv[0]
    return Vt[keep].T @ ((U[:, keep].T @ r) / sv[keep])


def sigma(tb, lam, A, b=None, c=None):
    """Sigma of eq. linear_q (m x p), from its formula in the header above."""
    G, gradG, H, gradH = tb["G"], tb["gradG"], tb["H"], tb["gradH"]
    d = gradG.shape[0]
    Sig = np.zeros((G.shape[1], H.shape[1]))
    for k in range(d):
        for l in range(d):
            Sig += gradG[k].T @ ((lam * A[:, k, l])[:, None] * gradH[l])
    if b is not None:
        Bh = sum(b[:, k][:, None] * gradH[k] for k in range(d))
        Sig += G.T @ (lam[:, None] * Bh)
    if c is not None:
        Sig += G.T @ ((lam * c)[:, None] * H)
    return Sig


def operators(tb, lam, A, b=None, c=None, rcond=DEFAULT_RCOND, alpha=None):
    """The Monte Carlo operator estimates that follow eq. linear_inversion (Sec. 3.1):
        Green operator     GL = G (Lambda + alpha I)^(-1) A^lam,       A^lam = G^T diag(lam)  [n x n],
        elliptic measure   HL = H - G (Lambda + alpha I)^(-1) Sigma                          [n x p],
    so that the linear solve of the same problem is u = GL f + HL g (the paper's -A and
    -A^lam are G and G^T diag(lam) here, with f -> -f as in the header).  Lambda + alpha I is
    the shifted matrix of solve_linear."""
    G = tb["G"]
    Lam = assemble(G, tb["gradG"], lam, A, b, c)
    alpha = shift(Lam, rcond) if alpha is None else float(alpha)
    F = factor(Lam + alpha * np.eye(Lam.shape[0]))
    Alam = G.T * lam[None, :]
    GL = G @ factor_solve(F, Alam)
    HL = tb["H"] - G @ factor_solve(F, sigma(tb, lam, A, b, c))
    return dict(GL=GL, HL=HL, alpha=alpha)


def adam_steps(grad, s0, alpha, beta1=0.9, beta2=0.999, eps=1e-10, iters=100):
    """The Adam algorithm of the paper's appendix ("ADAM"), written from its formulas:
        m_j = beta1 m_{j-1} + (1 - beta1) grad(s_{j-1}),
        v_j = beta2 v_{j-1} + (1 - beta2) grad(s_{j-1})^2   (element-wise square),
        alpha_j = alpha sqrt(1 - beta2^j) / (1 - beta1^j),
        s_j = s_{j-1} - alpha_j m_j / (sqrt(v_j) + eps),   j >= 1,   m_0 = v_0 = 0.
    grad is any callable s -> gradient (so the update can be checked on closed forms)."""
    s = np.array(s0, dtype=np.float64)
    m = np.zeros_like(s)
    v = np.zeros_like(s)
    for j in range(1, iters + 1):
        gr = grad(s)
        m = beta1 * m + (1.0 - beta1) * gr
        v = beta2 * v + (1.0 - beta2) * gr * gr
        aj = alpha * np.sqrt(1.0 - beta2 ** j) / (1.0 - beta1 ** j)
        s = s - aj * m / (np.sqrt(v) + eps)
    return s


def adam(tb, lam, A, b, c, f, g, s0, alpha, beta1=0.9, beta2=0.999, eps=1e-10, iters=100, nl=None):
    """Adam on the discrete functional J of Sec. 3.2: its gradient is R(s) (eq. gradJ)."""
    return adam_steps(lambda s: residual(tb, lam, A, b, c, f, g, s, nl), s0, alpha, beta1, beta2, eps, iters)


def errors(u, u_star, lam):
    """lambda-weighted discrete L2 error and max error against a manufactured solution."""
    e = np.asarray(u) - np.asarray(u_star)
    return dict(l2=float(np.sqrt(np.sum(lam * e * e))), linf=float(np.max(np.abs(e))))
