"""The tensor-core GEMM of the mixed-precision assembly (tcgen05 kind::tf32, FP32 accumulation)
against an FP64 matrix product.  Bound: TF32 keeps 10 explicit mantissa bits, so each product
carries a relative error below 2^-10 (both inputs rounded) and the FP32 accumulation adds
K * 2^-24; the test allows 2^-9 + K 2^-23 times sum_k |a_k b_k| per entry."""
import numpy as np
import pytest

from paper_2608_07017_b300 import ewos

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 256, 32), (256, 512, 1024), (200, 300, 100), (1, 7, 3), (520, 260, 1200)])
def test_tc_gemm_matches_fp64(M, N, K):
    from paper_2608_07017_b300 import build
    build.build()
    rng = np.random.default_rng(M * 1000 + N + K)
    A = rng.normal(size=(K, M)).astype(np.float32)
    B = rng.normal(size=(K, N)).astype(np.float32)
    C = ewos.debug_tc_gemm(A, B).astype(np.float64)
    ref = A.astype(np.float64).T @ B.astype(np.float64)
    bound = (2.0 ** -9 + K * 2.0 ** -23) * (np.abs(A).astype(np.float64).T @ np.abs(B).astype(np.float64))
    assert np.all(np.abs(C - ref) <= bound + 1e-30)
    # it is not plain FP32 arithmetic either: TF32 rounding is visible on random data
    if K >= 32:
        assert np.max(np.abs(C - ref) / bound) > 1e-4


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (300, 260, 1000), (4, 3, 70)])
def test_tc_gemm_split_tf32(M, N, K):
    """3xTF32: hi*hi + hi*lo + lo*hi with hi = round-to-TF32(x), lo = x - hi; the dropped lo*lo term
    and the truncation of lo leave about 2^-20 relative per product; bound 2^-19 + K 2^-23."""
    rng = np.random.default_rng(M + 7 * N + K)
    A = rng.normal(size=(K, M)).astype(np.float32)
    B = rng.normal(size=(K, N)).astype(np.float32)
    C = ewos.debug_tc_gemm(A, B, split=True).astype(np.float64)
    ref = A.astype(np.float64).T @ B.astype(np.float64)
    bound = (2.0 ** -19 + K * 2.0 ** -23) * (np.abs(A).astype(np.float64).T @ np.abs(B).astype(np.float64))
    assert np.all(np.abs(C - ref) <= bound + 1e-30)


@pytest.mark.parametrize("M,N,K,sym", [(128, 128, 64, False), (300, 260, 5000, False), (520, 520, 9000, True),
                                       (7, 5, 3, False)])
def test_tc_gemm_f16_split(M, N, K, sym):
    """The FP16 form of the long-K product (the Jacobian's G^T D G): A and B scaled by powers of two
    that put their largest entries in [2^13, 2^14), split into FP16 halves, three kind::f16
    products accumulated in chunks.  On normal data every operand entry keeps 22 bits (2^-21
    relative per product, plus the FP16 subnormal floor of 2^-25 / s per entry) and the chunked
    accumulation adds 2^-16 + K 2^-24 of sum |a b|."""
    rng = np.random.default_rng(M + N + K)
    A = rng.normal(size=(K, M)).astype(np.float32)
    B = (rng.uniform(0.5, 2.0, size=(K, 1)) * A[:, :N]).astype(np.float32) if sym else \
        rng.normal(size=(K, N)).astype(np.float32) * 1e-3
    C = ewos.debug_tc_gemm(A, B, f16=True, sym=sym).astype(np.float64)
    ref = A.astype(np.float64).T @ B.astype(np.float64)
    absref = np.abs(A).astype(np.float64).T @ np.abs(B).astype(np.float64)
    s_a = 2.0 ** (13 - np.floor(np.log2(np.abs(A).max())))
    s_b = 2.0 ** (13 - np.floor(np.log2(np.abs(B).max())))
    bound = (2.0 ** -19 + 2.0 ** -16 + K * 2.0 ** -24) * absref + \
        2.0 ** -24 / s_a * np.abs(B).astype(np.float64).sum(axis=0)[None, :] + \
        2.0 ** -24 / s_b * np.abs(A).astype(np.float64).sum(axis=0)[:, None]
    assert np.all(np.abs(C - ref) <= bound)
    if K >= 1000:
        assert np.linalg.norm(C - ref) < 4e-6 * np.linalg.norm(absref)


@pytest.mark.parametrize("M,K", [(128, 64), (300, 1000), (520, 96), (7, 5)])
def test_tc_gemm_symmetric_launch(M, K):
    """The symmetric launch of the assembly (A^T A, or A^T D A): only tiles on and below the
    diagonal are computed and each off-diagonal one is also stored transposed; the result equals
    the full 3xTF32 product within its bound, and the mirrored tiles are exact transposes (inside
    a diagonal tile the two halves come from different MMA lanes and round differently)."""
    rng = np.random.default_rng(M + K)
    A = rng.normal(size=(K, M)).astype(np.float32)
    d = rng.uniform(0.5, 2.0, size=(K, 1)).astype(np.float32)
    B = (d * A).astype(np.float32)
    C = ewos.debug_tc_gemm(A, B, sym=True).astype(np.float64)
    ref = A.astype(np.float64).T @ B.astype(np.float64)
    bound = (2.0 ** -19 + K * 2.0 ** -23) * (np.abs(A).astype(np.float64).T @ np.abs(B).astype(np.float64))
    assert np.all(np.abs(C - ref) <= bound + 1e-30)
    ti = np.arange(M)[:, None] // 128
    tj = np.arange(M)[None, :] // 128
    off = ti != tj
    assert np.array_equal(C[off], C.T[off])


def _pq_case(n, m, D, seed, spread, sym=False):
    """P [D+1][n][m] with magnitudes log-uniform over `spread` decades below 1e-2 and random
    signs (the bins of G and grad G range over several decades); M_i = lam_i [[A_i, 0], [b_i^T, c_i]]
    with A_i symmetric positive definite (sym: b_i = 0, so Q_i = M_i P_i gives a symmetric Lambda)."""
    rng = np.random.default_rng(seed)
    E = D + 1
    mag = 10.0 ** rng.uniform(-2.0 - spread, -2.0, size=(E, n, m))
    P = (mag * rng.choice([-1.0, 1.0], size=(E, n, m))).astype(np.float32)
    lam = rng.uniform(0.5, 1.5, size=n) / n
    R = rng.normal(size=(n, D, D))
    A = np.einsum("nij,nkj->nik", R, R) + np.eye(D)[None]
    M = np.zeros((n, E, E))
    M[:, :D, :D] = lam[:, None, None] * A
    M[:, D, D] = lam * rng.uniform(0.0, 2.0, size=n)
    if not sym:
        M[:, D, :D] = lam[:, None] * rng.normal(size=(n, D))
    return P, M


def _pq_ref(P, M):
    """Lambda = sum_{l, i} P[l][i]^T Q[l][i] with Q_i = M_i P_i in FP64, and sum |P|^T |Q|"""
    P64 = P.astype(np.float64)
    Q = np.einsum("ijk,kic->jic", M, P64)
    E, n, m = P.shape
    P2, Q2 = P64.reshape(E * n, m), Q.reshape(E * n, m)
    return P2.T @ Q2, np.abs(P2).T @ np.abs(Q2)


@pytest.mark.parametrize("f16", [True, False])
@pytest.mark.parametrize("n,m,D,sym,spread", [(200, 150, 2, False, 3.0), (300, 260, 3, True, 6.0),
                                              (1000, 520, 2, False, 9.0), (64, 33, 3, False, 1.0),
                                              (8000, 260, 3, True, 3.0)])
def test_tc_assemble_pq(n, m, D, sym, spread, f16):
    """Lambda = P^T (M P) as the mixed solve assembles it: FP16 halves of the scaled operands or
    three TF32 products.  Both keep about 22 significand bits per operand.  The tensor cores round
    their FP32 accumulation toward zero; the assembly accumulates chunks of 256 operand elements
    and adds the chunks in FP32 registers, so an entry carries the truncation of one chunk (at most
    48 MMAs of 2^-23 each, under 2^-16 of sum |P||Q|) and the rounding of the chunk sums (K 2^-24).
    In the FP16 form the entries far below the largest keep an absolute error of 2^-25 / s (s the
    power of two that scaled the operand): 2^-24 / s_P sum |Q| + 2^-24 / s_Q sum |P| more.  The
    matrix as a whole: ||C - Lambda||_F / ||Lambda||_F below 4e-6 at every K (measured 1e-6 to
    2e-6; one accumulator for all of K gave 5e-9 K), still a bias toward zero."""
    P, M = _pq_case(n, m, D, n + m + D, spread, sym)
    C = ewos.debug_tc_assemble(P, M, sym=sym, f16=f16).astype(np.float64)
    ref, absref = _pq_ref(P, M)
    K = (D + 1) * n
    bound = (2.0 ** -18 + 2.0 ** -16 + K * 2.0 ** -24) * absref
    if f16:
        E = D + 1
        Q = np.einsum("ijk,kic->jic", M, P.astype(np.float64)).reshape(E * n, m)
        P2 = np.abs(P.astype(np.float64)).reshape(E * n, m)
        s_p = 2.0 ** (13 - np.floor(np.log2(P2.max())))
        s_q = 2.0 ** (13 - np.floor(np.log2(np.abs(Q).max())))
        bound += 2.0 ** -24 / s_p * np.abs(Q).sum(axis=0)[None, :] + 2.0 ** -24 / s_q * P2.sum(axis=0)[:, None]
    err = np.abs(C - ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    rel = np.linalg.norm(C - ref) / np.linalg.norm(ref)
    assert rel < 4e-6
    assert np.linalg.norm(C) < np.linalg.norm(ref)


@pytest.mark.parametrize("f16", [True, False])
@pytest.mark.parametrize("M,N,K", [(389, 300, 512), (1000, 777, 512), (256, 256, 100), (130, 1100, 64), (3, 5, 7)])
def test_tc_update_per_row_and_column_scales(M, N, K, f16):
    """The LU's trailing update C - A B on the tensor cores.  In the FP16 form every row of A and
    every column of B gets its own power-of-two scale (largest entry in [2^13, 2^14)) before the
    split into FP16 halves, so rows and columns whose magnitudes differ by 2^40 keep their
    relative accuracy: per entry 2^-21 of sum |a b| from the halves, the truncating FP32
    accumulation (at most 2^-24 of the partial sums per step), the FP16 subnormal floor of
    2^-25 / s_i per entry of row i (2^-25 / t_j for column j), and the rounding of the result.
    The TF32 form splits without scales (FP32's range) and has no floor."""
    rng = np.random.default_rng(M * 7 + N + K)
    A = rng.normal(size=(M, K)) * 2.0 ** rng.integers(-20, 21, size=(M, 1))
    B = rng.normal(size=(K, N)) * 2.0 ** rng.integers(-20, 21, size=(1, N))
    A[M // 2, :] = 0.0               # a zero row and a zero column (scale 1)
    B[:, N // 2] = 0.0
    A = A.astype(np.float32)
    B = B.astype(np.float32)
    C = (A.astype(np.float64) @ B.astype(np.float64) * rng.uniform(0.5, 1.5, size=(M, N))).astype(np.float32)
    out = ewos.debug_tc_update(A, B, C, f16=f16).astype(np.float64)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = C.astype(np.float64) - A64 @ B64
    absref = np.abs(A64) @ np.abs(B64)
    bound = (2.0 ** -19 + K * 2.0 ** -24) * absref + 2.0 ** -23 * np.abs(ref)
    if f16:
        amax = np.abs(A64).max(axis=1, keepdims=True)
        bmax = np.abs(B64).max(axis=0, keepdims=True)
        s = np.where(amax > 0, 2.0 ** (13 - np.floor(np.log2(np.where(amax > 0, amax, 1.0)))), 1.0)
        t = np.where(bmax > 0, 2.0 ** (13 - np.floor(np.log2(np.where(bmax > 0, bmax, 1.0)))), 1.0)
        bound += 2.0 ** -24 / s * np.abs(B64).sum(axis=0, keepdims=True) + \
            2.0 ** -24 / t * np.abs(A64).sum(axis=1, keepdims=True)
    assert np.all(np.abs(out - ref) <= bound)
    # the zero row and column leave C as it was
    assert np.array_equal(out[M // 2, :], C[M // 2, :].astype(np.float64))
    assert np.array_equal(out[:, N // 2], C[:, N // 2].astype(np.float64))
    # relative accuracy of the rows and columns of smallest magnitude
    i = int(np.argmin(np.where(np.abs(A64).max(axis=1) > 0, np.abs(A64).max(axis=1), np.inf)))
    assert np.linalg.norm(out[i] - ref[i]) <= 1e-5 * np.linalg.norm(absref[i]) + 2.0 ** -23 * np.linalg.norm(ref[i])
