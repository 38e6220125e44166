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
