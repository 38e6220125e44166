// sgemm.cuh -- FP32 SIMT GEMM used by the low-precision LU (trailing updates) and, where the
// tensor-core path is not available, the low-precision assembly.
//   C[i][j] = alpha * sum_k opA(i,k) B[k][j] + beta * C[i][j]
//   opA(i,k) = A[k*lda + i] when A_KMAJOR (A stored K x M), else A[i*lda + k];  B is K x N.
// 128 x 128 block tiles, BK = 8, 256 threads, 8 x 8 outputs per thread (two 4-wide strips 64
// apart in each direction so shared-memory reads are conflict free), double-buffered stages.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace ewos {

template <bool A_KMAJOR>
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, float alpha, const float* __restrict__ A,
                                                    int64_t lda, const float* __restrict__ B, int64_t ldb, float beta,
                                                    float* __restrict__ C, int64_t ldc) {
    constexpr int BM = 128, BN = 128, BK = 8;
    __shared__ float As[2][BK][BM];
    __shared__ float Bs[2][BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;

    float ra[4], rb[4];
    auto load_global = [&](int k0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = tid + 256 * q;          // 0..1023 over the 8 x 128 tile
            int kk, ii;
            if (A_KMAJOR) { kk = t >> 7; ii = t & 127; } else { ii = t >> 3; kk = t & 7; }
            const int gi = i0 + ii, gk = k0 + kk;
            ra[q] = (gi < M && gk < K) ? (A_KMAJOR ? A[(int64_t)gk * lda + gi] : A[(int64_t)gi * lda + gk]) : 0.f;
            const int kb = t >> 7, jj = t & 127;
            const int gkb = k0 + kb, gj = j0 + jj;
            rb[q] = (gkb < K && gj < N) ? B[(int64_t)gkb * ldb + gj] : 0.f;
        }
    };
    auto store_shared = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = tid + 256 * q;
            int kk, ii;
            if (A_KMAJOR) { kk = t >> 7; ii = t & 127; } else { ii = t >> 3; kk = t & 7; }
            As[buf][kk][ii] = ra[q];
            Bs[buf][t >> 7][t & 127] = rb[q];
        }
    };
    int buf = 0;
    load_global(0);
    store_shared(0);
    __syncthreads();
    for (int k0 = 0; k0 < K; k0 += BK) {
        const bool more = k0 + BK < K;
        if (more) load_global(k0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[8], b[8];
#pragma unroll
            for (int r = 0; r < 4; ++r) { a[r] = As[buf][kk][ty * 4 + r]; a[4 + r] = As[buf][kk][64 + ty * 4 + r]; }
#pragma unroll
            for (int c = 0; c < 4; ++c) { b[c] = Bs[buf][kk][tx * 4 + c]; b[4 + c] = Bs[buf][kk][64 + tx * 4 + c]; }
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        if (more) {
            store_shared(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int gi = i0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
        if (gi >= M) continue;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int gj = j0 + (c < 4 ? tx * 4 + c : 64 + tx * 4 + (c - 4));
            if (gj >= N) continue;
            float* cp = C + (int64_t)gi * ldc + gj;
            *cp = alpha * acc[r][c] + (beta == 0.f ? 0.f : beta * *cp);
        }
    }
}

}  // namespace ewos
