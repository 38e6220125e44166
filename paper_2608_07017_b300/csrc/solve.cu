// solve.cu -- the finite-dimensional problems of Sec. 3 on the GPU.
//
// With the stacked toolbox P = [d_1 G, .., d_d G, G] ((d+1) n x m) and KH = [d_1 H, .., H]:
//   v_i  = (grad u_i, u_i) = P_i s + KH_i g                            (Sec. 3.1, u = G s + H g)
//   w_i  = M_i v_i + e_d lam_i (N(u_i) - f_i),    M_i = [[lam_i k_i A_i, 0], [lam_i b_i^T, lam_i c_i]]
//   R(s) = P^T w                                                        (Galerkin residual)
//   Lambda = P^T Q,  Q_i = M_i P_i                                      (eq. linear_q)
// so the assembly is one GEMM with K = (d+1) n and every residual is two passes over P.
// The linear system is (Lambda + alpha I) s = rhs, alpha = rcond ||Lambda||_F, rhs = -R_0(0).
// Dense LU with partial pivoting: blocked right-looking; the panel is a cooperative kernel
// (rows split over all SMs, one grid barrier per column, row swaps through published copies),
// then row interchanges, a unit-lower triangular solve for U12 and a GEMM for the trailing
// matrix.  Triangular solves with the factors are cooperative kernels as well.  Every grid
// barrier spins a bounded number of times; on a timeout the kernels return and the call
// reports EWOS_ETIMEOUT.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "sgemm.cuh"
#include "toolbox.hpp"

namespace ewos {

// ------------------------------------------------------------------ bounded grid barrier
struct GridBarrier {
    unsigned int count;
    unsigned int gen;
    int err;
    int singular;
};

constexpr long long kSpinLimit = 1ll << 24;   // about 10 s of L2 polling

__device__ __forceinline__ bool grid_sync(GridBarrier* b) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = &b->gen;
        const unsigned int g = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&b->count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            long long spins = 0;
            while (*vgen == g) {
                if (++spins > kSpinLimit) { atomicExch(&b->err, 1); break; }
            }
        }
        __threadfence();
        s_ok = (*(volatile int*)&b->err) == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// ------------------------------------------------------------------ small kernels
__global__ void coef_kernel(int n, int D, const double* __restrict__ lam, const double* __restrict__ A,
                            const double* __restrict__ b, const double* __restrict__ c,
                            const double* __restrict__ kap, int nkap, const double* __restrict__ u,
                            double* __restrict__ M) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int E = D + 1;
    double k = 1.0;
    if (kap && u) {
        double pw = 1.0;
        k = 0.0;
        for (int t = 0; t < nkap; ++t) { k += kap[t] * pw; pw *= u[i]; }
    }
    double* Mi = M + (size_t)i * E * E;
    for (int j = 0; j < D; ++j) {
        for (int q = 0; q < D; ++q) Mi[j * E + q] = lam[i] * k * A[((size_t)i * D + j) * D + q];
        Mi[j * E + D] = 0.0;
    }
    for (int q = 0; q < D; ++q) Mi[D * E + q] = b ? lam[i] * b[(size_t)i * D + q] : 0.0;
    Mi[D * E + D] = c ? lam[i] * c[i] : 0.0;
}

// Q[j][i][col] = sum_k M_i[j][k] P[k][i][col]
template <typename TP, typename TQ>
__global__ void formQ_kernel(const TP* __restrict__ P, const double* __restrict__ M, TQ* __restrict__ Q,
                             int n, int m, int D) {
    const int i = blockIdx.y;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= m) return;
    const int E = D + 1;
    const size_t nm = (size_t)n * m;
    double pv[4];
    for (int k = 0; k < E; ++k) pv[k] = (double)P[k * nm + (size_t)i * m + col];
    const double* Mi = M + (size_t)i * E * E;
    for (int j = 0; j < E; ++j) {
        double acc = 0.0;
        for (int k = 0; k < E; ++k) acc += Mi[j * E + k] * pv[k];
        Q[j * nm + (size_t)i * m + col] = (TQ)acc;
    }
}

// y = X v for a row-major X [rows][cols] (warp per row)
template <typename TP>
__global__ void rowdot_kernel(const TP* __restrict__ X, int64_t rows, int cols, const double* __restrict__ v,
                              double* __restrict__ y, int accumulate) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const TP* xr = X + r * cols;
    double acc = 0.0;
    for (int c = lane; c < cols; c += 32) acc += (double)xr[c] * v[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) y[r] = accumulate ? y[r] + acc : acc;
}

// y[col] += sum_{r in chunk} X[r][col] w[r]   (y zeroed beforehand)
template <typename TP>
__global__ void coltrans_kernel(const TP* __restrict__ X, int64_t rows, int cols, const double* __restrict__ w,
                                double* __restrict__ y, int64_t chunk) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= cols) return;
    const int64_t r0 = (int64_t)blockIdx.y * chunk;
    const int64_t r1 = min(rows, r0 + chunk);
    double acc = 0.0;
    for (int64_t r = r0; r < r1; ++r) acc += (double)X[r * cols + col] * w[r];
    atomicAdd(&y[col], acc);
}

// w_i = M_i v_i + e_D lam_i (N(u_i) - f_i); v laid out as [(D+1)][n]
__global__ void formw_kernel(int n, int D, const double* __restrict__ M, const double* __restrict__ v,
                             const double* __restrict__ lam, const double* __restrict__ f,
                             const double* __restrict__ nl, int nnl, double* __restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int E = D + 1;
    const double* Mi = M + (size_t)i * E * E;
    double vi[4];
    for (int k = 0; k < E; ++k) vi[k] = v[(size_t)k * n + i];
    for (int j = 0; j < E; ++j) {
        double acc = 0.0;
        for (int k = 0; k < E; ++k) acc += Mi[j * E + k] * vi[k];
        w[(size_t)j * n + i] = acc;
    }
    double extra = -f[i];
    if (nl) {
        double pw = 1.0, s = 0.0;
        for (int t = 0; t < nnl; ++t) { s += nl[t] * pw; pw *= vi[D]; }
        extra += s;
    }
    w[(size_t)D * n + i] += lam[i] * extra;
}

// Newton Jacobian term: Qn[i][col] = lam_i N'(u_i) G[i][col]
template <typename TP>
__global__ void jac_scale_kernel(const TP* __restrict__ Gm, const double* __restrict__ u, const double* __restrict__ lam,
                                 const double* __restrict__ nl, int nnl, double* __restrict__ out, int n, int m) {
    const int i = blockIdx.y;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= m) return;
    double d = 0.0, pw = 1.0;
    for (int t = 1; t < nnl; ++t) { d += t * nl[t] * pw; pw *= u[i]; }
    out[(size_t)i * m + col] = lam[i] * d * (double)Gm[(size_t)i * m + col];
}

__global__ void sumsq_kernel(const double* __restrict__ X, int64_t count, double* __restrict__ out) {
    double acc = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
        acc += X[t] * X[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

__global__ void narrow_f32_kernel(const double* __restrict__ in, float* __restrict__ out, int64_t count) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = (float)in[t];
}

__global__ void sumsq_f32_kernel(const float* __restrict__ X, int64_t count, double* __restrict__ out) {
    double acc = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
        acc += (double)X[t] * (double)X[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// Jacobian-vector product pieces of the Newton system: w_i = M_i v_i + e_D lam_i N'(u_i) v_{D,i}
__global__ void formw_jv_kernel(int n, int D, const double* __restrict__ M, const double* __restrict__ v,
                                const double* __restrict__ lam, const double* __restrict__ u,
                                const double* __restrict__ nl, int nnl, double* __restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int E = D + 1;
    const double* Mi = M + (size_t)i * E * E;
    double vi[4];
    for (int k = 0; k < E; ++k) vi[k] = v[(size_t)k * n + i];
    for (int j = 0; j < E; ++j) {
        double acc = 0.0;
        for (int k = 0; k < E; ++k) acc += Mi[j * E + k] * vi[k];
        w[(size_t)j * n + i] = acc;
    }
    double d = 0.0, pw = 1.0;
    for (int t = 1; t < nnl; ++t) { d += t * nl[t] * pw; pw *= u[i]; }
    w[(size_t)D * n + i] += lam[i] * d * vi[D];
}

template <typename T>
__global__ void add_diag_kernel(T* __restrict__ A, int m, int lda, double alpha) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) A[(size_t)i * lda + i] += (T)alpha;
}

__global__ void axpy_kernel(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += a * x[i];
}

__global__ void maxabsdiff_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                  unsigned long long* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < n) v = fabs(a[i] - b[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

// ------------------------------------------------------------------ FP64 tiled GEMM (SIMT)
// C[i][j] = alpha * sum_k opA(i,k) B[k][j] + beta * C[i][j];  opA(i,k) = A[k*lda + i] when
// A_KMAJOR (A stored K x M), else A[i*lda + k].  B is K x N row-major.  64 x 64 tiles, BK 16.
template <typename TA, bool A_KMAJOR>
__global__ void __launch_bounds__(256) gemm64_kernel(int M, int N, int K, double alpha, const TA* __restrict__ A,
                                                     int64_t lda, const double* __restrict__ B, int64_t ldb,
                                                     double beta, double* __restrict__ C, int64_t ldc) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int t = threadIdx.x; t < BK * BM; t += 256) {
            int kk, ii;
            if (A_KMAJOR) { kk = t / BM; ii = t % BM; } else { ii = t / BK; kk = t % BK; }
            const int gi = i0 + ii, gk = k0 + kk;
            double v = 0.0;
            if (gi < M && gk < K) v = A_KMAJOR ? (double)A[(int64_t)gk * lda + gi] : (double)A[(int64_t)gi * lda + gk];
            As[kk][ii] = v;
        }
        for (int t = threadIdx.x; t < BK * BN; t += 256) {
            const int kk = t / BN, jj = t % BN;
            const int gk = k0 + kk, gj = j0 + jj;
            Bs[kk][jj] = (gk < K && gj < N) ? B[(int64_t)gk * ldb + gj] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], bb[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
            for (int q = 0; q < 4; ++q) bb[q] = Bs[kk][tx + 16 * q];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = fma(a[r], bb[q], acc[r][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gi = i0 + ty + 16 * r, gj = j0 + tx + 16 * q;
            if (gi < M && gj < N) {
                double* cp = C + (int64_t)gi * ldc + gj;
                *cp = alpha * acc[r][q] + (beta == 0.0 ? 0.0 : beta * *cp);
            }
        }
}

template <typename TA, bool A_KMAJOR>
static void gemm64(cudaStream_t st, int M, int N, int K, double alpha, const TA* A, int64_t lda, const double* B,
                   int64_t ldb, double beta, double* C, int64_t ldc) {
    if (M <= 0 || N <= 0) return;
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    ::ewos::note_launch(), gemm64_kernel<TA, A_KMAJOR><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

template <typename T>
static void gemm_trailing(cudaStream_t st, int M, int N, int K, const T* A, int64_t lda, const T* B, int64_t ldb,
                          T* C, int64_t ldc);

template <>
void gemm_trailing<double>(cudaStream_t st, int M, int N, int K, const double* A, int64_t lda, const double* B,
                           int64_t ldb, double* C, int64_t ldc) {
    gemm64<double, false>(st, M, N, K, -1.0, A, lda, B, ldb, 1.0, C, ldc);
}

template <bool A_KMAJOR>
static void sgemm(cudaStream_t st, int M, int N, int K, float alpha, const float* A, int64_t lda, const float* B,
                  int64_t ldb, float beta, float* C, int64_t ldc) {
    if (M <= 0 || N <= 0) return;
    dim3 grid((N + 127) / 128, (M + 127) / 128);
    ::ewos::note_launch(), sgemm_kernel<A_KMAJOR><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

template <>
void gemm_trailing<float>(cudaStream_t st, int M, int N, int K, const float* A, int64_t lda, const float* B,
                          int64_t ldb, float* C, int64_t ldc) {
    sgemm<false>(st, M, N, K, -1.f, A, lda, B, ldb, 1.f, C, ldc);
}

// ------------------------------------------------------------------ LU with partial pivoting
constexpr int kNB = 64;

template <typename T>
struct PanelPub {
    T* val;       // [2][blocks]
    int* row;     // [2][blocks]
    T* vals;      // [2][blocks][nb]
    T* diag;      // [2][nb]
};

template <typename T>
__global__ void lu_panel_kernel(T* __restrict__ A, int lda, int mtot, int kb, int nb, int chunk, int* __restrict__ ipiv,
                                PanelPub<T> pub, GridBarrier* bar) {
    extern __shared__ __align__(16) unsigned char sm[];
    T* tile = reinterpret_cast<T*>(sm);               // [chunk][nb]
    __shared__ T s_best;
    __shared__ int s_brow;
    __shared__ int s_win;
    const int nblk = gridDim.x, b = blockIdx.x;
    const int r0 = kb + b * chunk;
    const int r1 = min(mtot, r0 + chunk);
    const int nr = max(0, r1 - r0);
    for (int t = threadIdx.x; t < nr * nb; t += blockDim.x) {
        const int rr = t / nb, cc = t % nb;
        tile[t] = A[(size_t)(r0 + rr) * lda + kb + cc];
    }
    __syncthreads();
    for (int jj = 0; jj < nb; ++jj) {
        const int par = jj & 1;
        const int prow0 = kb + jj;
        // local argmax over owned rows >= prow0 (ties: lowest row)
        if (threadIdx.x < 32) {
            T best = T(-1);
            int brow = 0x7fffffff;
            for (int rr = threadIdx.x; rr < nr; rr += 32) {
                const int gr = r0 + rr;
                if (gr < prow0) continue;
                const T v = fabs(tile[rr * nb + jj]);
                if (v > best || (v == best && gr < brow)) { best = v; brow = gr; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T ob = __shfl_down_sync(0xffffffffu, best, o);
                const int orw = __shfl_down_sync(0xffffffffu, brow, o);
                if (ob > best || (ob == best && orw < brow)) { best = ob; brow = orw; }
            }
            if (threadIdx.x == 0) { s_best = best; s_brow = brow; }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            pub.val[par * nblk + b] = s_best;
            pub.row[par * nblk + b] = s_brow;
        }
        if (s_brow != 0x7fffffff)
            for (int cc = threadIdx.x; cc < nb; cc += blockDim.x)
                pub.vals[((size_t)par * nblk + b) * nb + cc] = tile[(s_brow - r0) * nb + cc];
        if (prow0 >= r0 && prow0 < r1)
            for (int cc = threadIdx.x; cc < nb; cc += blockDim.x) pub.diag[par * nb + cc] = tile[(prow0 - r0) * nb + cc];
        if (!grid_sync(bar)) return;
        if (threadIdx.x == 0) {
            T best = T(-1);
            int brow = 0x7fffffff, win = 0;
            for (int q = 0; q < nblk; ++q) {
                const T v = pub.val[par * nblk + q];
                const int rw = pub.row[par * nblk + q];
                if (rw == 0x7fffffff) continue;
                if (v > best || (v == best && rw < brow)) { best = v; brow = rw; win = q; }
            }
            s_brow = brow;
            s_win = win;
            if (b == 0) {
                ipiv[prow0] = brow;
                if (best == T(0)) bar->singular = 1;
            }
        }
        __syncthreads();
        const int prow = s_brow;
        const T* pv = pub.vals + ((size_t)par * nblk + s_win) * nb;
        if (prow != prow0) {
            if (prow0 >= r0 && prow0 < r1)
                for (int cc = threadIdx.x; cc < nb; cc += blockDim.x) tile[(prow0 - r0) * nb + cc] = pv[cc];
            if (prow >= r0 && prow < r1)
                for (int cc = threadIdx.x; cc < nb; cc += blockDim.x) tile[(prow - r0) * nb + cc] = pub.diag[par * nb + cc];
        }
        __syncthreads();
        const T piv = pv[jj];
        const T inv = piv != T(0) ? T(1) / piv : T(0);
        for (int rr = threadIdx.x; rr < nr; rr += blockDim.x) {
            const int gr = r0 + rr;
            if (gr <= prow0) continue;
            T* rowp = tile + rr * nb;
            const T l = rowp[jj] * inv;
            rowp[jj] = l;
            for (int cc = jj + 1; cc < nb; ++cc) rowp[cc] -= l * pv[cc];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < nr * nb; t += blockDim.x) {
        const int rr = t / nb, cc = t % nb;
        A[(size_t)(r0 + rr) * lda + kb + cc] = tile[t];
    }
}

template <typename T>
__global__ void laswp_kernel(T* __restrict__ A, int lda, int m, int kb, int nb, const int* __restrict__ ipiv) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= m || (col >= kb && col < kb + nb)) return;
    for (int i = kb; i < kb + nb; ++i) {
        const int p = ipiv[i];
        if (p != i) {
            const T t = A[(size_t)i * lda + col];
            A[(size_t)i * lda + col] = A[(size_t)p * lda + col];
            A[(size_t)p * lda + col] = t;
        }
    }
}

// The row interchanges of one panel (ipiv[kb .. kb+nb)) composed into "row keys[t] receives the
// old row vals[t]" for the at most 2 nb rows they touch (one thread; shared-memory tables).
__global__ void perm_compose_kernel(const int* __restrict__ ipiv, int kb, int nb, int* __restrict__ keys,
                                    int* __restrict__ vals, int* __restrict__ count) {
    __shared__ int k[128], v[128];
    __shared__ int n;
    if (threadIdx.x != 0) return;
    n = 0;
    auto slot = [&](int row) {
        for (int t = 0; t < n; ++t)
            if (k[t] == row) return t;
        k[n] = row; v[n] = row;
        return n++;
    };
    for (int i = kb; i < kb + nb; ++i) {
        const int p = ipiv[i];
        if (p == i) continue;
        const int a = slot(i), b = slot(p);
        const int tv = v[a]; v[a] = v[b]; v[b] = tv;
    }
    int w = 0;
    for (int t = 0; t < n; ++t)
        if (k[t] != v[t]) { keys[w] = k[t]; vals[w] = v[t]; ++w; }
    *count = w;
}

// apply the composed interchanges to the columns outside the panel, 32 columns per block
template <typename T>
__global__ void rows_permute_kernel(T* __restrict__ A, int lda, int m, int kb, int nb, const int* __restrict__ keys,
                                    const int* __restrict__ vals, const int* __restrict__ count) {
    __shared__ T buf[128][32];
    const int cnt = *count;
    if (cnt == 0) return;
    int c0 = blockIdx.x * 32;
    if (c0 >= kb) c0 += nb;              // skip the panel's columns (kb is a multiple of 64)
    if (c0 >= m) return;
    const int cw = min(32, m - c0);
    for (int t = threadIdx.x; t < cnt * 32; t += blockDim.x) {
        const int r = t >> 5, c = t & 31;
        if (c < cw) buf[r][c] = A[(size_t)vals[r] * lda + c0 + c];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < cnt * 32; t += blockDim.x) {
        const int r = t >> 5, c = t & 31;
        if (c < cw) A[(size_t)keys[r] * lda + c0 + c] = buf[r][c];
    }
}

// final row order of P A = L U: perm[i] = original row at position i (one thread, shared table)
__global__ void perm_full_kernel(const int* __restrict__ ipiv, int m, int* __restrict__ perm) {
    extern __shared__ int pm[];
    for (int i = threadIdx.x; i < m; i += blockDim.x) pm[i] = i;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = 0; i < m; ++i) {
            const int p = ipiv[i];
            if (p != i) { const int t = pm[i]; pm[i] = pm[p]; pm[p] = t; }
        }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) perm[i] = pm[i];
}

__global__ void gather_rows_kernel(const double* __restrict__ in, double* __restrict__ out, const int* __restrict__ perm,
                                   int m, int nrhs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)m * nrhs) return;
    const int r = (int)(t / m), i = (int)(t % m);
    out[t] = in[(int64_t)r * m + perm[i]];
}

// U12 = L11^{-1} A12 (L11 unit lower nb x nb at (kb, kb))
template <typename T>
__global__ void trsm_unit_lower_kernel(T* __restrict__ A, int lda, int m, int kb, int nb) {
    extern __shared__ __align__(16) unsigned char sm[];
    T* L = reinterpret_cast<T*>(sm);
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) L[t] = A[(size_t)(kb + t / nb) * lda + kb + t % nb];
    __syncthreads();
    const int col = kb + nb + blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= m) return;
    T x[kNB];
#pragma unroll
    for (int i = 0; i < kNB; ++i) x[i] = i < nb ? A[(size_t)(kb + i) * lda + col] : T(0);
#pragma unroll
    for (int i = 1; i < kNB; ++i) {
        if (i >= nb) break;
        T acc = x[i];
#pragma unroll
        for (int k = 0; k < kNB; ++k)
            if (k < i) acc -= L[i * nb + k] * x[k];
        x[i] = acc;
    }
#pragma unroll
    for (int i = 0; i < kNB; ++i)
        if (i < nb) A[(size_t)(kb + i) * lda + col] = x[i];
}

// Panel factorisation on one thread-block cluster: the panel's rows are split over the
// cluster's CTAs and kept in their shared memory; per column, every CTA publishes its local
// pivot candidate, a cluster barrier, every CTA reads the candidates and the pivot and old rows
// through distributed shared memory, a second barrier, then the swap and the rank-1 update of
// the CTA's own rows.  Hardware cluster barriers replace the grid-wide barriers of the
// cooperative panel.
template <typename T>
__global__ void __launch_bounds__(256) lu_panel_cluster_kernel(T* __restrict__ A, int lda, int mtot, int kb, int nb,
                                                              int chunk, int* __restrict__ ipiv,
                                                              GridBarrier* __restrict__ bar) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int ncta = (int)cluster.num_blocks();
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* tile = reinterpret_cast<T*>(sm_raw);          // [chunk][nb]
    __shared__ T s_cval;
    __shared__ int s_crow;
    __shared__ T s_piv[64];
    __shared__ T s_old[64];
    __shared__ int s_prow;
    __shared__ T s_best;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int r0 = kb + rank * chunk;
    const int r1 = min(mtot, r0 + chunk);
    const int nr = max(0, r1 - r0);
    for (int t = threadIdx.x; t < nr * nb; t += blockDim.x) tile[t] = A[(size_t)(r0 + t / nb) * lda + kb + t % nb];
    __syncthreads();
    for (int jj = 0; jj < nb; ++jj) {
        const int prow0 = kb + jj;
        if (warp == 0) {
            T best = T(-1);
            int brow = 0x7fffffff;
            for (int rr = lane; rr < nr; rr += 32) {
                const int gr = r0 + rr;
                if (gr < prow0) continue;
                const T v = fabs(tile[rr * nb + jj]);
                if (v > best || (v == best && gr < brow)) { best = v; brow = gr; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T ob = __shfl_down_sync(0xffffffffu, best, o);
                const int orw = __shfl_down_sync(0xffffffffu, brow, o);
                if (ob > best || (ob == best && orw < brow)) { best = ob; brow = orw; }
            }
            if (lane == 0) { s_cval = best; s_crow = brow; }
        }
        cluster.sync();
        if (warp == 0) {
            T best = T(-1);
            int brow = 0x7fffffff;
            if (lane < ncta) {
                const T v = *cluster.map_shared_rank(&s_cval, lane);
                const int rw = *cluster.map_shared_rank(&s_crow, lane);
                if (rw != 0x7fffffff) { best = v; brow = rw; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T ob = __shfl_down_sync(0xffffffffu, best, o);
                const int orw = __shfl_down_sync(0xffffffffu, brow, o);
                if (ob > best || (ob == best && orw < brow)) { best = ob; brow = orw; }
            }
            if (lane == 0) {
                s_prow = brow;
                s_best = best;
                if (rank == 0) {
                    ipiv[prow0] = brow;
                    if (best == T(0)) bar->singular = 1;
                }
            }
        }
        __syncthreads();
        const int prow = s_prow;
        {
            const int ow = (prow - kb) / chunk, oi = (prow - kb) - ow * chunk;
            const int ow0 = (prow0 - kb) / chunk, oi0 = (prow0 - kb) - ow0 * chunk;
            const T* rp = cluster.map_shared_rank(tile, ow) + (size_t)oi * nb;
            const T* rp0 = cluster.map_shared_rank(tile, ow0) + (size_t)oi0 * nb;
            for (int cc = threadIdx.x; cc < nb; cc += blockDim.x) { s_piv[cc] = rp[cc]; s_old[cc] = rp0[cc]; }
        }
        cluster.sync();
        if (prow != prow0) {
            if (prow0 >= r0 && prow0 < r1)
                for (int cc = threadIdx.x; cc < nb; cc += blockDim.x) tile[(prow0 - r0) * nb + cc] = s_piv[cc];
            if (prow >= r0 && prow < r1)
                for (int cc = threadIdx.x; cc < nb; cc += blockDim.x) tile[(prow - r0) * nb + cc] = s_old[cc];
        }
        __syncthreads();
        const T piv = s_piv[jj];
        const T inv = piv != T(0) ? T(1) / piv : T(0);
        for (int rr = warp; rr < nr; rr += nw) {
            const int gr = r0 + rr;
            if (gr <= prow0) continue;
            T* rowp = tile + rr * nb;
            const T l = rowp[jj] * inv;
            for (int cc = jj + 1 + lane; cc < nb; cc += 32) rowp[cc] -= l * s_piv[cc];
            __syncwarp();
            if (lane == 0) rowp[jj] = l;
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < nr * nb; t += blockDim.x) A[(size_t)(r0 + t / nb) * lda + kb + t % nb] = tile[t];
    cluster.sync();
}

struct LuScratch {
    void* pub = nullptr;
    size_t pub_bytes = 0;
    GridBarrier* bar = nullptr;
    int* ipiv = nullptr;
    int* perm = nullptr;        // [m] final row order
    int* swp = nullptr;         // [2 * 128 + 1] composed interchanges of one panel
    double* tmp = nullptr;      // [m * nrhs] permuted right-hand sides
    int panel_blocks = 0;
};

template <typename T>
static ewos_status lu_factor_device(T* A, int m, int lda, LuScratch& S, cudaStream_t st, bool* singular) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256;
    EWOS_CUDA_TRY(cudaMemsetAsync(S.bar, 0, sizeof(GridBarrier), st));
    for (int kb = 0; kb < m; kb += kNB) {
        const int nb = std::min(kNB, m - kb);
        const int rows = m - kb;
        int blocks = std::min(nsm, std::max(1, (rows + 7) / 8));
        const int chunk = (rows + blocks - 1) / blocks;
        blocks = (rows + chunk - 1) / chunk;
        // cluster panel when the panel fits in the shared memory of one cluster
        bool done_cluster = false;
        for (int cl : {16, 8}) {
            const int cchunk = (rows + cl - 1) / cl;
            const size_t csmem = sizeof(T) * (size_t)cchunk * nb;
            if (csmem > 200 * 1024) continue;
            auto kfn = lu_panel_cluster_kernel<T>;
            if (cl > 8 && cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(csmem, 16)) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            cudaLaunchConfig_t lc = {};
            lc.gridDim = dim3(cl);
            lc.blockDim = dim3(256);
            lc.dynamicSmemBytes = csmem;
            lc.stream = st;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = cl;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            lc.attrs = at;
            lc.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, kfn, &lc) != cudaSuccess || nclusters < 1) {
                cudaGetLastError();
                continue;
            }
            ::ewos::note_launch();
            if (cudaLaunchKernelEx(&lc, kfn, A, lda, m, kb, nb, cchunk, S.ipiv, S.bar) == cudaSuccess) {
                done_cluster = true;
                break;
            }
            cudaGetLastError();
        }
        if (!done_cluster) {
        const size_t smem = sizeof(T) * (size_t)chunk * nb;
        int per_sm = 0;
        cudaFuncSetAttribute(lu_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 1));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lu_panel_kernel<T>, threads, smem);
        if (per_sm * nsm < blocks) { set_error("LU panel: blocks not co-resident"); return EWOS_EINVAL; }
        PanelPub<T> pub;
        char* base = (char*)S.pub;
        pub.val = (T*)base;
        pub.row = (int*)(base + sizeof(T) * 2 * nsm);
        pub.vals = (T*)(base + sizeof(T) * 2 * nsm + sizeof(int) * 2 * nsm + 64);
        pub.diag = pub.vals + (size_t)2 * nsm * kNB;
        T* Ap = A;
        int ldai = lda, mt = m, kbi = kb, nbi = nb, chi = chunk;
        int* ip = S.ipiv;
        GridBarrier* bar = S.bar;
        void* args[] = {&Ap, &ldai, &mt, &kbi, &nbi, &chi, &ip, &pub, &bar};
        ::ewos::note_launch();
        EWOS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)lu_panel_kernel<T>, blocks, threads, args, smem, st));
        }
        ::ewos::note_launch(), perm_compose_kernel<<<1, 32, 0, st>>>(S.ipiv, kb, nb, S.swp, S.swp + 128, S.swp + 256);
        {
            const int ncols = m - nb;
            if (ncols > 0)
                ::ewos::note_launch(), rows_permute_kernel<T><<<(ncols + 31) / 32, 256, 0, st>>>(A, lda, m, kb, nb, S.swp,
                                                                                                S.swp + 128, S.swp + 256);
        }
        const int rest = m - kb - nb;
        if (rest > 0) {
            ::ewos::note_launch(), trsm_unit_lower_kernel<T><<<(rest + 127) / 128, 128, sizeof(T) * nb * nb, st>>>(A, lda, m, kb, nb);
            // A22 -= L21 U12
            gemm_trailing<T>(st, rest, rest, nb, A + (size_t)(kb + nb) * lda + kb, lda,
                             A + (size_t)kb * lda + kb + nb, lda, A + (size_t)(kb + nb) * lda + kb + nb, lda);
        }
        EWOS_CUDA_TRY(cudaGetLastError());
    }
    EWOS_CUDA_TRY(cudaFuncSetAttribute(perm_full_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(int) * m)));
    ::ewos::note_launch(), perm_full_kernel<<<1, 1024, sizeof(int) * m, st>>>(S.ipiv, m, S.perm);
    GridBarrier hb{};
    EWOS_CUDA_TRY(cudaMemcpyAsync(&hb, S.bar, sizeof(hb), cudaMemcpyDeviceToHost, st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(st));
    if (hb.err) { set_error("LU panel: grid barrier timed out"); return EWOS_ETIMEOUT; }
    *singular = hb.singular != 0;
    return EWOS_OK;
}


// Solve with the factors of P A = L U for nrhs right-hand sides x [nrhs][m] (in place; x arrives
// already permuted).  Block 0 owns the 64-row diagonal blocks and solves each from shared memory;
// per diagonal block one grid barrier: block 0 first updates the next diagonal block's rows and
// solves it while the other blocks update the rows further down (the same in reverse for U).
constexpr int kTB = 64;

template <typename T>
__global__ void lu_solve_kernel(const T* __restrict__ LU, int lda, int m, const int* __restrict__ ipiv,
                                double* __restrict__ x, int nrhs, GridBarrier* bar) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nblk = gridDim.x;
    const int nbk = (m + kTB - 1) / kTB;
    (void)ipiv;
    __shared__ T sL[kTB][kTB + 1];
    __shared__ double sx[kTB];
    auto update_rows = [&](int kb, int ke, int rlo, int rhi, int worker, int nworkers) {
        // x[r][i] -= sum_{k in [kb, ke)} LU[i][k] x[r][k] for rows i in [rlo, rhi)
        const int64_t total = (int64_t)(rhi - rlo) * nrhs;
        for (int64_t t = worker; t < total; t += nworkers) {
            const int i = rlo + (int)(t / nrhs), r = (int)(t % nrhs);
            double* xr = x + (size_t)r * m;
            double acc = 0.0;
            for (int k = kb + lane; k < ke; k += 32) acc += (double)LU[(size_t)i * lda + k] * xr[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane == 0) xr[i] -= acc;
        }
    };
    auto diag = [&](int t, bool lower) {
        const int ib = t * kTB, ie = min(m, ib + kTB), w = ie - ib;
        for (int q = threadIdx.x; q < w * w; q += blockDim.x) sL[q / w][q % w] = LU[(size_t)(ib + q / w) * lda + ib + q % w];
        for (int r = 0; r < nrhs; ++r) {
            double* xr = x + (size_t)r * m;
            __syncthreads();
            for (int i = threadIdx.x; i < w; i += blockDim.x) sx[i] = xr[ib + i];
            __syncthreads();
            if (warp == 0) {
                if (lower) {
                    for (int i = 0; i < w; ++i) {
                        double acc = 0.0;
                        for (int k = lane; k < i; k += 32) acc += (double)sL[i][k] * sx[k];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
                        if (lane == 0) sx[i] -= acc;
                        __syncwarp();
                    }
                } else {
                    for (int i = w - 1; i >= 0; --i) {
                        double acc = 0.0;
                        for (int k = i + 1 + lane; k < w; k += 32) acc += (double)sL[i][k] * sx[k];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
                        if (lane == 0) sx[i] = (sx[i] - acc) / (double)sL[i][i];
                        __syncwarp();
                    }
                }
            }
            __syncthreads();
            for (int i = threadIdx.x; i < w; i += blockDim.x) xr[ib + i] = sx[i];
        }
        __syncthreads();
    };
    // ---- forward, unit lower
    if (blockIdx.x == 0) diag(0, true);
    if (!grid_sync(bar)) return;
    for (int t = 0; t + 1 < nbk; ++t) {
        const int ib = t * kTB, ie = ib + kTB;
        const int nxt_hi = min(m, ie + kTB);
        if (blockIdx.x == 0) {
            update_rows(ib, ie, ie, nblk == 1 ? m : nxt_hi, warp, nw);
            __syncthreads();
            diag(t + 1, true);
        } else if (nxt_hi < m) {
            update_rows(ib, ie, nxt_hi, m, (blockIdx.x - 1) * nw + warp, (nblk - 1) * nw);
        }
        if (!grid_sync(bar)) return;
    }
    // ---- backward, upper with diagonal
    if (blockIdx.x == 0) diag(nbk - 1, false);
    if (!grid_sync(bar)) return;
    for (int t = nbk - 1; t > 0; --t) {
        const int ib = t * kTB, ie = min(m, ib + kTB);
        const int prv_lo = ib - kTB;
        if (blockIdx.x == 0) {
            update_rows(ib, ie, nblk == 1 ? 0 : prv_lo, ib, warp, nw);
            __syncthreads();
            diag(t - 1, false);
        } else if (prv_lo > 0) {
            update_rows(ib, ie, 0, prv_lo, (blockIdx.x - 1) * nw + warp, (nblk - 1) * nw);
        }
        if (!grid_sync(bar)) return;
    }
}

// ------------------------------------------------------------------ workspace
struct SolveWorkspace {
    int D = 0;
    int64_t n = 0, m = 0, p = 0;
    double *Q = nullptr, *Lam = nullptr, *LUm = nullptr, *M = nullptr, *Jx = nullptr;
    double *A = nullptr, *b = nullptr, *c = nullptr, *f = nullptr, *g = nullptr, *nl = nullptr;
    double *s = nullptr, *x = nullptr, *v = nullptr, *w = nullptr, *y = nullptr, *u = nullptr, *u2 = nullptr;
    double* scal = nullptr;                   // [4] reductions
    unsigned long long* umax = nullptr;
    LuScratch lu;
    int64_t cap_rhs = 0;
    // mixed precision
    float *Q32 = nullptr, *L32 = nullptr, *LU32 = nullptr, *J32 = nullptr, *Jx32 = nullptr, *P32 = nullptr;
    double *rhs = nullptr, *r = nullptr, *dx = nullptr;
};

void free_workspace(SolveWorkspace* ws) {
    if (!ws) return;
    ::ewos::dev_free(ws->Q); ::ewos::dev_free(ws->Lam); ::ewos::dev_free(ws->LUm); ::ewos::dev_free(ws->M); ::ewos::dev_free(ws->Jx);
    ::ewos::dev_free(ws->A); ::ewos::dev_free(ws->b); ::ewos::dev_free(ws->c); ::ewos::dev_free(ws->f); ::ewos::dev_free(ws->g); ::ewos::dev_free(ws->nl);
    ::ewos::dev_free(ws->s); ::ewos::dev_free(ws->x); ::ewos::dev_free(ws->v); ::ewos::dev_free(ws->w); ::ewos::dev_free(ws->y); ::ewos::dev_free(ws->u); ::ewos::dev_free(ws->u2);
    ::ewos::dev_free(ws->scal); ::ewos::dev_free(ws->umax);
    ::ewos::dev_free(ws->lu.pub); ::ewos::dev_free(ws->lu.bar); ::ewos::dev_free(ws->lu.ipiv);
    ::ewos::dev_free(ws->lu.perm); ::ewos::dev_free(ws->lu.swp); ::ewos::dev_free(ws->lu.tmp);
    ::ewos::dev_free(ws->Q32); ::ewos::dev_free(ws->L32); ::ewos::dev_free(ws->LU32); ::ewos::dev_free(ws->J32);
    ::ewos::dev_free(ws->Jx32); ::ewos::dev_free(ws->P32);
    ::ewos::dev_free(ws->rhs); ::ewos::dev_free(ws->r); ::ewos::dev_free(ws->dx);
    delete ws;
}

static ewos_status ensure_workspace(ewos_toolbox* tb, int64_t nrhs, bool mixed) {
    if (tb->ws && tb->ws->cap_rhs < nrhs) { free_workspace(tb->ws); tb->ws = nullptr; }
    const int D = tb->dim, E = D + 1;
    const int64_t n = tb->n, m = tb->m, p = tb->p;
    if (!tb->ws) {
        SolveWorkspace* ws = new SolveWorkspace();
        tb->ws = ws;
        ws->D = D; ws->n = n; ws->m = m; ws->p = p; ws->cap_rhs = nrhs;
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->M, sizeof(double) * n * E * E));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->A, sizeof(double) * n * D * D));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->b, sizeof(double) * n * D));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->c, sizeof(double) * n));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->f, sizeof(double) * n * nrhs));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->g, sizeof(double) * p * nrhs));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->nl, sizeof(double) * 64));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->s, sizeof(double) * m * nrhs));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->x, sizeof(double) * m * nrhs));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->rhs, sizeof(double) * m * nrhs));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->r, sizeof(double) * m * nrhs));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->dx, sizeof(double) * m * nrhs));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->v, sizeof(double) * E * n));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->w, sizeof(double) * E * n));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->y, sizeof(double) * m));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->u, sizeof(double) * n * nrhs));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->u2, sizeof(double) * n));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->scal, sizeof(double) * 4));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->umax, sizeof(unsigned long long)));
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        ws->lu.pub_bytes = (size_t)2 * nsm * (sizeof(double) + sizeof(int)) + 64 + sizeof(double) * ((size_t)2 * nsm * kNB + 2 * kNB);
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->lu.pub, ws->lu.pub_bytes));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->lu.bar, sizeof(GridBarrier)));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->lu.ipiv, sizeof(int) * m));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->lu.perm, sizeof(int) * m));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->lu.swp, sizeof(int) * 260));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->lu.tmp, sizeof(double) * m * nrhs));
    }
    SolveWorkspace* ws = tb->ws;
    if (!mixed && !ws->Q) {
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Q, sizeof(double) * E * n * m));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Lam, sizeof(double) * m * m));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->LUm, sizeof(double) * m * m));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Jx, sizeof(double) * n * m));
    }
    if (mixed && !ws->Q32) {
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Q32, sizeof(float) * E * n * m));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->L32, sizeof(float) * m * m));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->LU32, sizeof(float) * m * m));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Jx32, sizeof(float) * n * m));
        if (tb->precision == 64) EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->P32, sizeof(float) * E * n * m));
    }
    return EWOS_OK;
}

template <typename T>
static ewos_status lu_solve_device(const T* LU, int m, int lda, LuScratch& S, double* x, int nrhs, cudaStream_t st) {
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lu_solve_kernel<T>, threads, 0);
    const int blocks = std::max(1, std::min(nsm, per_sm * nsm));
    EWOS_CUDA_TRY(cudaMemsetAsync(S.bar, 0, sizeof(GridBarrier), st));
    {
        const int64_t cnt = (int64_t)m * nrhs;
        ::ewos::note_launch(), gather_rows_kernel<<<(int)((cnt + 255) / 256), 256, 0, st>>>(x, S.tmp, S.perm, m, nrhs);
        EWOS_CUDA_TRY(cudaMemcpyAsync(x, S.tmp, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, st));
    }
    const T* a0 = LU;
    int lda_ = lda, m_ = m, nr = nrhs;
    const int* ip = S.ipiv;
    GridBarrier* bar = S.bar;
    void* args[] = {&a0, &lda_, &m_, &ip, &x, &nr, &bar};
    ::ewos::note_launch();
        EWOS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)lu_solve_kernel<T>, blocks, threads, args, 0, st));
    GridBarrier hb{};
    EWOS_CUDA_TRY(cudaMemcpyAsync(&hb, S.bar, sizeof(hb), cudaMemcpyDeviceToHost, st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(st));
    if (hb.err) { set_error("LU solve: grid barrier timed out"); return EWOS_ETIMEOUT; }
    return EWOS_OK;
}

// ------------------------------------------------------------------ operator pieces
struct Ctx {
    ewos_toolbox* tb;
    SolveWorkspace* ws;
    cudaStream_t st;
    int D, E;
    int64_t n, m, p;
};

template <typename TP>
static void apply_v(const Ctx& C, const double* s, const double* g) {
    // v = P s + KH g  ([(D+1)][n]); s may be NULL (= 0)
    const TP* P = (const TP*)C.tb->P;
    const TP* KH = (const TP*)C.tb->KH;
    const int64_t rows = (int64_t)C.E * C.n;
    const int blocks = (int)((rows * 32 + 255) / 256);
    if (s) {
        ::ewos::note_launch(), rowdot_kernel<TP><<<blocks, 256, 0, C.st>>>(P, rows, (int)C.m, s, C.ws->v, 0);
        ::ewos::note_launch(), rowdot_kernel<TP><<<blocks, 256, 0, C.st>>>(KH, rows, (int)C.p, g, C.ws->v, 1);
    } else {
        ::ewos::note_launch(), rowdot_kernel<TP><<<blocks, 256, 0, C.st>>>(KH, rows, (int)C.p, g, C.ws->v, 0);
    }
}

template <typename TP>
static void apply_PT(const Ctx& C, const double* w, double* y) {
    const TP* P = (const TP*)C.tb->P;
    const int64_t rows = (int64_t)C.E * C.n;
    const int64_t chunk = 256;
    cudaMemsetAsync(y, 0, sizeof(double) * C.m, C.st);
    dim3 grid((unsigned)((C.m + 255) / 256), (unsigned)((rows + chunk - 1) / chunk));
    ::ewos::note_launch(), coltrans_kernel<TP><<<grid, 256, 0, C.st>>>(P, rows, (int)C.m, w, y, chunk);
}

// y = R(s) = P^T w(P s + KH g)  (+ alpha s when alpha != 0); f, nl as in formw_kernel
template <typename TP>
static void residual(const Ctx& C, const double* s, const double* g, const double* f, const double* nl, int nnl,
                     double alpha, double* y) {
    apply_v<TP>(C, s, g);
    ::ewos::note_launch(), formw_kernel<<<(int)((C.n + 127) / 128), 128, 0, C.st>>>((int)C.n, C.D, C.ws->M, C.ws->v, C.tb->lambda, f, nl, nnl,
                                                             C.ws->w);
    apply_PT<TP>(C, C.ws->w, y);
    if (alpha != 0.0 && s) ::ewos::note_launch(), axpy_kernel<<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.m, alpha, s, y);
}

static double norm2(const Ctx& C, const double* v, int64_t len) {
    cudaMemsetAsync(C.ws->scal, 0, sizeof(double), C.st);
    ::ewos::note_launch(), sumsq_kernel<<<std::max<int64_t>(1, std::min<int64_t>(1024, (len + 255) / 256)), 256, 0, C.st>>>(v, len, C.ws->scal);
    double h = 0;
    cudaMemcpyAsync(&h, C.ws->scal, sizeof(double), cudaMemcpyDeviceToHost, C.st);
    cudaStreamSynchronize(C.st);
    return std::sqrt(h);
}

// Lambda = P^T Q with Q = M P (coefficients already in ws->M)
template <typename TP>
static void assemble_fp64(const Ctx& C) {
    const TP* P = (const TP*)C.tb->P;
    dim3 g((unsigned)((C.m + 255) / 256), (unsigned)C.n);
    ::ewos::note_launch(), formQ_kernel<TP, double><<<g, 256, 0, C.st>>>(P, C.ws->M, C.ws->Q, (int)C.n, (int)C.m, C.D);
    gemm64<TP, true>(C.st, (int)C.m, (int)C.m, (int)(C.E * C.n), 1.0, P, C.m, C.ws->Q, C.m, 0.0, C.ws->Lam, C.m);
}

static void u_from_s(const Ctx& C, const void* P, const void* KH, bool fp64, const double* s, const double* g, double* u) {
    const int blocks = (int)((C.n * 32 + 255) / 256);
    const size_t e = fp64 ? 8 : 4;
    const char* Gm = (const char*)P + e * C.D * C.n * C.m;
    const char* Hm = (const char*)KH + e * C.D * C.n * C.p;
    if (fp64) {
        ::ewos::note_launch(), rowdot_kernel<double><<<blocks, 256, 0, C.st>>>((const double*)Gm, C.n, (int)C.m, s, u, 0);
        ::ewos::note_launch(), rowdot_kernel<double><<<blocks, 256, 0, C.st>>>((const double*)Hm, C.n, (int)C.p, g, u, 1);
    } else {
        ::ewos::note_launch(), rowdot_kernel<float><<<blocks, 256, 0, C.st>>>((const float*)Gm, C.n, (int)C.m, s, u, 0);
        ::ewos::note_launch(), rowdot_kernel<float><<<blocks, 256, 0, C.st>>>((const float*)Hm, C.n, (int)C.p, g, u, 1);
    }
}

static double frob_shift(const Ctx& C, double rcond) {
    if (rcond == 0.0) return 0.0;
    return rcond * norm2(C, C.ws->Lam, C.m * C.m);
}

template <typename TP>
static ewos_status factor_shifted(const Ctx& C, double alpha, const double* extra_gemm_B) {
    // LU <- Lambda (+ G^T extra) + alpha I, factorised in place
    cudaMemcpyAsync(C.ws->LUm, C.ws->Lam, sizeof(double) * C.m * C.m, cudaMemcpyDeviceToDevice, C.st);
    if (extra_gemm_B) {
        const TP* Gm = (const TP*)C.tb->P + (size_t)C.D * C.n * C.m;
        gemm64<TP, true>(C.st, (int)C.m, (int)C.m, (int)C.n, 1.0, Gm, C.m, extra_gemm_B, C.m, 1.0, C.ws->LUm, C.m);
    }
    ::ewos::note_launch(), add_diag_kernel<double><<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.ws->LUm, (int)C.m, (int)C.m, alpha);
    bool sing = false;
    ewos_status s = lu_factor_device<double>(C.ws->LUm, (int)C.m, (int)C.m, C.ws->lu, C.st, &sing);
    if (s != EWOS_OK) return s;
    if (sing) { set_error("LU: zero pivot"); return EWOS_ESINGULAR; }
    return EWOS_OK;
}

static double elapsed_ms(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

template <typename TP>
static ewos_status solve_fp64(ewos_toolbox* tb, const ewos_problem* pb, double rcond, double tol, int max_iter,
                              ewos_solve_report* rep) {
    Ctx C{tb, tb->ws, pb->stream ? (cudaStream_t)pb->stream : tb->stream, tb->dim, tb->dim + 1, tb->n, tb->m, tb->p};
    SolveWorkspace* ws = tb->ws;
    const int64_t nrhs = pb->nrhs;
    auto t0 = std::chrono::steady_clock::now();
    const bool quasi = pb->nl_kind == EWOS_NL_QUASILINEAR, semi = pb->nl_kind == EWOS_NL_SEMILINEAR;
    ::ewos::note_launch(), coef_kernel<<<(int)((C.n + 127) / 128), 128, 0, C.st>>>((int)C.n, C.D, tb->lambda, ws->A, pb->b ? ws->b : nullptr,
                                                           pb->c ? ws->c : nullptr, nullptr, 0, nullptr, ws->M);
    rep->iters = 0;
    rep->converged = 1;
    if (!quasi) {
        assemble_fp64<TP>(C);
        const double alpha = frob_shift(C, rcond);
        rep->alpha = alpha;
        rep->ms_assemble = elapsed_ms(t0);
        if (!semi) {
            auto t1 = std::chrono::steady_clock::now();
            ewos_status s = factor_shifted<TP>(C, alpha, nullptr);
            if (s != EWOS_OK) return s;
            rep->ms_factor = elapsed_ms(t1);
            auto t2 = std::chrono::steady_clock::now();
            for (int64_t r = 0; r < nrhs; ++r) {       // rhs = -R_0(0)
                residual<TP>(C, nullptr, ws->g + r * C.p, ws->f + r * C.n, nullptr, 0, 0.0, ws->y);
                cudaMemsetAsync(ws->x + r * C.m, 0, sizeof(double) * C.m, C.st);
                ::ewos::note_launch(), axpy_kernel<<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.m, -1.0, ws->y, ws->x + r * C.m);
            }
            s = lu_solve_device<double>(ws->LUm, (int)C.m, (int)C.m, ws->lu, ws->x, (int)nrhs, C.st);
            if (s != EWOS_OK) return s;
            cudaMemcpyAsync(ws->s, ws->x, sizeof(double) * C.m * nrhs, cudaMemcpyDeviceToDevice, C.st);
            rep->iters = 1;
            rep->ms_solve = elapsed_ms(t2);
        } else {
            // Newton on R(s) + alpha s = 0
            const double* nl = ws->nl;
            for (int64_t r = 0; r < nrhs; ++r) {
                double* s = ws->s + r * C.m;
                const double* g = ws->g + r * C.p;
                const double* f = ws->f + r * C.n;
                cudaMemsetAsync(s, 0, sizeof(double) * C.m, C.st);
                residual<TP>(C, s, g, f, nl, pb->nl_ncoef, alpha, ws->y);
                const double r0 = norm2(C, ws->y, C.m);
                double rn = r0;
                int it = 0;
                while (it < max_iter && rn > tol * r0) {
                    // u at the current s, Jacobian term G^T diag(lam N'(u)) G
                    u_from_s(C, tb->P, tb->KH, tb->precision == 64, s, g, ws->u2);
                    dim3 gj((unsigned)((C.m + 255) / 256), (unsigned)C.n);
                    const TP* Gm = (const TP*)tb->P + (size_t)C.D * C.n * C.m;
                    ::ewos::note_launch(), jac_scale_kernel<TP><<<gj, 256, 0, C.st>>>(Gm, ws->u2, tb->lambda, nl, pb->nl_ncoef, ws->Jx, (int)C.n, (int)C.m);
                    auto t1 = std::chrono::steady_clock::now();
                    ewos_status st = factor_shifted<TP>(C, alpha, ws->Jx);
                    if (st != EWOS_OK) return st;
                    rep->ms_factor += elapsed_ms(t1);
                    cudaMemcpyAsync(ws->x, ws->y, sizeof(double) * C.m, cudaMemcpyDeviceToDevice, C.st);
                    st = lu_solve_device<double>(ws->LUm, (int)C.m, (int)C.m, ws->lu, ws->x, 1, C.st);
                    if (st != EWOS_OK) return st;
                    ::ewos::note_launch(), axpy_kernel<<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.m, -1.0, ws->x, s);
                    residual<TP>(C, s, g, f, nl, pb->nl_ncoef, alpha, ws->y);
                    rn = norm2(C, ws->y, C.m);
                    ++it;
                }
                rep->iters = std::max(rep->iters, it);
                if (!(rn <= tol * r0)) rep->converged = 0;
            }
        }
    } else {
        // Picard: A_i <- kappa(u_i) A_i, u_0 = H g
        for (int64_t r = 0; r < nrhs; ++r) {
            const double* g = ws->g + r * C.p;
            const double* f = ws->f + r * C.n;
            double* s = ws->s + r * C.m;
            double* u = ws->u + r * C.n;
            cudaMemsetAsync(s, 0, sizeof(double) * C.m, C.st);
            u_from_s(C, tb->P, tb->KH, tb->precision == 64, s, g, u);
            int it = 0;
            bool conv = false;
            while (it < max_iter) {
                ::ewos::note_launch(), coef_kernel<<<(int)((C.n + 127) / 128), 128, 0, C.st>>>((int)C.n, C.D, tb->lambda, ws->A,
                                                                       pb->b ? ws->b : nullptr, pb->c ? ws->c : nullptr,
                                                                       ws->nl, pb->nl_ncoef, u, ws->M);
                auto ta = std::chrono::steady_clock::now();
                assemble_fp64<TP>(C);
                const double alpha = frob_shift(C, rcond);
                rep->alpha = alpha;
                rep->ms_assemble += elapsed_ms(ta);
                auto t1 = std::chrono::steady_clock::now();
                ewos_status st = factor_shifted<TP>(C, alpha, nullptr);
                if (st != EWOS_OK) return st;
                rep->ms_factor += elapsed_ms(t1);
                residual<TP>(C, nullptr, g, f, nullptr, 0, 0.0, ws->y);
                cudaMemsetAsync(ws->x, 0, sizeof(double) * C.m, C.st);
                ::ewos::note_launch(), axpy_kernel<<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.m, -1.0, ws->y, ws->x);
                st = lu_solve_device<double>(ws->LUm, (int)C.m, (int)C.m, ws->lu, ws->x, 1, C.st);
                if (st != EWOS_OK) return st;
                cudaMemcpyAsync(s, ws->x, sizeof(double) * C.m, cudaMemcpyDeviceToDevice, C.st);
                u_from_s(C, tb->P, tb->KH, tb->precision == 64, s, g, ws->u2);
                cudaMemsetAsync(ws->umax, 0, sizeof(unsigned long long), C.st);
                ::ewos::note_launch(), maxabsdiff_kernel<<<(int)((C.n + 255) / 256), 256, 0, C.st>>>(C.n, ws->u2, u, ws->umax);
                unsigned long long hm = 0;
                cudaMemcpyAsync(&hm, ws->umax, sizeof(hm), cudaMemcpyDeviceToHost, C.st);
                cudaMemcpyAsync(u, ws->u2, sizeof(double) * C.n, cudaMemcpyDeviceToDevice, C.st);
                cudaStreamSynchronize(C.st);
                ++it;
                double du;
                memcpy(&du, &hm, sizeof(du));
                if (du <= tol) { conv = true; break; }
            }
            rep->iters = std::max(rep->iters, it);
            if (!conv) rep->converged = 0;
        }
    }
    // u = G s + H g, and the final FP64 residual of the last right-hand side
    for (int64_t r = 0; r < nrhs; ++r)
        u_from_s(C, tb->P, tb->KH, tb->precision == 64, ws->s + r * C.m, ws->g + r * C.p, ws->u + r * C.n);
    if (!quasi) {
        const int64_t r = nrhs - 1;
        residual<TP>(C, ws->s + r * C.m, ws->g + r * C.p, ws->f + r * C.n, semi ? ws->nl : nullptr,
                     semi ? pb->nl_ncoef : 0, rep->alpha, ws->y);
        rep->residual = norm2(C, ws->y, C.m);
    }
    EWOS_CUDA_TRY(cudaStreamSynchronize(C.st));
    EWOS_CUDA_TRY(cudaGetLastError());
    rep->ms_total = elapsed_ms(t0);
    return rep->converged ? EWOS_OK : EWOS_ENOCONV;
}

// ------------------------------------------------------------------ mixed precision
// Low-precision side: Lambda in FP32 (assembled by tc_assemble on the tensor cores, TF32 inputs
// with FP32 accumulation, or by the FP32 SIMT GEMM), LU of Lambda + alpha I in FP32 (the same
// blocked kernels, trailing updates in FP32).  FP64 side: the residual of every correction is
// the matrix-free FP64 operator (two passes over P), so iterative refinement converges to the
// FP64 solution of the same system while the O(m^3) work runs in 32-bit.
bool tc_assemble_available();
ewos_status tc_assemble(const float* A_km, const float* B_km, float* C, int M, int N, int K, cudaStream_t st,
                        bool split);
constexpr bool kSplitTF32 = true;     // 3xTF32 assembly: Lambda to ~1e-6, fewer refinement sweeps

template <typename TP>
__global__ void jac_scale32_kernel(const TP* __restrict__ Gm, const double* __restrict__ u, const double* __restrict__ lam,
                                   const double* __restrict__ nl, int nnl, float* __restrict__ out, int n, int m) {
    const int i = blockIdx.y;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= m) return;
    double d = 0.0, pw = 1.0;
    for (int t = 1; t < nnl; ++t) { d += t * nl[t] * pw; pw *= u[i]; }
    out[(size_t)i * m + col] = (float)(lam[i] * d * (double)Gm[(size_t)i * m + col]);
}

static double frob32(const Ctx& C, const float* X, int64_t count) {
    cudaMemsetAsync(C.ws->scal, 0, sizeof(double), C.st);
    ::ewos::note_launch(), sumsq_f32_kernel<<<1024, 256, 0, C.st>>>(X, count, C.ws->scal);
    double h = 0;
    cudaMemcpyAsync(&h, C.ws->scal, sizeof(double), cudaMemcpyDeviceToHost, C.st);
    cudaStreamSynchronize(C.st);
    return std::sqrt(h);
}

template <typename TP>
static const float* p_f32(const Ctx& C) {
    if (C.tb->precision == 32) return (const float*)C.tb->P;
    const int64_t cnt = (int64_t)C.E * C.n * C.m;
    ::ewos::note_launch(), narrow_f32_kernel<<<1024, 256, 0, C.st>>>((const double*)C.tb->P, C.ws->P32, cnt);
    return C.ws->P32;
}

// Lambda32 = P^T Q with Q = M P in FP32
template <typename TP>
static void assemble_mixed(const Ctx& C, const float* P32) {
    dim3 g((unsigned)((C.m + 255) / 256), (unsigned)C.n);
    ::ewos::note_launch(), formQ_kernel<float, float><<<g, 256, 0, C.st>>>(P32, C.ws->M, C.ws->Q32, (int)C.n, (int)C.m, C.D);
    sgemm<true>(C.st, (int)C.m, (int)C.m, (int)(C.E * C.n), 1.f, P32, C.m, C.ws->Q32, C.m, 0.f, C.ws->L32, C.m);
}

// y = (Lambda + alpha I) x with Lambda applied matrix-free in FP64; with u != NULL the Newton
// Jacobian term G^T diag(lam N'(u)) G is included
template <typename TP>
static void apply_op(const Ctx& C, const double* x, double alpha, const double* u, const double* nl, int nnl,
                     double* y) {
    const TP* P = (const TP*)C.tb->P;
    const int64_t rows = (int64_t)C.E * C.n;
    ::ewos::note_launch(), rowdot_kernel<TP><<<(int)((rows * 32 + 255) / 256), 256, 0, C.st>>>(P, rows, (int)C.m, x, C.ws->v, 0);
    ::ewos::note_launch(), formw_jv_kernel<<<(int)((C.n + 127) / 128), 128, 0, C.st>>>((int)C.n, C.D, C.ws->M, C.ws->v,
                                                                                      C.tb->lambda, u, u ? nl : nullptr,
                                                                                      u ? nnl : 0, C.ws->w);
    apply_PT<TP>(C, C.ws->w, y);
    if (alpha != 0.0) ::ewos::note_launch(), axpy_kernel<<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.m, alpha, x, y);
}

// x <- solution of (A) x = b by the FP32 factors plus FP64 refinement; A applied by apply_op
template <typename TP>
static ewos_status refine(const Ctx& C, const double* b, double* x, double alpha, const double* u, const double* nl,
                          int nnl, double rel_tol, int max_sweeps, int* sweeps, double* final_rel) {
    SolveWorkspace* ws = C.ws;
    const double nb = norm2(C, b, C.m);
    cudaMemsetAsync(x, 0, sizeof(double) * C.m, C.st);
    cudaMemcpyAsync(ws->r, b, sizeof(double) * C.m, cudaMemcpyDeviceToDevice, C.st);
    double rel = 1.0;
    int it = 0;
    while (it < max_sweeps) {
        cudaMemcpyAsync(ws->dx, ws->r, sizeof(double) * C.m, cudaMemcpyDeviceToDevice, C.st);
        ewos_status st = lu_solve_device<float>(ws->LU32, (int)C.m, (int)C.m, ws->lu, ws->dx, 1, C.st);
        if (st != EWOS_OK) return st;
        ::ewos::note_launch(), axpy_kernel<<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.m, 1.0, ws->dx, x);
        apply_op<TP>(C, x, alpha, u, nl, nnl, ws->y);
        cudaMemcpyAsync(ws->r, b, sizeof(double) * C.m, cudaMemcpyDeviceToDevice, C.st);
        ::ewos::note_launch(), axpy_kernel<<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.m, -1.0, ws->y, ws->r);
        ++it;
        rel = nb > 0 ? norm2(C, ws->r, C.m) / nb : 0.0;
        if (rel <= rel_tol) break;
    }
    *sweeps += it;
    if (final_rel) *final_rel = rel;
    return EWOS_OK;
}

static ewos_status factor32(const Ctx& C, const float* src, double alpha) {
    cudaMemcpyAsync(C.ws->LU32, src, sizeof(float) * C.m * C.m, cudaMemcpyDeviceToDevice, C.st);
    ::ewos::note_launch(), add_diag_kernel<float><<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.ws->LU32, (int)C.m, (int)C.m, alpha);
    bool sing = false;
    ewos_status s = lu_factor_device<float>(C.ws->LU32, (int)C.m, (int)C.m, C.ws->lu, C.st, &sing);
    if (s != EWOS_OK) return s;
    if (sing) { set_error("LU (FP32): zero pivot"); return EWOS_ESINGULAR; }
    return EWOS_OK;
}

constexpr double kRefineTol = 1e-10;
constexpr int kRefineMax = 40;

template <typename TP>
static ewos_status solve_mixed_t(ewos_toolbox* tb, const ewos_problem* pb, double rcond, double tol, int max_iter,
                                 ewos_solve_report* rep) {
    Ctx C{tb, tb->ws, pb->stream ? (cudaStream_t)pb->stream : tb->stream, tb->dim, tb->dim + 1, tb->n, tb->m, tb->p};
    SolveWorkspace* ws = tb->ws;
    const int64_t nrhs = pb->nrhs;
    auto t0 = std::chrono::steady_clock::now();
    const bool quasi = pb->nl_kind == EWOS_NL_QUASILINEAR, semi = pb->nl_kind == EWOS_NL_SEMILINEAR;
    const float* P32 = p_f32<TP>(C);
    ::ewos::note_launch(), coef_kernel<<<(int)((C.n + 127) / 128), 128, 0, C.st>>>((int)C.n, C.D, tb->lambda, ws->A,
                                                                                pb->b ? ws->b : nullptr,
                                                                                pb->c ? ws->c : nullptr, nullptr, 0,
                                                                                nullptr, ws->M);
    rep->iters = 0;
    rep->converged = 1;
    int sweeps = 0;
    double rel = 0.0;
    if (!quasi) {
        auto ta = std::chrono::steady_clock::now();
        if (tc_assemble_available()) {
            dim3 g((unsigned)((C.m + 255) / 256), (unsigned)C.n);
            ::ewos::note_launch(), formQ_kernel<float, float><<<g, 256, 0, C.st>>>(P32, ws->M, ws->Q32, (int)C.n, (int)C.m, C.D);
            ewos_status st = tc_assemble(P32, ws->Q32, ws->L32, (int)C.m, (int)C.m, (int)(C.E * C.n), C.st, kSplitTF32);
            if (st != EWOS_OK) return st;
        } else {
            assemble_mixed<TP>(C, P32);
        }
        const double alpha = rcond * frob32(C, ws->L32, C.m * C.m);
        rep->alpha = alpha;
        rep->ms_assemble = elapsed_ms(ta);
        if (!semi) {
            auto t1 = std::chrono::steady_clock::now();
            ewos_status st = factor32(C, ws->L32, alpha);
            if (st != EWOS_OK) return st;
            rep->ms_factor = elapsed_ms(t1);
            auto t2 = std::chrono::steady_clock::now();
            for (int64_t r = 0; r < nrhs; ++r) {
                residual<TP>(C, nullptr, ws->g + r * C.p, ws->f + r * C.n, nullptr, 0, 0.0, ws->y);   // -rhs
                cudaMemsetAsync(ws->rhs, 0, sizeof(double) * C.m, C.st);
                ::ewos::note_launch(), axpy_kernel<<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.m, -1.0, ws->y, ws->rhs);
                st = refine<TP>(C, ws->rhs, ws->s + r * C.m, alpha, nullptr, nullptr, 0, kRefineTol, kRefineMax, &sweeps,
                                &rel);
                if (st != EWOS_OK) return st;
                if (!(rel <= kRefineTol)) rep->converged = 0;
            }
            rep->iters = 1;
            rep->ms_solve = elapsed_ms(t2);
        } else {
            // Newton on R(s) + alpha s = 0; each step solved by the FP32 factors of the Jacobian
            // with FP64 refinement of the Jacobian system
            const double* nl = ws->nl;
            for (int64_t r = 0; r < nrhs; ++r) {
                double* s = ws->s + r * C.m;
                const double* g = ws->g + r * C.p;
                const double* f = ws->f + r * C.n;
                cudaMemsetAsync(s, 0, sizeof(double) * C.m, C.st);
                residual<TP>(C, s, g, f, nl, pb->nl_ncoef, alpha, ws->y);
                const double r0 = norm2(C, ws->y, C.m);
                double rn = r0;
                int it = 0;
                while (it < max_iter && rn > tol * r0) {
                    u_from_s(C, tb->P, tb->KH, tb->precision == 64, s, g, ws->u2);
                    dim3 gj((unsigned)((C.m + 255) / 256), (unsigned)C.n);
                    const TP* Gm = (const TP*)tb->P + (size_t)C.D * C.n * C.m;
                    ::ewos::note_launch(), jac_scale32_kernel<TP><<<gj, 256, 0, C.st>>>(Gm, ws->u2, tb->lambda, nl, pb->nl_ncoef,
                                                                                      ws->Jx32, (int)C.n, (int)C.m);
                    cudaMemcpyAsync(ws->LU32, ws->L32, sizeof(float) * C.m * C.m, cudaMemcpyDeviceToDevice, C.st);
                    const float* Gm32 = P32 + (size_t)C.D * C.n * C.m;
                    sgemm<true>(C.st, (int)C.m, (int)C.m, (int)C.n, 1.f, Gm32, C.m, ws->Jx32, C.m, 1.f, ws->LU32, C.m);
                    ::ewos::note_launch(), add_diag_kernel<float><<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(ws->LU32, (int)C.m, (int)C.m, alpha);
                    bool sing = false;
                    auto t1 = std::chrono::steady_clock::now();
                    ewos_status st = lu_factor_device<float>(ws->LU32, (int)C.m, (int)C.m, ws->lu, C.st, &sing);
                    if (st != EWOS_OK) return st;
                    if (sing) { set_error("LU (FP32): zero pivot"); return EWOS_ESINGULAR; }
                    rep->ms_factor += elapsed_ms(t1);
                    cudaMemcpyAsync(ws->rhs, ws->y, sizeof(double) * C.m, cudaMemcpyDeviceToDevice, C.st);
                    st = refine<TP>(C, ws->rhs, ws->x, alpha, ws->u2, nl, pb->nl_ncoef, 1e-10, 8, &sweeps, nullptr);
                    if (st != EWOS_OK) return st;
                    ::ewos::note_launch(), axpy_kernel<<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.m, -1.0, ws->x, s);
                    residual<TP>(C, s, g, f, nl, pb->nl_ncoef, alpha, ws->y);
                    rn = norm2(C, ws->y, C.m);
                    ++it;
                }
                rep->iters = std::max(rep->iters, it);
                if (!(rn <= tol * r0)) rep->converged = 0;
            }
        }
    } else {
        for (int64_t r = 0; r < nrhs; ++r) {
            const double* g = ws->g + r * C.p;
            const double* f = ws->f + r * C.n;
            double* s = ws->s + r * C.m;
            double* u = ws->u + r * C.n;
            cudaMemsetAsync(s, 0, sizeof(double) * C.m, C.st);
            u_from_s(C, tb->P, tb->KH, tb->precision == 64, s, g, u);
            int it = 0;
            bool conv = false;
            while (it < max_iter) {
                ::ewos::note_launch(), coef_kernel<<<(int)((C.n + 127) / 128), 128, 0, C.st>>>((int)C.n, C.D, tb->lambda, ws->A,
                                                                                            pb->b ? ws->b : nullptr,
                                                                                            pb->c ? ws->c : nullptr,
                                                                                            ws->nl, pb->nl_ncoef, u, ws->M);
                auto ta = std::chrono::steady_clock::now();
                if (tc_assemble_available()) {
                    dim3 gq((unsigned)((C.m + 255) / 256), (unsigned)C.n);
                    ::ewos::note_launch(), formQ_kernel<float, float><<<gq, 256, 0, C.st>>>(P32, ws->M, ws->Q32, (int)C.n, (int)C.m, C.D);
                    ewos_status st = tc_assemble(P32, ws->Q32, ws->L32, (int)C.m, (int)C.m, (int)(C.E * C.n), C.st, kSplitTF32);
                    if (st != EWOS_OK) return st;
                } else {
                    assemble_mixed<TP>(C, P32);
                }
                const double alpha = rcond * frob32(C, ws->L32, C.m * C.m);
                rep->alpha = alpha;
                rep->ms_assemble += elapsed_ms(ta);
                auto t1 = std::chrono::steady_clock::now();
                ewos_status st = factor32(C, ws->L32, alpha);
                if (st != EWOS_OK) return st;
                rep->ms_factor += elapsed_ms(t1);
                residual<TP>(C, nullptr, g, f, nullptr, 0, 0.0, ws->y);
                cudaMemsetAsync(ws->rhs, 0, sizeof(double) * C.m, C.st);
                ::ewos::note_launch(), axpy_kernel<<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.m, -1.0, ws->y, ws->rhs);
                st = refine<TP>(C, ws->rhs, s, alpha, nullptr, nullptr, 0, kRefineTol, kRefineMax, &sweeps, nullptr);
                if (st != EWOS_OK) return st;
                u_from_s(C, tb->P, tb->KH, tb->precision == 64, s, g, ws->u2);
                cudaMemsetAsync(ws->umax, 0, sizeof(unsigned long long), C.st);
                ::ewos::note_launch(), maxabsdiff_kernel<<<(int)((C.n + 255) / 256), 256, 0, C.st>>>(C.n, ws->u2, u, ws->umax);
                unsigned long long hm = 0;
                cudaMemcpyAsync(&hm, ws->umax, sizeof(hm), cudaMemcpyDeviceToHost, C.st);
                cudaMemcpyAsync(u, ws->u2, sizeof(double) * C.n, cudaMemcpyDeviceToDevice, C.st);
                cudaStreamSynchronize(C.st);
                ++it;
                double du;
                memcpy(&du, &hm, sizeof(du));
                if (du <= tol) { conv = true; break; }
            }
            rep->iters = std::max(rep->iters, it);
            if (!conv) rep->converged = 0;
        }
    }
    for (int64_t r = 0; r < nrhs; ++r)
        u_from_s(C, tb->P, tb->KH, tb->precision == 64, ws->s + r * C.m, ws->g + r * C.p, ws->u + r * C.n);
    if (!quasi) {
        const int64_t r = nrhs - 1;
        residual<TP>(C, ws->s + r * C.m, ws->g + r * C.p, ws->f + r * C.n, semi ? ws->nl : nullptr,
                     semi ? pb->nl_ncoef : 0, rep->alpha, ws->y);
        rep->residual = norm2(C, ws->y, C.m);
    }
    rep->refine_iters = sweeps;
    EWOS_CUDA_TRY(cudaStreamSynchronize(C.st));
    EWOS_CUDA_TRY(cudaGetLastError());
    rep->ms_total = elapsed_ms(t0);
    return rep->converged ? EWOS_OK : EWOS_ENOCONV;
}

ewos_status solve_mixed(ewos_toolbox* tb, const ewos_problem* pb, double rcond, double tol, int max_iter,
                        ewos_solve_report* rep) {
    return tb->precision == 64 ? solve_mixed_t<double>(tb, pb, rcond, tol, max_iter, rep)
                               : solve_mixed_t<float>(tb, pb, rcond, tol, max_iter, rep);
}

}  // namespace ewos

using namespace ewos;

extern "C" ewos_status ewos_solve(ewos_toolbox* tb, const ewos_problem* pb, double* u_out, double* s_out,
                                  int outputs_on_device, ewos_solve_report* rep_out) {
    if (!tb || !pb || !u_out || !pb->A || !pb->f || !pb->g || pb->nrhs < 1) {
        set_error("ewos_solve: need toolbox, problem with A, f, g, nrhs >= 1, and u_out");
        return EWOS_EINVAL;
    }
    if (pb->nl_kind < 0 || pb->nl_kind > 2 || (pb->nl_kind != EWOS_NL_NONE && (!pb->nl_coef || pb->nl_ncoef < 1 || pb->nl_ncoef > 64))) {
        set_error("ewos_solve: nonlinearity needs 1..64 coefficients");
        return EWOS_EINVAL;
    }
    if (pb->mode != EWOS_SOLVE_FP64 && pb->mode != EWOS_SOLVE_MIXED) { set_error("ewos_solve: unknown mode"); return EWOS_EINVAL; }
    cudaStream_t st = pb->stream ? (cudaStream_t)pb->stream : tb->stream;
    AllocStream as(st);
    ewos_status s = ensure_workspace(tb, pb->nrhs, pb->mode == EWOS_SOLVE_MIXED);
    if (s != EWOS_OK) return s;
    SolveWorkspace* ws = tb->ws;
    const cudaMemcpyKind k = pb->inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const int D = tb->dim;
    EWOS_CUDA_TRY(cudaMemcpyAsync(ws->A, pb->A, sizeof(double) * tb->n * D * D, k, st));
    if (pb->b) EWOS_CUDA_TRY(cudaMemcpyAsync(ws->b, pb->b, sizeof(double) * tb->n * D, k, st));
    if (pb->c) EWOS_CUDA_TRY(cudaMemcpyAsync(ws->c, pb->c, sizeof(double) * tb->n, k, st));
    EWOS_CUDA_TRY(cudaMemcpyAsync(ws->f, pb->f, sizeof(double) * tb->n * pb->nrhs, k, st));
    EWOS_CUDA_TRY(cudaMemcpyAsync(ws->g, pb->g, sizeof(double) * tb->p * pb->nrhs, k, st));
    if (pb->nl_kind != EWOS_NL_NONE)
        EWOS_CUDA_TRY(cudaMemcpyAsync(ws->nl, pb->nl_coef, sizeof(double) * pb->nl_ncoef, cudaMemcpyHostToDevice, st));
    const double rcond = pb->rcond < 0 ? 3e-2 : pb->rcond;
    const double tol = pb->tol > 0 ? pb->tol : 1e-10;
    const int max_iter = pb->max_iter > 0 ? pb->max_iter : (pb->nl_kind == EWOS_NL_QUASILINEAR ? 100 : 30);
    ewos_solve_report rep{};
    if (pb->mode == EWOS_SOLVE_FP64)
        s = tb->precision == 64 ? solve_fp64<double>(tb, pb, rcond, tol, max_iter, &rep)
                                : solve_fp64<float>(tb, pb, rcond, tol, max_iter, &rep);
    else
        s = solve_mixed(tb, pb, rcond, tol, max_iter, &rep);
    if (s != EWOS_OK && s != EWOS_ENOCONV) return s;
    const cudaMemcpyKind ko = outputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    EWOS_CUDA_TRY(cudaMemcpyAsync(u_out, ws->u, sizeof(double) * tb->n * pb->nrhs, ko, st));
    if (s_out) EWOS_CUDA_TRY(cudaMemcpyAsync(s_out, ws->s, sizeof(double) * tb->m * pb->nrhs, ko, st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(st));
    if (rep_out) *rep_out = rep;
    return s;
}
