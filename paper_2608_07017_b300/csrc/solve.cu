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
// matrix.  Triangular solves with the factors are one dataflow launch (row blocks published
// through flags, CTAs ordered by tickets).  Every grid barrier and flag wait spins a bounded
// number of times; on a timeout the kernels return and the call reports EWOS_ETIMEOUT.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "pdl.cuh"
#include "tf32.cuh"
#include "sgemm.cuh"
#include "solve_internal.hpp"
#include "toolbox.hpp"

namespace ewos {

// ------------------------------------------------------------------ bounded grid barrier
struct GridBarrier {
    unsigned int count;
    unsigned int gen;
    int err;
    int singular;
    unsigned long long maxl_bits;   // largest |multiplier| of an unpivoted factorisation (double bits)
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

struct TcScratch;   // mixed.cu: operand transposes of one caller
void tc_scratch_free(TcScratch* t);
ewos_status tc_assemble(const float* A_km, const float* B_km, float* C, int M, int N, int K, cudaStream_t st,
                        bool split, TcScratch** owned, bool sym = false, bool f16 = false, uint64_t akey = 0,
                        const float* dscale = nullptr, const float* amax = nullptr);
ewos_status tc_update_enqueue(const float* A, int64_t lda, const float* B, int64_t ldb, float* C, int64_t ldc, int M,
                              int N, int K, cudaStream_t st, TcScratch** owned, bool presplit = false, int a_off = 0,
                              int b_off = 0, bool f16 = true);
ewos_status tc_update_reserve(int max_mn, int k, cudaStream_t st, TcScratch** owned);
ewos_status tc_update_lshape_enqueue(float* C, int64_t ldc, int rest, int band, int K, cudaStream_t st,
                                     TcScratch** owned);
ewos_status tc_assemble_pq(const float* P, const double* Mc, int n, int m, int D, float* C, cudaStream_t st,
                           TcScratch** owned, bool sym = false, bool f16 = true, uint64_t pkey = 0,
                           const float* pmax = nullptr);
void tc_update_operands(TcScratch* t, float** a_hi, float** a_lo, float** b_hi, float** b_lo);
ewos_status tc_update_check(TcScratch* t, cudaStream_t st);
bool tc_assemble_available();

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

// Q[j][i][col] = sum_k M_i[j][k] P[k][i][col], computed in TQ: FP64 for the FP64 path; FP32 for
// the FP32 copy of the mixed path (Q is stored in FP32 there, and FP64 arithmetic would make
// this pass over P compute-bound on a part whose FP64 rate is a small fraction of its FP32 rate)
template <typename TP, typename TQ>
__global__ void formQ_kernel(const TP* __restrict__ P, const double* __restrict__ M, TQ* __restrict__ Q,
                             int n, int m, int D) {
    const int i = blockIdx.y;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= m) return;
    const int E = D + 1;
    const size_t nm = (size_t)n * m;
    TQ pv[4];
    for (int k = 0; k < E; ++k) pv[k] = (TQ)P[k * nm + (size_t)i * m + col];
    const double* Mi = M + (size_t)i * E * E;
    for (int j = 0; j < E; ++j) {
        TQ acc = TQ(0);
        for (int k = 0; k < E; ++k) acc += (TQ)Mi[j * E + k] * pv[k];
        Q[j * nm + (size_t)i * m + col] = acc;
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

// sum of squares of an FP32 array (for alpha = rcond ||Lambda||_F): each thread's partial sum in
// FP32 (a few dozen terms; FP64 per element made this pass FP64-bound), widened for the reduction
__global__ void sumsq_f32_kernel(const float* __restrict__ X, int64_t count, double* __restrict__ out) {
    float part = 0.f;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
        part = fmaf(X[t], X[t], part);
    double acc = part;
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
// cluster's CTAs and kept in their shared memory.  Per column, every CTA publishes (parity double
// buffered) its pivot candidate, a copy of that candidate row and, for the CTA owning it, a copy
// of the row the pivot will replace; one hardware cluster barrier; then every CTA reads the
// candidates and the two rows through distributed shared memory, swaps locally and applies the
// rank-1 update to its own rows.
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
    __shared__ T s_cval[2];
    __shared__ int s_crow[2];
    __shared__ T s_pub[2][64];      // published candidate row
    __shared__ T s_old[2][64];      // published copy of row prow0 (owner only)
    __shared__ T s_piv[64];
    __shared__ T s_rep[64];
    __shared__ int s_prow;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int r0 = kb + rank * chunk;
    const int r1 = min(mtot, r0 + chunk);
    const int nr = max(0, r1 - r0);
    for (int t = threadIdx.x; t < nr * nb; t += blockDim.x) tile[t] = A[(size_t)(r0 + t / nb) * lda + kb + t % nb];
    __syncthreads();
    for (int jj = 0; jj < nb; ++jj) {
        const int par = jj & 1;
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
            best = __shfl_sync(0xffffffffu, best, 0);
            brow = __shfl_sync(0xffffffffu, brow, 0);
            if (lane == 0) { s_cval[par] = best; s_crow[par] = brow; }
            if (brow != 0x7fffffff)
                for (int cc = lane; cc < nb; cc += 32) s_pub[par][cc] = tile[(brow - r0) * nb + cc];
        } else if (warp == 1 && prow0 >= r0 && prow0 < r1) {
            for (int cc = lane; cc < nb; cc += 32) s_old[par][cc] = tile[(prow0 - r0) * nb + cc];
        }
        cluster.sync();
        if (warp == 0) {
            T best = T(-1);
            int brow = 0x7fffffff, win = 0;
            if (lane < ncta) {
                const T v = cluster.map_shared_rank(s_cval, lane)[par];
                const int rw = cluster.map_shared_rank(s_crow, lane)[par];
                if (rw != 0x7fffffff) { best = v; brow = rw; win = lane; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T ob = __shfl_down_sync(0xffffffffu, best, o);
                const int orw = __shfl_down_sync(0xffffffffu, brow, o);
                const int ow = __shfl_down_sync(0xffffffffu, win, o);
                if (ob > best || (ob == best && orw < brow)) { best = ob; brow = orw; win = ow; }
            }
            win = __shfl_sync(0xffffffffu, win, 0);
            brow = __shfl_sync(0xffffffffu, brow, 0);
            const T* pr = &cluster.map_shared_rank(s_pub, win)[par][0];
            const int ow0 = (prow0 - kb) / chunk;
            const T* orow = &cluster.map_shared_rank(s_old, ow0)[par][0];
            for (int cc = lane; cc < nb; cc += 32) { s_piv[cc] = pr[cc]; s_rep[cc] = orow[cc]; }
            if (lane == 0) {
                s_prow = brow;
                if (rank == 0) {
                    ipiv[prow0] = brow;
                    if (best == T(0)) bar->singular = 1;
                }
            }
        }
        __syncthreads();
        const int prow = s_prow;
        if (prow != prow0) {
            if (prow0 >= r0 && prow0 < r1)
                for (int cc = threadIdx.x; cc < nb; cc += blockDim.x) tile[(prow0 - r0) * nb + cc] = s_piv[cc];
            if (prow >= r0 && prow < r1)
                for (int cc = threadIdx.x; cc < nb; cc += blockDim.x) tile[(prow - r0) * nb + cc] = s_rep[cc];
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

// FP32 panel factorisation with one panel row per thread.  The cluster's CTAs own consecutive
// chunks of at most kRegThreads rows; each thread holds its row's 64 panel entries in registers.
// Rows are not moved during the panel: each thread tracks the position its row occupies under
// the interchanges so far (the interchange of column j swaps the positions j and that of the
// pivot row), and writes its row to that position at the end.  A row's multipliers go to shared
// memory as they are formed, so the rank-1 update can run over all 64 registers unmasked (the
// entries left of the current column are dead).  Per column: arg-max over the warp by shuffles,
// the warp winners' rows staged in shared memory, arg-max over the warps by warp 0, which pushes
// its CTA's candidate (value, position, row) into every CTA of the cluster by distributed shared
// memory stores (parity double buffered); one cluster barrier; every warp then picks the winner
// from its own shared memory.
constexpr int kRegThreads = 512;
constexpr int kRegCluster = 16;

__device__ __forceinline__ void argmax_step(float& v, int& r, int& w, int o) {
    const float ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int orow = __shfl_xor_sync(0xffffffffu, r, o);
    const int ow = __shfl_xor_sync(0xffffffffu, w, o);
    if (ov > v || (ov == v && orow < r)) { v = ov; r = orow; w = ow; }
}

// row[j] for a run-time j: a binary tree of selects on the bits of j
__device__ __forceinline__ float pick64(const float (&row)[kNB], int j) {
    float t32[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) t32[c] = (j & 1) ? row[2 * c + 1] : row[2 * c];
#pragma unroll
    for (int c = 0; c < 16; ++c) t32[c] = (j & 2) ? t32[2 * c + 1] : t32[2 * c];
#pragma unroll
    for (int c = 0; c < 8; ++c) t32[c] = (j & 4) ? t32[2 * c + 1] : t32[2 * c];
#pragma unroll
    for (int c = 0; c < 4; ++c) t32[c] = (j & 8) ? t32[2 * c + 1] : t32[2 * c];
#pragma unroll
    for (int c = 0; c < 2; ++c) t32[c] = (j & 16) ? t32[2 * c + 1] : t32[2 * c];
    return (j & 32) ? t32[1] : t32[0];
}

constexpr size_t panel_reg_smem(int threads) { return sizeof(float) * (size_t)kNB * threads; }

__global__ void __launch_bounds__(kRegThreads, 1) lu_panel_reg_kernel(float* __restrict__ A, int lda, int mtot, int kb,
                                                                     int nb, int chunk, int* __restrict__ ipiv,
                                                                     GridBarrier* __restrict__ bar) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int ncta = (int)cluster.num_blocks();
    constexpr int kW = kRegThreads / 32;
    extern __shared__ __align__(16) float s_l[];                    // [64][blockDim] multipliers
    __shared__ __align__(16) float s_wrow[kW][kNB];                 // warp winners' rows (local)
    __shared__ float s_wval[kW];
    __shared__ int s_wrw[kW];
    __shared__ __align__(16) float s_cand[2][kRegCluster][kNB];     // CTA candidates' rows (pushed)
    __shared__ float s_cval[2][kRegCluster];
    __shared__ int s_crow[2][kRegCluster];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5, nt = blockDim.x;
    const int r0 = kb + rank * chunk;
    const int gr = r0 + tid;
    const bool mine = tid < chunk && gr < mtot;
    float row[kNB];
#pragma unroll
    for (int c = 0; c < kNB; ++c) row[c] = (mine && c < nb) ? A[(size_t)gr * lda + kb + c] : 0.f;
    int pos = gr;          // current position of this thread's row
    int mycol = nb;        // column at which the row became a pivot row
    float cur = row[0];    // row[jj] of the current column
    for (int jj = 0; jj < nb; ++jj) {
        const int par = jj & 1;
        const int prow0 = kb + jj;
        const bool cand = mine && pos >= prow0;
        float bv = cand ? fabsf(cur) : -1.f;
        int br = cand ? pos : 0x7fffffff, bw = warp;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) argmax_step(bv, br, bw, o);
        if (cand && br == pos) {
            float4* dst = reinterpret_cast<float4*>(&s_wrow[warp][0]);
#pragma unroll
            for (int q = 0; q < kNB / 4; ++q) dst[q] = make_float4(row[4 * q], row[4 * q + 1], row[4 * q + 2], row[4 * q + 3]);
        }
        if (lane == 0) { s_wval[warp] = bv; s_wrw[warp] = br; }
        __syncthreads();
        if (warp == 0) {
            float v = lane < nw ? s_wval[lane] : -1.f;
            int r = lane < nw ? s_wrw[lane] : 0x7fffffff, w = lane;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) argmax_step(v, r, w, o);
            if (lane < ncta) {
                cluster.map_shared_rank(&s_cval[par][0], lane)[rank] = v;
                cluster.map_shared_rank(&s_crow[par][0], lane)[rank] = r;
            }
            const float4* src = reinterpret_cast<const float4*>(&s_wrow[w < nw ? w : 0][0]);
            for (int i = lane; i < ncta * (kNB / 4); i += 32) {
                const int d = i / (kNB / 4), q = i % (kNB / 4);
                reinterpret_cast<float4*>(cluster.map_shared_rank(&s_cand[par][rank][0], d))[q] = src[q];
            }
        }
        cluster.sync();
        float v = lane < ncta ? s_cval[par][lane] : -1.f;
        int r = lane < ncta ? s_crow[par][lane] : 0x7fffffff, src = lane;
        if (r == 0x7fffffff) v = -1.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) argmax_step(v, r, src, o);
        if (tid == 0 && rank == 0) {
            ipiv[prow0] = r;
            if (v == 0.f) bar->singular = 1;
        }
        if (mine) {
            if (pos == r) { pos = prow0; mycol = jj; }
            else if (pos == prow0) pos = r;
        }
        const float* p = &s_cand[par][src][0];
        if (mine && pos > prow0) {
            const float piv = p[jj];
            const float l = cur * (piv != 0.f ? 1.f / piv : 0.f);
            s_l[jj * nt + tid] = l;
            const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
            for (int q = 0; q < kNB / 4; ++q) {
                const float4 pv = p4[q];
                row[4 * q] = fmaf(-l, pv.x, row[4 * q]);
                row[4 * q + 1] = fmaf(-l, pv.y, row[4 * q + 1]);
                row[4 * q + 2] = fmaf(-l, pv.z, row[4 * q + 2]);
                row[4 * q + 3] = fmaf(-l, pv.w, row[4 * q + 3]);
            }
        }
        cur = pick64(row, (jj + 1) & (kNB - 1));
    }
    __syncthreads();
    if (mine) {
        float* out = A + (size_t)pos * lda + kb;
#pragma unroll
        for (int c = 0; c < kNB; ++c)
            if (c < nb) out[c] = c < mycol ? s_l[c * nt + tid] : row[c];
    }
    cluster.sync();
}

static bool launch_panel_reg(float* A, int lda, int m, int kb, int nb, int rows, int* ipiv, GridBarrier* bar,
                             cudaStream_t st, bool check) {
    constexpr int cl = kRegCluster;
    const int chunk = (rows + cl - 1) / cl;
    const int threads = std::max(32, (chunk + 31) / 32 * 32);
    const size_t smem = panel_reg_smem(threads);
    auto kfn = lu_panel_reg_kernel;
    if (check && (cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
                  cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_reg_smem(kRegThreads)) !=
                      cudaSuccess)) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cl);
    lc.blockDim = dim3(threads);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    int nclusters = 0;
    if (check && (cudaOccupancyMaxActiveClusters(&nclusters, kfn, &lc) != cudaSuccess || nclusters < 1)) {
        cudaGetLastError();
        return false;
    }
    ::ewos::note_launch();
    if (cudaLaunchKernelEx(&lc, kfn, A, lda, m, kb, nb, chunk, ipiv, bar) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// Inverses of the 64 x 64 diagonal blocks of the factors (unit lower part and upper part), one CTA
// per block: thread j solves the block against e_j.  Dinv [nbk][2][64][64].
template <typename T>
__global__ void diag_inverse_kernel(const T* __restrict__ LU, int lda, int m, T* __restrict__ Dinv) {
    __shared__ T B[64][65];
    const int t = blockIdx.x, ib = t * 64, w = min(64, m - ib);
    for (int q = threadIdx.x; q < 64 * 64; q += blockDim.x) {
        const int i = q >> 6, k = q & 63;
        B[i][k] = (i < w && k < w) ? LU[(size_t)(ib + i) * lda + ib + k] : T(0);
    }
    __syncthreads();
    const int j = threadIdx.x;
    T* Li = Dinv + (size_t)t * 2 * 64 * 64;
    T* Ui = Li + 64 * 64;
    if (j < 64) {
        T col[64];
        // unit lower: solve L y = e_j
        for (int i = 0; i < 64; ++i) {
            T acc = (i == j) ? T(1) : T(0);
            for (int k = 0; k < i; ++k) acc -= B[i][k] * col[k];
            col[i] = i < w ? acc : T(0);
        }
        for (int i = 0; i < 64; ++i) Li[i * 64 + j] = col[i];
        // upper with diagonal: solve U y = e_j
        for (int i = 63; i >= 0; --i) {
            if (i >= w) { col[i] = T(0); continue; }
            T acc = (i == j) ? T(1) : T(0);
            for (int k = i + 1; k < w; ++k) acc -= B[i][k] * col[k];
            col[i] = acc / B[i][i];
        }
        for (int i = 0; i < 64; ++i) Ui[i * 64 + j] = col[i];
    }
}

struct LuScratch {
    void* pub = nullptr;
    size_t pub_bytes = 0;
    GridBarrier* bar = nullptr;
    int* ipiv = nullptr;
    int* perm = nullptr;        // [m] final row order
    int* swp = nullptr;         // [2 * 128 + 1] composed interchanges of one panel
    double* tmp = nullptr;      // [m * nrhs] permuted right-hand sides
    void* dinv = nullptr;       // [nbk][2][64][64] inverses of the diagonal blocks (T)
    void* diagb = nullptr;      // [nbk][64][64] factored diagonal blocks of the unpivoted path (T)
    unsigned int* flow = nullptr;   // state of the dataflow triangular solve (flow_state_words)
    int panel_blocks = 0;
};

template <typename T>
static ewos_status lu_factor_device(T* A, int m, int lda, LuScratch& S, cudaStream_t st, bool* singular) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256;
    EWOS_CUDA_TRY(cudaMemsetAsync(S.bar, 0, sizeof(GridBarrier), st));
    // Panel variant, chosen (attributes set, co-residency checked) on the first and largest panel
    // and kept for the rest: 0 register panel, 16 / 8 shared-memory cluster panel, -1 cooperative.
    int plan = -2;
    for (int kb = 0; kb < m; kb += kNB) {
        const int nb = std::min(kNB, m - kb);
        const int rows = m - kb;
        int blocks = std::min(nsm, std::max(1, (rows + 7) / 8));
        const int chunk = (rows + blocks - 1) / blocks;
        blocks = (rows + chunk - 1) / chunk;
        const bool first = plan == -2;
        bool done_cluster = false;
        if (std::is_same<T, float>::value && (first || plan == 0) &&
            (rows + kRegCluster - 1) / kRegCluster <= kRegThreads) {
            done_cluster = launch_panel_reg(reinterpret_cast<float*>(A), lda, m, kb, nb, rows, S.ipiv, S.bar, st, first);
            if (done_cluster) plan = 0;
        }
        for (int cl : {16, 8}) {
            if (done_cluster) break;
            if (!first && plan != cl) continue;
            if (!first) {
                const int cchunk = (rows + cl - 1) / cl;
                const size_t csmem = sizeof(T) * (size_t)cchunk * nb;
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
                ::ewos::note_launch();
                EWOS_CUDA_TRY(cudaLaunchKernelEx(&lc, lu_panel_cluster_kernel<T>, A, lda, m, kb, nb, cchunk, S.ipiv, S.bar));
                done_cluster = true;
                break;
            }
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
                plan = cl;
                break;
            }
            cudaGetLastError();
        }
        if (!done_cluster) {
        plan = -1;
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
    ::ewos::note_launch(), diag_inverse_kernel<T><<<(m + 63) / 64, 64, 0, st>>>(A, lda, m, (T*)S.dinv);
    GridBarrier hb{};
    EWOS_CUDA_TRY(cudaMemcpyAsync(&hb, S.bar, sizeof(hb), cudaMemcpyDeviceToHost, st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(st));
    if (hb.err) { set_error("LU panel: grid barrier timed out"); return EWOS_ETIMEOUT; }
    *singular = hb.singular != 0;
    return EWOS_OK;
}


// ------------------------------------------------------------------ LU without interchanges
// Blocked LU with the diagonal pivots, accepted only when it equals the partial-pivoting
// factorisation: partial pivoting picks the diagonal at every column exactly when every
// multiplier satisfies |l| <= 1, so the largest |l| is tracked and the caller refactors with
// interchanges when it exceeds 1 (or a pivot is zero).  Per 64-column panel: one CTA factors the
// diagonal block and forms the inverses of its two triangles; many CTAs then form
// L21 = A21 U11^-1 and U12 = L11^-1 A12 as products with those inverses; the trailing update is
// a GEMM (tensor cores for FP32 from 256 rows).  Factored diagonal blocks go to a side buffer and
// are written into the matrix after the last panel; their inverses go straight to the buffer
// the triangular solves use.
constexpr int kNpThreads = 256;

// max that keeps a NaN (fmax drops it): a NaN multiplier must reject the unpivoted factors.
// Kept in the factors' precision per element (FP64 arithmetic is slow on this part) and widened
// once per warp for the device-wide maximum.
template <typename T>
__device__ __forceinline__ T nanmax(T m, T v) { return (v > m || v != v) ? v : m; }

template <typename T>
__device__ __forceinline__ void publish_maxl(T mx, GridBarrier* bar) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = nanmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const double w = (double)mx;
    if ((threadIdx.x & 31) == 0 && (w > 0.0 || w != w)) atomicMax(&bar->maxl_bits, (unsigned long long)__double_as_longlong(w));
}

// Diagonal block of one panel, factored with the diagonal pivots by one CTA in shared memory,
// blocked by 16 columns so that few CTA-wide barriers sit on this latency-bound path:
//   for each 16-column sub-panel: one warp eliminates it (rows from the sub-panel's diagonal
//   down, two rows per lane, pivot rows passed by shuffles; multipliers l = a / u_jj), the
//   16 x 16 unit lower triangle is applied to the sub-panel's row to the right (U12, a thread
//   per column), and the rows and columns beyond it get the rank-16 update a -= L21 U12.
// Then the inverses of the unit lower and of the upper triangle by recursive doubling: each
// 16 x 16 diagonal tile inverted by substitution (a lane per column), then the off-diagonal
// blocks at 32 and 64 from  X21 = -inv(L22) L21 inv(L11)  and  X12 = -inv(U11) U12 inv(U22).
// Writes the factored block to diag_out [64][64] and the inverses to dinv_blk [2][64][64].
template <typename T>
constexpr size_t diag_smem() { return sizeof(T) * (3 * kNB * (kNB + 1) + 2 * 32 * 33); }

template <typename T>
__global__ void __launch_bounds__(kNpThreads) lu_diag_factor_kernel(const T* __restrict__ A, int lda, int kb, int nb,
                                                                    T* __restrict__ diag_out, T* __restrict__ dinv_blk,
                                                                    GridBarrier* __restrict__ bar) {
    constexpr int LD = kNB + 1;              // row stride of the shared tiles
    extern __shared__ __align__(16) unsigned char df_sm[];
    T* F = reinterpret_cast<T*>(df_sm);      // [64][65] the block, factored in place
    T* Li = F + kNB * LD;                    // [64][65] inverse of the unit lower triangle
    T* Ui = Li + kNB * LD;                   // [64][65] inverse of the upper triangle
    T* Tb = Ui + kNB * LD;                   // [2][32][33] products of the doubling steps
    __shared__ T rU[kNB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    pdl_trigger();
    pdl_wait();                               // the block comes from the preceding update
    {
        // element e = tid + 256 s: row tid / 64 + 4 s, column tid % 64; all loads in flight first
        constexpr int kE = kNB * kNB / kNpThreads;
        const int c = tid & 63, i0 = tid >> 6;
        T v[kE];
#pragma unroll
        for (int s2 = 0; s2 < kE; ++s2) {
            const int i = i0 + 4 * s2;
            v[s2] = (i < nb && c < nb) ? A[(size_t)(kb + i) * lda + kb + c] : (i == c ? T(1) : T(0));
        }
#pragma unroll
        for (int s2 = 0; s2 < kE; ++s2) {
            const int i = i0 + 4 * s2;
            F[i * LD + c] = v[s2];
            Li[i * LD + c] = T(0);
            Ui[i * LD + c] = T(0);
        }
    }
    __syncthreads();
    T mx = T(0);
    int zero = 0;
    for (int p = 0; p < 4; ++p) {
        const int c0 = 16 * p, nr = kNB - c0;
        if (warp == 0) {
            // rows c0 + lane and c0 + lane + 32 of columns c0 .. c0 + 15
            const bool v0 = lane < nr, v1 = lane + 32 < nr;
            T a0[16], a1[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                a0[k] = v0 ? F[(c0 + lane) * LD + c0 + k] : T(0);
                a1[k] = v1 ? F[(c0 + lane + 32) * LD + c0 + k] : T(0);
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const T piv = __shfl_sync(0xffffffffu, a0[j], j);
                const T r = piv != T(0) ? T(1) / piv : T(0);
                if (lane == 0) {
                    rU[c0 + j] = r;
                    zero |= piv == T(0);
                }
                const bool b0 = v0 && lane > j;
                if (b0) {
                    a0[j] *= r;
                    mx = nanmax(mx, fabs(a0[j]));
                }
                if (v1) {
                    a1[j] *= r;
                    mx = nanmax(mx, fabs(a1[j]));
                }
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    if (jj > j) {
                        const T u = __shfl_sync(0xffffffffu, a0[jj], j);
                        if (b0) a0[jj] = fma(-a0[j], u, a0[jj]);
                        if (v1) a1[jj] = fma(-a1[j], u, a1[jj]);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                if (v0) F[(c0 + lane) * LD + c0 + k] = a0[k];
                if (v1) F[(c0 + lane + 32) * LD + c0 + k] = a1[k];
            }
        }
        __syncthreads();
        const int ncol = kNB - c0 - 16;
        if (tid < ncol) {                     // U12 = inv(L11) A12, a thread per column
            const int col = c0 + 16 + tid;
            T x[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) x[k] = F[(c0 + k) * LD + col];
#pragma unroll
            for (int k = 0; k < 16; ++k)
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (i > k) x[i] = fma(-F[(c0 + i) * LD + c0 + k], x[k], x[i]);
#pragma unroll
            for (int k = 0; k < 16; ++k) F[(c0 + k) * LD + col] = x[k];
        }
        __syncthreads();
        if (ncol > 0) {                       // A22 -= L21 U12 over rows and columns c0 + 16 ..
            const int col = tid & 63;
            if (col >= c0 + 16) {
                T u[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) u[k] = F[(c0 + k) * LD + col];
                for (int i = c0 + 16 + (tid >> 6); i < kNB; i += kNpThreads / kNB) {
                    T acc = F[i * LD + col];
#pragma unroll
                    for (int k = 0; k < 16; ++k) acc = fma(-F[i * LD + c0 + k], u[k], acc);
                    F[i * LD + col] = acc;
                }
            }
            __syncthreads();
        }
    }
    for (int e = tid; e < kNB * kNB; e += kNpThreads) diag_out[e] = F[(e >> 6) * LD + (e & 63)];
    // inverses of the 16 x 16 diagonal tiles: warps 0-3 the lower ones, 4-7 the upper ones
    {
        const int t = warp & 3, o = 16 * t, c = lane;
        if (c < 16) {
            T x[16];
            if (warp < 4) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    T sum = (i == c) ? T(1) : T(0);
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        if (k < i) sum = fma(-F[(o + i) * LD + o + k], x[k], sum);
                    x[i] = sum;
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) Li[(o + i) * LD + o + c] = x[i];
            } else {
#pragma unroll
                for (int ii = 0; ii < 16; ++ii) {
                    const int i = 15 - ii;
                    T sum = (i == c) ? T(1) : T(0);
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        if (k > i) sum = fma(-F[(o + i) * LD + o + k], x[k], sum);
                    x[i] = sum * rU[o + i];
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) Ui[(o + i) * LD + o + c] = x[i];
            }
        }
    }
    __syncthreads();
    // doubling to 32: four 16 x 16 tasks (lower pairs 0, 1 and upper pairs 0, 1), four elements
    // per thread (rows r0 + 4 s of column c); T = L21 inv(L11) (T = U12 inv(U22)), then
    // X21 = -inv(L22) T (X12 = -inv(U11) T).  The k loop is outside the thread's rows, so each
    // value of the right factor is read once for all of them (the row values are broadcasts):
    // these products are bound by shared-memory reads.  Each sum keeps its order over k.
    {
        const int task = tid >> 6, up = task >> 1, a = 32 * (task & 1), b = a + 16;
        const int r0 = (tid & 63) >> 4, c = tid & 15;
        T* Tt = Tb + task * 16 * 17;
        {
            const T* Fr = up ? F + a * LD + b : F + b * LD + a;          // rows of L21 (U12)
            const T* Xc = up ? Ui + b * LD + b + c : Li + a * LD + a + c; // column c of inv(L11) (inv(U22))
            T sum[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const T x = Xc[k * LD];
#pragma unroll
                for (int s4 = 0; s4 < 4; ++s4) sum[s4] = fma(Fr[(r0 + 4 * s4) * LD + k], x, sum[s4]);
            }
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4) Tt[(r0 + 4 * s4) * 17 + c] = sum[s4];
        }
        __syncthreads();
        {
            T* Xi = up ? Ui + a * LD + a : Li + b * LD + b;                // inv(U11) (inv(L22))
            T* Xo = up ? Ui + a * LD + b + c : Li + b * LD + a + c;        // the block written
            T sum[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const T t = Tt[k * 17 + c];
#pragma unroll
                for (int s4 = 0; s4 < 4; ++s4) sum[s4] = fma(Xi[(r0 + 4 * s4) * LD + k], t, sum[s4]);
            }
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4) Xo[(r0 + 4 * s4) * LD] = -sum[s4];
        }
        __syncthreads();
    }
    // doubling to 64: the lower and the upper 32 x 32 task, eight elements per thread (rows
    // r0 + 4 s of column c), as above
    {
        const int up = tid >> 7, a = 0, b = 32;
        const int r0 = (tid & 127) >> 5, c = tid & 31;
        T* Tt = Tb + up * 32 * 33;
        {
            const T* Fr = up ? F + a * LD + b : F + b * LD + a;
            const T* Xc = up ? Ui + b * LD + b + c : Li + a * LD + a + c;
            T sum[8];
#pragma unroll
            for (int s8 = 0; s8 < 8; ++s8) sum[s8] = T(0);
#pragma unroll 8
            for (int k = 0; k < 32; ++k) {
                const T x = Xc[k * LD];
#pragma unroll
                for (int s8 = 0; s8 < 8; ++s8) sum[s8] = fma(Fr[(r0 + 4 * s8) * LD + k], x, sum[s8]);
            }
#pragma unroll
            for (int s8 = 0; s8 < 8; ++s8) Tt[(r0 + 4 * s8) * 33 + c] = sum[s8];
        }
        __syncthreads();
        {
            T* Xi = up ? Ui + a * LD + a : Li + b * LD + b;
            T* Xo = up ? Ui + a * LD + b + c : Li + b * LD + a + c;
            T sum[8];
#pragma unroll
            for (int s8 = 0; s8 < 8; ++s8) sum[s8] = T(0);
#pragma unroll 8
            for (int k = 0; k < 32; ++k) {
                const T t = Tt[k * 33 + c];
#pragma unroll
                for (int s8 = 0; s8 < 8; ++s8) sum[s8] = fma(Xi[(r0 + 4 * s8) * LD + k], t, sum[s8]);
            }
#pragma unroll
            for (int s8 = 0; s8 < 8; ++s8) Xo[(r0 + 4 * s8) * LD] = -sum[s8];
        }
        __syncthreads();
    }
    for (int e = tid; e < kNB * kNB; e += kNpThreads) {
        const int i = e >> 6, c = e & 63;
        dinv_blk[e] = Li[i * LD + c];
        dinv_blk[kNB * kNB + e] = Ui[i * LD + c];
    }
    if (tid == 0 && zero) bar->singular = 1;
    publish_maxl(mx, bar);
}

// L21 = A21 U11^-1 and U12 = L11^-1 A12 of one panel, as 64 x 64 x 64 products with the
// inverses of the diagonal block's triangles (the first half of the grid does 64-row tiles of
// A21, the second 64-column tiles of A12, in place); tracks the largest |l| of L21.  Both tiles
// are fetched into registers first (all loads in flight together), then staged in shared memory.
// When the trailing update runs on the tensor cores (FP32 factors), the kernel also writes L21
// and U12 split into TF32 hi + lo parts in the update's operand layout (K = 64: A [rest][64] by
// rows of L21, B [rest][64] by columns of U12), so the update needs no separate split pass.
struct TcOperands {
    float* a_hi = nullptr;
    float* a_lo = nullptr;
    float* b_hi = nullptr;
    float* b_lo = nullptr;
};
template <typename T>
constexpr size_t panel_smem() { return sizeof(T) * 2 * kNB * (kNB + 1); }

template <typename T>
__global__ void __launch_bounds__(kNpThreads) lu_panel_gemm_kernel(T* __restrict__ A, int lda, int m, int kb,
                                                                   const T* __restrict__ dinv_blk,
                                                                   GridBarrier* __restrict__ bar, TcOperands ops) {
    constexpr int kS = kNB * kNB / kNpThreads;   // elements of a tile per thread (16)
    extern __shared__ __align__(16) unsigned char pg_sm[];
    T (*X)[kNB + 1] = reinterpret_cast<T (*)[kNB + 1]>(pg_sm);     // the A21 or A12 tile
    T (*V)[kNB + 1] = X + kNB;                                       // U11^-1 or L11^-1
    const int tid = threadIdx.x, a = tid & (kNB - 1), g = (tid >> 6) & 3;
    pdl_trigger();
    pdl_wait();                               // the inverses come from the diagonal-block launch
    const int rest = m - kb - kNB;
    const int ntl = (rest + kNB - 1) / kNB;
    const bool rows = (int)blockIdx.x < ntl;
    const int t0 = kb + kNB + (rows ? (int)blockIdx.x : (int)blockIdx.x - ntl) * kNB;
    const int ext = min(kNB, m - t0);
    const T* inv = dinv_blk + (rows ? kNB * kNB : 0);
    // element e = tid + 256 s of a 64 x 64 tile: row e / 64 = g + 4 s, column a
    T xv[kS], vv[kS];
#pragma unroll
    for (int s = 0; s < kS; ++s) {
        const int i = g + 4 * s;
        vv[s] = inv[i * kNB + a];
        if (rows) xv[s] = i < ext ? A[(size_t)(t0 + i) * lda + kb + a] : T(0);
        else xv[s] = a < ext ? A[(size_t)(kb + i) * lda + t0 + a] : T(0);
    }
#pragma unroll
    for (int s = 0; s < kS; ++s) {
        V[g + 4 * s][a] = vv[s];
        X[g + 4 * s][a] = xv[s];
    }
    __syncthreads();
    T mx = T(0);
    T acc[kS];
#pragma unroll
    for (int k = 0; k < kS; ++k) acc[k] = T(0);
    if (rows) {
        // row a of the tile, columns g + 4 k:  sum_t X[a][t] U^-1[t][col]
        for (int t = 0; t < kNB; ++t) {
            const T x = X[a][t];
#pragma unroll
            for (int k = 0; k < kS; ++k) acc[k] = fma(x, V[t][g + 4 * k], acc[k]);
        }
        __syncthreads();                      // staged in X for row-contiguous stores
#pragma unroll
        for (int k = 0; k < kS; ++k) X[a][g + 4 * k] = acc[k];
        __syncthreads();
        const int64_t o0 = (int64_t)(t0 - kb - kNB) * kNB;        // first operand row of this tile
#pragma unroll
        for (int s = 0; s < kS; ++s) {
            const int i = g + 4 * s;
            if (i < ext) {
                const T l = X[i][a];
                A[(size_t)(t0 + i) * lda + kb + a] = l;
                mx = nanmax(mx, fabs(l));
                if constexpr (std::is_same<T, float>::value) {
                    if (ops.a_hi) {
                        float hv, lv;
                        tf32_split(l, hv, lv);
                        ops.a_hi[o0 + (int64_t)i * kNB + a] = hv;
                        ops.a_lo[o0 + (int64_t)i * kNB + a] = lv;
                    }
                }
            }
        }
    } else {
        // column a of the tile, rows g + 4 k:  sum_t L^-1[row][t] X[t][a]
        for (int t = 0; t < kNB; ++t) {
            const T x = X[t][a];
#pragma unroll
            for (int k = 0; k < kS; ++k) acc[k] = fma(V[g + 4 * k][t], x, acc[k]);
        }
        if (a < ext) {
#pragma unroll
            for (int k = 0; k < kS; ++k) A[(size_t)(kb + g + 4 * k) * lda + t0 + a] = acc[k];
        }
        if constexpr (std::is_same<T, float>::value) {
            if (ops.b_hi) {
                // B operand: column t0 + e / 64 of U12, row e % 64, contiguous; staged transposed
                __syncthreads();                  // every thread is done reading X
#pragma unroll
                for (int k = 0; k < kS; ++k) X[g + 4 * k][a] = acc[k];
                __syncthreads();
                const int64_t o0 = (int64_t)(t0 - kb - kNB) * kNB;
#pragma unroll
                for (int s = 0; s < kS; ++s) {
                    const int col = g + 4 * s, row = a;
                    if (col < ext) {
                        float hv, lv;
                        tf32_split(X[row][col], hv, lv);
                        ops.b_hi[o0 + (int64_t)col * kNB + row] = hv;
                        ops.b_lo[o0 + (int64_t)col * kNB + row] = lv;
                    }
                }
            }
        }
    }
    publish_maxl(mx, bar);
}

template <typename T>
__global__ void diag_writeback_kernel(T* __restrict__ A, int lda, int m, const T* __restrict__ diag) {
    const int t = blockIdx.x, kb = t * kNB, nb = min(kNB, m - kb);
    const T* d = diag + (size_t)t * kNB * kNB;      // [64][64] (rows and columns beyond nb unused)
    for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) A[(size_t)(kb + q / nb) * lda + kb + q % nb] = d[(q / nb) * kNB + q % nb];
}

__global__ void iota_kernel(int* __restrict__ v, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) v[i] = i;
}

// Returns EWOS_OK with *accepted false when a multiplier exceeds 1 or a pivot is zero (the
// caller then refactors the original matrix with interchanges).
// Trailing updates of at least this many rows go to the tensor cores (FP32 factors; three TF32
// products on the halves the panel kernel splits, three FP16 products on per-row and per-column
// scaled halves for the rank-512 updates); smaller ones stay on the FP32 SIMT GEMM.
constexpr int kTcUpdateMin = 256;
constexpr int kSuper = 8;           // 64-column panels per super panel of the unpivoted LU

template <typename T>
static ewos_status lu_factor_nopiv(T* A, int m, int lda, LuScratch& S, cudaStream_t st, bool* accepted,
                                   TcScratch** tc = nullptr) {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(lu_panel_gemm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)panel_smem<T>());
        if (attr == cudaSuccess)
            attr = cudaFuncSetAttribute(lu_diag_factor_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)diag_smem<T>());
    });
    EWOS_CUDA_TRY(attr);
    EWOS_CUDA_TRY(cudaMemsetAsync(S.bar, 0, sizeof(GridBarrier), st));
    T* diagb = reinterpret_cast<T*>(S.diagb);
    T* dinv = reinterpret_cast<T*>(S.dinv);
    // tensor-core updates take their operands split by the panel kernel
    TcOperands tc_ops;
    const bool use_tc = std::is_same<T, float>::value && tc != nullptr && m - kNB >= kTcUpdateMin;
    if (use_tc) {
        // room for the rank-kSuper*64 updates' operands too (split by the update itself)
        ewos_status e = tc_update_reserve(m - kNB, kSuper * kNB, st, tc);
        if (e != EWOS_OK) return e;
        tc_update_operands(*tc, &tc_ops.a_hi, &tc_ops.a_lo, &tc_ops.b_hi, &tc_ops.b_lo);
    }
    // C[row0 .., col0 ..] (M x N) -= L[row0 .., kcol .. kcol + K] U[krow .. krow + K, col0 ..], in place;
    // with `split` the operands are the panel's split ones, starting at operand rows a_off, b_off
    auto update = [&](int M, int N, int K, int row0, int col0, int kcol, int krow, bool split, int a_off,
                      int b_off) -> ewos_status {
        if (M <= 0 || N <= 0 || K <= 0) return EWOS_OK;
        T* C = A + (size_t)row0 * lda + col0;
        const T* L = A + (size_t)row0 * lda + kcol;
        const T* U = A + (size_t)krow * lda + col0;
        if constexpr (std::is_same<T, float>::value) {
            if (split || (use_tc && M >= kTcUpdateMin && N >= kTcUpdateMin))
                return tc_update_enqueue(reinterpret_cast<const float*>(L), lda, reinterpret_cast<const float*>(U), lda,
                                         reinterpret_cast<float*>(C), lda, M, N, K, st, tc, split, a_off, b_off);
        }
        gemm_trailing<T>(st, M, N, K, L, lda, U, lda, C, lda);
        return EWOS_OK;
    };
    // Super panels of kSuper 64-column panels.  Inside a super panel each panel updates only the
    // rows of the super panel's later panels (across every column to its right: the band) and the
    // super panel's later columns (for every row below the super panel); the trailing matrix
    // below and right of the super panel gets one rank-(kSuper * 64) update at its end, which
    // reads and writes that matrix once instead of kSuper times.
    for (int KB = 0; KB < m; KB += kSuper * kNB) {
        const int KE = std::min(m, KB + kSuper * kNB);
        for (int kb = KB; kb < KE; kb += kNB) {
            const int nb = std::min(kNB, m - kb);
            const int rest = m - kb - nb;
            T* dblk = diagb + (size_t)(kb / kNB) * kNB * kNB;
            T* iblk = dinv + (size_t)(kb / kNB) * 2 * kNB * kNB;
            ::ewos::note_launch();
            EWOS_CUDA_TRY(launch_pdl(lu_diag_factor_kernel<T>, dim3(1), dim3(kNpThreads), diag_smem<T>(), st, (const T*)A,
                                     lda, kb, nb, dblk, iblk, S.bar));
            if (rest > 0) {
                // nb == 64 whenever rows remain below the diagonal block
                const int ntl = (rest + kNB - 1) / kNB;
                const bool tc_here = use_tc && rest >= kTcUpdateMin;
                ::ewos::note_launch();
                EWOS_CUDA_TRY(launch_pdl(lu_panel_gemm_kernel<T>, dim3(2 * ntl), dim3(kNpThreads), panel_smem<T>(), st, A,
                                         lda, m, kb, (const T*)iblk, S.bar, tc_here ? tc_ops : TcOperands{}));
                const int band = KE - (kb + nb);       // rows (and columns) of the super panel's later panels
                const int below = m - KE;
                ewos_status e = EWOS_OK;
                if constexpr (std::is_same<T, float>::value) {
                    // on the tensor cores both updates are one launch over their L-shaped region
                    if (tc_here && band > 0 && (lda & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0) {
                        e = tc_update_lshape_enqueue(reinterpret_cast<float*>(A + (size_t)(kb + nb) * lda + kb + nb), lda,
                                                     rest, band, nb, st, tc);
                        if (e != EWOS_OK) return e;
                        continue;
                    }
                }
                e = update(band, rest, nb, kb + nb, kb + nb, kb, kb, tc_here, 0, 0);
                if (e == EWOS_OK) e = update(below, band, nb, KE, kb + nb, kb, kb, tc_here, band, 0);
                if (e != EWOS_OK) return e;
            }
        }
        ewos_status e = update(m - KE, m - KE, KE - KB, KE, KE, KB, KB, false, 0, 0);
        if (e != EWOS_OK) return e;
    }
    if (tc && *tc) {
        ewos_status e = tc_update_check(*tc, st);
        if (e != EWOS_OK) return e;
    }
    const int nbk = (m + kNB - 1) / kNB;
    ::ewos::note_launch(), diag_writeback_kernel<T><<<nbk, 256, 0, st>>>(A, lda, m, diagb);
    ::ewos::note_launch(), iota_kernel<<<(m + 255) / 256, 256, 0, st>>>(S.ipiv, m);
    ::ewos::note_launch(), iota_kernel<<<(m + 255) / 256, 256, 0, st>>>(S.perm, m);
    GridBarrier hb{};
    EWOS_CUDA_TRY(cudaMemcpyAsync(&hb, S.bar, sizeof(hb), cudaMemcpyDeviceToHost, st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(st));
    EWOS_CUDA_TRY(cudaGetLastError());
    const double one = 1.0;
    unsigned long long one_bits;
    memcpy(&one_bits, &one, sizeof(one));
    *accepted = !hb.singular && hb.maxl_bits <= one_bits;
    return EWOS_OK;
}

// Triangular solves with the factors of P A = L U in ONE launch, as a dataflow over 64-row
// blocks.  X [m][rc] holds rc right-hand sides per row, in place, rows in pivot order.  The
// CTA with ticket t (tickets are taken in the order the CTAs start) owns block row i = t of
// the forward solve (t < nbk) or block row i = 2 nbk - 1 - t of the backward solve:
//   forward   Y_i = L_ii^{-1} (X_i - sum_{j<i} L_ij Y_j)
//   backward  X_i = U_ii^{-1} (Y_i - sum_{j>i} U_ij X_j)
// with the inverses of the diagonal blocks precomputed.  A row block publishes its result with
// a release flag; a CTA waits only on flags of smaller tickets, which belong to CTAs that have
// already started, so the launch completes whatever else runs on the device (no co-residency
// assumption; several streams may solve at once).  Every backward write of X_i comes after the
// last forward read (the backward chain starts from the last forward row block).  Every wait
// is bounded; a timeout sets the error word, on which all other waits give up too.  A row block
// is published by a release store of one thread after a CTA barrier (cumulative over the CTA's
// writes) and read after an acquire load of one thread followed by a barrier; flags are polled
// without sleeping (each poll is an L2 round trip).
// state: [0] ticket counter, [1] error word, [2, 2 + nbk) forward flags, [2 + nbk, 2 + 2 nbk)
// backward flags; zeroed before each launch.
constexpr long long kFlowSpinLimit = 1ll << 22;
// the limit the kernels use (a test hook lowers it to make the waits run out)
__device__ long long g_flow_spin_limit = kFlowSpinLimit;

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// thread 0 waits for *flag != 0; the result is the CTA's (false: give up and return)
__device__ __forceinline__ bool flow_wait(const unsigned int* flag, unsigned int* err, int* s_ok) {
    if (threadIdx.x == 0) {
        int ok = 1;
        long long spins = 0;
        const long long limit = g_flow_spin_limit;
        while (ld_acquire_u32(flag) == 0) {
            if ((++spins & 63) == 0 && ld_acquire_u32(err) != 0) { ok = 0; break; }   // another CTA gave up
            if (spins > limit) { atomicExch(err, 1u); ok = 0; break; }
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// dst[a][b] = src[a * ld + b] for a < h, b < w, else 0 (a 64 x 64 tile, 256 threads): all 16
// loads of a thread are issued before the shared-memory stores
template <typename T, bool L2_ONLY>
__device__ __forceinline__ void stage_tile(T (*dst)[65], const T* src, size_t ld, int h, int w) {
    const int b = threadIdx.x & 63, a0 = threadIdx.x >> 6;
    T v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int a = a0 + 4 * s;
        v[s] = (a < h && b < w) ? (L2_ONLY ? __ldcg(src + a * ld + b) : src[a * ld + b]) : T(0);
    }
#pragma unroll
    for (int s = 0; s < 16; ++s) dst[a0 + 4 * s][b] = v[s];
}

// 4 consecutive values of a shared-memory row (16-byte aligned for FP32)
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T* v) {
    if constexpr (std::is_same<T, float>::value) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = p[e];
    }
}

// Many right-hand sides: the same dataflow over 64-row blocks, 64 right-hand sides at a time.
// A thread owns a 4 x 4 piece of the block's 64 x 64 accumulator in registers; each preceding
// block's contribution L_ij X_j is a 64 x 64 x 64 product from shared memory (L_ij staged
// transposed), 16 multiply-adds per two 4-wide loads, and the diagonal inverse is applied the
// same way at the end.
constexpr int kFlowLd = 68;                   // shared row stride (16-byte aligned rows)
template <typename T>
__global__ void __launch_bounds__(256) trsm_flow_kernel(const T* __restrict__ LU, int lda, int m,
                                                       const T* __restrict__ Dinv, T* X, int rc,
                                                       unsigned int* state) {
    extern __shared__ __align__(16) unsigned char flow_sm[];
    T (*Lt)[kFlowLd] = reinterpret_cast<T (*)[kFlowLd]>(flow_sm);   // [k][row]: L_ij (U_ij) transposed
    T (*Xs)[kFlowLd] = Lt + 64;                                       // [k][col]: X_j
    T (*Dt)[kFlowLd] = Xs + 64;                                       // [k][row]: the diagonal inverse, transposed
    T (*As)[kFlowLd] = Dt + 64;                                       // [row][col]: the accumulator
    __shared__ unsigned int s_ticket;
    __shared__ int s_ok;
    const int nbk = (m + 63) / 64;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;     // rows 4 ty .. 4 ty + 3, columns 4 tx ..
    if (tid == 0) s_ticket = atomicAdd(state, 1u);
    __syncthreads();
    const int t = (int)s_ticket;
    if (t >= 2 * nbk) return;
    const bool lower = t < nbk;
    const int i = lower ? t : 2 * nbk - 1 - t;
    unsigned int* err = state + 1;
    unsigned int* const fl = state + 2;
    unsigned int* const fu = state + 2 + nbk;
    unsigned int* const mine = lower ? fl : fu;
    const int r0 = i * 64, h = min(64, m - r0);
    const T* Di = Dinv + (size_t)i * 2 * 64 * 64 + (lower ? 0 : 64 * 64);
    // the diagonal inverse, transposed: Dt[k][a] = D[a][k]
    for (int e = tid; e < 64 * 64; e += 256) Dt[e & 63][e >> 6] = Di[e];
    if (!lower && !flow_wait(fl + i, err, &s_ok)) return;      // Y_i from the forward solve
    const int nj = lower ? i : nbk - 1 - i;
    for (int q0 = 0; q0 < rc; q0 += 64) {
        const int rw = min(64, rc - q0);
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int row = 4 * ty + a, col = 4 * tx + c;
                acc[a][c] = (row < h && col < rw) ? __ldcg(X + (size_t)(r0 + row) * rc + q0 + col) : T(0);
            }
        for (int q = 0; q < nj; ++q) {
            const int j = lower ? q : nbk - 1 - q;
            const int c0 = j * 64, w = min(64, m - c0);
            // L_ij transposed (rows of the block, columns of block j), fetched before the flag wait
            for (int e = tid; e < 64 * 64; e += 256) {
                const int a = e >> 6, k = e & 63;
                Lt[k][a] = (a < h && k < w) ? LU[(size_t)(r0 + a) * lda + c0 + k] : T(0);
            }
            if (!flow_wait(mine + j, err, &s_ok)) return;
            for (int e = tid; e < 64 * 64; e += 256) {
                const int k = e >> 6, c = e & 63;
                Xs[k][c] = (k < w && c < rw) ? __ldcg(X + (size_t)(c0 + k) * rc + q0 + c) : T(0);
            }
            __syncthreads();
#pragma unroll 8
            for (int k = 0; k < 64; ++k) {
                T l4[4], x4[4];
                ld4(&Lt[k][4 * ty], l4);
                ld4(&Xs[k][4 * tx], x4);
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[a][c] = fma(-l4[a], x4[c], acc[a][c]);
            }
            __syncthreads();
        }
        // X_i = D (B_i - sum_j L_ij X_j)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) As[4 * ty + a][4 * tx + c] = acc[a][c];
        __syncthreads();
        T out[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) out[a][c] = T(0);
#pragma unroll 8
        for (int k = 0; k < 64; ++k) {
            T d4[4], a4[4];
            ld4(&Dt[k][4 * ty], d4);
            ld4(&As[k][4 * tx], a4);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) out[a][c] = fma(d4[a], a4[c], out[a][c]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int row = 4 * ty + a, col = 4 * tx + c;
                if (row < h && col < rw) X[(size_t)(r0 + row) * rc + q0 + col] = out[a][c];
            }
        __syncthreads();
    }
    if (tid == 0) st_release_u32(mine + i, 1u);     // after the barrier: publishes the CTA's writes
}

// The same dataflow for one right-hand side (rc = 1), built for throughput of each CTA: the CTA
// waits for the next block it needs and then takes every later block whose flag is already set
// (up to 8 at once), so it never falls behind the chain.  Warp w owns rows w, w + 8, .. of the
// row block; lanes stride over the columns of the ready blocks (row segments of L or U read
// contiguously, all loads of a chunk in flight), partial sums are reduced across the warp at
// the end, and the inverse of the diagonal block is applied from shared memory.
template <typename T>
__global__ void __launch_bounds__(256) trsm_flow_vec_kernel(const T* __restrict__ LU, int lda, int m,
                                                           const T* __restrict__ Dinv, T* X, unsigned int* state) {
    __shared__ T Ds[64][65];
    __shared__ T ys[64];
    __shared__ unsigned int s_ticket;
    __shared__ int s_ok, s_cnt;
    const int nbk = (m + 63) / 64;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) s_ticket = atomicAdd(state, 1u);
    __syncthreads();
    const int t = (int)s_ticket;
    if (t >= 2 * nbk) return;
    const bool lower = t < nbk;
    const int i = lower ? t : 2 * nbk - 1 - t;
    unsigned int* err = state + 1;
    unsigned int* const fl = state + 2;
    unsigned int* const fu = state + 2 + nbk;
    unsigned int* const mine = lower ? fl : fu;
    const int r0 = i * 64, h = min(64, m - r0);
    stage_tile<T, false>(Ds, Dinv + (size_t)i * 2 * 64 * 64 + (lower ? 0 : 64 * 64), 64, 64, 64);
    if (!lower && !flow_wait(fl + i, err, &s_ok)) return;      // Y_i from the forward solve
    __syncthreads();                                          // s_ok is rewritten below
    T own[8];                                                 // this block's right-hand side, fetched early
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int row = w + 8 * r;
        own[r] = (lane == 0 && row < h) ? __ldcg(X + r0 + row) : T(0);
    }
    T acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = T(0);
    const int nj = lower ? i : nbk - 1 - i;
    int q = 0;
    while (q < nj) {
        // the next block this CTA needs: its rows of L (U) are fetched before its flag is polled
        const int j0 = lower ? q : nbk - 1 - q;
        const int cj = 64 * j0;
        T pre[16];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int row = w + 8 * r;
            const T* src = LU + (size_t)(r0 + row) * lda + cj;
            pre[2 * r] = (row < h && cj + lane < m) ? src[lane] : T(0);
            pre[2 * r + 1] = (row < h && cj + lane + 32 < m) ? src[lane + 32] : T(0);
        }
        if (tid == 0) {
            int ok = 1, cnt = 0;
            const unsigned int* f0 = mine + j0;
            long long spins = 0;
            const long long limit = g_flow_spin_limit;
            while (ld_acquire_u32(f0) == 0) {
                if ((++spins & 63) == 0 && ld_acquire_u32(err) != 0) { ok = 0; break; }
                if (spins > limit) { atomicExch(err, 1u); ok = 0; break; }
            }
            if (ok) {
                cnt = 1;
                while (cnt < 8 && q + cnt < nj && ld_acquire_u32(mine + (lower ? q + cnt : nbk - 1 - q - cnt)) != 0) ++cnt;
            }
            s_ok = ok;
            s_cnt = cnt;
        }
        __syncthreads();
        if (!s_ok) return;
        const int cnt = s_cnt;
        {
            const T x0 = cj + lane < m ? __ldcg(X + cj + lane) : T(0);
            const T x1 = cj + lane + 32 < m ? __ldcg(X + cj + lane + 32) : T(0);
#pragma unroll
            for (int r = 0; r < 8; ++r) acc[r] = fma(pre[2 * r + 1], x1, fma(pre[2 * r], x0, acc[r]));
        }
        // the other ready blocks: forward j0 + 1 .. j0 + cnt - 1, backward j0 - cnt + 1 .. j0 - 1
        const int c_lo = lower ? cj + 64 : 64 * (j0 - cnt + 1);
        const int c_hi = lower ? cj + 64 * cnt : cj;
#pragma unroll 2
        for (int k = c_lo + lane; k < c_hi; k += 32) {
            const T xk = __ldcg(X + k);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int row = w + 8 * r;
                if (row < h) acc[r] = fma(LU[(size_t)(r0 + row) * lda + k], xk, acc[r]);
            }
        }
        q += cnt;
        __syncthreads();                      // s_ok and s_cnt are rewritten by the next round
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        T v = acc[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int row = w + 8 * r;
        if (lane == 0) ys[row] = row < h ? own[r] - v : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int row = w + 8 * r;
        T v = fma(Ds[row][lane], ys[lane], Ds[row][lane + 32] * ys[lane + 32]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && row < h) X[r0 + row] = v;
    }
    __syncthreads();
    if (tid == 0) st_release_u32(mine + i, 1u);     // after the barrier: publishes the CTA's writes
}

template <typename T>
constexpr size_t flow_smem() { return sizeof(T) * 4 * 64 * kFlowLd; }

constexpr size_t flow_state_words(int64_t m) { return 2 + 2 * (size_t)((m + 63) / 64); }

template <typename T>
static cudaError_t trsm_prepare() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        err = cudaFuncSetAttribute(trsm_flow_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)flow_smem<T>());
    });
    return err;
}

// L U X = X (rows already in pivot order), enqueued on st: the state reset and the one launch
template <typename T>
static void trsm_flow(const T* LU, int m, int lda, const T* Dinv, T* X, int rc, unsigned int* state, cudaStream_t st) {
    const int nbk = (m + 63) / 64;
    cudaMemsetAsync(state, 0, sizeof(unsigned int) * flow_state_words(m), st);
    if (rc == 1)
        ::ewos::note_launch(), trsm_flow_vec_kernel<T><<<2 * nbk, 256, 0, st>>>(LU, lda, m, Dinv, X, state);
    else
        ::ewos::note_launch(), trsm_flow_kernel<T><<<2 * nbk, 256, flow_smem<T>(), st>>>(LU, lda, m, Dinv, X, rc, state);
}

// the error word of the last triangular solve on st (synchronises st)
static ewos_status flow_check(const unsigned int* state, cudaStream_t st) {
    unsigned int herr = 0;
    EWOS_CUDA_TRY(cudaMemcpyAsync(&herr, state + 1, sizeof(herr), cudaMemcpyDeviceToHost, st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr) {
        set_error("triangular solve: a wait on a preceding row block timed out");
        return EWOS_ETIMEOUT;
    }
    return EWOS_OK;
}

// out[i][r] = (T) x[r][perm[i]]  /  x[r][i] = out[i][r]
template <typename T>
__global__ void gather_cols_kernel(const double* __restrict__ x, const int* __restrict__ perm, T* __restrict__ out,
                                   int m, int nrhs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)m * nrhs) return;
    const int i = (int)(t / nrhs), r = (int)(t % nrhs);
    out[t] = (T)x[(size_t)r * m + perm[i]];
}

template <typename T>
__global__ void scatter_cols_kernel(const T* __restrict__ in, double* __restrict__ x, int m, int nrhs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)m * nrhs) return;
    const int r = (int)(t / m), i = (int)(t % m);
    x[t] = (double)in[(size_t)i * nrhs + r];
}

// ------------------------------------------------------------------ workspace
static inline int64_t pad4(int64_t x) { return (x + 3) & ~(int64_t)3; }   // 16-byte segments of F2one

struct SolveWorkspace {
    double last_alpha = 0.0;                  // shift of the last linear factorisation (factor reuse)
    int D = 0;
    int64_t n = 0, m = 0, p = 0;
    double *Q = nullptr, *Lam = nullptr, *LUm = nullptr, *M = nullptr, *Jx = nullptr;
    double *A = nullptr, *b = nullptr, *c = nullptr, *f = nullptr, *g = nullptr, *nl = nullptr;
    double *s = nullptr, *x = nullptr, *v = nullptr, *w = nullptr, *y = nullptr, *u = nullptr, *u2 = nullptr;
    // KH g of the right-hand side being solved ([(D+1)][n]), valid while vg_for == that g (set and
    // cleared around one right-hand side's iteration by VgScope): the residuals of Newton and
    // Picard iterations start from it instead of reading KH again
    double* vg = nullptr;
    const double* vg_for = nullptr;
    double* scal = nullptr;                   // [4] reductions
    unsigned long long* umax = nullptr;
    LuScratch lu;
    int64_t cap_rhs = 0;
    // mixed precision
    float *Q32 = nullptr, *L32 = nullptr, *LU32 = nullptr, *J32 = nullptr, *Jx32 = nullptr, *P32 = nullptr;
    double *rhs = nullptr, *r = nullptr, *dx = nullptr;
    TcScratch* tc = nullptr;
    // all right-hand sides at once: [rows][bcap] layouts (bcap = a power-of-two bucket)
    int64_t bcap = 0;
    double *Sb = nullptr, *Yb = nullptr, *Vb = nullptr, *Wb = nullptr, *Fb = nullptr, *Gb = nullptr, *Ub = nullptr;
    double *nrm = nullptr, *alpha_dev = nullptr;
    float *D32 = nullptr, *D32p = nullptr;
    float* F2buf = nullptr;          // hi/lo FP32 pairs of Sb [m][bcap], Gb [p][bcap], Wb [rows][bcap]
    double* Ypart = nullptr;         // per-CTA partials of the fused one-column residual [ypart_grid][m]
    double* ctpart = nullptr;        // per-CTA partials of the whole-row column products [parts][m]
    int64_t ctpart_cap = 0;          // doubles
    float* F2one = nullptr;          // FP32 toolboxes: hi/lo pairs of one column of s [m], g [p], w [rows]
    int ypart_grid = 0;
    struct Graph {
        uint64_t tb;     // serial of the toolbox whose buffers the graph reads
        int64_t rc;
        int nl;          // number of nonlinearity coefficients (0: linear)
        cudaGraphExec_t exec;
        int launches;
    };
    std::vector<Graph> graphs;
    cudaStream_t cap_st = nullptr;   // capture stream of the graphs
};

void free_workspace(SolveWorkspace* ws) {
    if (!ws) return;
    ::ewos::dev_free(ws->Q); ::ewos::dev_free(ws->Lam); ::ewos::dev_free(ws->LUm); ::ewos::dev_free(ws->M); ::ewos::dev_free(ws->Jx);
    ::ewos::dev_free(ws->A); ::ewos::dev_free(ws->b); ::ewos::dev_free(ws->c); ::ewos::dev_free(ws->f); ::ewos::dev_free(ws->g); ::ewos::dev_free(ws->nl);
    ::ewos::dev_free(ws->vg);
    ::ewos::dev_free(ws->s); ::ewos::dev_free(ws->x); ::ewos::dev_free(ws->v); ::ewos::dev_free(ws->w); ::ewos::dev_free(ws->y); ::ewos::dev_free(ws->u); ::ewos::dev_free(ws->u2);
    ::ewos::dev_free(ws->scal); ::ewos::dev_free(ws->umax);
    ::ewos::dev_free(ws->lu.pub); ::ewos::dev_free(ws->lu.bar); ::ewos::dev_free(ws->lu.ipiv);
    ::ewos::dev_free(ws->lu.perm); ::ewos::dev_free(ws->lu.swp); ::ewos::dev_free(ws->lu.tmp);
    ::ewos::dev_free(ws->lu.dinv); ::ewos::dev_free(ws->lu.diagb); ::ewos::dev_free(ws->lu.flow);
    ::ewos::dev_free(ws->Q32); ::ewos::dev_free(ws->L32); ::ewos::dev_free(ws->LU32); ::ewos::dev_free(ws->J32);
    ::ewos::dev_free(ws->Jx32); ::ewos::dev_free(ws->P32);
    ::ewos::dev_free(ws->rhs); ::ewos::dev_free(ws->r); ::ewos::dev_free(ws->dx);
    tc_scratch_free(ws->tc);
    ::ewos::dev_free(ws->Sb); ::ewos::dev_free(ws->Yb); ::ewos::dev_free(ws->Vb); ::ewos::dev_free(ws->Wb);
    ::ewos::dev_free(ws->Fb); ::ewos::dev_free(ws->Gb); ::ewos::dev_free(ws->Ub); ::ewos::dev_free(ws->nrm);
    ::ewos::dev_free(ws->alpha_dev); ::ewos::dev_free(ws->D32); ::ewos::dev_free(ws->D32p); ::ewos::dev_free(ws->F2buf);
    ::ewos::dev_free(ws->Ypart); ::ewos::dev_free(ws->F2one); ::ewos::dev_free(ws->ctpart);
    for (auto& g : ws->graphs) cudaGraphExecDestroy(g.exec);
    if (ws->cap_st) cudaStreamDestroy(ws->cap_st);
    delete ws;
}

static ewos_status ensure_workspace(const ewos_toolbox* tb, SolveWorkspace*& slot, int64_t nrhs, bool mixed,
                                    bool matrices = true) {
    if (slot && (slot->cap_rhs < nrhs || slot->n != tb->n || slot->m != tb->m || slot->p != tb->p || slot->D != tb->dim)) {
        free_workspace(slot);
        slot = nullptr;
    }
    const int D = tb->dim, E = D + 1;
    const int64_t n = tb->n, m = tb->m, p = tb->p;
    // a failed allocation leaves no half-built workspace behind: the next call starts afresh
    struct Undo {
        SolveWorkspace*& slot;
        bool armed = true;
        ~Undo() { if (armed && slot) { free_workspace(slot); slot = nullptr; } }
    };
    if (!slot) {
        SolveWorkspace* ws = new SolveWorkspace();
        slot = ws;
        Undo undo{slot};
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
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->vg, sizeof(double) * E * n));
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
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->lu.dinv, sizeof(double) * ((m + 63) / 64) * 2 * 64 * 64));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->lu.diagb, sizeof(double) * ((m + 63) / 64) * 64 * 64));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->lu.flow, sizeof(unsigned int) * flow_state_words(m)));
        if (tb->precision == 32)
            EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->F2one, sizeof(float) * 2 * (pad4(m) + pad4(p) + pad4((int64_t)E * n))));
        undo.armed = false;
    }
    SolveWorkspace* ws = slot;
    if (!matrices) return EWOS_OK;            // the vectors suffice (gradient, Adam)
    if (!mixed && !ws->Q) {
        Undo undo{slot};
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Lam, sizeof(double) * m * m));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->LUm, sizeof(double) * m * m));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Jx, sizeof(double) * n * m));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Q, sizeof(double) * E * n * m));     // last: marks the set complete
        undo.armed = false;
    }
    if (mixed && !ws->Q32) {
        Undo undo{slot};
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->L32, sizeof(float) * m * m));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->LU32, sizeof(float) * m * m));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Jx32, sizeof(float) * n * m));
        if (tb->precision == 64) EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->P32, sizeof(float) * E * n * m));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Q32, sizeof(float) * E * n * m));   // last: marks the set complete
        undo.armed = false;
    }
    return EWOS_OK;
}

template <typename T>
static ewos_status lu_solve_device(const T* LU, int m, int lda, LuScratch& S, double* x, int nrhs, cudaStream_t st,
                                   bool check = true) {
    EWOS_CUDA_TRY(trsm_prepare<T>());
    T* X = reinterpret_cast<T*>(S.tmp);   // [m][nrhs] in the precision of the factors
    const int64_t cnt = (int64_t)m * nrhs;
    const int nb = (int)((cnt + 255) / 256);
    ::ewos::note_launch(), gather_cols_kernel<T><<<nb, 256, 0, st>>>(x, S.perm, X, m, nrhs);
    trsm_flow<T>(LU, m, lda, (const T*)S.dinv, X, nrhs, S.flow, st);
    ::ewos::note_launch(), scatter_cols_kernel<T><<<nb, 256, 0, st>>>(X, x, m, nrhs);
    EWOS_CUDA_TRY(cudaGetLastError());
    return check ? flow_check(S.flow, st) : EWOS_OK;
}

// ------------------------------------------------------------------ operator pieces
struct Ctx {
    ewos_toolbox* tb;
    SolveWorkspace* ws;
    cudaStream_t st;
    int D, E;
    int64_t n, m, p;
};

// FP32-pair products (defined with the batched solves below)
static void multi_rowdot_f2(cudaStream_t st, const float* X, int64_t rows, int cols, const float* Vhi, const float* Vlo,
                            double* Vout, int rc, int accumulate);
static void multi_coltrans_f2(cudaStream_t st, const float* X, int64_t rows, int cols, const float* Whi, const float* Wlo,
                              double* Y, int rc);
static void split_f2(cudaStream_t st, const double* v, float* hi, float* lo, int64_t count);
static bool coltrans_rows(const Ctx& C, const float* X, int64_t rows, int cols, const float* Whi, const float* Wlo,
                          double* Y);

// FP32 toolboxes: v = P s (+ KH g) and y = P^T w with FP64-accurate products on the FP32 pipes:
// s, g, w split into unevaluated FP32 pairs, products summed in FP32 pairs (two-sum), reduced in
// FP64 (the same arithmetic as the batched solves' residual; about 1e-14 relative)
static void apply_v_f2(const Ctx& C, const double* s, const double* g) {
    float* sh = C.ws->F2one;
    float* sl = sh + pad4(C.m);
    float* gh = sl + pad4(C.m);
    float* gl = gh + pad4(C.p);
    const int64_t rows = (int64_t)C.E * C.n;
    if (g && g == C.ws->vg_for) {
        // v = KH g + P s: the same two sums as P s + KH g, in the other (exact) order
        cudaMemcpyAsync(C.ws->v, C.ws->vg, sizeof(double) * rows, cudaMemcpyDeviceToDevice, C.st);
        if (s) {
            split_f2(C.st, s, sh, sl, C.m);
            multi_rowdot_f2(C.st, (const float*)C.tb->P, rows, (int)C.m, sh, sl, C.ws->v, 1, 1);
        }
        return;
    }
    if (s) {
        split_f2(C.st, s, sh, sl, C.m);
        multi_rowdot_f2(C.st, (const float*)C.tb->P, rows, (int)C.m, sh, sl, C.ws->v, 1, 0);
    }
    if (g) {
        split_f2(C.st, g, gh, gl, C.p);
        multi_rowdot_f2(C.st, (const float*)C.tb->KH, rows, (int)C.p, gh, gl, C.ws->v, 1, s ? 1 : 0);
    }
}

static void apply_PT_f2(const Ctx& C, const double* w, double* y) {
    float* wh = C.ws->F2one + 2 * (pad4(C.m) + pad4(C.p));
    float* wl = wh + pad4((int64_t)C.E * C.n);
    const int64_t rows = (int64_t)C.E * C.n;
    split_f2(C.st, w, wh, wl, rows);
    if (coltrans_rows(C, (const float*)C.tb->P, rows, (int)C.m, wh, wl, y)) return;
    cudaMemsetAsync(y, 0, sizeof(double) * C.m, C.st);
    multi_coltrans_f2(C.st, (const float*)C.tb->P, rows, (int)C.m, wh, wl, y, 1);
}

template <typename TP>
static void apply_v(const Ctx& C, const double* s, const double* g) {
    // v = P s + KH g  ([(D+1)][n]); s may be NULL (= 0)
    const TP* P = (const TP*)C.tb->P;
    const TP* KH = (const TP*)C.tb->KH;
    const int64_t rows = (int64_t)C.E * C.n;
    const int blocks = (int)((rows * 32 + 255) / 256);
    if (g && g == C.ws->vg_for) {
        cudaMemcpyAsync(C.ws->v, C.ws->vg, sizeof(double) * rows, cudaMemcpyDeviceToDevice, C.st);
        if (s) ::ewos::note_launch(), rowdot_kernel<TP><<<blocks, 256, 0, C.st>>>(P, rows, (int)C.m, s, C.ws->v, 1);
        return;
    }
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
    const bool f2 = sizeof(TP) == 4 && C.ws->F2one && g;
    if (f2) apply_v_f2(C, s, g);
    else apply_v<TP>(C, s, g);
    ::ewos::note_launch(), formw_kernel<<<(int)((C.n + 127) / 128), 128, 0, C.st>>>((int)C.n, C.D, C.ws->M, C.ws->v, C.tb->lambda, f, nl, nnl,
                                                             C.ws->w);
    if (f2) apply_PT_f2(C, C.ws->w, y);
    else apply_PT<TP>(C, C.ws->w, y);
    if (alpha != 0.0 && s) ::ewos::note_launch(), axpy_kernel<<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.m, alpha, s, y);
}

// KH g of one right-hand side kept for the residuals of its iterations (ws->vg), cleared when the
// scope ends: computed here as the residual's own v with s = 0
template <typename TP>
struct VgScope {
    const Ctx& C;
    VgScope(const Ctx& c, const double* g) : C(c) {
        C.ws->vg_for = nullptr;
        if (sizeof(TP) == 4 && C.ws->F2one) apply_v_f2(C, nullptr, g);
        else apply_v<TP>(C, nullptr, g);
        cudaMemcpyAsync(C.ws->vg, C.ws->v, sizeof(double) * C.E * C.n, cudaMemcpyDeviceToDevice, C.st);
        C.ws->vg_for = g;
    }
    ~VgScope() { C.ws->vg_for = nullptr; }
};

// u = G s + H g after a residual at s: the last plane of that residual's v = P s + KH g (the
// same FP32-pair or FP64 row products, in the same order, as u_from_s), while nothing else has
// written ws->v since
static void u_from_v(const Ctx& C, double* u) {
    cudaMemcpyAsync(u, C.ws->v + (size_t)C.D * C.n, sizeof(double) * C.n, cudaMemcpyDeviceToDevice, C.st);
}

// ||v||; with flag, the word *flag on the device is read in the same synchronisation (into *flag_h)
static double norm2(const Ctx& C, const double* v, int64_t len, const unsigned int* flag = nullptr,
                    unsigned int* flag_h = nullptr) {
    cudaMemsetAsync(C.ws->scal, 0, sizeof(double), C.st);
    ::ewos::note_launch(), sumsq_kernel<<<std::max<int64_t>(1, std::min<int64_t>(1024, (len + 255) / 256)), 256, 0, C.st>>>(v, len, C.ws->scal);
    double h = 0;
    cudaMemcpyAsync(&h, C.ws->scal, sizeof(double), cudaMemcpyDeviceToHost, C.st);
    if (flag) cudaMemcpyAsync(flag_h, flag, sizeof(unsigned int), cudaMemcpyDeviceToHost, C.st);
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
    } else if (C.ws->F2one) {
        // FP32 matrices, FP64 vectors: the FP32-pair products (as in the residual)
        float* sh = C.ws->F2one;
        float* sl = sh + pad4(C.m);
        float* gh = sl + pad4(C.m);
        float* gl = gh + pad4(C.p);
        split_f2(C.st, s, sh, sl, C.m);
        multi_rowdot_f2(C.st, (const float*)Gm, C.n, (int)C.m, sh, sl, u, 1, 0);
        split_f2(C.st, g, gh, gl, C.p);
        multi_rowdot_f2(C.st, (const float*)Hm, C.n, (int)C.p, gh, gl, u, 1, 1);
    } else {
        ::ewos::note_launch(), rowdot_kernel<float><<<blocks, 256, 0, C.st>>>((const float*)Gm, C.n, (int)C.m, s, u, 0);
        ::ewos::note_launch(), rowdot_kernel<float><<<blocks, 256, 0, C.st>>>((const float*)Hm, C.n, (int)C.p, g, u, 1);
    }
}

static double frob_shift(const Ctx& C, double rcond) {
    if (rcond == 0.0) return 0.0;
    return rcond * norm2(C, C.ws->Lam, C.m * C.m);
}

// LU <- Lambda (+ G^T extra) + alpha I, factorised in place: with the diagonal pivots when that
// equals partial pivoting (pivoting == 0), else rebuilt and factored with row interchanges.
template <typename TP>
static ewos_status factor_shifted(const Ctx& C, double alpha, const double* extra_gemm_B, int pivoting,
                                  ewos_solve_report* rep) {
    auto build = [&] {
        cudaMemcpyAsync(C.ws->LUm, C.ws->Lam, sizeof(double) * C.m * C.m, cudaMemcpyDeviceToDevice, C.st);
        if (extra_gemm_B) {
            const TP* Gm = (const TP*)C.tb->P + (size_t)C.D * C.n * C.m;
            gemm64<TP, true>(C.st, (int)C.m, (int)C.m, (int)C.n, 1.0, Gm, C.m, extra_gemm_B, C.m, 1.0, C.ws->LUm, C.m);
        }
        ::ewos::note_launch(), add_diag_kernel<double><<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.ws->LUm, (int)C.m,
                                                                                                (int)C.m, alpha);
    };
    build();
    ++rep->factorizations;
    if (pivoting == 0) {
        bool accepted = false;
        ewos_status s = lu_factor_nopiv<double>(C.ws->LUm, (int)C.m, (int)C.m, C.ws->lu, C.st, &accepted);
        if (s != EWOS_OK) return s;
        if (accepted) return EWOS_OK;
        build();
    }
    ++rep->pivoted_factorizations;
    bool sing = false;
    ewos_status s = lu_factor_device<double>(C.ws->LUm, (int)C.m, (int)C.m, C.ws->lu, C.st, &sing);
    if (s != EWOS_OK) return s;
    if (sing) { set_error("LU: zero pivot"); return EWOS_ESINGULAR; }
    return EWOS_OK;
}

static double elapsed_ms(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// device time of a stretch of work on a stream, added to *acc (CUDA events; waits for the end
// event, which the solve's stages do anyway when they read their results back)
struct DevSpan {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st;
    double* acc;
    DevSpan(cudaStream_t s, double* a) : st(s), acc(a) {
        if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) cudaEventRecord(e0, st);
    }
    ~DevSpan() {
        if (e0 && e1 && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) *acc += ms;
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

template <typename TP>
static ewos_status solve_fp64(ewos_toolbox* tb, SolveWorkspace* ws, const ewos_problem* pb, double rcond, double tol, int max_iter,
                              ewos_solve_report* rep, bool reuse = false) {
    Ctx C{tb, ws, pb->stream ? (cudaStream_t)pb->stream : tb->stream, tb->dim, tb->dim + 1, tb->n, tb->m, tb->p};
    const int64_t nrhs = pb->nrhs;
    auto t0 = std::chrono::steady_clock::now();
    const bool quasi = pb->nl_kind == EWOS_NL_QUASILINEAR, semi = pb->nl_kind == EWOS_NL_SEMILINEAR;
    ::ewos::note_launch(), coef_kernel<<<(int)((C.n + 127) / 128), 128, 0, C.st>>>((int)C.n, C.D, tb->lambda, ws->A, pb->b ? ws->b : nullptr,
                                                           pb->c ? ws->c : nullptr, nullptr, 0, nullptr, ws->M);
    rep->iters = 0;
    rep->converged = 1;
    if (!quasi) {
        const bool keep = reuse && !semi;     // the factors of the previous linear solve
        if (!keep) {
            assemble_fp64<TP>(C);
            ws->last_alpha = frob_shift(C, rcond);
        }
        const double alpha = ws->last_alpha;
        rep->alpha = alpha;
        rep->ms_assemble = elapsed_ms(t0);
        if (!semi) {
            auto t1 = std::chrono::steady_clock::now();
            if (!keep) {
                ewos_status s = factor_shifted<TP>(C, alpha, nullptr, pb->pivoting, rep);
                if (s != EWOS_OK) return s;
            }
            rep->ms_factor = elapsed_ms(t1);
            auto t2 = std::chrono::steady_clock::now();
            for (int64_t r = 0; r < nrhs; ++r) {       // rhs = -R_0(0)
                residual<TP>(C, nullptr, ws->g + r * C.p, ws->f + r * C.n, nullptr, 0, 0.0, ws->y);
                cudaMemsetAsync(ws->x + r * C.m, 0, sizeof(double) * C.m, C.st);
                ::ewos::note_launch(), axpy_kernel<<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.m, -1.0, ws->y, ws->x + r * C.m);
            }
            ewos_status s = lu_solve_device<double>(ws->LUm, (int)C.m, (int)C.m, ws->lu, ws->x, (int)nrhs, C.st);
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
                VgScope<TP> vgs(C, g);
                residual<TP>(C, s, g, f, nl, pb->nl_ncoef, alpha, ws->y);
                const double r0 = norm2(C, ws->y, C.m);
                double rn = r0;
                int it = 0;
                while (it < max_iter && rn > tol * r0) {
                    // u at the current s (from the residual just evaluated there), Jacobian term
                    // G^T diag(lam N'(u)) G
                    u_from_v(C, ws->u2);
                    dim3 gj((unsigned)((C.m + 255) / 256), (unsigned)C.n);
                    const TP* Gm = (const TP*)tb->P + (size_t)C.D * C.n * C.m;
                    ::ewos::note_launch(), jac_scale_kernel<TP><<<gj, 256, 0, C.st>>>(Gm, ws->u2, tb->lambda, nl, pb->nl_ncoef, ws->Jx, (int)C.n, (int)C.m);
                    auto t1 = std::chrono::steady_clock::now();
                    ewos_status st = factor_shifted<TP>(C, alpha, ws->Jx, pb->pivoting, rep);
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
            VgScope<TP> vgs(C, g);               // the residual at s = 0 of every iteration
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
                ewos_status st = factor_shifted<TP>(C, alpha, nullptr, pb->pivoting, rep);
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
constexpr bool kSplitTF32 = true;     // 3xTF32 assembly: Lambda to ~1e-6, fewer refinement sweeps

// LU = LU + L + alpha I  (m x m, grid-stride)
__global__ void add_shifted_kernel(float* __restrict__ LU, const float* __restrict__ L, int64_t count, int m,
                                   double alpha) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
        float v = LU[t] + L[t];
        if (t / m == t % m) v += (float)alpha;
        LU[t] = v;
    }
}

// the same in 16-byte pieces (m a multiple of 4, both matrices 16-byte aligned): row i's diagonal
// element sits in piece (i m + i) / 4
__global__ void add_shifted4_kernel(float4* __restrict__ LU, const float4* __restrict__ L, int64_t count4, int m,
                                    float alpha) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count4; t += (int64_t)gridDim.x * blockDim.x) {
        float4 v = __ldcs(LU + t);
        const float4 l = __ldcs(L + t);
        v.x += l.x; v.y += l.y; v.z += l.z; v.w += l.w;
        const int64_t e = 4 * t, row = e / m, col = e - row * m;
        if (row >= col && row < col + 4) {
            const int k = (int)(row - col);
            if (k == 0) v.x += alpha; else if (k == 1) v.y += alpha; else if (k == 2) v.z += alpha; else v.w += alpha;
        }
        __stcs(LU + t, v);
    }
}

// d_i = lam_i N'(u_i) in FP64, stored in FP32 (the factor jac_scale32_kernel applies to row i of G)
__global__ void jac_diag_kernel(const double* __restrict__ u, const double* __restrict__ lam, const double* __restrict__ nl,
                                int nnl, float* __restrict__ d, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double dd = 0.0, pw = 1.0;
    for (int t = 1; t < nnl; ++t) { dd += t * nl[t] * pw; pw *= u[i]; }
    d[i] = (float)(lam[i] * dd);
}

template <typename TP>
__global__ void jac_scale32_kernel(const TP* __restrict__ Gm, const double* __restrict__ u, const double* __restrict__ lam,
                                   const double* __restrict__ nl, int nnl, float* __restrict__ out, int n, int m,
                                   int vec) {
    // the row's factor lam_i N'(u_i) once per block in FP64, the scaling on the FP32 pipes (the
    // factors only precondition the FP64-refined Newton systems)
    // (block per row; 16-byte loads and stores when the rows are FP32 and 16-byte aligned)
    __shared__ float s_scale;
    const int i = blockIdx.x;
    if (threadIdx.x == 0) {
        double d = 0.0, pw = 1.0;
        for (int t = 1; t < nnl; ++t) { d += t * nl[t] * pw; pw *= u[i]; }
        s_scale = (float)(lam[i] * d);
    }
    __syncthreads();
    const float sc = s_scale;
    const TP* g = Gm + (size_t)i * m;
    float* o = out + (size_t)i * m;
    if (std::is_same<TP, float>::value && vec) {
        const float4* g4 = reinterpret_cast<const float4*>(g);
        float4* o4 = reinterpret_cast<float4*>(o);
        for (int c = threadIdx.x; c < (m >> 2); c += blockDim.x) {
            const float4 v = __ldcs(g4 + c);
            __stcs(o4 + c, make_float4(sc * v.x, sc * v.y, sc * v.z, sc * v.w));
        }
    } else {
        for (int c = threadIdx.x; c < m; c += blockDim.x) o[c] = sc * (float)g[c];
    }
}

static double frob32(const Ctx& C, const float* X, int64_t count) {
    cudaMemsetAsync(C.ws->scal, 0, sizeof(double), C.st);
    ::ewos::note_launch(), sumsq_f32_kernel<<<4 * 148 * 4, 256, 0, C.st>>>(X, count, C.ws->scal);
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
    const bool f2 = sizeof(TP) == 4 && C.ws->F2one;
    if (f2) apply_v_f2(C, x, nullptr);
    else ::ewos::note_launch(), rowdot_kernel<TP><<<(int)((rows * 32 + 255) / 256), 256, 0, C.st>>>(P, rows, (int)C.m, x, C.ws->v, 0);
    ::ewos::note_launch(), formw_jv_kernel<<<(int)((C.n + 127) / 128), 128, 0, C.st>>>((int)C.n, C.D, C.ws->M, C.ws->v,
                                                                                      C.tb->lambda, u, u ? nl : nullptr,
                                                                                      u ? nnl : 0, C.ws->w);
    if (f2) apply_PT_f2(C, C.ws->w, y);
    else apply_PT<TP>(C, C.ws->w, y);
    if (alpha != 0.0) ::ewos::note_launch(), axpy_kernel<<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.m, alpha, x, y);
}

// x <- solution of (A) x = b by the FP32 factors plus FP64 refinement; A applied by apply_op
template <typename TP>
static ewos_status refine(const Ctx& C, const double* b, double* x, double alpha, const double* u, const double* nl,
                          int nnl, double rel_tol, int max_sweeps, int* sweeps, double* final_rel, double b_norm = -1.0) {
    SolveWorkspace* ws = C.ws;
    const double nb = b_norm >= 0.0 ? b_norm : norm2(C, b, C.m);
    cudaMemsetAsync(x, 0, sizeof(double) * C.m, C.st);
    cudaMemcpyAsync(ws->r, b, sizeof(double) * C.m, cudaMemcpyDeviceToDevice, C.st);
    double rel = 1.0;
    int it = 0;
    while (it < max_sweeps) {
        cudaMemcpyAsync(ws->dx, ws->r, sizeof(double) * C.m, cudaMemcpyDeviceToDevice, C.st);
        // the triangular solves' error word is read with the residual's norm (one synchronisation)
        ewos_status st = lu_solve_device<float>(ws->LU32, (int)C.m, (int)C.m, ws->lu, ws->dx, 1, C.st, false);
        if (st != EWOS_OK) return st;
        ::ewos::note_launch(), axpy_kernel<<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.m, 1.0, ws->dx, x);
        apply_op<TP>(C, x, alpha, u, nl, nnl, ws->y);
        cudaMemcpyAsync(ws->r, b, sizeof(double) * C.m, cudaMemcpyDeviceToDevice, C.st);
        ::ewos::note_launch(), axpy_kernel<<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.m, -1.0, ws->y, ws->r);
        ++it;
        unsigned int flow_err = 0;
        const double nr = norm2(C, ws->r, C.m, ws->lu.flow + 1, &flow_err);
        if (flow_err) {
            cudaMemsetAsync(ws->lu.flow + 1, 0, sizeof(unsigned int), C.st);
            set_error("triangular solve: a wait on a preceding row block timed out");
            return EWOS_ETIMEOUT;
        }
        rel = nb > 0 ? nr / nb : 0.0;
        if (rel <= rel_tol) break;
    }
    *sweeps += it;
    if (final_rel) *final_rel = rel;
    return EWOS_OK;
}

// FP32 factors of the matrix that build() writes into LU32: first with the diagonal pivots
// (pivoting == 0; kept when it equals the partial-pivoting factorisation), else rebuilt and
// factored with row interchanges.
template <typename Build>
static ewos_status factor32_with(const Ctx& C, Build build, int pivoting, ewos_solve_report* rep) {
    build();
    ++rep->factorizations;
    DevSpan span(C.st, &rep->dev_ms_lu);
    if (pivoting == 0) {
        bool accepted = false;
        ewos_status s = lu_factor_nopiv<float>(C.ws->LU32, (int)C.m, (int)C.m, C.ws->lu, C.st, &accepted,
                                               tc_assemble_available() ? &C.ws->tc : nullptr);
        if (s != EWOS_OK) return s;
        if (accepted) return EWOS_OK;
        build();
    }
    ++rep->pivoted_factorizations;
    bool sing = false;
    ewos_status s = lu_factor_device<float>(C.ws->LU32, (int)C.m, (int)C.m, C.ws->lu, C.st, &sing);
    if (s != EWOS_OK) return s;
    if (sing) { set_error("LU (FP32): zero pivot"); return EWOS_ESINGULAR; }
    return EWOS_OK;
}

static ewos_status factor32(const Ctx& C, const float* src, double alpha, int pivoting, ewos_solve_report* rep) {
    return factor32_with(
        C,
        [&] {
            cudaMemcpyAsync(C.ws->LU32, src, sizeof(float) * C.m * C.m, cudaMemcpyDeviceToDevice, C.st);
            ::ewos::note_launch(), add_diag_kernel<float><<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.ws->LU32, (int)C.m,
                                                                                                   (int)C.m, alpha);
        },
        pivoting, rep);
}

// ------------------------------------------------------------------ all right-hand sides at once
// Layouts [rows][rc]: the rc right-hand sides of one row are contiguous (rc = the request's
// count rounded up to a power of two; the padding columns carry zeros).  The FP64 operator is
// applied to all of them with one pass over P (FP64 FMAs, the residual's precision); the FP32
// triangular solves run as one launch per 64-row block step (no grid barrier), so that the
// sweep can be captured in a CUDA graph and several requests can share the GPU.

// in [r][len] (r < R) -> out [len][rc] (zero columns r >= R)
__global__ void to_cols_kernel(const double* __restrict__ in, double* __restrict__ out, int64_t len, int R, int rc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= len * rc) return;
    const int64_t l = t / rc;
    const int r = (int)(t % rc);
    out[t] = r < R ? in[(size_t)r * len + l] : 0.0;
}

__global__ void from_cols_kernel(const double* __restrict__ in, double* __restrict__ out, int64_t len, int R, int rc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= len * R) return;
    const int r = (int)(t / len);
    const int64_t l = t % len;
    out[t] = in[l * rc + r];
}

// Vout[row][r] (+)= sum_c X[row][c] Vin[c][r]   (warp per row, RB right-hand sides per pass;
// rc is a power of two, RB = min(rc, 8); the FP32-pair version below takes RB = min(rc, 16))
template <typename TP, int RB>
__global__ void multi_rowdot_kernel(const TP* __restrict__ X, int64_t rows, int cols, const double* __restrict__ Vin,
                                    double* __restrict__ Vout, int rc, int accumulate) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const TP* xr = X + row * cols;
    for (int r0 = 0; r0 < rc; r0 += RB) {
        double acc[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) acc[q] = 0.0;
        for (int c = lane; c < cols; c += 32) {
            const double xv = (double)xr[c];
            const double* vr = Vin + (size_t)c * rc + r0;
#pragma unroll
            for (int q = 0; q < RB; ++q) acc[q] = fma(xv, vr[q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < RB; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
        }
        if (lane < RB) {
            double v = acc[0];
#pragma unroll
            for (int q = 1; q < RB; ++q)
                if (lane == q) v = acc[q];
            double* o = Vout + row * rc + r0 + lane;
            *o = accumulate ? *o + v : v;
        }
    }
}

// Y[c][r] += sum_{row in chunk} X[row][c] Win[row][r]   (thread per column; Y zeroed before;
// RB = min(rc, 8) right-hand sides per pass)
template <typename TP, int RB>
__global__ void multi_coltrans_kernel(const TP* __restrict__ X, int64_t rows, int cols, const double* __restrict__ Win,
                                      double* __restrict__ Y, int rc, int64_t chunk) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    const int64_t a = (int64_t)blockIdx.y * chunk;
    const int64_t b = min(rows, a + chunk);
    for (int r0 = 0; r0 < rc; r0 += RB) {
        double acc[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) acc[q] = 0.0;
        for (int64_t row = a; row < b; ++row) {
            const double xv = (double)X[row * cols + c];
            const double* wr = Win + row * rc + r0;
#pragma unroll
            for (int q = 0; q < RB; ++q) acc[q] = fma(xv, wr[q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < RB; ++q) atomicAdd(&Y[(size_t)c * rc + r0 + q], acc[q]);
    }
}

// W[e*n + i][r] = sum_k M_i[e][k] V[k*n + i][r] + [e == D] lam_i (N(u_ir) - F[i][r]),
// u_ir = V[D*n + i][r]   (thread per (i, r))
__global__ void formw_multi_kernel(int n, int D, const double* __restrict__ M, const double* __restrict__ V,
                                   const double* __restrict__ lam, const double* __restrict__ F,
                                   const double* __restrict__ nl, int nnl, double* __restrict__ W, int rc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * rc) return;
    const int i = (int)(t / rc), r = (int)(t % rc);
    const int E = D + 1;
    const double* Mi = M + (size_t)i * E * E;
    double vi[4];
    for (int k = 0; k < E; ++k) vi[k] = V[((size_t)k * n + i) * rc + r];
    for (int j = 0; j < E; ++j) {
        double acc = 0.0;
        for (int k = 0; k < E; ++k) acc += Mi[j * E + k] * vi[k];
        W[((size_t)j * n + i) * rc + r] = acc;
    }
    double extra = -F[(size_t)i * rc + r];
    if (nl) {
        double pw = 1.0, sv = 0.0;
        for (int q = 0; q < nnl; ++q) { sv += nl[q] * pw; pw *= vi[D]; }
        extra += sv;
    }
    W[((size_t)D * n + i) * rc + r] += lam[i] * extra;
}

__global__ void axpy_dev_kernel(int64_t count, const double* __restrict__ a, const double* __restrict__ x,
                                double* __restrict__ y) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] += a[0] * x[t];
}

// D[i][r] = -(float) Y[perm[i]][r]   (right-hand side of the correction, rows in pivot order)
__global__ void neg_gather32_kernel(const double* __restrict__ Y, const int* __restrict__ perm, float* __restrict__ D,
                                    int64_t m, int rc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * rc) return;
    const int64_t i = t / rc;
    const int r = (int)(t % rc);
    D[t] = (float)(-Y[(size_t)perm[i] * rc + r]);
}

__global__ void add_widen_kernel(int64_t count, const float* __restrict__ d, double* __restrict__ s) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) s[t] += (double)d[t];
}

// nrm[r] = sum_i Y[i][r]^2  (nrm zeroed before)
__global__ void colsumsq_kernel(const double* __restrict__ Y, int64_t m, int rc, double* __restrict__ nrm) {
    const int r = blockIdx.y;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = Y[i * rc + r];
        acc += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&nrm[r], acc);
}

__global__ void set_scalar_kernel(double* __restrict__ out, double v) {
    if (threadIdx.x == 0) out[0] = v;
}

__global__ void alpha_from_sumsq_kernel(const double* __restrict__ sumsq, double rcond, double* __restrict__ alpha) {
    if (threadIdx.x == 0) alpha[0] = rcond * sqrt(sumsq[0]);
}

__global__ void add_diag_dev_kernel(float* __restrict__ A, int m, int lda, const double* __restrict__ alpha) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) A[(size_t)i * lda + i] += (float)alpha[0];
}

// ------------------------------------------------------------------ FP64-accurate FP32 products
// P is FP32 (exact); a FP64 vector s enters as s_hi + s_lo (FP32 pair, s_lo = fp32(s - s_hi):
// 48 bits of s).  x * s_hi is split exactly into p + pe by one FMA, x * s_lo is second order;
// partial sums are unevaluated FP32 pairs (hi + lo, by TwoSum) and become FP64 for the final
// reduction.  A partial sum of k terms is exact to about k * 2^-48 relative, far below the
// refinement's 1e-10, at the FP32 issue rate (B300 runs FP64 FMAs at 1/64 of it).
// (the _rn intrinsics keep the compiler from contracting the error-free steps into FMAs)
__device__ __forceinline__ void f2_add_prod(float& hi, float& lo, float x, float shi, float slo) {
    const float p = __fmul_rn(x, shi);
    const float pe = __fmaf_rn(x, shi, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fmaf_rn(x, slo, __fadd_rn(lo, __fadd_rn(err, pe)));
}

__global__ void split_f2_kernel(const double* __restrict__ v, float* __restrict__ hi, float* __restrict__ lo,
                                int64_t count) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
        const double d = v[t];
        const float h = (float)d;
        hi[t] = h;
        lo[t] = (float)(d - (double)h);
    }
}

// hi/lo pair of v [cols][rc], stored transposed [rc][cols] (coalesced reads in the row products)
__global__ void split_f2_t_kernel(const double* __restrict__ v, float* __restrict__ hi, float* __restrict__ lo,
                                  int64_t cols, int rc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cols * rc) return;
    const int64_t c = t / rc;
    const int r = (int)(t % rc);
    const double d = v[t];
    const float h = (float)d;
    hi[(size_t)r * cols + c] = h;
    lo[(size_t)r * cols + c] = (float)(d - (double)h);
}

// Vout[row][r] (+)= sum_c X[row][c] V[c][r] with V = Vhi + Vlo given as [rc][cols]   (warp per
// row; lanes walk the columns, so every load is coalesced)
template <int RB>
__global__ void multi_rowdot_f2_kernel(const float* __restrict__ X, int64_t rows, int cols, const float* __restrict__ Vhi,
                                       const float* __restrict__ Vlo, double* __restrict__ Vout, int rc, int accumulate) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const float* xr = X + row * cols;
    for (int r0 = 0; r0 < rc; r0 += RB) {
        float hi[RB], lo[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) hi[q] = lo[q] = 0.f;
        for (int c = lane; c < cols; c += 32) {
            const float xv = xr[c];
#pragma unroll
            for (int q = 0; q < RB; ++q)
                f2_add_prod(hi[q], lo[q], xv, Vhi[(size_t)(r0 + q) * cols + c], Vlo[(size_t)(r0 + q) * cols + c]);
        }
        double acc[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            acc[q] = (double)hi[q] + (double)lo[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
        }
        if (lane < RB) {
            double v = acc[0];
#pragma unroll
            for (int q = 1; q < RB; ++q)
                if (lane == q) v = acc[q];
            double* o = Vout + row * rc + r0 + lane;
            *o = accumulate ? *o + v : v;
        }
    }
}

// Y[c][r] += sum_{row in chunk} X[row][c] W[row][r] with W = Whi + Wlo   (thread per column)
template <int RB>
__global__ void multi_coltrans_f2_kernel(const float* __restrict__ X, int64_t rows, int cols, const float* __restrict__ Whi,
                                         const float* __restrict__ Wlo, double* __restrict__ Y, int rc, int64_t chunk) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    const int64_t a = (int64_t)blockIdx.y * chunk;
    const int64_t b = min(rows, a + chunk);
    for (int r0 = 0; r0 < rc; r0 += RB) {
        float hi[RB], lo[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) hi[q] = lo[q] = 0.f;
        for (int64_t row = a; row < b; ++row) {
            const float xv = X[row * cols + c];
            float wh[RB], wl[RB];
            if (RB >= 4) {
#pragma unroll
                for (int q = 0; q < RB; q += 4) {
                    const float4 h4 = *reinterpret_cast<const float4*>(Whi + row * rc + r0 + q);
                    const float4 l4 = *reinterpret_cast<const float4*>(Wlo + row * rc + r0 + q);
                    wh[q] = h4.x; wh[q + 1] = h4.y; wh[q + 2] = h4.z; wh[q + 3] = h4.w;
                    wl[q] = l4.x; wl[q + 1] = l4.y; wl[q + 2] = l4.z; wl[q + 3] = l4.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < RB; ++q) { wh[q] = Whi[row * rc + r0 + q]; wl[q] = Wlo[row * rc + r0 + q]; }
            }
#pragma unroll
            for (int q = 0; q < RB; ++q) f2_add_prod(hi[q], lo[q], xv, wh[q], wl[q]);
        }
#pragma unroll
        for (int q = 0; q < RB; ++q) atomicAdd(&Y[(size_t)c * rc + r0 + q], (double)hi[q] + (double)lo[q]);
    }
}

// Single-column forms for 16-byte aligned operands with cols % 4 == 0.  The kernels above keep
// one load of X in flight per lane and a single pair chain, which leaves P's stream waiting on
// HBM latency (about a third of the copy rate); here every lane issues kU 16-byte streaming loads
// before it uses them and keeps four independent pairs (one per float4 component).
__device__ __forceinline__ void f2_add_prod4(float* hi, float* lo, const float4 x, const float4 h, const float4 l) {
    f2_add_prod(hi[0], lo[0], x.x, h.x, l.x);
    f2_add_prod(hi[1], lo[1], x.y, h.y, l.y);
    f2_add_prod(hi[2], lo[2], x.z, h.z, l.z);
    f2_add_prod(hi[3], lo[3], x.w, h.w, l.w);
}

// Vout[row] (+)= sum_c X[row][c] (Vhi[c] + Vlo[c])   (warp per row)
template <int kU>
__global__ void __launch_bounds__(256, 6) rowdot_f2_vec_kernel(const float* __restrict__ X, int64_t rows, int cols, const float* __restrict__ Vhi,
                                     const float* __restrict__ Vlo, double* __restrict__ Vout, int accumulate) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const float4* xr = reinterpret_cast<const float4*>(X + row * cols);
    const float4* vh = reinterpret_cast<const float4*>(Vhi);
    const float4* vl = reinterpret_cast<const float4*>(Vlo);
    const int c4 = cols >> 2;
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    int c = lane;
    for (; c + 32 * (kU - 1) < c4; c += 32 * kU) {
        float4 x[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) x[u] = __ldcs(xr + c + 32 * u);
#pragma unroll
        for (int u = 0; u < kU; ++u) f2_add_prod4(hi, lo, x[u], __ldg(vh + c + 32 * u), __ldg(vl + c + 32 * u));
    }
    for (; c < c4; c += 32) f2_add_prod4(hi, lo, __ldcs(xr + c), __ldg(vh + c), __ldg(vl + c));
    double acc = ((double)hi[0] + (double)lo[0]) + ((double)hi[1] + (double)lo[1]) + ((double)hi[2] + (double)lo[2]) +
                 ((double)hi[3] + (double)lo[3]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) Vout[row] = accumulate ? Vout[row] + acc : acc;
}

// Y[c] += sum_{row in chunk} X[row][c] (Whi[row] + Wlo[row])   (thread per four columns); with
// Ypart the chunk's sums are stored to row blockIdx.y of Ypart [chunks][cols] instead (summed in
// order by sum_parts_kernel: no atomics, the result independent of the order the CTAs run in)
template <int kU>
__global__ void coltrans_f2_vec_kernel(const float* __restrict__ X, int64_t rows, int cols, const float* __restrict__ Whi,
                                       const float* __restrict__ Wlo, double* __restrict__ Y, int64_t chunk,
                                       double* __restrict__ Ypart = nullptr) {
    const int c4 = blockIdx.x * blockDim.x + threadIdx.x;
    if (c4 >= (cols >> 2)) return;
    const int64_t a = (int64_t)blockIdx.y * chunk;
    const int64_t b = min(rows, a + chunk);
    const float4* xc = reinterpret_cast<const float4*>(X) + c4;
    const int64_t rs = cols >> 2;
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    int64_t r = a;
    for (; r + kU <= b; r += kU) {
        float4 x[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) x[u] = __ldcs(xc + (r + u) * rs);
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const float wh = __ldg(Whi + r + u), wl = __ldg(Wlo + r + u);
            f2_add_prod4(hi, lo, x[u], make_float4(wh, wh, wh, wh), make_float4(wl, wl, wl, wl));
        }
    }
    for (; r < b; ++r) {
        const float wh = __ldg(Whi + r), wl = __ldg(Wlo + r);
        f2_add_prod4(hi, lo, __ldcs(xc + r * rs), make_float4(wh, wh, wh, wh), make_float4(wl, wl, wl, wl));
    }
    if (Ypart) {
        double* yp = Ypart + (size_t)blockIdx.y * cols + (size_t)c4 * 4;
#pragma unroll
        for (int k = 0; k < 4; ++k) yp[k] = (double)hi[k] + (double)lo[k];
        return;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) atomicAdd(&Y[(size_t)c4 * 4 + k], (double)hi[k] + (double)lo[k]);
}

// Y[c] = sum over b of Ypart[b][c] in a fixed order: a CTA takes 32 columns, warp w sums parts
// w, w + 8, .. (eight loads in flight), and the eight warp sums are added in warp order
__global__ void __launch_bounds__(256) sum_parts_kernel(const double* __restrict__ Ypart, int parts, int cols,
                                                        double* __restrict__ Y) {
    __shared__ double red[8][33];
    const int tx = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + tx;
    double a = 0.0;
    if (c < cols) {
        int b = w;
        for (; b + 56 < parts; b += 64) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = Ypart[(size_t)(b + 8 * u) * cols + c];
#pragma unroll
            for (int u = 0; u < 8; ++u) a += v[u];
        }
        for (; b < parts; b += 8) a += Ypart[(size_t)b * cols + c];
    }
    red[w][tx] = a;
    __syncthreads();
    if (w == 0 && c < cols) {
        double t = red[0][tx];
#pragma unroll
        for (int k = 1; k < 8; ++k) t += red[k][tx];
        Y[c] = t;
    }
}

static inline bool aligned16(const void* q) { return ((uintptr_t)q & 15) == 0; }

// Many columns (rc >= 8): the products are small GEMMs on the FP32 pipes in FP32 pairs.  A CTA
// stages 32-column (32-row) slices of X and of the vector block in shared memory and every
// thread accumulates RW x 4 outputs as FP32 pairs, so each element of X is read once from HBM
// for all the CTA's columns (the kernels above read the vectors from L1/L2 once per product).
template <int RCT>
struct F2Tile {
    static constexpr int TX = RCT / 4;                 // threads across vector columns (4 each)
    static constexpr int TY = 256 / TX;                // threads across matrix rows (columns)
    static constexpr int RW = TY >= 64 ? 1 : 64 / TY;  // rows per thread
    static constexpr int TR = TY * RW;                 // rows per CTA
    static constexpr int CK = 32;                      // slice depth
};

// Vout[row][r] (+)= sum_c X[row][c] V[r][c], V = Vhi + Vlo given as [rc][cols]
template <int RCT>
__global__ void __launch_bounds__(256) rowdot_f2_tile_kernel(const float* __restrict__ X, int64_t rows, int cols,
                                                            const float* __restrict__ Vhi, const float* __restrict__ Vlo,
                                                            double* __restrict__ Vout, int rc, int accumulate) {
    using F = F2Tile<RCT>;
    constexpr int TX = F::TX, TY = F::TY, RW = F::RW, TR = F::TR, CK = F::CK;
    __shared__ float Xs[CK][TR + 1];
    __shared__ __align__(16) float Hs[CK][RCT + 4];
    __shared__ __align__(16) float Ls[CK][RCT + 4];
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int64_t row0 = (int64_t)blockIdx.x * TR;
    const int r0 = blockIdx.y * RCT;
    float hi[RW][4], lo[RW][4];
#pragma unroll
    for (int i = 0; i < RW; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) hi[i][j] = lo[i][j] = 0.f;
    for (int c0 = 0; c0 < cols; c0 += CK) {
        for (int e = threadIdx.x; e < TR * CK; e += 256) {
            const int r = e / CK, c = e % CK;
            const int64_t gr = row0 + r;
            Xs[c][r] = (gr < rows && c0 + c < cols) ? __ldcs(X + gr * cols + c0 + c) : 0.f;
        }
        for (int e = threadIdx.x; e < RCT * CK; e += 256) {
            const int j = e / CK, c = e % CK;
            const bool ok = r0 + j < rc && c0 + c < cols;
            Hs[c][j] = ok ? Vhi[(size_t)(r0 + j) * cols + c0 + c] : 0.f;
            Ls[c][j] = ok ? Vlo[(size_t)(r0 + j) * cols + c0 + c] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int c = 0; c < CK; ++c) {
            float x[RW];
#pragma unroll
            for (int i = 0; i < RW; ++i) x[i] = Xs[c][ty + TY * i];
            const float4 h = *reinterpret_cast<const float4*>(&Hs[c][tx * 4]);
            const float4 l = *reinterpret_cast<const float4*>(&Ls[c][tx * 4]);
#pragma unroll
            for (int i = 0; i < RW; ++i) {
                f2_add_prod(hi[i][0], lo[i][0], x[i], h.x, l.x);
                f2_add_prod(hi[i][1], lo[i][1], x[i], h.y, l.y);
                f2_add_prod(hi[i][2], lo[i][2], x[i], h.z, l.z);
                f2_add_prod(hi[i][3], lo[i][3], x[i], h.w, l.w);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < RW; ++i) {
        const int64_t row = row0 + ty + TY * i;
        if (row >= rows) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = r0 + tx * 4 + j;
            if (r >= rc) continue;
            const double v = (double)hi[i][j] + (double)lo[i][j];
            double* o = Vout + row * rc + r;
            *o = accumulate ? *o + v : v;
        }
    }
}

// Y[c][r] += sum_{row in chunk} X[row][c] W[row][r], W = Whi + Wlo given as [rows][rc]
template <int RCT>
__global__ void __launch_bounds__(256) coltrans_f2_tile_kernel(const float* __restrict__ X, int64_t rows, int cols,
                                                              const float* __restrict__ Whi, const float* __restrict__ Wlo,
                                                              double* __restrict__ Y, int rc, int64_t chunk) {
    using F = F2Tile<RCT>;
    constexpr int TX = F::TX, TY = F::TY, RW = F::RW, TR = F::TR, CK = F::CK;
    __shared__ float Xs[CK][TR + 1];
    __shared__ __align__(16) float Hs[CK][RCT + 4];
    __shared__ __align__(16) float Ls[CK][RCT + 4];
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int col0 = blockIdx.x * TR;
    const int r0 = blockIdx.y * RCT;
    const int64_t a = (int64_t)blockIdx.z * chunk;
    const int64_t b = min(rows, a + chunk);
    float hi[RW][4], lo[RW][4];
#pragma unroll
    for (int i = 0; i < RW; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) hi[i][j] = lo[i][j] = 0.f;
    for (int64_t k0 = a; k0 < b; k0 += CK) {
        for (int e = threadIdx.x; e < TR * CK; e += 256) {
            const int k = e / TR, c = e % TR;
            Xs[k][c] = (k0 + k < b && col0 + c < cols) ? __ldcs(X + (k0 + k) * cols + col0 + c) : 0.f;
        }
        for (int e = threadIdx.x; e < RCT * CK; e += 256) {
            const int k = e / RCT, j = e % RCT;
            const bool ok = k0 + k < b && r0 + j < rc;
            Hs[k][j] = ok ? Whi[(k0 + k) * rc + r0 + j] : 0.f;
            Ls[k][j] = ok ? Wlo[(k0 + k) * rc + r0 + j] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < CK; ++k) {
            float x[RW];
#pragma unroll
            for (int i = 0; i < RW; ++i) x[i] = Xs[k][ty + TY * i];
            const float4 h = *reinterpret_cast<const float4*>(&Hs[k][tx * 4]);
            const float4 l = *reinterpret_cast<const float4*>(&Ls[k][tx * 4]);
#pragma unroll
            for (int i = 0; i < RW; ++i) {
                f2_add_prod(hi[i][0], lo[i][0], x[i], h.x, l.x);
                f2_add_prod(hi[i][1], lo[i][1], x[i], h.y, l.y);
                f2_add_prod(hi[i][2], lo[i][2], x[i], h.z, l.z);
                f2_add_prod(hi[i][3], lo[i][3], x[i], h.w, l.w);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < RW; ++i) {
        const int c = col0 + ty + TY * i;
        if (c >= cols) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = r0 + tx * 4 + j;
            if (r < rc) atomicAdd(&Y[(size_t)c * rc + r], (double)hi[i][j] + (double)lo[i][j]);
        }
    }
}

template <int RCT>
static void rowdot_f2_tile(cudaStream_t st, const float* X, int64_t rows, int cols, const float* Vhi, const float* Vlo,
                           double* Vout, int rc, int accumulate) {
    using F = F2Tile<RCT>;
    dim3 grid((unsigned)((rows + F::TR - 1) / F::TR), (unsigned)((rc + RCT - 1) / RCT));
    ::ewos::note_launch(), rowdot_f2_tile_kernel<RCT><<<grid, 256, 0, st>>>(X, rows, cols, Vhi, Vlo, Vout, rc, accumulate);
}

template <int RCT>
static void coltrans_f2_tile(cudaStream_t st, const float* X, int64_t rows, int cols, const float* Whi, const float* Wlo,
                             double* Y, int rc) {
    using F = F2Tile<RCT>;
    const int64_t chunk = 1024;
    dim3 grid((unsigned)((cols + F::TR - 1) / F::TR), (unsigned)((rc + RCT - 1) / RCT), (unsigned)((rows + chunk - 1) / chunk));
    ::ewos::note_launch(), coltrans_f2_tile_kernel<RCT><<<grid, 256, 0, st>>>(X, rows, cols, Whi, Wlo, Y, rc, chunk);
}

static void multi_rowdot_f2(cudaStream_t st, const float* X, int64_t rows, int cols, const float* Vhi, const float* Vlo,
                            double* Vout, int rc, int accumulate) {
    const int rb = (int)std::max<int64_t>(1, (rows * 32 + 255) / 256);
    if (rc == 1 && cols % 4 == 0 && aligned16(X) && aligned16(Vhi) && aligned16(Vlo)) {
        ::ewos::note_launch(), rowdot_f2_vec_kernel<4><<<rb, 256, 0, st>>>(X, rows, cols, Vhi, Vlo, Vout, accumulate);
        return;
    }
    if (rc >= 64) return rowdot_f2_tile<64>(st, X, rows, cols, Vhi, Vlo, Vout, rc, accumulate);
    if (rc >= 32) return rowdot_f2_tile<32>(st, X, rows, cols, Vhi, Vlo, Vout, rc, accumulate);
    if (rc >= 16) return rowdot_f2_tile<16>(st, X, rows, cols, Vhi, Vlo, Vout, rc, accumulate);
    if (rc >= 8) return rowdot_f2_tile<8>(st, X, rows, cols, Vhi, Vlo, Vout, rc, accumulate);
    if (rc == 1) ::ewos::note_launch(), multi_rowdot_f2_kernel<1><<<rb, 256, 0, st>>>(X, rows, cols, Vhi, Vlo, Vout, rc, accumulate);
    else if (rc == 2) ::ewos::note_launch(), multi_rowdot_f2_kernel<2><<<rb, 256, 0, st>>>(X, rows, cols, Vhi, Vlo, Vout, rc, accumulate);
    else if (rc == 4) ::ewos::note_launch(), multi_rowdot_f2_kernel<4><<<rb, 256, 0, st>>>(X, rows, cols, Vhi, Vlo, Vout, rc, accumulate);
    else if (rc == 8) ::ewos::note_launch(), multi_rowdot_f2_kernel<8><<<rb, 256, 0, st>>>(X, rows, cols, Vhi, Vlo, Vout, rc, accumulate);
    else ::ewos::note_launch(), multi_rowdot_f2_kernel<16><<<rb, 256, 0, st>>>(X, rows, cols, Vhi, Vlo, Vout, rc, accumulate);
}

static void multi_coltrans_f2(cudaStream_t st, const float* X, int64_t rows, int cols, const float* Whi, const float* Wlo,
                              double* Y, int rc) {
    if (rc >= 64) return coltrans_f2_tile<64>(st, X, rows, cols, Whi, Wlo, Y, rc);
    if (rc >= 32) return coltrans_f2_tile<32>(st, X, rows, cols, Whi, Wlo, Y, rc);
    if (rc >= 16) return coltrans_f2_tile<16>(st, X, rows, cols, Whi, Wlo, Y, rc);
    if (rc >= 8) return coltrans_f2_tile<8>(st, X, rows, cols, Whi, Wlo, Y, rc);
    if (rc == 1 && cols % 4 == 0 && aligned16(X)) {
        const int64_t vchunk = 256;
        dim3 vgrid((unsigned)((cols / 4 + 127) / 128), (unsigned)((rows + vchunk - 1) / vchunk));
        ::ewos::note_launch(), coltrans_f2_vec_kernel<8><<<vgrid, 128, 0, st>>>(X, rows, cols, Whi, Wlo, Y, vchunk);
        return;
    }
    const int64_t chunk = 512;
    dim3 grid((unsigned)((cols + 127) / 128), (unsigned)((rows + chunk - 1) / chunk));
    if (rc == 1) ::ewos::note_launch(), multi_coltrans_f2_kernel<1><<<grid, 128, 0, st>>>(X, rows, cols, Whi, Wlo, Y, rc, chunk);
    else if (rc == 2) ::ewos::note_launch(), multi_coltrans_f2_kernel<2><<<grid, 128, 0, st>>>(X, rows, cols, Whi, Wlo, Y, rc, chunk);
    else if (rc == 4) ::ewos::note_launch(), multi_coltrans_f2_kernel<4><<<grid, 128, 0, st>>>(X, rows, cols, Whi, Wlo, Y, rc, chunk);
    else if (rc == 8) ::ewos::note_launch(), multi_coltrans_f2_kernel<8><<<grid, 128, 0, st>>>(X, rows, cols, Whi, Wlo, Y, rc, chunk);
    else ::ewos::note_launch(), multi_coltrans_f2_kernel<16><<<grid, 128, 0, st>>>(X, rows, cols, Whi, Wlo, Y, rc, chunk);
}

// Y = X^T (Whi + Wlo) for one column: the 256-row x 512-column tiles of coltrans_f2_vec_kernel
// with their sums stored as partials and added in order (no atomics); X 16-byte aligned, cols a
// multiple of 4; false when it does not apply or the partials cannot be allocated (the caller
// then takes the atomic form)
static bool coltrans_rows(const Ctx& C, const float* X, int64_t rows, int cols, const float* Whi, const float* Wlo,
                          double* Y) {
    if (cols % 4 != 0 || !aligned16(X) || rows < 1) return false;
    // row chunks sized so that the grid is one full wave of resident CTAs: with fixed 256-row
    // chunks the ball's 2000 CTAs made 1.13 waves, and the last 13 % took as long as a full wave
    static int slots = 0;
    if (slots == 0) {
        int dev = 0, nsm = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coltrans_f2_vec_kernel<8>, 128, 0);
        slots = std::max(1, nsm * std::max(1, per_sm));
    }
    const int gx = (cols / 4 + 127) / 128;
    const int64_t want = std::max<int64_t>(1, slots / gx);
    const int64_t vchunk = std::max<int64_t>(8, (rows + want - 1) / want);
    const int parts = (int)((rows + vchunk - 1) / vchunk);
    SolveWorkspace* ws = C.ws;
    if (ws->ctpart_cap < (int64_t)parts * cols) {
        ::ewos::dev_free(ws->ctpart);
        ws->ctpart = nullptr;
        ws->ctpart_cap = 0;
        if (::ewos::dev_alloc((void**)&ws->ctpart, sizeof(double) * (size_t)parts * cols) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        ws->ctpart_cap = (int64_t)parts * cols;
    }
    dim3 vgrid((unsigned)((cols / 4 + 127) / 128), (unsigned)parts);
    ::ewos::note_launch(), coltrans_f2_vec_kernel<8><<<vgrid, 128, 0, C.st>>>(X, rows, cols, Whi, Wlo, Y, vchunk, ws->ctpart);
    ::ewos::note_launch(), sum_parts_kernel<<<(cols + 31) / 32, 256, 0, C.st>>>(ws->ctpart, parts, cols, Y);
    return true;
}

static void split_f2(cudaStream_t st, const double* v, float* hi, float* lo, int64_t count) {
    ::ewos::note_launch(), split_f2_kernel<<<(int)std::min<int64_t>(4096, (count + 255) / 256), 256, 0, st>>>(v, hi, lo, count);
}

template <typename TP>
static void multi_rowdot(cudaStream_t st, const TP* X, int64_t rows, int cols, const double* Vin, double* Vout, int rc,
                         int accumulate) {
    const int rb = (int)std::max<int64_t>(1, (rows * 32 + 255) / 256);
    if (rc == 1) ::ewos::note_launch(), multi_rowdot_kernel<TP, 1><<<rb, 256, 0, st>>>(X, rows, cols, Vin, Vout, rc, accumulate);
    else if (rc == 2) ::ewos::note_launch(), multi_rowdot_kernel<TP, 2><<<rb, 256, 0, st>>>(X, rows, cols, Vin, Vout, rc, accumulate);
    else if (rc == 4) ::ewos::note_launch(), multi_rowdot_kernel<TP, 4><<<rb, 256, 0, st>>>(X, rows, cols, Vin, Vout, rc, accumulate);
    else ::ewos::note_launch(), multi_rowdot_kernel<TP, 8><<<rb, 256, 0, st>>>(X, rows, cols, Vin, Vout, rc, accumulate);
}

template <typename TP>
static void multi_coltrans(cudaStream_t st, const TP* X, int64_t rows, int cols, const double* Win, double* Y, int rc) {
    const int64_t chunk = 512;
    dim3 grid((unsigned)((cols + 127) / 128), (unsigned)((rows + chunk - 1) / chunk));
    if (rc == 1) ::ewos::note_launch(), multi_coltrans_kernel<TP, 1><<<grid, 128, 0, st>>>(X, rows, cols, Win, Y, rc, chunk);
    else if (rc == 2) ::ewos::note_launch(), multi_coltrans_kernel<TP, 2><<<grid, 128, 0, st>>>(X, rows, cols, Win, Y, rc, chunk);
    else if (rc == 4) ::ewos::note_launch(), multi_coltrans_kernel<TP, 4><<<grid, 128, 0, st>>>(X, rows, cols, Win, Y, rc, chunk);
    else ::ewos::note_launch(), multi_coltrans_kernel<TP, 8><<<grid, 128, 0, st>>>(X, rows, cols, Win, Y, rc, chunk);
}

static int64_t bucket_of(int64_t R) {
    int64_t b = 1;
    while (b < R) b <<= 1;
    return b;
}

size_t workspace_bytes(const ewos_toolbox* tb, int64_t nrhs, bool mixed) {
    const size_t n = (size_t)tb->n, m = (size_t)tb->m, p = (size_t)tb->p, E = (size_t)tb->dim + 1;
    const size_t rc = (size_t)bucket_of(std::max<int64_t>(1, nrhs));
    size_t b = 8 * (n * E * E + n * E * E + n * (E + 1) + (n + p + 5 * m) * nrhs + 4 * E * n + 3 * m);   // vectors
    b += 8 * ((m + 63) / 64) * 2 * 64 * 64 + 4 * ((m + 63) / 64) * 64 * 64 + 16 * m + 4 * flow_state_words(m);   // LU side
    if (mixed) {
        const size_t Kp = (E * n + 31) / 32 * 32;
        b += 4 * (E * n * m + 3 * m * m + n * m);                 // Q32, L32, LU32, Jx32
        b += 4 * 4 * std::max(m, m) * Kp;                          // TF32 hi/lo transposes
        if (tb->precision == 64) b += 4 * E * n * m;               // FP32 copy of P
        b += 8 * rc * (2 * m + 2 * E * n + 2 * n + p + 1) + 8 * rc * m;   // batched columns
    } else {
        b += 8 * (E * n * m + 2 * m * m + n * m);                  // Q, Lambda, LU, Jx
    }
    return b;
}

static constexpr size_t kMaxSweepGraphs = 16;
// columns of m and of p per thread in the fused one-column residual (m <= 4096, p <= 1024)
constexpr int kFusedCols = 16, kFusedColsH = 4;

static ewos_status ensure_batched(const Ctx& C, int64_t rc) {
    SolveWorkspace* ws = C.ws;
    if (ws->bcap >= rc && ws->Sb) return EWOS_OK;
    for (auto& g : ws->graphs) cudaGraphExecDestroy(g.exec);
    ws->graphs.clear();
    // every buffer of the set is freed and cleared first, and the capacity is set only once all
    // of them exist: a failed allocation leaves an empty set that the next call rebuilds
    ws->bcap = 0;
    for (double** b : {&ws->Sb, &ws->Yb, &ws->Vb, &ws->Wb, &ws->Fb, &ws->Gb, &ws->Ub, &ws->nrm}) {
        ::ewos::dev_free(*b);
        *b = nullptr;
    }
    for (float** b : {&ws->D32, &ws->D32p, &ws->F2buf}) {
        ::ewos::dev_free(*b);
        *b = nullptr;
    }
    const int64_t rows = (int64_t)C.E * C.n;
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->F2buf, sizeof(float) * 2 * (C.m + C.p + rows) * rc));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Sb, sizeof(double) * C.m * rc));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Yb, sizeof(double) * C.m * rc));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Vb, sizeof(double) * rows * rc));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Wb, sizeof(double) * rows * rc));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Fb, sizeof(double) * C.n * rc));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Gb, sizeof(double) * C.p * rc));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Ub, sizeof(double) * C.n * rc));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->nrm, sizeof(double) * rc));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->D32, sizeof(float) * C.m * rc));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->D32p, sizeof(float) * C.m * rc));
    if (!ws->alpha_dev) EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->alpha_dev, sizeof(double)));
    if (!ws->Ypart && C.tb->precision == 32 && C.m <= 256 * kFusedCols && C.p <= 256 * kFusedColsH && (C.E == 3 || C.E == 4)) {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        ws->ypart_grid = std::max(1, std::min(nsm, (int)C.n));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ws->Ypart, sizeof(double) * ws->ypart_grid * C.m));
    }
    ws->bcap = rc;
    return EWOS_OK;
}

static int nblocks(int64_t count, int tpb = 256) { return (int)std::max<int64_t>(1, (count + tpb - 1) / tpb); }

// (h, l) += (h2, l2) for unevaluated FP32 pairs (two-sum of the high parts)
__device__ __forceinline__ void f2_merge(float& h, float& l, float h2, float l2) {
    const float sum = __fadd_rn(h, h2);
    const float bb = __fsub_rn(sum, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(sum, bb)), __fsub_rn(h2, bb));
    h = sum;
    l = __fadd_rn(__fadd_rn(l, l2), err);
}

// One right-hand side, FP32 toolbox, m <= 4096, p <= 1024: the residual's two passes over P in
// one.  A CTA takes nodes i = b, b + grid, ..; for each it holds the node's d+1 rows of P in
// registers (16 columns per thread; the next node's rows are loaded meanwhile), forms v_i = P_i s + KH_i g (FP32 pairs, reduced over the
// CTA), w_i = M_i v_i + e_d lam_i (N(v_{d,i}) - f_i) (FP64, by d+1 threads), and adds P_i^T w_i
// to its own partial of Y (FP32 pairs per column); Ypart [grid][m] is summed by
// reduce_partials_kernel.  s, g arrive split into FP32 pairs.
template <int E>
__global__ void __launch_bounds__(256, 1) residual1_f2_kernel(const float* __restrict__ P, const float* __restrict__ KH,
                                                              int n, int m, int p, const float* __restrict__ Shi,
                                                              const float* __restrict__ Slo, const float* __restrict__ Ghi,
                                                              const float* __restrict__ Glo, const double* __restrict__ M,
                                                              const double* __restrict__ lam, const double* __restrict__ F,
                                                              const double* __restrict__ nl, int nnl,
                                                              double* __restrict__ Ypart) {
    constexpr int D = E - 1;
    __shared__ float red_h[8][E], red_l[8][E];
    __shared__ float w_h[E], w_l[E];
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    const size_t nm = (size_t)n * m, np = (size_t)n * p;
    float sh[kFusedCols], sl[kFusedCols], yh[kFusedCols], yl[kFusedCols];
#pragma unroll
    for (int k = 0; k < kFusedCols; ++k) {
        const int c = tid + 256 * k;
        sh[k] = c < m ? Shi[c] : 0.f;
        sl[k] = c < m ? Slo[c] : 0.f;
        yh[k] = yl[k] = 0.f;
    }
    float gh[kFusedColsH], gl[kFusedColsH];
#pragma unroll
    for (int k = 0; k < kFusedColsH; ++k) {
        const int c = tid + 256 * k;
        gh[k] = c < p ? Ghi[c] : 0.f;
        gl[k] = c < p ? Glo[c] : 0.f;
    }
    // the rows of the next node are loaded while the current one is reduced and applied
    float pn[E][kFusedCols];
    auto load_rows = [&](int i) {
#pragma unroll
        for (int l = 0; l < E; ++l)
#pragma unroll
            for (int k = 0; k < kFusedCols; ++k) {
                const int c = tid + 256 * k;
                pn[l][k] = (i < n && c < m) ? P[l * nm + (size_t)i * m + c] : 0.f;
            }
    };
    load_rows(blockIdx.x);
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        float pv[E][kFusedCols];
#pragma unroll
        for (int l = 0; l < E; ++l)
#pragma unroll
            for (int k = 0; k < kFusedCols; ++k) pv[l][k] = pn[l][k];
        load_rows(i + gridDim.x);
        float vh[E], vl[E];
#pragma unroll
        for (int l = 0; l < E; ++l) {
            vh[l] = vl[l] = 0.f;
#pragma unroll
            for (int k = 0; k < kFusedCols; ++k) f2_add_prod(vh[l], vl[l], pv[l][k], sh[k], sl[k]);
#pragma unroll
            for (int k = 0; k < kFusedColsH; ++k) {
                const int c = tid + 256 * k;
                if (c < p) f2_add_prod(vh[l], vl[l], KH[l * np + (size_t)i * p + c], gh[k], gl[k]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                f2_merge(vh[l], vl[l], __shfl_xor_sync(0xffffffffu, vh[l], o), __shfl_xor_sync(0xffffffffu, vl[l], o));
            if (lane == 0) {
                red_h[wp][l] = vh[l];
                red_l[wp][l] = vl[l];
            }
        }
        __syncthreads();
        if (tid < E) {
            double vi[E];
#pragma unroll
            for (int l = 0; l < E; ++l) {
                double a = 0.0;
#pragma unroll
                for (int q = 0; q < 8; ++q) a += (double)red_h[q][l] + (double)red_l[q][l];
                vi[l] = a;
            }
            const double* Mi = M + (size_t)i * E * E;
            double wj = 0.0;
#pragma unroll
            for (int l = 0; l < E; ++l) wj += Mi[tid * E + l] * vi[l];
            if (tid == D) {
                double extra = -F[i];
                if (nl) {
                    double pw = 1.0, sv = 0.0;
                    for (int q = 0; q < nnl; ++q) { sv += nl[q] * pw; pw *= vi[D]; }
                    extra += sv;
                }
                wj += lam[i] * extra;
            }
            const float h = (float)wj;
            w_h[tid] = h;
            w_l[tid] = (float)(wj - (double)h);
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < E; ++l) {
            const float wh = w_h[l], wl = w_l[l];
#pragma unroll
            for (int k = 0; k < kFusedCols; ++k) f2_add_prod(yh[k], yl[k], pv[l][k], wh, wl);
        }
    }
#pragma unroll
    for (int k = 0; k < kFusedCols; ++k) {
        const int c = tid + 256 * k;
        if (c < m) Ypart[(size_t)blockIdx.x * m + c] = (double)yh[k] + (double)yl[k];
    }
}

// Y[c] = sum over the parts of Ypart[b][c] + alpha S[c]
__global__ void reduce_partials_kernel(const double* __restrict__ Ypart, int parts, int m, const double* __restrict__ alpha,
                                       const double* __restrict__ S, double* __restrict__ Y) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    double a = 0.0;
    for (int b = 0; b < parts; ++b) a += Ypart[(size_t)b * m + c];
    Y[c] = a + alpha[0] * S[c];
}

// Yb = R(Sb) + alpha Sb for all columns (f, g of the request in Fb, Gb; nl may be NULL)
template <typename TP>
static void residual_multi(const Ctx& C, int64_t rc, int R, const double* nl, int nnl) {
    SolveWorkspace* ws = C.ws;
    const TP* P = (const TP*)C.tb->P;
    const TP* KH = (const TP*)C.tb->KH;
    const int64_t rows = (int64_t)C.E * C.n;
    float* Shi = ws->F2buf;
    float* Slo = Shi + C.m * rc;
    float* Ghi = Slo + C.m * rc;
    float* Glo = Ghi + C.p * rc;
    float* Whi = Glo + C.p * rc;
    float* Wlo = Whi + rows * rc;
    if (sizeof(TP) == 4 && rc == 1 && ws->Ypart) {
        ::ewos::note_launch(), split_f2_t_kernel<<<nblocks(C.m), 256, 0, C.st>>>(ws->Sb, Shi, Slo, C.m, 1);
        ::ewos::note_launch(), split_f2_t_kernel<<<nblocks(C.p), 256, 0, C.st>>>(ws->Gb, Ghi, Glo, C.p, 1);
        const float* P32 = (const float*)P;
        const float* KH32 = (const float*)KH;
        if (C.E == 3)
            ::ewos::note_launch(), residual1_f2_kernel<3><<<ws->ypart_grid, 256, 0, C.st>>>(
                                       P32, KH32, (int)C.n, (int)C.m, (int)C.p, Shi, Slo, Ghi, Glo, ws->M, C.tb->lambda,
                                       ws->Fb, nl, nnl, ws->Ypart);
        else
            ::ewos::note_launch(), residual1_f2_kernel<4><<<ws->ypart_grid, 256, 0, C.st>>>(
                                       P32, KH32, (int)C.n, (int)C.m, (int)C.p, Shi, Slo, Ghi, Glo, ws->M, C.tb->lambda,
                                       ws->Fb, nl, nnl, ws->Ypart);
        ::ewos::note_launch(), reduce_partials_kernel<<<nblocks(C.m), 256, 0, C.st>>>(ws->Ypart, ws->ypart_grid, (int)C.m,
                                                                                    ws->alpha_dev, ws->Sb, ws->Yb);
        return;
    }
    if (sizeof(TP) == 4) {
        ::ewos::note_launch(), split_f2_t_kernel<<<nblocks(C.m * rc), 256, 0, C.st>>>(ws->Sb, Shi, Slo, C.m, (int)rc);
        ::ewos::note_launch(), split_f2_t_kernel<<<nblocks(C.p * rc), 256, 0, C.st>>>(ws->Gb, Ghi, Glo, C.p, (int)rc);
        multi_rowdot_f2(C.st, (const float*)P, rows, (int)C.m, Shi, Slo, ws->Vb, (int)rc, 0);
        multi_rowdot_f2(C.st, (const float*)KH, rows, (int)C.p, Ghi, Glo, ws->Vb, (int)rc, 1);
    } else {
        multi_rowdot<TP>(C.st, P, rows, (int)C.m, ws->Sb, ws->Vb, (int)rc, 0);
        multi_rowdot<TP>(C.st, KH, rows, (int)C.p, ws->Gb, ws->Vb, (int)rc, 1);
    }
    (void)R;   // padding columns are processed like the others (zero data); graphs depend on rc only
    ::ewos::note_launch(), formw_multi_kernel<<<nblocks(C.n * rc, 128), 128, 0, C.st>>>(
        (int)C.n, C.D, ws->M, ws->Vb, C.tb->lambda, ws->Fb, nl, nnl, ws->Wb, (int)rc);
    cudaMemsetAsync(ws->Yb, 0, sizeof(double) * C.m * rc, C.st);
    if (sizeof(TP) == 4) {
        split_f2(C.st, ws->Wb, Whi, Wlo, rows * rc);
        multi_coltrans_f2(C.st, (const float*)P, rows, (int)C.m, Whi, Wlo, ws->Yb, (int)rc);
    } else {
        multi_coltrans<TP>(C.st, P, rows, (int)C.m, ws->Wb, ws->Yb, (int)rc);
    }
    ::ewos::note_launch(), axpy_dev_kernel<<<nblocks(C.m * rc), 256, 0, C.st>>>(C.m * rc, ws->alpha_dev, ws->Sb, ws->Yb);
}

static void colnorms(const Ctx& C, int64_t rc) {
    cudaMemsetAsync(C.ws->nrm, 0, sizeof(double) * rc, C.st);
    dim3 g((unsigned)std::min<int64_t>(64, (C.m + 255) / 256), (unsigned)rc);
    ::ewos::note_launch(), colsumsq_kernel<<<g, 256, 0, C.st>>>(C.ws->Yb, C.m, (int)rc, C.ws->nrm);
}

// One sweep: correction from the FP32 factors for every column, s += correction, new residual
// and its column norms.  Launch count returned for the launch counter of graph replays.
template <typename TP>
static int sweep_multi(const Ctx& C, int64_t rc, int R, const double* nl, int nnl) {
    SolveWorkspace* ws = C.ws;
    const unsigned long long l0 = ewos_launch_count();
    const int m = (int)C.m;
    ::ewos::note_launch(), neg_gather32_kernel<<<nblocks(C.m * rc), 256, 0, C.st>>>(ws->Yb, ws->lu.perm, ws->D32, C.m, (int)rc);
    trsm_flow<float>(ws->LU32, m, m, (const float*)ws->lu.dinv, ws->D32, (int)rc, ws->lu.flow, C.st);
    ::ewos::note_launch(), add_widen_kernel<<<nblocks(C.m * rc), 256, 0, C.st>>>(C.m * rc, ws->D32, ws->Sb);
    residual_multi<TP>(C, rc, R, nl, nnl);
    colnorms(C, rc);
    return (int)(ewos_launch_count() - l0);
}

// Batched refinement (linear) or chord iteration (semilinear) for the R right-hand sides of the
// request on factors already in LU32; returns false (nothing reported) when it does not reach
// tol so that the caller takes the per-right-hand-side path.
template <typename TP>
static ewos_status solve_batched(const Ctx& C, int R, const double* nl, int nnl, double tol, int max_sweeps,
                                 int* sweeps, bool* ok, double* final_rel, double* last_norm = nullptr) {
    SolveWorkspace* ws = C.ws;
    const int64_t rc = bucket_of(R);
    *ok = false;
    ewos_status s = ensure_batched(C, rc);
    if (s != EWOS_OK) return s;
    ::ewos::note_launch(), to_cols_kernel<<<nblocks(C.n * rc), 256, 0, C.st>>>(ws->f, ws->Fb, C.n, R, (int)rc);
    ::ewos::note_launch(), to_cols_kernel<<<nblocks(C.p * rc), 256, 0, C.st>>>(ws->g, ws->Gb, C.p, R, (int)rc);
    EWOS_CUDA_TRY(cudaMemsetAsync(ws->Sb, 0, sizeof(double) * C.m * rc, C.st));
    residual_multi<TP>(C, rc, R, nl, nnl);
    colnorms(C, rc);
    std::vector<double> r0(rc), rk(rc);
    EWOS_CUDA_TRY(cudaMemcpyAsync(r0.data(), ws->nrm, sizeof(double) * rc, cudaMemcpyDeviceToHost, C.st));
    // the sweep as a CUDA graph, captured once per (workspace, toolbox, bucket, nonlinearity)
    const int nlk = nl ? nnl : 0;
    SolveWorkspace::Graph* gr = nullptr;
    for (auto& g : ws->graphs)
        if (g.tb == C.tb->serial && g.rc == rc && g.nl == nlk) gr = &g;
    EWOS_CUDA_TRY(trsm_prepare<float>());
    double worst = 1.0;
    int it = 0;
    while (it < max_sweeps) {
        const bool capture = gr == nullptr;
        if (capture) {
            sweep_multi<TP>(C, rc, R, nl, nnl);   // first sweep of a new key: launched directly
        } else {
            EWOS_CUDA_TRY(cudaGraphLaunch(gr->exec, C.st));
            for (int q = 0; q < gr->launches; ++q) ::ewos::note_launch();
        }
        ++it;
        EWOS_CUDA_TRY(cudaMemcpyAsync(rk.data(), ws->nrm, sizeof(double) * rc, cudaMemcpyDeviceToHost, C.st));
        unsigned int flow_err = 0;
        EWOS_CUDA_TRY(cudaMemcpyAsync(&flow_err, ws->lu.flow + 1, sizeof(flow_err), cudaMemcpyDeviceToHost, C.st));
        if (capture) {
            // captured while the first sweep runs, on the workspace's own stream (the caller's may
            // be the legacy default stream, which cannot be captured); launched on the caller's
            if (!ws->cap_st) EWOS_CUDA_TRY(cudaStreamCreateWithFlags(&ws->cap_st, cudaStreamNonBlocking));
            Ctx Cc = C;
            Cc.st = ws->cap_st;
            cudaGraph_t graph = nullptr;
            EWOS_CUDA_TRY(cudaStreamBeginCapture(Cc.st, cudaStreamCaptureModeThreadLocal));
            const int launches = sweep_multi<TP>(Cc, rc, R, nl, nnl);
            ::ewos::unnote_launches(launches);    // recorded, not run: counted at each replay
            cudaError_t e = cudaStreamEndCapture(Cc.st, &graph);
            if (e != cudaSuccess) { set_error(std::string("graph capture: ") + cudaGetErrorString(e)); return EWOS_ECUDA; }
            cudaGraphExec_t exec = nullptr;
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) { set_error(std::string("graph instantiate: ") + cudaGetErrorString(e)); return EWOS_ECUDA; }
            // a server slot's workspace serves many toolboxes: keep the most recent few graphs
            if (ws->graphs.size() >= kMaxSweepGraphs) {
                cudaGraphExecDestroy(ws->graphs.front().exec);
                ws->graphs.erase(ws->graphs.begin());
            }
            ws->graphs.push_back(SolveWorkspace::Graph{C.tb->serial, rc, nlk, exec, launches});
            gr = &ws->graphs.back();
        }
        EWOS_CUDA_TRY(cudaStreamSynchronize(C.st));
        if (flow_err) {
            set_error("triangular solve: a wait on a preceding row block timed out");
            return EWOS_ETIMEOUT;
        }
        worst = 0.0;
        bool bad = false;
        for (int r = 0; r < R; ++r) {
            const double rel = r0[r] > 0 ? std::sqrt(rk[r] / r0[r]) : 0.0;
            if (!(rel == rel) || rel > 1e3) bad = true;
            worst = std::max(worst, rel);
        }
        if (bad) break;
        if (worst <= tol) break;
    }
    *sweeps += it;
    if (final_rel) *final_rel = worst;
    if (last_norm) *last_norm = std::sqrt(rk[R - 1]);   // ||R(s) + alpha s|| of the last column, from the last sweep
    *ok = worst <= tol;
    if (!*ok) return EWOS_OK;
    // s and u = G s + H g for every column
    ::ewos::note_launch(), from_cols_kernel<<<nblocks(C.m * R), 256, 0, C.st>>>(ws->Sb, ws->s, C.m, R, (int)rc);
    const TP* Gm = (const TP*)C.tb->P + (size_t)C.D * C.n * C.m;
    const TP* Hm = (const TP*)C.tb->KH + (size_t)C.D * C.n * C.p;
    if (sizeof(TP) == 4) {
        // FP32 matrices: the FP32-pair products, as in the sweeps
        float* Shi = ws->F2buf;
        float* Slo = Shi + C.m * rc;
        float* Ghi = Slo + C.m * rc;
        float* Glo = Ghi + C.p * rc;
        ::ewos::note_launch(), split_f2_t_kernel<<<nblocks(C.m * rc), 256, 0, C.st>>>(ws->Sb, Shi, Slo, C.m, (int)rc);
        ::ewos::note_launch(), split_f2_t_kernel<<<nblocks(C.p * rc), 256, 0, C.st>>>(ws->Gb, Ghi, Glo, C.p, (int)rc);
        multi_rowdot_f2(C.st, (const float*)Gm, C.n, (int)C.m, Shi, Slo, ws->Ub, (int)rc, 0);
        multi_rowdot_f2(C.st, (const float*)Hm, C.n, (int)C.p, Ghi, Glo, ws->Ub, (int)rc, 1);
    } else {
        multi_rowdot<TP>(C.st, Gm, C.n, (int)C.m, ws->Sb, ws->Ub, (int)rc, 0);
        multi_rowdot<TP>(C.st, Hm, C.n, (int)C.p, ws->Gb, ws->Ub, (int)rc, 1);
    }
    ::ewos::note_launch(), from_cols_kernel<<<nblocks(C.n * R), 256, 0, C.st>>>(ws->Ub, ws->u, C.n, R, (int)rc);
    return EWOS_OK;
}

constexpr double kRefineTol = 1e-10;
constexpr int kRefineMax = 40;
constexpr int kStaleSweeps = 24;     // refinement sweeps allowed on the factors of an older Jacobian
// Inexact Newton: each Newton system is solved to the relative residual eta_k (the forcing term,
// Eisenstat and Walker's second choice with gamma = 0.9, alpha = 2, capped at kEtaMax), and never
// more accurately than the outer tolerance needs (eta_k >= 0.5 tol r_0 / r_k).  The outer test is
// on the true residual, so the converged solution meets the same tolerance as with exact solves.
constexpr double kEtaMax = 1e-3;
constexpr double kEtaMin = 1e-12;
constexpr int kChordMax = 80;    // chord sweeps before the semilinear batch falls back to Newton

template <typename TP>
static ewos_status solve_mixed_t(ewos_toolbox* tb, SolveWorkspace* ws, const ewos_problem* pb, double rcond, double tol, int max_iter,
                                 ewos_solve_report* rep, const SolveOptions& opt) {
    Ctx C{tb, ws, pb->stream ? (cudaStream_t)pb->stream : tb->stream, tb->dim, tb->dim + 1, tb->n, tb->m, tb->p};
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
    bool u_done = false;
    double batched_res = -1.0;      // residual norm of the last column from the batched sweeps
    if (!quasi) {
        auto ta = std::chrono::steady_clock::now();
        const bool keep = opt.reuse_factors && !semi;     // the factors of the previous linear solve
        if (!keep) {
            if (tc_assemble_available()) {
                DevSpan span(C.st, &rep->dev_ms_gemm);
                // a symmetric system is computed as its lower triangle: m (m + 1) K
                rep->gemm_flop += (pb->b == nullptr ? (double)C.m * (double)(C.m + 1) : 2.0 * (double)C.m * (double)C.m) *
                                  (double)(C.E * C.n);
                ewos_status st = tc_assemble_pq(P32, ws->M, (int)C.n, (int)C.m, C.D, ws->L32, C.st, &ws->tc,
                                                    pb->b == nullptr, pb->assembly != 1, tb->serial,
                                                    tb->pmax_valid ? tb->pmax : nullptr);
                if (st != EWOS_OK) return st;
            } else {
                assemble_mixed<TP>(C, P32);
            }
            ws->last_alpha = rcond * frob32(C, ws->L32, C.m * C.m);
        }
        const double alpha = ws->last_alpha;
        rep->alpha = alpha;
        rep->ms_assemble = elapsed_ms(ta);
        bool batched_done = false;
        if (opt.batched) {
            // one factorisation of Lambda + alpha I; all right-hand sides refined together
            // (linear) or the chord iteration on R(s) + alpha s = 0 (semilinear)
            auto t1 = std::chrono::steady_clock::now();
            if (!keep) {
                ewos_status st = factor32(C, ws->L32, alpha, pb->pivoting, rep);
                if (st != EWOS_OK) return st;
            }
            rep->ms_factor = elapsed_ms(t1);
            auto t2 = std::chrono::steady_clock::now();
            ewos_status st = EWOS_OK;
            EWOS_CUDA_TRY(cudaMemsetAsync(ws->scal, 0, sizeof(double), C.st));
            st = ensure_batched(C, bucket_of(nrhs));
            if (st != EWOS_OK) return st;
            ::ewos::note_launch(), set_scalar_kernel<<<1, 32, 0, C.st>>>(ws->alpha_dev, alpha);
            bool ok = false;
            double rel = 0.0;
            st = solve_batched<TP>(C, (int)nrhs, semi ? ws->nl : nullptr, semi ? pb->nl_ncoef : 0,
                                   semi ? tol : kRefineTol, semi ? kChordMax : kRefineMax, &sweeps, &ok, &rel,
                                   &batched_res);
            if (st != EWOS_OK) return st;
            rep->ms_solve = elapsed_ms(t2);
            if (ok) {
                batched_done = true;
                u_done = true;
                rep->iters = semi ? sweeps : 1;
            } else {
                batched_res = -1.0;               // the fallback below computes another s
            }
        }
        if (batched_done) {
        } else if (!semi) {
            auto t1 = std::chrono::steady_clock::now();
            ewos_status st = EWOS_OK;
            if (!keep) {
                st = factor32(C, ws->L32, alpha, pb->pivoting, rep);
                if (st != EWOS_OK) return st;
            }
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
            // Newton on R(s) + alpha s = 0.  Each Newton system J(u) x = R is solved to its forcing
            // term eta_k by FP64 refinement (J applied matrix-free) preconditioned by FP32 factors
            // of a Jacobian: the current one when factored at this step, else the last one
            // factored, kept while the refinement still reaches eta_k within kStaleSweeps sweeps
            // (the step is the Newton step either way; only the preconditioner is older),
            // refactored otherwise.
            const double* nl = ws->nl;
            for (int64_t r = 0; r < nrhs; ++r) {
                double* s = ws->s + r * C.m;
                const double* g = ws->g + r * C.p;
                const double* f = ws->f + r * C.n;
                cudaMemsetAsync(s, 0, sizeof(double) * C.m, C.st);
                VgScope<TP> vgs(C, g);
                residual<TP>(C, s, g, f, nl, pb->nl_ncoef, alpha, ws->y);
                const double r0 = norm2(C, ws->y, C.m);
                double rn = r0, rn_prev = r0;
                int it = 0;
                bool have_factors = false;
                while (it < max_iter && rn > tol * r0) {
                    double eta = kEtaMax;
                    if (it > 0) eta = std::min(kEtaMax, 0.9 * (rn / rn_prev) * (rn / rn_prev));
                    eta = std::max(eta, std::max(kEtaMin, 0.5 * tol * r0 / rn));
                    rn_prev = rn;
                    u_from_v(C, ws->u2);         // u at the current s, from the residual just evaluated
                    if (have_factors && opt.newton_reuse) {
                        cudaMemcpyAsync(ws->rhs, ws->y, sizeof(double) * C.m, cudaMemcpyDeviceToDevice, C.st);
                        double rel = 1.0;
                        ewos_status st = refine<TP>(C, ws->rhs, ws->x, alpha, ws->u2, nl, pb->nl_ncoef, eta,
                                                    kStaleSweeps, &sweeps, &rel, rn);
                        if (st != EWOS_OK) return st;
                        if (rel <= eta) {
                            ::ewos::note_launch(), axpy_kernel<<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(C.m, -1.0, ws->x, s);
                            residual<TP>(C, s, g, f, nl, pb->nl_ncoef, alpha, ws->y);
                            rn = norm2(C, ws->y, C.m);
                            ++it;
                            continue;
                        }
                        // the refinement used y as scratch: put the Newton residual back
                        cudaMemcpyAsync(ws->y, ws->rhs, sizeof(double) * C.m, cudaMemcpyDeviceToDevice, C.st);
                    }
                    have_factors = true;
                    const TP* Gm = (const TP*)tb->P + (size_t)C.D * C.n * C.m;
                    const float* Gm32 = P32 + (size_t)C.D * C.n * C.m;
                    // Jacobian Lambda + alpha I + G^T diag(lam N'(u)) G: the product on the tensor
                    // cores (three products of FP16 halves, or of TF32 parts) when available.  The
                    // FP16 form takes d = lam N'(u) as a vector and splits G and diag(d) G in one pass
                    // over G; the others scale a copy of G first
                    const bool tcj = tc_assemble_available();
                    const bool jrow = tcj && pb->assembly != 1;
                    if (jrow)
                        ::ewos::note_launch(), jac_diag_kernel<<<(unsigned)((C.n + 255) / 256), 256, 0, C.st>>>(
                                                   ws->u2, tb->lambda, nl, pb->nl_ncoef, ws->Jx32, (int)C.n);
                    else
                        ::ewos::note_launch(), jac_scale32_kernel<TP><<<(unsigned)C.n, 256, 0, C.st>>>(
                                                   Gm, ws->u2, tb->lambda, nl, pb->nl_ncoef, ws->Jx32, (int)C.n, (int)C.m,
                                                   (int)(C.m % 4 == 0 && aligned16(Gm) && aligned16(ws->Jx32)));
                    auto t1 = std::chrono::steady_clock::now();
                    ewos_status tst = EWOS_OK;
                    ewos_status st = factor32_with(
                        C,
                        [&] {
                            if (tcj) {
                                DevSpan span(C.st, &rep->dev_ms_gemm);
                                rep->gemm_flop += (double)C.m * (double)(C.m + 1) * (double)C.n;   // symmetric: lower triangle
                                ewos_status e = jrow ? tc_assemble(Gm32, nullptr, ws->LU32, (int)C.m, (int)C.m, (int)C.n, C.st,
                                                                   kSplitTF32, &ws->tc, true, true, tb->serial, ws->Jx32,
                                                                   tb->pmax_valid ? tb->pmax + 1 : nullptr)
                                                     : tc_assemble(Gm32, ws->Jx32, ws->LU32, (int)C.m, (int)C.m, (int)C.n, C.st,
                                                                   kSplitTF32, &ws->tc, true, false, tb->serial);
                                if (e != EWOS_OK) tst = e;
                                const int64_t cnt = C.m * C.m;
                                if (C.m % 4 == 0 && aligned16(ws->LU32) && aligned16(ws->L32))
                                    ::ewos::note_launch(), add_shifted4_kernel<<<4 * 148 * 8, 256, 0, C.st>>>(
                                        reinterpret_cast<float4*>(ws->LU32), reinterpret_cast<const float4*>(ws->L32), cnt / 4,
                                        (int)C.m, (float)alpha);
                                else
                                    ::ewos::note_launch(), add_shifted_kernel<<<(int)std::min<int64_t>(65535, (cnt + 255) / 256), 256, 0, C.st>>>(
                                        ws->LU32, ws->L32, cnt, (int)C.m, alpha);
                            } else {
                                cudaMemcpyAsync(ws->LU32, ws->L32, sizeof(float) * C.m * C.m, cudaMemcpyDeviceToDevice, C.st);
                                sgemm<true>(C.st, (int)C.m, (int)C.m, (int)C.n, 1.f, Gm32, C.m, ws->Jx32, C.m, 1.f, ws->LU32, C.m);
                                ::ewos::note_launch(), add_diag_kernel<float><<<(int)((C.m + 255) / 256), 256, 0, C.st>>>(
                                    ws->LU32, (int)C.m, (int)C.m, alpha);
                            }
                        },
                        pb->pivoting, rep);
                    if (tst != EWOS_OK) return tst;
                    if (st != EWOS_OK) return st;
                    rep->ms_factor += elapsed_ms(t1);
                    cudaMemcpyAsync(ws->rhs, ws->y, sizeof(double) * C.m, cudaMemcpyDeviceToDevice, C.st);
                    st = refine<TP>(C, ws->rhs, ws->x, alpha, ws->u2, nl, pb->nl_ncoef, eta, 8, &sweeps, nullptr, rn);
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
            VgScope<TP> vgs(C, g);               // the residual at s = 0 of every iteration
            int it = 0;
            bool conv = false;
            while (it < max_iter) {
                ::ewos::note_launch(), coef_kernel<<<(int)((C.n + 127) / 128), 128, 0, C.st>>>((int)C.n, C.D, tb->lambda, ws->A,
                                                                                            pb->b ? ws->b : nullptr,
                                                                                            pb->c ? ws->c : nullptr,
                                                                                            ws->nl, pb->nl_ncoef, u, ws->M);
                auto ta = std::chrono::steady_clock::now();
                if (tc_assemble_available()) {
                    DevSpan span(C.st, &rep->dev_ms_gemm);
                    // a symmetric system is computed as its lower triangle: m (m + 1) K
                rep->gemm_flop += (pb->b == nullptr ? (double)C.m * (double)(C.m + 1) : 2.0 * (double)C.m * (double)C.m) *
                                  (double)(C.E * C.n);
                    ewos_status st = tc_assemble_pq(P32, ws->M, (int)C.n, (int)C.m, C.D, ws->L32, C.st, &ws->tc,
                                                    pb->b == nullptr, pb->assembly != 1, tb->serial,
                                                    tb->pmax_valid ? tb->pmax : nullptr);
                    if (st != EWOS_OK) return st;
                } else {
                    assemble_mixed<TP>(C, P32);
                }
                const double alpha = rcond * frob32(C, ws->L32, C.m * C.m);
                rep->alpha = alpha;
                rep->ms_assemble += elapsed_ms(ta);
                auto t1 = std::chrono::steady_clock::now();
                ewos_status st = factor32(C, ws->L32, alpha, pb->pivoting, rep);
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
    if (!u_done)
        for (int64_t r = 0; r < nrhs; ++r)
            u_from_s(C, tb->P, tb->KH, tb->precision == 64, ws->s + r * C.m, ws->g + r * C.p, ws->u + r * C.n);
    if (batched_res >= 0.0) {
        rep->residual = batched_res;          // the last sweep evaluated it at the final s
    } else if (!quasi) {
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

ewos_status solve_mixed(ewos_toolbox* tb, SolveWorkspace* ws, const ewos_problem* pb, double rcond, double tol,
                        int max_iter, ewos_solve_report* rep, const SolveOptions& opt) {
    return tb->precision == 64 ? solve_mixed_t<double>(tb, ws, pb, rcond, tol, max_iter, rep, opt)
                               : solve_mixed_t<float>(tb, ws, pb, rcond, tol, max_iter, rep, opt);
}

}  // namespace ewos

using namespace ewos;

namespace ewos {

// One solve on a given workspace (the toolbox's own for ewos_solve, a server slot's otherwise).
ewos_status solve_on(ewos_toolbox* tb, SolveWorkspace*& wslot, const ewos_problem* pb, double* u_out, double* s_out,
                     int outputs_on_device, ewos_solve_report* rep_out, const SolveOptions& opt) {
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
    ewos_status s = ensure_workspace(tb, wslot, pb->nrhs, pb->mode == EWOS_SOLVE_MIXED);
    if (s != EWOS_OK) return s;
    SolveWorkspace* ws = wslot;
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
        s = tb->precision == 64 ? solve_fp64<double>(tb, ws, pb, rcond, tol, max_iter, &rep, opt.reuse_factors)
                                : solve_fp64<float>(tb, ws, pb, rcond, tol, max_iter, &rep, opt.reuse_factors);
    else
        s = solve_mixed(tb, ws, pb, rcond, tol, max_iter, &rep, opt);
    if (s != EWOS_OK && s != EWOS_ENOCONV) return s;
    const cudaMemcpyKind ko = outputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    EWOS_CUDA_TRY(cudaMemcpyAsync(u_out, ws->u, sizeof(double) * tb->n * pb->nrhs, ko, st));
    if (s_out) EWOS_CUDA_TRY(cudaMemcpyAsync(s_out, ws->s, sizeof(double) * tb->m * pb->nrhs, ko, st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(st));
    if (rep_out) *rep_out = rep;
    return s;
}

// ------------------------------------------------------------------ gradient of J and Adam
// grad J(s) = R(s) (eq. gradJ, Sec. 3.2: the Galerkin residual of the variational form), evaluated
// matrix-free in FP64 with the coefficient blocks M_i; Adam as in the paper's appendix algorithm:
//   m_j = b1 m_{j-1} + (1 - b1) grad J,  v_j = b2 v_{j-1} + (1 - b2) (grad J)^2,
//   alpha_j = alpha sqrt(1 - b2^j) / (1 - b1^j),  s_j = s_{j-1} - alpha_j m_j / (sqrt(v_j) + eps).
__global__ void adam_kernel(int64_t m, const double* __restrict__ g, double* __restrict__ mo, double* __restrict__ vo,
                            double* __restrict__ s, double alpha_j, double b1, double b2, double eps) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const double gt = g[t];
    const double mj = b1 * mo[t] + (1.0 - b1) * gt;
    const double vj = b2 * vo[t] + (1.0 - b2) * gt * gt;
    mo[t] = mj;
    vo[t] = vj;
    s[t] -= alpha_j * mj / (sqrt(vj) + eps);
}

// sum_i w_i y_i^2 (w = NULL: all weights 1)
__global__ void wsumsq_kernel(const double* __restrict__ y, const double* __restrict__ w, int64_t len,
                              double* __restrict__ out) {
    double acc = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (int64_t)gridDim.x * blockDim.x)
        acc += (w ? w[t] : 1.0) * y[t] * y[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// the problem's first column and coefficients on the device, M_i formed (semilinear or linear)
static ewos_status prepare_gradient(ewos_toolbox* tb, SolveWorkspace*& wslot, const ewos_problem* pb, Ctx& C) {
    if (!pb->A || !pb->f || !pb->g) { set_error("gradient: need a problem with A, f, g"); return EWOS_EINVAL; }
    if (pb->nl_kind == EWOS_NL_QUASILINEAR) {
        set_error("gradient: a quasilinear equation is not the Euler-Lagrange equation of a functional");
        return EWOS_EINVAL;
    }
    if (pb->nl_kind == EWOS_NL_SEMILINEAR && (!pb->nl_coef || pb->nl_ncoef < 1 || pb->nl_ncoef > 64)) {
        set_error("gradient: the nonlinearity needs 1..64 coefficients");
        return EWOS_EINVAL;
    }
    AllocStream as(C.st);
    ewos_status s = ensure_workspace(tb, wslot, 1, false, false);
    if (s != EWOS_OK) return s;
    SolveWorkspace* ws = wslot;
    C.ws = ws;
    const cudaMemcpyKind k = pb->inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const int D = tb->dim;
    EWOS_CUDA_TRY(cudaMemcpyAsync(ws->A, pb->A, sizeof(double) * tb->n * D * D, k, C.st));
    if (pb->b) EWOS_CUDA_TRY(cudaMemcpyAsync(ws->b, pb->b, sizeof(double) * tb->n * D, k, C.st));
    if (pb->c) EWOS_CUDA_TRY(cudaMemcpyAsync(ws->c, pb->c, sizeof(double) * tb->n, k, C.st));
    EWOS_CUDA_TRY(cudaMemcpyAsync(ws->f, pb->f, sizeof(double) * tb->n, k, C.st));
    EWOS_CUDA_TRY(cudaMemcpyAsync(ws->g, pb->g, sizeof(double) * tb->p, k, C.st));
    if (pb->nl_kind == EWOS_NL_SEMILINEAR)
        EWOS_CUDA_TRY(cudaMemcpyAsync(ws->nl, pb->nl_coef, sizeof(double) * pb->nl_ncoef, cudaMemcpyHostToDevice, C.st));
    ::ewos::note_launch(), coef_kernel<<<(int)((C.n + 127) / 128), 128, 0, C.st>>>((int)C.n, C.D, tb->lambda, ws->A,
                                                                                pb->b ? ws->b : nullptr,
                                                                                pb->c ? ws->c : nullptr, nullptr, 0,
                                                                                nullptr, ws->M);
    if (tb->precision == 32) {
        // FP32 toolbox: the refinement's residual (FP32-pair products, one pass over P where it
        // fits) on the single-column buffers: s in Sb, the gradient in Yb, shift 0
        s = ensure_batched(C, 1);
        if (s != EWOS_OK) return s;
        EWOS_CUDA_TRY(cudaMemcpyAsync(ws->Fb, ws->f, sizeof(double) * tb->n, cudaMemcpyDeviceToDevice, C.st));
        EWOS_CUDA_TRY(cudaMemcpyAsync(ws->Gb, ws->g, sizeof(double) * tb->p, cudaMemcpyDeviceToDevice, C.st));
        ::ewos::note_launch(), set_scalar_kernel<<<1, 32, 0, C.st>>>(ws->alpha_dev, 0.0);
    }
    return EWOS_OK;
}

// the iterate and gradient buffers of the gradient evaluation
static double* grad_s(const Ctx& C) { return C.tb->precision == 32 ? C.ws->Sb : C.ws->s; }
static double* grad_y(const Ctx& C) { return C.tb->precision == 32 ? C.ws->Yb : C.ws->y; }

// grad_y = R(grad_s)
static void gradient_at(const Ctx& C, const ewos_problem* pb) {
    const double* nl = pb->nl_kind == EWOS_NL_SEMILINEAR ? C.ws->nl : nullptr;
    const int nnl = pb->nl_kind == EWOS_NL_SEMILINEAR ? pb->nl_ncoef : 0;
    if (C.tb->precision == 64) residual<double>(C, C.ws->s, C.ws->g, C.ws->f, nl, nnl, 0.0, C.ws->y);
    else residual_multi<float>(C, 1, 1, nl, nnl);
}

// (sum_i w_i y_i^2)^(1/2), w = lambda when the V-centres are the nodes, else 1 (synchronises)
static double grad_norm(const Ctx& C, const double* y) {
    cudaMemsetAsync(C.ws->scal, 0, sizeof(double), C.st);
    const double* w = C.tb->y ? nullptr : C.tb->lambda;
    ::ewos::note_launch(), wsumsq_kernel<<<std::max<int64_t>(1, std::min<int64_t>(1024, (C.m + 255) / 256)), 256, 0, C.st>>>(
                               y, w, C.m, C.ws->scal);
    double h = 0;
    cudaMemcpyAsync(&h, C.ws->scal, sizeof(double), cudaMemcpyDeviceToHost, C.st);
    cudaStreamSynchronize(C.st);
    return std::sqrt(h);
}

}  // namespace ewos

extern "C" ewos_status ewos_gradient(ewos_toolbox* tb, const ewos_problem* pb, const double* s, double* grad) {
    using namespace ewos;
    if (!tb || !pb || !s || !grad) { set_error("ewos_gradient: NULL argument"); return EWOS_EINVAL; }
    Ctx C{tb, nullptr, pb->stream ? (cudaStream_t)pb->stream : tb->stream, tb->dim, tb->dim + 1, tb->n, tb->m, tb->p};
    ewos_status st = prepare_gradient(tb, tb->ws, pb, C);
    if (st != EWOS_OK) return st;
    const cudaMemcpyKind k = pb->inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    EWOS_CUDA_TRY(cudaMemcpyAsync(grad_s(C), s, sizeof(double) * tb->m, k, C.st));
    gradient_at(C, pb);
    const cudaMemcpyKind ko = pb->inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    EWOS_CUDA_TRY(cudaMemcpyAsync(grad, grad_y(C), sizeof(double) * tb->m, ko, C.st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(C.st));
    return EWOS_OK;
}

extern "C" ewos_status ewos_minimize_adam(ewos_toolbox* tb, const ewos_problem* pb, const ewos_adam_opts* opts,
                                         double* s_inout, double* u_out, ewos_adam_report* rep) {
    using namespace ewos;
    if (!tb || !pb || !opts || !s_inout) { set_error("ewos_minimize_adam: NULL argument"); return EWOS_EINVAL; }
    if (!(opts->alpha > 0) || !(opts->beta1 >= 0 && opts->beta1 < 1) || !(opts->beta2 >= 0 && opts->beta2 < 1) ||
        !(opts->eps > 0) || opts->max_iter < 0) {
        set_error("ewos_minimize_adam: need alpha > 0, beta1 and beta2 in [0, 1), eps > 0, max_iter >= 0");
        return EWOS_EINVAL;
    }
    auto t0 = std::chrono::steady_clock::now();
    Ctx C{tb, nullptr, pb->stream ? (cudaStream_t)pb->stream : tb->stream, tb->dim, tb->dim + 1, tb->n, tb->m, tb->p};
    ewos_status st = prepare_gradient(tb, tb->ws, pb, C);
    if (st != EWOS_OK) return st;
    SolveWorkspace* ws = C.ws;
    double* sv = grad_s(C);
    double* gv = grad_y(C);
    const cudaMemcpyKind k = pb->inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    EWOS_CUDA_TRY(cudaMemcpyAsync(sv, s_inout, sizeof(double) * tb->m, k, C.st));
    EWOS_CUDA_TRY(cudaMemsetAsync(ws->r, 0, sizeof(double) * tb->m, C.st));     // first moment
    EWOS_CUDA_TRY(cudaMemsetAsync(ws->dx, 0, sizeof(double) * tb->m, C.st));    // second moment
    const int check = opts->check_every > 0 ? opts->check_every : 10;
    double p1 = 1.0, p2 = 1.0, gn = 0.0;
    int64_t j = 0;
    bool conv = false;
    while (j < opts->max_iter) {
        gradient_at(C, pb);
        if (opts->tol > 0 && j % check == 0) {
            gn = grad_norm(C, gv);
            if (gn <= opts->tol) { conv = true; break; }
        }
        ++j;
        p1 *= opts->beta1;
        p2 *= opts->beta2;
        const double aj = opts->alpha * std::sqrt(1.0 - p2) / (1.0 - p1);
        ::ewos::note_launch(), adam_kernel<<<(int)((tb->m + 255) / 256), 256, 0, C.st>>>(tb->m, gv, ws->r, ws->dx, sv, aj,
                                                                                       opts->beta1, opts->beta2, opts->eps);
    }
    if (!conv) {                              // the gradient at the final iterate
        gradient_at(C, pb);
        gn = grad_norm(C, gv);
        conv = opts->tol > 0 && gn <= opts->tol;
    }
    const cudaMemcpyKind ko = pb->inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    EWOS_CUDA_TRY(cudaMemcpyAsync(s_inout, sv, sizeof(double) * tb->m, ko, C.st));
    if (u_out) {
        u_from_s(C, tb->P, tb->KH, tb->precision == 64, sv, ws->g, ws->u);
        EWOS_CUDA_TRY(cudaMemcpyAsync(u_out, ws->u, sizeof(double) * tb->n, ko, C.st));
    }
    EWOS_CUDA_TRY(cudaStreamSynchronize(C.st));
    EWOS_CUDA_TRY(cudaGetLastError());
    if (rep) {
        rep->iters = j;
        rep->grad_norm = gn;
        rep->converged = conv ? 1 : 0;
        rep->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return EWOS_OK;
}

extern "C" ewos_status ewos_solve(ewos_toolbox* tb, const ewos_problem* pb, double* u_out, double* s_out,
                                  int outputs_on_device, ewos_solve_report* rep_out) {
    if (!tb) {
        set_error("ewos_solve: need a toolbox");
        return EWOS_EINVAL;
    }
    ewos::SolveOptions opt;
    opt.batched = pb && pb->batched != 0;
    opt.newton_reuse = !(pb && pb->newton_refactor != 0);
    return ewos::solve_on(tb, tb->ws, pb, u_out, s_out, outputs_on_device, rep_out, opt);
}

// ------------------------------------------------------------------ operator estimates
namespace ewos {

// unit right-hand sides of the columns [k0, k0 + cols) of the solve map: column k < n is f = e_k,
// column n + j is g = e_j (F [cols][n] and Gb [cols][p] zeroed before)
__global__ void unit_rhs_kernel(double* __restrict__ F, double* __restrict__ Gb, int64_t n, int64_t p, int64_t k0,
                                int64_t cols) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cols) return;
    const int64_t k = k0 + t;
    if (k < n) F[t * n + k] = 1.0;
    else if (k < n + p) Gb[t * p + (k - n)] = 1.0;
}

// out[i][col0 + k] = U[t0 + k][i] for k < cols, i < n; out has row length ldo (32 x 32 tiles
// through shared memory)
__global__ void transpose_cols_kernel(const double* __restrict__ U, int64_t n, int64_t t0, int64_t cols,
                                      double* __restrict__ out, int64_t ldo, int64_t col0) {
    __shared__ double tile[32][33];
    const int64_t kb = (int64_t)blockIdx.y * 32, ib = (int64_t)blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t k = kb + r, i = ib + threadIdx.x;
        if (k < cols && i < n) tile[r][threadIdx.x] = U[(t0 + k) * n + i];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = ib + r, k = kb + threadIdx.x;
        if (i < n && k < cols) out[i * ldo + col0 + k] = tile[threadIdx.x][r];
    }
}

static void transpose_cols(const double* U, int64_t n, int64_t t0, int64_t cols, double* out, int64_t ldo,
                           int64_t col0, cudaStream_t st) {
    if (!out || cols <= 0) return;
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((cols + 31) / 32));
    ::ewos::note_launch(), transpose_cols_kernel<<<grid, dim3(32, 8), 0, st>>>(U, n, t0, cols, out, ldo, col0);
}

// right-hand sides per solve of the operator estimates: the dataflow triangular solves give every
// wait a bounded spin, and their work grows as m^2 per column, so the columns go in chunks of at
// most ~2^31 multiply-adds per triangular solve (FP64 runs at 1/32 of that; all at once when
// they fit); the chunks after the first reuse the factors
static int64_t operator_chunk(int64_t m, int64_t R, bool mixed) {
    const int64_t cap = std::max<int64_t>(1, (int64_t(1) << 31) / (m * m * (mixed ? 1 : 32)));
    if (R <= cap) return R;
    int64_t c = 1;
    while (c * 2 <= cap) c *= 2;
    return c;
}

}  // namespace ewos

extern "C" ewos_status ewos_operators(ewos_toolbox* tb, const ewos_problem* pb, double* GL, double* HL,
                                      int outputs_on_device, ewos_solve_report* rep) {
    using namespace ewos;
    if (!tb || !pb || !pb->A || (!GL && !HL)) { set_error("ewos_operators: need toolbox, problem with A, and an output"); return EWOS_EINVAL; }
    if (pb->nl_kind != EWOS_NL_NONE) { set_error("ewos_operators: the operator estimates are for the linear problem"); return EWOS_EINVAL; }
    if (pb->mode != EWOS_SOLVE_FP64 && pb->mode != EWOS_SOLVE_MIXED) { set_error("ewos_operators: unknown mode"); return EWOS_EINVAL; }
    const cudaStream_t st = pb->stream ? (cudaStream_t)pb->stream : tb->stream;
    const bool mixed = pb->mode == EWOS_SOLVE_MIXED;
    const int64_t n = tb->n, p = tb->p, R = n + p, D = tb->dim;
    const int64_t CH = operator_chunk(tb->m, R, mixed);
    double *F = nullptr, *Gb = nullptr, *U = nullptr, *Ad = nullptr, *bd = nullptr, *cd = nullptr;
    double *GLd = outputs_on_device ? GL : nullptr, *HLd = outputs_on_device ? HL : nullptr;
    SolveWorkspace* ws = nullptr;
    auto cleanup = [&]() {
        AllocStream as(st);
        ::ewos::dev_free(F); ::ewos::dev_free(Gb); ::ewos::dev_free(U); ::ewos::dev_free(Ad);
        ::ewos::dev_free(bd); ::ewos::dev_free(cd);
        if (!outputs_on_device) { ::ewos::dev_free(GLd); ::ewos::dev_free(HLd); }
        if (ws) free_workspace(ws);
    };
    const bool host = pb->inputs_on_device == 0;
    {
        AllocStream as(st);
        cudaError_t e = ::ewos::dev_alloc((void**)&F, sizeof(double) * CH * n);
        if (e == cudaSuccess) e = ::ewos::dev_alloc((void**)&Gb, sizeof(double) * CH * p);
        if (e == cudaSuccess) e = ::ewos::dev_alloc((void**)&U, sizeof(double) * CH * n);
        if (e == cudaSuccess && !outputs_on_device && GL) e = ::ewos::dev_alloc((void**)&GLd, sizeof(double) * n * n);
        if (e == cudaSuccess && !outputs_on_device && HL) e = ::ewos::dev_alloc((void**)&HLd, sizeof(double) * n * p);
        if (e == cudaSuccess && host) e = ::ewos::dev_alloc((void**)&Ad, sizeof(double) * n * D * D);
        if (e == cudaSuccess && host && pb->b) e = ::ewos::dev_alloc((void**)&bd, sizeof(double) * n * D);
        if (e == cudaSuccess && host && pb->c) e = ::ewos::dev_alloc((void**)&cd, sizeof(double) * n);
        if (e == cudaSuccess && host) {
            e = cudaMemcpyAsync(Ad, pb->A, sizeof(double) * n * D * D, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess && pb->b) e = cudaMemcpyAsync(bd, pb->b, sizeof(double) * n * D, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess && pb->c) e = cudaMemcpyAsync(cd, pb->c, sizeof(double) * n, cudaMemcpyHostToDevice, st);
        }
        if (e != cudaSuccess) {
            set_error(std::string("ewos_operators: ") + cudaGetErrorString(e));
            cleanup();
            return e == cudaErrorMemoryAllocation ? EWOS_ENOMEM : EWOS_ECUDA;
        }
    }
    ewos_problem q = *pb;
    q.A = host ? Ad : pb->A;
    q.b = host ? bd : pb->b;
    q.c = host ? cd : pb->c;
    q.f = F;
    q.g = Gb;
    q.inputs_on_device = 1;
    q.stream = st;
    // mixed mode: the columns of a chunk are refined together (graph-captured sweeps)
    q.batched = mixed ? 1 : 0;
    SolveOptions opt;
    opt.batched = mixed;
    ewos_status s = EWOS_OK;
    ewos_solve_report r{}, total{};
    for (int64_t k0 = 0; k0 < R && s == EWOS_OK; k0 += CH) {
        const int64_t cols = std::min(CH, R - k0);
        {
            AllocStream as(st);
            if (cudaMemsetAsync(F, 0, sizeof(double) * cols * n, st) != cudaSuccess ||
                cudaMemsetAsync(Gb, 0, sizeof(double) * cols * p, st) != cudaSuccess) {
                set_error("ewos_operators: memset");
                s = EWOS_ECUDA;
                break;
            }
            ::ewos::note_launch(), unit_rhs_kernel<<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(F, Gb, n, p, k0, cols);
        }
        q.nrhs = cols;
        opt.reuse_factors = k0 > 0;
        s = solve_on(tb, ws, &q, U, nullptr, 1, &r, opt);
        if (s != EWOS_OK) break;
        if (k0 == 0) total = r;
        else {
            total.ms_total += r.ms_total;
            total.ms_solve += r.ms_solve;
            total.refine_iters = std::max(total.refine_iters, r.refine_iters);
            total.converged = total.converged && r.converged;
            total.residual = r.residual;
        }
        const int64_t g1 = std::max<int64_t>(0, std::min(cols, n - k0));      // local columns of GL
        transpose_cols(U, n, 0, g1, GLd, n, k0, st);
        transpose_cols(U, n, g1, cols - g1, HLd, p, k0 + g1 - n, st);
    }
    if (s == EWOS_OK && !outputs_on_device) {
        cudaError_t e = cudaSuccess;
        if (GL) e = cudaMemcpyAsync(GL, GLd, sizeof(double) * n * n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && HL) e = cudaMemcpyAsync(HL, HLd, sizeof(double) * n * p, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) { set_error(std::string("ewos_operators: ") + cudaGetErrorString(e)); s = EWOS_ECUDA; }
    }
    if (s == EWOS_OK && cudaStreamSynchronize(st) != cudaSuccess) { set_error("ewos_operators: stream"); s = EWOS_ECUDA; }
    if (rep && s == EWOS_OK) *rep = total;
    cleanup();
    return s;
}

// Test hook (no counterpart in the paper): the dataflow triangular solves' flag waits give up
// after `polls` polls on the current device (polls < 0: the default, 2^22).
extern "C" ewos_status ewos_debug_set_flow_wait_limit(int64_t polls) {
    using namespace ewos;
    const long long v = polls < 0 ? kFlowSpinLimit : (long long)polls;
    EWOS_CUDA_TRY(cudaMemcpyToSymbol(g_flow_spin_limit, &v, sizeof(v)));
    EWOS_CUDA_TRY(cudaDeviceSynchronize());
    return EWOS_OK;
}
