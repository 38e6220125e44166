// wos_build.cu -- toolbox build on the GPU: Voronoi lookup structures, Monte Carlo cell
// weights, and the persistent walk kernel that fuses the four matrix estimators of Sec. 2.3
// (eqs. Estimator_A, Estimator_B, Estimator_H, Estimator_K) the way Algorithm 5 does, one
// CTA per node row at a time.
//
// Walk of node i, walk l (G := A/2, gradG := B/2; w = X_1 - x_i = r0 U_0):
//   ball    ball term of Prop. 2.6 (ii): S = 1 - sqrt(u), point x_i + r0 S Z,
//           gradG += (r0/2) (sum_{k<d} S^k) Z.
//   step 0  X_0 = x_i, r = r0: source x_i + r0 Y_0 (Green density, Prop. 2.6 (i)):
//           G += r0^2/(2d);  X_1 = x_i + r0 U_0.
//   step k  r = r(X_k); stop if r < eps (or k > max_steps); source X_k + r Y_k:
//           G += r^2/(2d), gradG_c += w_c r^2/(2 r0^2);  X_{k+1} = X_k + r U_k.
//   exit    boundary cell of the stopping point: H += 1, gradH_c += (d/r0^2) w_c.
//
// Layout in HBM: P = [d_1 G, .., d_d G, G] as [(d+1)][n][m] and KH = [d_1 H, .., d_d H, H] as
// [(d+1)][n][p] (T = float or double), Hc [n][p] uint32 exit counts.  The stacked P is the
// operand of the Galerkin assembly Lambda = P^T Q (solve.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "toolbox.hpp"

namespace ewos {

constexpr int kMaxPolygonVertices = 256;
constexpr int kCandidateCap = 96;         // longer lists fall back to a scan of all centres

// ------------------------------------------------------------------ lookup construction
struct GridSpec {
    double lo[3];
    double h;
    int dims[3];
    int64_t ncell;
};

// For grid cell Q: R_Q = min_c maxdist(c, Q); candidates = { c : mindist(c, Q) <= R_Q }.
// Computed in FP64 with a small relative margin, so the list is a superset of the exact
// candidates and FP32 queries still see the true nearest centre.
template <int D>
__device__ void cell_box(const GridSpec& g, int64_t cell, double* blo, double* bhi) {
    int64_t rem = cell;
    for (int c = 0; c < D; ++c) {
        const int k = (int)(rem % g.dims[c]);
        rem /= g.dims[c];
        blo[c] = g.lo[c] + k * g.h;
        bhi[c] = blo[c] + g.h;
    }
}

// Candidate lists are computed in FP32 (FP64 is a small fraction of B300's arithmetic) with a
// margin that keeps them supersets of the exact lists: lim = R_Q^2 (1 + 1e-4) + slack, where
// slack (host: 1e-6 x squared extent of the domain) dominates the FP32 rounding of squared
// distances.  One warp per grid cell; lanes scan the centres.
template <int D>
__device__ __forceinline__ void cell_box_f(const GridSpec& g, int64_t cell, float* blo, float* bhi) {
    int64_t rem = cell;
    for (int c = 0; c < D; ++c) {
        const int k = (int)(rem % g.dims[c]);
        rem /= g.dims[c];
        blo[c] = (float)(g.lo[c] + k * g.h);
        bhi[c] = (float)(g.lo[c] + (k + 1) * g.h);
    }
}

template <int D>
__device__ __forceinline__ float mind2(const float* __restrict__ pts, int j, const float* blo, const float* bhi) {
    float mn = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const float v = pts[j * D + c];
        const float t = v < blo[c] ? blo[c] - v : (v > bhi[c] ? v - bhi[c] : 0.f);
        mn += t * t;
    }
    return mn;
}

// Per grid cell Q: the centre c_b minimising maxdist(c, Q) and lim = R_Q^2 with margin.  A centre
// is listed when mindist(c, Q)^2 <= lim and Q does not lie entirely on c_b's side of the bisector
// of c and c_b (every corner of Q strictly closer to c_b, with a margin): both tests only drop
// centres that cannot be nearest anywhere in Q, so the lists stay exact supersets.
template <int D>
struct CellTest {
    float blo[3], bhi[3];
    float lim;
    int best;             // index of the centre c_b that bounds the cell
    float cb[3];
    float dcb[8];         // squared distance of each corner to c_b
    float slack;
};

template <int D>
__device__ __forceinline__ void corner(const CellTest<D>& t, int k, float* x) {
#pragma unroll
    for (int c = 0; c < D; ++c) x[c] = (k >> c) & 1 ? t.bhi[c] : t.blo[c];
}

template <int D>
__device__ __forceinline__ void cell_setup(const float* __restrict__ pts, int np, CellTest<D>& t) {
    const int lane = threadIdx.x & 31;
    float R2 = 3.0e38f;
    int bj = 0x7fffffff;
    for (int j = lane; j < np; j += 32) {
        float mx = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float v = pts[j * D + c];
            const float u = fmaxf(fabsf(v - t.blo[c]), fabsf(v - t.bhi[c]));
            mx += u * u;
        }
        if (mx < R2 || (mx == R2 && j < bj)) { R2 = mx; bj = j; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oR = __shfl_xor_sync(0xffffffffu, R2, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (oR < R2 || (oR == R2 && oj < bj)) { R2 = oR; bj = oj; }
    }
    t.lim = R2 * (1.0f + 1e-4f) + t.slack;
    t.best = bj;
#pragma unroll
    for (int c = 0; c < D; ++c) t.cb[c] = pts[bj * D + c];
#pragma unroll
    for (int k = 0; k < (1 << D); ++k) {
        float x[3];
        corner(t, k, x);
        float d2 = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) { const float u = x[c] - t.cb[c]; d2 += u * u; }
        t.dcb[k] = d2;
    }
}

// the cell test from the bound and centre a previous pass found (same values as cell_setup)
template <int D>
__device__ __forceinline__ void cell_setup_stored(const float* __restrict__ pts, int best, float lim, CellTest<D>& t) {
    t.lim = lim;
    t.best = best;
#pragma unroll
    for (int c = 0; c < D; ++c) t.cb[c] = pts[best * D + c];
#pragma unroll
    for (int k = 0; k < (1 << D); ++k) {
        float x[3];
        corner(t, k, x);
        float d2 = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) { const float u = x[c] - t.cb[c]; d2 += u * u; }
        t.dcb[k] = d2;
    }
}

template <int D>
__device__ __forceinline__ bool cell_candidate(const float* __restrict__ pts, int j, const CellTest<D>& t) {
    if (mind2<D>(pts, j, t.blo, t.bhi) > t.lim) return false;
    bool all_closer = true;
#pragma unroll
    for (int k = 0; k < (1 << D); ++k) {
        float x[3];
        corner(t, k, x);
        float d2 = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) { const float u = x[c] - pts[j * D + c]; d2 += u * u; }
        all_closer = all_closer && (t.dcb[k] < d2 * (1.0f - 1e-4f) - t.slack);
    }
    return !all_closer;
}

template <int D>
__global__ void lookup_count_kernel(const float* __restrict__ pts, int np, GridSpec g, float slack,
                                    int* __restrict__ count, float* __restrict__ radius, int* __restrict__ maxcount,
                                    int* __restrict__ best) {
    const int64_t cell = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= g.ncell) return;
    CellTest<D> t;
    cell_box_f<D>(g, cell, t.blo, t.bhi);
    t.slack = slack;
    cell_setup<D>(pts, np, t);
    int cnt = 0;
    for (int j = lane; j < np; j += 32) cnt += cell_candidate<D>(pts, j, t);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) {
        count[cell] = cnt > kCandidateCap ? 0 : cnt;   // empty list = scan all centres
        radius[cell] = t.lim;
        if (best) best[cell] = t.best;
        if (maxcount) atomicMax(maxcount, cnt);
    }
}

// ordered fill: ballot per 32 centres keeps the increasing index order
template <int D, typename I>
__device__ __forceinline__ void fill_cell(const float* __restrict__ pts, int np, const CellTest<D>& t,
                                          I* __restrict__ out, int cap) {
    const int lane = threadIdx.x & 31;
    int w = 0;
    for (int base = 0; base < np && w < cap; base += 32) {
        const int j = base + lane;
        const bool in = j < np && cell_candidate<D>(pts, j, t);
        const unsigned msk = __ballot_sync(0xffffffffu, in);
        const int off = w + __popc(msk & ((1u << lane) - 1u));
        if (in && off < cap) out[off] = (I)j;
        w += __popc(msk);
    }
}

template <int D>
__global__ void lookup_fill_kernel(const float* __restrict__ pts, int np, GridSpec g, float slack,
                                   const int* __restrict__ start, int* __restrict__ cand) {
    const int64_t cell = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (cell >= g.ncell) return;
    const int w = start[cell], e = start[cell + 1];
    if (w == e) return;
    CellTest<D> t;
    cell_box_f<D>(g, cell, t.blo, t.bhi);
    t.slack = slack;
    cell_setup<D>(pts, np, t);
    fill_cell<D, int>(pts, np, t, cand + w, e - w);
}

// Both candidate tables of a cell from one ordered scan, with the bound and centre the count pass
// stored: the list [start[cell], start[cell + 1]) and, when candK is given, the fixed-stride row
// of K slots padded with the sentinel np (a point placed far away, never nearest).  Same
// contents as filling each table on its own.
template <int D>
__global__ void lookup_fill_both_kernel(const float* __restrict__ pts, int np, GridSpec g, float slack,
                                        const float* __restrict__ radius, const int* __restrict__ best,
                                        const int* __restrict__ start, int* __restrict__ cand, int K,
                                        uint16_t* __restrict__ candK) {
    const int64_t cell = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= g.ncell) return;
    const int s0 = start[cell], cap = start[cell + 1] - s0;
    const int capK = candK ? K : 0;
    if (candK)
        for (int q = lane; q < K; q += 32) candK[cell * K + q] = (uint16_t)np;
    if (cap == 0 && capK == 0) return;
    CellTest<D> t;
    cell_box_f<D>(g, cell, t.blo, t.bhi);
    t.slack = slack;
    cell_setup_stored<D>(pts, best[cell], radius[cell], t);
    __syncwarp();
    const int lim = max(cap, capK);
    int w = 0;
    for (int base = 0; base < np && w < lim; base += 32) {
        const int j = base + lane;
        const bool in = j < np && cell_candidate<D>(pts, j, t);
        const unsigned msk = __ballot_sync(0xffffffffu, in);
        const int off = w + __popc(msk & ((1u << lane) - 1u));
        if (in && off < cap) cand[s0 + off] = j;
        if (in && off < capK) candK[cell * K + off] = (uint16_t)j;
        w += __popc(msk);
    }
}

// Candidate lists of a grid refined 2x from a coarser one (same origin, half the spacing,
// twice the cells per axis): a point of a fine cell lies in its parent cell, so its nearest
// centre is on the parent's list, and the fine cell's list is the parent's list filtered by the
// same tests (bound R_Q and the bisector test taken over the parent's candidates: a larger
// bound and any bounding centre keep the list a superset of the exact candidates).  One thread
// per fine cell; lists stay in increasing centre index.  A parent that scans all centres (empty
// list) gives an empty fine list.  count pass: counts (and the largest count) or, with start
// given, fill pass: the CSR lists and, when candK is given, the fixed-stride rows (K slots, the
// unused ones holding the sentinel np).
template <int D>
__global__ void lookup_refine_kernel(const float* __restrict__ pts, int np, GridSpec coarse, GridSpec fine, float slack,
                                     const int* __restrict__ cstart, const int* __restrict__ ccand,
                                     int* __restrict__ count, int* __restrict__ maxcount, const int* __restrict__ start,
                                     int* __restrict__ cand, int K, uint16_t* __restrict__ candK) {
    const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= fine.ncell) return;
    int64_t rem = cell, pc = 0, mul = 1;
    for (int c = 0; c < D; ++c) {
        const int k = (int)(rem % fine.dims[c]);
        rem /= fine.dims[c];
        pc += (int64_t)(k >> 1) * mul;
        mul *= coarse.dims[c];
    }
    const int s0 = cstart[pc], e0 = cstart[pc + 1];
    if (candK)
        for (int q = 0; q < K; ++q) candK[cell * K + q] = (uint16_t)np;
    if (s0 == e0) {                 // the parent scans all centres: so does this cell
        if (count) count[cell] = 0;
        if (maxcount) atomicMax(maxcount, kCandidateCap + 1);
        return;
    }
    CellTest<D> t;
    cell_box_f<D>(fine, cell, t.blo, t.bhi);
    t.slack = slack;
    float R2 = 3.0e38f;
    int bj = 0x7fffffff;
    for (int q = s0; q < e0; ++q) {
        const int j = ccand[q];
        float mx = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float v = pts[j * D + c];
            const float u = fmaxf(fabsf(v - t.blo[c]), fabsf(v - t.bhi[c]));
            mx += u * u;
        }
        if (mx < R2 || (mx == R2 && j < bj)) { R2 = mx; bj = j; }
    }
    cell_setup_stored<D>(pts, bj, R2 * (1.0f + 1e-4f) + slack, t);
    if (!start) {
        int cnt = 0;
        for (int q = s0; q < e0; ++q) cnt += cell_candidate<D>(pts, ccand[q], t);
        count[cell] = cnt;
        atomicMax(maxcount, cnt);
        return;
    }
    int w = start[cell];
    int wk = 0;
    for (int q = s0; q < e0; ++q) {
        const int j = ccand[q];
        if (!cell_candidate<D>(pts, j, t)) continue;
        cand[w++] = j;
        if (candK && wk < K) candK[cell * K + wk++] = (uint16_t)j;
    }
}

// exclusive scan of count[0..len) into start[0..len], single block (len is at most a few 10^5)
__global__ void exclusive_scan_kernel(const int* __restrict__ count, int64_t len, int* __restrict__ start) {
    __shared__ int warp_sums[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < len; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        int v = i < len ? count[i] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_sums[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += t;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const int before = (wid > 0 ? warp_sums[wid - 1] : 0) + carry;
        if (i < len) start[i] = before + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[len] = carry;
}

// Exclusive scan over many blocks: per-block sums of `chunk` entries, one block scans the sums,
// then every block scans its chunk from its offset (fine lookup grids have millions of cells,
// which the single-block scan above walks through sequentially).
constexpr int kScanChunk = 4096;      // 1024 threads x 4 entries

__global__ void __launch_bounds__(1024) block_sums_kernel(const int* __restrict__ count, int64_t len,
                                                          int* __restrict__ sums) {
    __shared__ int ws[32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
    int v = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t i = base + threadIdx.x * 4 + q;
        if (i < len) v += count[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        int t = ws[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) sums[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) block_scan_kernel(const int* __restrict__ count, int64_t len,
                                                          const int* __restrict__ offs, int* __restrict__ start) {
    __shared__ int ws[32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + threadIdx.x * 4;
    int v[4];
    int tsum = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = base + q < len ? count[base + q] : 0;
        tsum += v[q];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) ws[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int t = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        ws[lane] = t;
    }
    __syncthreads();
    int run = offs[blockIdx.x] + (wid > 0 ? ws[wid - 1] : 0) + incl - tsum;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (base + q < len) start[base + q] = run;
        run += v[q];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) start[len] = offs[gridDim.x];
}

// start[0..len] = exclusive scan of count[0..len) (start[len] = total) on the stream
static ewos_status exclusive_scan(const int* count, int64_t len, int* start, cudaStream_t st) {
    const int64_t nb = (len + kScanChunk - 1) / kScanChunk;
    if (nb <= 1) {
        ::ewos::note_launch(), exclusive_scan_kernel<<<1, 1024, 0, st>>>(count, len, start);
        return EWOS_OK;
    }
    int* sums = nullptr;
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&sums, sizeof(int) * (2 * nb + 1)));
    int* offs = sums + nb;
    ::ewos::note_launch(), block_sums_kernel<<<(unsigned)nb, 1024, 0, st>>>(count, len, sums);
    ::ewos::note_launch(), exclusive_scan_kernel<<<1, 1024, 0, st>>>(sums, nb, offs);
    ::ewos::note_launch(), block_scan_kernel<<<(unsigned)nb, 1024, 0, st>>>(count, len, offs, start);
    ::ewos::dev_free(sums);
    EWOS_CUDA_TRY(cudaGetLastError());
    return EWOS_OK;
}

template <typename T, int D>
__global__ void convert_points_kernel(const double* __restrict__ in, T* __restrict__ out, int64_t count) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) out[t] = (T)in[t];
    if (t < D) out[count + t] = T(1.0e18f);            // sentinel point of the fixed-stride table
}

struct DeviceLookup {
    void* pts = nullptr;     // T [np + 1][D] (last: sentinel)
    int* start = nullptr;
    int* cand = nullptr;
    uint16_t* candK = nullptr;   // [ncell][K] when K > 0
    int K = 0;
    GridSpec grid{};
    int64_t ncand = 0;
    int np = 0;
    void release() {
        ::ewos::dev_free(pts); ::ewos::dev_free(start); ::ewos::dev_free(cand); ::ewos::dev_free(candK);
        pts = nullptr; start = nullptr; cand = nullptr; candK = nullptr;
    }
};

constexpr int kFixedCandMax = 32;

static GridSpec make_grid(int dim, const double* lo, const double* hi, double h) {
    GridSpec g{};
    g.h = h;
    g.ncell = 1;
    for (int c = 0; c < 3; ++c) {
        if (c < dim) {
            const double ext = hi[c] - lo[c];
            g.dims[c] = std::max(1, (int)std::ceil(ext / h - 1e-9));
            const double pad = 0.5 * (g.dims[c] * h - ext);
            g.lo[c] = lo[c] - pad;
            g.ncell *= g.dims[c];
        } else {
            g.dims[c] = 1;
            g.lo[c] = 0;
        }
    }
    return g;
}

template <typename T>
static ewos_status build_lookup_refined(int dim, const double* d_pts, int np, const double* lo, const double* hi,
                                        double h, double h_direct, cudaStream_t st, DeviceLookup& out,
                                        bool want_fixed);

// Lookup grid of spacing h over [lo, hi].  Grids finer than h_direct are refined 2x (repeatedly)
// from a grid of spacing >= h_direct, whose lists are computed directly from all centres.
template <typename T>
static ewos_status build_lookup(int dim, const double* d_pts, int np, const double* lo, const double* hi,
                                double h, cudaStream_t st, DeviceLookup& out, bool want_fixed, double h_direct = 0.0) {
    if (h_direct > 0.0 && h < h_direct)
        return build_lookup_refined<T>(dim, d_pts, np, lo, hi, h, h_direct, st, out, want_fixed);
    out.np = np;
    out.grid = make_grid(dim, lo, hi, h);
    const int64_t nc = out.grid.ncell;
    double ext = 0;
    for (int c = 0; c < dim; ++c) ext = std::max(ext, std::max(std::fabs(lo[c]), std::fabs(hi[c])) + (hi[c] - lo[c]));
    const float slack = (float)(1e-6 * ext * ext);
    int* d_count = nullptr;
    float* d_rad = nullptr;
    float* d_pf = nullptr;
    int* d_best = nullptr;
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&d_count, sizeof(int) * (nc + 1)));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&d_rad, sizeof(float) * nc));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&d_best, sizeof(int) * nc));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&d_pf, sizeof(float) * (np + 1) * dim));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&out.start, sizeof(int) * (nc + 1)));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&out.pts, sizeof(T) * (np + 1) * dim));
    EWOS_CUDA_TRY(cudaMemsetAsync(d_count + nc, 0, sizeof(int), st));
    const int64_t ne = (int64_t)np * dim;
    const int cb = (int)((ne + 255) / 256);
    if (dim == 2) {
        ::ewos::note_launch(), convert_points_kernel<float, 2><<<cb, 256, 0, st>>>(d_pts, d_pf, ne);
        ::ewos::note_launch(), convert_points_kernel<T, 2><<<cb, 256, 0, st>>>(d_pts, (T*)out.pts, ne);
    } else {
        ::ewos::note_launch(), convert_points_kernel<float, 3><<<cb, 256, 0, st>>>(d_pts, d_pf, ne);
        ::ewos::note_launch(), convert_points_kernel<T, 3><<<cb, 256, 0, st>>>(d_pts, (T*)out.pts, ne);
    }
    const int tb = 256;
    const int nb = (int)((nc * 32 + tb - 1) / tb);
    if (dim == 2) ::ewos::note_launch(), lookup_count_kernel<2><<<nb, tb, 0, st>>>(d_pf, np, out.grid, slack, d_count, d_rad, d_count + nc, d_best);
    else ::ewos::note_launch(), lookup_count_kernel<3><<<nb, tb, 0, st>>>(d_pf, np, out.grid, slack, d_count, d_rad, d_count + nc, d_best);
    if (ewos_status ss = exclusive_scan(d_count, nc, out.start, st); ss != EWOS_OK) return ss;
    int hv[2] = {0, 0};
    EWOS_CUDA_TRY(cudaMemcpyAsync(&hv[0], out.start + nc, sizeof(int), cudaMemcpyDeviceToHost, st));
    EWOS_CUDA_TRY(cudaMemcpyAsync(&hv[1], d_count + nc, sizeof(int), cudaMemcpyDeviceToHost, st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(st));
    const int total = hv[0], kmax = hv[1];
    out.ncand = total;
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&out.cand, sizeof(int) * std::max(1, total)));
    if (want_fixed && kmax >= 1 && kmax <= kFixedCandMax && np < 65535) {
        out.K = kmax;
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&out.candK, sizeof(uint16_t) * nc * kmax));
    }
    if (dim == 2)
        ::ewos::note_launch(), lookup_fill_both_kernel<2><<<nb, tb, 0, st>>>(d_pf, np, out.grid, slack, d_rad, d_best, out.start,
                                                                          out.cand, out.K, out.candK);
    else
        ::ewos::note_launch(), lookup_fill_both_kernel<3><<<nb, tb, 0, st>>>(d_pf, np, out.grid, slack, d_rad, d_best, out.start,
                                                                          out.cand, out.K, out.candK);
    EWOS_CUDA_TRY(cudaGetLastError());
    ::ewos::dev_free(d_count);
    ::ewos::dev_free(d_rad);
    ::ewos::dev_free(d_best);
    ::ewos::dev_free(d_pf);
    return EWOS_OK;
}

template <typename T>
static ewos_status build_lookup_refined(int dim, const double* d_pts, int np, const double* lo, const double* hi,
                                        double h, double h_direct, cudaStream_t st, DeviceLookup& out,
                                        bool want_fixed) {
    DeviceLookup coarse;
    struct Rel { DeviceLookup* L; ~Rel() { L->release(); } } rel{&coarse};
    ewos_status s = build_lookup<float>(dim, d_pts, np, lo, hi, 2.0 * h, st, coarse, false, h_direct);
    if (s != EWOS_OK) return s;
    out.np = np;
    out.grid = coarse.grid;
    out.grid.h = coarse.grid.h * 0.5;
    out.grid.ncell = 1;
    for (int c = 0; c < 3; ++c) {
        if (c < dim) { out.grid.dims[c] = 2 * coarse.grid.dims[c]; out.grid.ncell *= out.grid.dims[c]; }
        else out.grid.dims[c] = 1;
    }
    const int64_t nc = out.grid.ncell;
    double ext = 0;
    for (int c = 0; c < dim; ++c) ext = std::max(ext, std::max(std::fabs(lo[c]), std::fabs(hi[c])) + (hi[c] - lo[c]));
    const float slack = (float)(1e-6 * ext * ext);
    int* d_count = nullptr;
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&d_count, sizeof(int) * (nc + 1)));
    struct Fr { int** p; ~Fr() { ::ewos::dev_free(*p); } } fr{&d_count};
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&out.start, sizeof(int) * (nc + 1)));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&out.pts, sizeof(T) * (np + 1) * dim));
    EWOS_CUDA_TRY(cudaMemsetAsync(d_count + nc, 0, sizeof(int), st));
    const int64_t ne = (int64_t)np * dim;
    const int cb = (int)((ne + 255) / 256);
    if (dim == 2) ::ewos::note_launch(), convert_points_kernel<T, 2><<<cb, 256, 0, st>>>(d_pts, (T*)out.pts, ne);
    else ::ewos::note_launch(), convert_points_kernel<T, 3><<<cb, 256, 0, st>>>(d_pts, (T*)out.pts, ne);
    const float* pf = (const float*)coarse.pts;          // the coarse lookup's FP32 centres
    const int tb = 128;
    const int nb = (int)((nc + tb - 1) / tb);
    if (dim == 2)
        ::ewos::note_launch(), lookup_refine_kernel<2><<<nb, tb, 0, st>>>(pf, np, coarse.grid, out.grid, slack, coarse.start,
                                                                        coarse.cand, d_count, d_count + nc, nullptr,
                                                                        nullptr, 0, nullptr);
    else
        ::ewos::note_launch(), lookup_refine_kernel<3><<<nb, tb, 0, st>>>(pf, np, coarse.grid, out.grid, slack, coarse.start,
                                                                        coarse.cand, d_count, d_count + nc, nullptr,
                                                                        nullptr, 0, nullptr);
    if (ewos_status ss = exclusive_scan(d_count, nc, out.start, st); ss != EWOS_OK) return ss;
    int hv[2] = {0, 0};
    EWOS_CUDA_TRY(cudaMemcpyAsync(&hv[0], out.start + nc, sizeof(int), cudaMemcpyDeviceToHost, st));
    EWOS_CUDA_TRY(cudaMemcpyAsync(&hv[1], d_count + nc, sizeof(int), cudaMemcpyDeviceToHost, st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(st));
    const int total = hv[0], kmax = hv[1];
    out.ncand = total;
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&out.cand, sizeof(int) * std::max(1, total)));
    if (want_fixed && kmax >= 1 && kmax <= kFixedCandMax && np < 65535) {
        out.K = kmax;
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&out.candK, sizeof(uint16_t) * nc * kmax));
    }
    if (dim == 2)
        ::ewos::note_launch(), lookup_refine_kernel<2><<<nb, tb, 0, st>>>(pf, np, coarse.grid, out.grid, slack, coarse.start,
                                                                        coarse.cand, nullptr, nullptr, out.start,
                                                                        out.cand, out.K, out.candK);
    else
        ::ewos::note_launch(), lookup_refine_kernel<3><<<nb, tb, 0, st>>>(pf, np, coarse.grid, out.grid, slack, coarse.start,
                                                                        coarse.cand, nullptr, nullptr, out.start,
                                                                        out.cand, out.K, out.candK);
    EWOS_CUDA_TRY(cudaGetLastError());
    return EWOS_OK;
}

template <typename T, int D>
static Lookup<T, D> lookup_view(const DeviceLookup& L) {
    Lookup<T, D> v{};
    v.pts = (const T*)L.pts;
    v.start = L.start;
    v.cand = L.cand;
    for (int c = 0; c < D; ++c) { v.lo[c] = (T)L.grid.lo[c]; v.dims[c] = L.grid.dims[c]; }
    v.inv_h = (T)(1.0 / L.grid.h);
    return v;
}

// nearest centre with the fallback scan for cells whose list was too long
template <typename T, int D>
__device__ __forceinline__ int nearest_or_scan(const Lookup<T, D>& L, int np, const T* q) {
    const int cell = lookup_cell(L, q);
    const int s = L.start[cell], e = L.start[cell + 1];
    T best = T(3.0e38f);
    int bi = 0;
    if (s == e) {
        for (int j = 0; j < np; ++j) {
            T d2 = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) { const T dd = q[c] - L.pts[j * D + c]; d2 += dd * dd; }
            if (d2 < best) { best = d2; bi = j; }
        }
        return bi;
    }
    for (int t = s; t < e; ++t) {
        const int j = L.cand[t];
        T d2 = 0;
#pragma unroll
        for (int c = 0; c < D; ++c) { const T dd = q[c] - L.pts[j * D + c]; d2 += dd * dd; }
        if (d2 < best) { best = d2; bi = j; }
    }
    return bi;
}

// ------------------------------------------------------------------ cell weights
template <typename T, int D, int KIND>
__global__ void cell_count_kernel(Lookup<T, D> V, int m, const T* __restrict__ sdf_prm, int nsdf,
                                  T lo0, T lo1, T lo2, T ex0, T ex1, T ex2, int64_t nsamples,
                                  uint32_t k0, uint32_t k1, uint32_t inst, unsigned int* __restrict__ counts) {
    extern __shared__ unsigned int s_cnt[];
    for (int j = threadIdx.x; j < m; j += blockDim.x) s_cnt[j] = 0;
    __syncthreads();
    const T lo[3] = {lo0, lo1, lo2}, ex[3] = {ex0, ex1, ex2};
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nsamples;
         j += (int64_t)gridDim.x * blockDim.x) {
        const u32x4 q = philox4x32_10(u32x4{(uint32_t)j, (uint32_t)((uint64_t)j >> 32), 0u,
                                            (1u << 24) | (inst << 8)}, k0, k1);
        const uint32_t w[4] = {q.a, q.b, q.c, q.d};
        T pt[D];
#pragma unroll
        for (int c = 0; c < D; ++c) pt[c] = lo[c] + ex[c] * u01<T>(w[c]);
        if (Sdf<T, D, KIND>::eval(sdf_prm, nsdf, pt) > T(0)) atomicAdd(&s_cnt[nearest_or_scan(V, m, pt)], 1u);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x)
        if (s_cnt[j]) atomicAdd(&counts[j], s_cnt[j]);
}

__global__ void counts_to_lambda_kernel(const unsigned int* __restrict__ counts, int m, double* __restrict__ lam) {
    __shared__ unsigned long long tot;
    if (threadIdx.x == 0) tot = 0;
    __syncthreads();
    unsigned long long s = 0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) s += counts[j];
    atomicAdd(&tot, s);
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) lam[j] = (double)counts[j] / (double)tot;
}

template <typename T, int D>
__global__ void node_radius_kernel(const double* __restrict__ x, int n, int kind, const T* __restrict__ prm,
                                   int nsdf, T* __restrict__ xT, T* __restrict__ r0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T p[D];
#pragma unroll
    for (int c = 0; c < D; ++c) { p[c] = (T)x[i * D + c]; xT[i * D + c] = p[c]; }
    T r;
    if (kind == SDF_BALL) r = Sdf<T, D, SDF_BALL>::eval(prm, nsdf, p);
    else if (kind == SDF_BOX) r = Sdf<T, D, SDF_BOX>::eval(prm, nsdf, p);
    else r = Sdf<T, 2, SDF_POLYGON>::eval(prm, nsdf, p);
    r0[i] = r;
}

// ------------------------------------------------------------------ the walk kernel
template <typename T, int D>
struct WalkArgs {
    int n, m, p;
    int64_t N;
    T eps;
    uint32_t k0, k1, inst;
    uint32_t rk[20];   // Philox key schedule of (k0, k1): rk[r] = k0 + r W0, rk[10 + r] = k1 + r W1
    int64_t max_steps;
    const T* x;        // [n][D]
    const T* r0;       // [n]
    const T* sdf;      // params
    int nsdf;          // polygon vertices (else unused)
    int sdf_len;       // number of T in sdf
    Lookup<T, D> V;
    Lookup<T, D> Z;
    int v_in_smem;
    int v_ncell;
    int64_t v_ncand;
    const uint16_t* v_candK;   // fixed-stride table [ncell][v_K] or NULL
    int v_K;
    T* P;              // [(D+1)][n][m]
    T* KH;             // [(D+1)][n][p]
    uint32_t* Hc;      // [n][p]
    float* pmax;       // [2] max |P| and max |G| of the rows written (FP32 bits, atomic max; may be NULL)
    int* row_counter;
    unsigned long long* stat_steps;
    unsigned long long* stat_capped;
    // G and grad G accumulators of the rows in flight, in global memory (L2-resident): CTA b owns
    // acc_g[b * acc_cells * 4 ..) as [cell][4] = (G, d_1 G, .., d_D G) (NULL: the shared-memory form)
    T* acc_g;
    int acc_cells;
    int64_t acc_len;                    // elements of acc_g
    // indexes the kernel found out of range and skipped (a bin, a row, the accumulator region;
    // none expected: the host reports any as an error); may be NULL
    unsigned long long* stat_bad;
    int32_t* rec_exit;
    int32_t* rec_steps;
    T* rec_mass;
    uint32_t* rec_vhash;   // XOR over the walk's interior binnings of cellmix(step tag, cell)
    T* rec_xexit;          // [n][N][D] stopping point
    // autotuner trials: fetched row t < trial_rows is row (t * trial_step) mod n (0: all rows in order)
    int trial_rows;
    int trial_step;
    // polygon edge grid (walk steps): candidate edges per cell, records (ax, ay, ex, ey, 1/|e|^2)
    // at sdf[e_off + 5 e]; NULL for other domains (and the full scan is used)
    const uint8_t* e_cnt;
    const uint8_t* e_list;  // [ncell][nsdf]
    T e_lo0, e_lo1, e_inv_h;
    int e_nx, e_ny, e_off;
};

// walk-record digest of one interior binning: the splitmix64 output function applied to
// (tag << 32 | cell), folded to 32 bits (Vigna's SplitMix64 finaliser)
__device__ __forceinline__ uint32_t cellmix(uint32_t tag, uint32_t cell) {
    unsigned long long x = ((unsigned long long)tag << 32) | cell;
    x ^= x >> 30; x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27; x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return (uint32_t)(x ^ (x >> 32));
}

// One walk point's binning (G += G_add, grad G += g[0..D)) into cell j of the CTA's accumulator
// row.  Global form: the 1 + D values sit together in a 16-byte (FP32) cell and go to L2 as one
// vector reduction; FP32 atomics in shared memory cost about 20 % of the walk (a
// compare-and-swap loop per value on the L1 data pipe), the reduction next to nothing.
// Shared form: one shared-memory atomic per value, planar rows acc[c * m + j].
template <typename T, int D, bool L2ACC>
__device__ __forceinline__ void bin_point(T* acc, int m, int j, T G_add, const T* g, bool grad) {
    if constexpr (L2ACC) {
        T* dst = acc + (size_t)j * 4;
        if constexpr (std::is_same<T, float>::value) {
            const float g0 = grad ? g[0] : 0.0f, g1 = grad ? g[1] : 0.0f, g2 = (grad && D == 3) ? g[D - 1] : 0.0f;
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(G_add), "f"(g0), "f"(g1),
                         "f"(g2)
                         : "memory");
        } else {
            if (G_add != T(0)) atomicAdd(dst, G_add);
            if (grad) {
#pragma unroll
                for (int c = 0; c < D; ++c) atomicAdd(dst + 1 + c, g[c]);
            }
        }
    } else {
        if (G_add != T(0)) atomicAdd(&acc[(size_t)D * m + j], G_add);
        if (grad) {
#pragma unroll
            for (int c = 0; c < D; ++c) atomicAdd(&acc[(size_t)c * m + j], g[c]);
        }
    }
}

// Random-number layout (shared with the oracle through its published definition):
//   ball term   counter (l, 0xFFFFFFFF, i, inst|0): (S, angle or z, phi, -)
//   step k >= 0 counter (l, k, i, inst|slot): d = 2 slot 0 = (radius of Y, angle of Y, angle of U, -);
//               d = 3 slot 0 = (median uniforms x3, z of Y), slot 1 = (phi of Y, z of U, phi of U, -)
// Philox block of counter c: from the precomputed key schedule rk (single builds: the schedule sits
// in the kernel's parameters) or from the key (batched builds read their arguments from shared
// memory, where the schedule would cost loads)
template <bool PRK>
__device__ __forceinline__ u32x4 walk_philox(u32x4 c, uint32_t k0, uint32_t k1, const uint32_t* rk) {
    if constexpr (PRK) return philox4x32_10_rk(c, rk);
    else return philox4x32_10(c, k0, k1);
}

template <typename T, int D, bool PRK = false>
__device__ __forceinline__ void draw_ball(uint32_t l, uint32_t row, uint32_t inst, uint32_t k0, uint32_t k1,
                                          T& S, T* Zb, const uint32_t* rk = nullptr) {
    const u32x4 q = walk_philox<PRK>(u32x4{l, 0xFFFFFFFFu, row, inst}, k0, k1, rk);
    S = T(1) - m_sqrt(u01<T>(q.a));
    if (D == 2) dir2<T>(u01<T>(q.b), Zb);
    else dir3<T>(u01<T>(q.b), u01<T>(q.c), Zb);
}

template <typename T, int D, bool PRK = false>
__device__ __forceinline__ void draw_step(uint32_t l, uint32_t k, uint32_t row, uint32_t inst, uint32_t k0,
                                          uint32_t k1, T& R, T* Zs, T* U, const uint32_t* rk = nullptr) {
    if (D == 2) {
        const u32x4 q = walk_philox<PRK>(u32x4{l, k, row, inst | 0u}, k0, k1, rk);
        R = green_radius_2d<T>(u01<T>(q.a));
        dir2<T>(u01<T>(q.b), Zs);
        dir2<T>(u01<T>(q.c), U);
    } else {
        const u32x4 q = walk_philox<PRK>(u32x4{l, k, row, inst | 0u}, k0, k1, rk);
        const u32x4 v = walk_philox<PRK>(u32x4{l, k, row, inst | 1u}, k0, k1, rk);
        R = med3(u01<T>(q.a), u01<T>(q.b), u01<T>(q.c));
        dir3<T>(u01<T>(q.d), u01<T>(v.a), Zs);
        dir3<T>(u01<T>(v.b), u01<T>(v.c), U);
    }
}

// nearest V centre through the fixed-stride table (K slots per grid cell, uniform trip count)
template <typename T, int D>
__device__ __forceinline__ int nearest_fixed(const Lookup<T, D>& L, const uint16_t* __restrict__ candK, int K,
                                             const T* q, int sentinel) {
    const int cell = lookup_cell(L, q);
    const uint16_t* c = candK + (size_t)cell * K;
    // a cell with one candidate lies inside that centre's Voronoi cell: no distance needed
    const int j0 = c[0];
    if (K == 1 || c[1] >= sentinel) return j0;
    T best = T(3.0e38f);
    int bi = 0;
    for (int t = 0; t < K; ++t) {
        const int j = c[t];
        if (j >= sentinel) break;             // the list ends where the sentinel padding starts
        T d2 = 0;
#pragma unroll
        for (int cc = 0; cc < D; ++cc) { const T dd = q[cc] - L.pts[j * D + cc]; d2 += dd * dd; }
        if (d2 < best) { best = d2; bi = j; }
    }
    return bi;
}

constexpr int kQueue = 64;   // per-warp queue of stopped walks awaiting their boundary binning

// A stopped walk's first direction U_0 is not queued: the binning draws it again from the
// walk's step-0 counter (one Philox block), which leaves more of the SM's unified L1 / shared
// memory to the L1 (the ball's queue shrinks from 48 to 32 KB).
template <typename T, int D>
struct WalkQueue {
    T* X;          // [warps][kQueue][D] stopping point
    uint32_t* L;   // [warps][kQueue] walk index
    uint32_t* vh;  // [warps][kQueue] binning digest  (records only)
    uint32_t* K;   // [warps][kQueue] steps           (records only)
    T* mass;       // [warps][kQueue] G mass          (records only)
};

// bytes of the per-warp queues in shared memory
template <typename T, int D>
__host__ __device__ constexpr size_t queue_bytes(int nwarps, bool record) {
    return (size_t)nwarps * kQueue * (D * sizeof(T) + sizeof(uint32_t) + (record ? 2 * sizeof(uint32_t) + sizeof(T) : 0));
}

// U_0 of walk l of a row, as draw_step draws it at step 0
template <typename T, int D, bool PRK = false>
__device__ __forceinline__ void draw_first_direction(uint32_t l, uint32_t row, uint32_t inst, uint32_t k0, uint32_t k1,
                                                     T* U, const uint32_t* rk = nullptr) {
    if (D == 2) {
        const u32x4 q = walk_philox<PRK>(u32x4{l, 0u, row, inst | 0u}, k0, k1, rk);
        dir2<T>(u01<T>(q.c), U);
    } else {
        const u32x4 v = walk_philox<PRK>(u32x4{l, 0u, row, inst | 1u}, k0, k1, rk);
        dir3<T>(u01<T>(v.b), u01<T>(v.c), U);
    }
}

template <typename T, int D, bool RECORD, bool PRK>
__device__ __forceinline__ void bin_stopped(const WalkArgs<T, D>& a, const WalkQueue<T, D>& q, int slot, int row,
                                            T* accKH, uint32_t* accH) {
    T X[D], U[D];
#pragma unroll
    for (int c = 0; c < D; ++c) X[c] = q.X[slot * D + c];
    draw_first_direction<T, D, PRK>(q.L[slot], (uint32_t)row, a.inst, a.k0, a.k1, U, a.rk);
    const int jz = nearest_or_scan(a.Z, a.p, X);
    atomicAdd(&accH[jz], 1u);
#pragma unroll
    for (int c = 0; c < D; ++c) atomicAdd(&accKH[(size_t)c * a.p + jz], U[c]);
    if (RECORD) {
        const size_t ri = (size_t)row * a.N + q.L[slot];
        a.rec_exit[ri] = jz;
#pragma unroll
        for (int c = 0; c < D; ++c) a.rec_xexit[ri * D + c] = X[c];
        a.rec_mass[ri] = q.mass[slot];
        a.rec_steps[ri] = (int32_t)q.K[slot];
        atomicXor(&a.rec_vhash[ri], q.vh[slot]);
    }
}

// Distance from a point of the polygon to its boundary through the edge grid: only the cell's
// candidate edges are measured (a superset of the edges that can be nearest to a point of the
// cell, with a margin above the rounding of this arithmetic, so the minimum is the full scan's).
// Walk points lie in the domain, so the distance is returned without the crossing-rule sign.
template <typename T, int D>
__device__ __forceinline__ T polygon_dist_grid(const WalkArgs<T, D>& a, const T* s_prm, const T* x) {
    int cx = (int)floorf((float)((x[0] - a.e_lo0) * a.e_inv_h));
    int cy = (int)floorf((float)((x[1] - a.e_lo1) * a.e_inv_h));
    cx = min(max(cx, 0), a.e_nx - 1);
    cy = min(max(cy, 0), a.e_ny - 1);
    const int cell = cy * a.e_nx + cx;
    const int n = a.e_cnt[cell];
    const uint8_t* L = a.e_list + (size_t)cell * a.nsdf;
    const T* rec = s_prm + a.e_off;
    T best = T(3.0e38f);
    for (int i = 0; i < n; ++i) {
        const T* r = rec + 5 * L[i];
        const T px = x[0] - r[0], py = x[1] - r[1];
        T t = (px * r[2] + py * r[3]) * r[4];
        t = fmin(fmax(t, T(0)), T(1));
        const T dx = px - t * r[2], dy = py - t * r[3];
        best = fmin(best, dx * dx + dy * dy);
    }
    return m_sqrt(best);
}

// The persistent row loop of one toolbox (instance).  Single builds fetch rows from the
// instance's own counter; batched builds fetch global rows g from one counter shared by all
// instances (rows of instance k are [gbase, gend)) and return the first fetched row that belongs
// to a later instance.
template <typename T, int D, int KIND, bool RECORD, bool BATCH, bool L2ACC>
__device__ __forceinline__ int walk_rows(const WalkArgs<T, D>& a, int g_first, int gbase, int gend, int* gcounter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // shared layout: [acc [(D+1)][m] T, shared form only] | accKH [D][p] T | accH [p] u32 | sdf
    // params | per-warp queues | V lookup (points, then the fixed-stride table or the CSR lists)
    T* acc = L2ACC ? a.acc_g + (size_t)blockIdx.x * a.acc_cells * 4 : reinterpret_cast<T*>(smem_raw);
    T* accKH = L2ACC ? reinterpret_cast<T*>(smem_raw) : acc + (size_t)(D + 1) * a.m;
    uint32_t* accH = reinterpret_cast<uint32_t*>(accKH + (size_t)D * a.p);
    T* s_sdf = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(accH + a.p) + 15) & ~uintptr_t(15));
    const int nwarps = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WalkQueue<T, D> q;
    q.X = s_sdf + ((a.sdf_len + 3) & ~3);
    q.L = reinterpret_cast<uint32_t*>(q.X + (size_t)nwarps * kQueue * D);
    const size_t qr = RECORD ? (size_t)nwarps * kQueue : 0;
    q.vh = q.L + (size_t)nwarps * kQueue;
    q.K = q.vh + qr;
    q.mass = reinterpret_cast<T*>(q.K + qr);
    unsigned char* s_v = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(q.mass + qr) + 15) & ~uintptr_t(15));
    __shared__ int s_row;
    __shared__ unsigned int s_walk;

    for (int t = threadIdx.x; t < a.sdf_len; t += blockDim.x) s_sdf[t] = a.sdf[t];
    Lookup<T, D> V = a.V;
    const uint16_t* candK = a.v_candK;
    if (a.v_in_smem) {
        T* vp = reinterpret_cast<T*>(s_v);
        for (int t = threadIdx.x; t < (a.m + 1) * D; t += blockDim.x) vp[t] = a.V.pts[t];
        V.pts = vp;
        if (a.v_K > 0) {
            uint16_t* vk = reinterpret_cast<uint16_t*>(vp + (size_t)(a.m + 1) * D);
            for (int64_t t = threadIdx.x; t < (int64_t)a.v_ncell * a.v_K; t += blockDim.x) vk[t] = a.v_candK[t];
            candK = vk;
        } else {
            int* vs = reinterpret_cast<int*>(vp + (size_t)(a.m + 1) * D);
            int* vc = vs + a.v_ncell + 1;
            for (int t = threadIdx.x; t <= a.v_ncell; t += blockDim.x) vs[t] = a.V.start[t];
            for (int64_t t = threadIdx.x; t < a.v_ncand; t += blockDim.x) vc[t] = a.V.cand[t];
            V.start = vs; V.cand = vc;
        }
    }
    const int K = a.v_K;
    if (L2ACC && ((int64_t)(blockIdx.x + 1) * a.acc_cells * 4 > a.acc_len || a.m > a.acc_cells)) {
        if (threadIdx.x == 0 && a.stat_bad) atomicAdd(a.stat_bad, 1ull);
        return BATCH ? gend : 0;              // (the CTA as a whole, before any barrier)
    }
    const int accN = L2ACC ? 4 * a.acc_cells : (D + 1) * a.m;
    for (int t = threadIdx.x; t < accN; t += blockDim.x) acc[t] = T(0);
    for (int t = threadIdx.x; t < D * a.p; t += blockDim.x) accKH[t] = T(0);
    for (int t = threadIdx.x; t < a.p; t += blockDim.x) accH[t] = 0u;

    unsigned long long my_steps = 0, my_capped = 0;
    const T invN = T(1) / (T)a.N;
    bool first = true;
    int g_next = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            if (BATCH) s_row = first ? g_first : atomicAdd(gcounter, 1);
            else s_row = atomicAdd(a.row_counter, 1);
            s_walk = 0u;
        }
        first = false;
        __syncthreads();
        int row = s_row;
        if (BATCH) {
            if (row >= gend) { g_next = row; break; }
            row -= gbase;
            if (row < 0 || row >= a.n) {
                if (threadIdx.x == 0 && a.stat_bad) atomicAdd(a.stat_bad, 1ull);
                g_next = gend;
                break;
            }
        } else if (a.trial_rows > 0) {
            if (row >= a.trial_rows) break;
            row = (int)(((int64_t)row * a.trial_step) % a.n);
        } else if (row >= a.n) {
            break;
        }
        T xi[D];
#pragma unroll
        for (int c = 0; c < D; ++c) xi[c] = a.x[(size_t)row * D + c];
        const T r0 = a.r0[row];
        const T r02 = r0 * r0;

        // ---- ball term of the first sphere (path independent, Prop. 2.6 (ii))
        for (int64_t l = threadIdx.x; l < a.N; l += blockDim.x) {
            T S, Zb[D], pt[D];
            draw_ball<T, D, !BATCH>((uint32_t)l, (uint32_t)row, a.inst, a.k0, a.k1, S, Zb, a.rk);
            const T wsum = (D == 2) ? T(1) + S : T(1) + S + S * S;
#pragma unroll
            for (int c = 0; c < D; ++c) pt[c] = xi[c] + r0 * S * Zb[c];
            const int jb = K > 0 ? nearest_fixed(V, candK, K, pt, a.m) : nearest_or_scan(V, a.m, pt);
            T gb[D];
#pragma unroll
            for (int c = 0; c < D; ++c) gb[c] = r02 * wsum * Zb[c];
            if ((unsigned)jb < (unsigned)a.m) bin_point<T, D, L2ACC>(acc, a.m, jb, T(0), gb, true);
            else if (a.stat_bad) atomicAdd(a.stat_bad, 1ull);
            if (RECORD) atomicXor(&a.rec_vhash[(size_t)row * a.N + l], cellmix(0xFFFFFFFFu, jb));
        }

        // ---- the chains.  The warp iterates until none of its lanes holds a walk; a lane whose
        // walk stops queues its stopping point for boundary binning (slots assigned from a ballot,
        // the queue length kept warp-uniform in a register) and takes the next walk of the row,
        // doing that walk's step 0 (at x_i, radius r0) in the same iteration as the other lanes'
        // steps; the warp bins 32 queued walks together whenever it holds that many.
        uint32_t l = atomicAdd(&s_walk, 1u);
        bool have = l < (uint64_t)a.N;
        T X[D], U0[D], mass = T(0);
        uint32_t k = 0, vh = 0u;
        int qn = 0;
        const unsigned below = (1u << lane) - 1u;
#pragma unroll
        for (int c = 0; c < D; ++c) { X[c] = xi[c]; U0[c] = T(0); }
        for (;;) {
            if (!__any_sync(0xffffffffu, have)) break;
            T r = r0;
            if (have && k > 0) {
                if (KIND == SDF_POLYGON && a.e_cnt) r = polygon_dist_grid<T, D>(a, s_sdf, X);
                else r = Sdf<T, D, KIND>::eval(s_sdf, a.nsdf, X);
            }
            const bool stop = have && k > 0 && (r < a.eps || (int64_t)k > a.max_steps);
            const unsigned sm = __ballot_sync(0xffffffffu, stop);
            if (stop) {
                const int slot = wid * kQueue + qn + __popc(sm & below);
#pragma unroll
                for (int c = 0; c < D; ++c) q.X[slot * D + c] = X[c];
                q.L[slot] = l;
                if (RECORD) {
                    q.mass[slot] = mass / T(2 * D); q.vh[slot] = vh; q.K[slot] = k - 1;
                    vh = 0u; mass = T(0);
                }
                my_steps += k;
                my_capped += (r >= a.eps);
                l = atomicAdd(&s_walk, 1u);
                have = l < (uint64_t)a.N;
#pragma unroll
                for (int c = 0; c < D; ++c) X[c] = xi[c];
                k = 0;
                r = r0;
            }
            qn += __popc(sm);
            if (have) {
                T R, Zs[D], U[D], pt[D];
                draw_step<T, D, !BATCH>(l, k, (uint32_t)row, a.inst, a.k0, a.k1, R, Zs, U, a.rk);
                const T rR = r * R;
#pragma unroll
                for (int c = 0; c < D; ++c) pt[c] = X[c] + rR * Zs[c];
                const int j = K > 0 ? nearest_fixed(V, candK, K, pt, a.m) : nearest_or_scan(V, a.m, pt);
                const T r2 = r * r;
                T gs[D];
#pragma unroll
                for (int c = 0; c < D; ++c) gs[c] = U0[c] * r2;     // (not added at step 0)
                if ((unsigned)j < (unsigned)a.m) bin_point<T, D, L2ACC>(acc, a.m, j, r2, gs, k > 0);
                else if (a.stat_bad) atomicAdd(a.stat_bad, 1ull);
                if (k == 0) {
#pragma unroll
                    for (int c = 0; c < D; ++c) U0[c] = U[c];
                }
#pragma unroll
                for (int c = 0; c < D; ++c) X[c] += r * U[c];
                if (RECORD) { mass += r2; vh ^= cellmix(k, (uint32_t)j); }
                ++k;
            }
            // converged boundary binning of queued walks (queue < 32 + 32 <= kQueue entries)
            __syncwarp();
            while (qn >= 32) {
                bin_stopped<T, D, RECORD, !BATCH>(a, q, wid * kQueue + qn - 1 - lane, row, accKH, accH);
                qn -= 32;
            }
            __syncwarp();
        }
        // drain this warp's queue
        for (int e = lane; e < qn; e += 32) bin_stopped<T, D, RECORD, !BATCH>(a, q, wid * kQueue + e, row, accKH, accH);
        __syncwarp();
        __syncthreads();

        // ---- flush the row: scale and write coalesced, then clear the accumulators.  The output
        // rows (1.3 GB per ball launch) are written with the streaming (evict-first) policy, so
        // that they do not push the V lookup's candidate table (74 MB) out of L2
        const T sG = invN / T(2 * D);
        const T sGG = invN / (T(2) * r0);
        const T sKH = T(D) * invN / r0;
        const size_t nm = (size_t)a.n * a.m, np = (size_t)a.n * a.p;
        float my_pmax = 0.f, my_gmax = 0.f;   // largest |value| of P (of G) this thread writes in the row
        for (int t = threadIdx.x; t < a.m; t += blockDim.x) {
            if constexpr (L2ACC) {
                // the reductions of the row are complete at the barrier above; read past L1
                T v[4];
                if constexpr (std::is_same<T, float>::value) {
                    const float4 q4 = __ldcg(reinterpret_cast<const float4*>(acc) + t);
                    v[0] = q4.x; v[1] = q4.y; v[2] = q4.z; v[3] = q4.w;
                    __stcg(reinterpret_cast<float4*>(acc) + t, make_float4(0.f, 0.f, 0.f, 0.f));
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) { v[c] = __ldcg(acc + (size_t)t * 4 + c); acc[(size_t)t * 4 + c] = T(0); }
                }
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const T o = v[1 + c] * sGG;
                    __stcs(a.P + c * nm + (size_t)row * a.m + t, o);
                    my_pmax = fmaxf(my_pmax, fabsf((float)o));
                }
                const T og = v[0] * sG;
                __stcs(a.P + D * nm + (size_t)row * a.m + t, og);
                my_gmax = fmaxf(my_gmax, fabsf((float)og));
            } else {
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const T o = acc[(size_t)c * a.m + t] * sGG;
                    __stcs(a.P + c * nm + (size_t)row * a.m + t, o);
                    my_pmax = fmaxf(my_pmax, fabsf((float)o));
                    acc[(size_t)c * a.m + t] = T(0);
                }
                const T og = acc[(size_t)D * a.m + t] * sG;
                __stcs(a.P + D * nm + (size_t)row * a.m + t, og);
                my_gmax = fmaxf(my_gmax, fabsf((float)og));
                acc[(size_t)D * a.m + t] = T(0);
            }
        }
        if (a.pmax) {                         // (non-negative floats compare as their bits)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                my_pmax = fmaxf(my_pmax, __shfl_xor_sync(0xffffffffu, my_pmax, o));
                my_gmax = fmaxf(my_gmax, __shfl_xor_sync(0xffffffffu, my_gmax, o));
            }
            my_pmax = fmaxf(my_pmax, my_gmax);
            if (lane == 0 && my_pmax > 0.f) atomicMax(reinterpret_cast<unsigned int*>(a.pmax), __float_as_uint(my_pmax));
            if (lane == 0 && my_gmax > 0.f) atomicMax(reinterpret_cast<unsigned int*>(a.pmax + 1), __float_as_uint(my_gmax));
        }
        for (int t = threadIdx.x; t < a.p; t += blockDim.x) {
#pragma unroll
            for (int c = 0; c < D; ++c) {
                __stcs(a.KH + c * np + (size_t)row * a.p + t, accKH[(size_t)c * a.p + t] * sKH);
                accKH[(size_t)c * a.p + t] = T(0);
            }
            const uint32_t h = accH[t];
            __stcs(a.KH + D * np + (size_t)row * a.p + t, (T)h * invN);
            __stcs(a.Hc + (size_t)row * a.p + t, h);
            accH[t] = 0u;
        }
    }
    // totals
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_steps += __shfl_down_sync(0xffffffffu, my_steps, o);
        my_capped += __shfl_down_sync(0xffffffffu, my_capped, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(a.stat_steps, my_steps);
        if (my_capped) atomicAdd(a.stat_capped, my_capped);
    }
    return g_next;
}

// the row kernel with its G / grad G accumulators in global memory (walk_kernel 1, the default)
template <typename T, int D, int KIND, bool RECORD>
__global__ void __launch_bounds__(1024, 1) wos_walk_kernel(WalkArgs<T, D> a) {
    walk_rows<T, D, KIND, RECORD, false, true>(a, 0, 0, 0, nullptr);
}

// the same with the accumulators in shared memory (walk_kernel 2; the build without allocation)
template <typename T, int D, int KIND, bool RECORD>
__global__ void __launch_bounds__(1024, 1) wos_walk_smem_kernel(WalkArgs<T, D> a) {
    walk_rows<T, D, KIND, RECORD, false, false>(a, 0, 0, 0, nullptr);
}

// Several toolboxes in one persistent launch: the rows of all instances form one index space
// (instance k owns [row_off[k], row_off[k+1])); a CTA takes the next global row, loads that
// instance's arguments into shared memory when the instance changes, and runs the instance's
// row loop until it draws a row of a later instance.
template <typename T, int D, int KIND>
__global__ void __launch_bounds__(1024, 1) wos_walk_batch_kernel(const WalkArgs<T, D>* __restrict__ batch,
                                                                 const int* __restrict__ row_off, int nb,
                                                                 int* __restrict__ gcounter) {
    __shared__ WalkArgs<T, D> s_a;
    __shared__ int s_g;
    if (threadIdx.x == 0) s_g = atomicAdd(gcounter, 1);
    __syncthreads();
    int g = s_g;
    const int total = row_off[nb];
    while (g < total) {
        int lo = 0, hi = nb - 1;              // last instance whose first row is <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (row_off[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_a = batch[lo];
        __syncthreads();
        g = walk_rows<T, D, KIND, false, true, true>(s_a, g, row_off[lo], row_off[lo + 1], gcounter);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host side
static double host_sdf(int dim, int kind, const double* prm, int64_t nprm, const double* x) {
    if (kind == SDF_BALL) {
        double s = 0;
        for (int c = 0; c < dim; ++c) s += (x[c] - prm[c]) * (x[c] - prm[c]);
        return prm[dim] - std::sqrt(s);
    }
    if (kind == SDF_BOX) {
        double r = 1e300;
        for (int c = 0; c < dim; ++c) r = std::min(r, std::min(x[c] - prm[c], prm[dim + c] - x[c]));
        return r;
    }
    const int64_t nv = nprm / 2;
    double best = 1e300;
    bool inside = false;
    for (int64_t e = 0; e < nv; ++e) {
        const double ax = prm[2 * e], ay = prm[2 * e + 1];
        const int64_t f = (e + 1) % nv;
        const double bx = prm[2 * f], by = prm[2 * f + 1];
        const double ex = bx - ax, ey = by - ay, px = x[0] - ax, py = x[1] - ay;
        double t = (px * ex + py * ey) / (ex * ex + ey * ey);
        t = std::min(1.0, std::max(0.0, t));
        const double dx = px - t * ex, dy = py - t * ey;
        best = std::min(best, dx * dx + dy * dy);
        if ((ay > x[1]) != (by > x[1])) {
            const double xc = ax + (x[1] - ay) / (by - ay) * ex;
            if (x[0] < xc) inside = !inside;
        }
    }
    return inside ? std::sqrt(best) : -std::sqrt(best);
}

static void domain_bbox(int dim, int kind, const double* prm, int64_t nprm, double* lo, double* hi) {
    if (kind == SDF_BALL) {
        for (int c = 0; c < dim; ++c) { lo[c] = prm[c] - prm[dim]; hi[c] = prm[c] + prm[dim]; }
    } else if (kind == SDF_BOX) {
        for (int c = 0; c < dim; ++c) { lo[c] = prm[c]; hi[c] = prm[dim + c]; }
    } else {
        lo[0] = lo[1] = 1e300; hi[0] = hi[1] = -1e300;
        for (int64_t e = 0; e < nprm / 2; ++e)
            for (int c = 0; c < 2; ++c) {
                lo[c] = std::min(lo[c], prm[2 * e + c]);
                hi[c] = std::max(hi[c], prm[2 * e + c]);
            }
    }
}

// ------------------------------------------------------------------ polygon edge grid
__device__ __forceinline__ double seg_point_dist(double px, double py, double ax, double ay, double bx, double by) {
    const double ex = bx - ax, ey = by - ay, ee = ex * ex + ey * ey;
    double t = ee > 0 ? ((px - ax) * ex + (py - ay) * ey) / ee : 0.0;
    t = fmin(fmax(t, 0.0), 1.0);
    const double dx = px - ax - t * ex, dy = py - ay - t * ey;
    return sqrt(dx * dx + dy * dy);
}

__device__ __forceinline__ double box_point_dist(double px, double py, double x0, double x1, double y0, double y1) {
    const double dx = fmax(fmax(x0 - px, px - x1), 0.0), dy = fmax(fmax(y0 - py, py - y1), 0.0);
    return sqrt(dx * dx + dy * dy);
}

// the segment meets the closed box (parametric clipping against the four slabs)
__device__ __forceinline__ bool seg_meets_box(double ax, double ay, double bx, double by, double x0, double x1,
                                              double y0, double y1) {
    double t0 = 0.0, t1 = 1.0;
    const double d[2] = {bx - ax, by - ay}, o[2] = {ax, ay}, lo[2] = {x0, y0}, hi[2] = {x1, y1};
    for (int c = 0; c < 2; ++c) {
        if (d[c] == 0.0) {
            if (o[c] < lo[c] || o[c] > hi[c]) return false;
        } else {
            double ta = (lo[c] - o[c]) / d[c], tb = (hi[c] - o[c]) / d[c];
            if (ta > tb) { const double t = ta; ta = tb; tb = t; }
            t0 = fmax(t0, ta);
            t1 = fmin(t1, tb);
            if (t0 > t1) return false;
        }
    }
    return true;
}

// Candidate edges of each cell of a uniform grid over the polygon's box: every edge whose
// distance to the cell is at most R = min_f maxdist(cell, f) + margin (the nearest edge of any
// point of the cell is at most R away from it).  One CTA per cell, one thread per edge (edge e
// joins vertex e-1 to vertex e), FP64; the list is written in increasing edge order.
__global__ void polygon_grid_kernel(const double* __restrict__ V, int nv, double lo0, double lo1, double h, int nx,
                                   double margin, uint8_t* __restrict__ cnt, uint8_t* __restrict__ list) {
    __shared__ double s_max[256];
    __shared__ unsigned char s_flag[256];
    const int cell = blockIdx.x, cx = cell % nx, cy = cell / nx, e = threadIdx.x;
    const double x0 = lo0 + cx * h, x1 = x0 + h, y0 = lo1 + cy * h, y1 = y0 + h;
    double mx = 1e300, mn = 1e300;
    if (e < nv) {
        const int a = (e + nv - 1) % nv;
        const double ax = V[2 * a], ay = V[2 * a + 1], bx = V[2 * e], by = V[2 * e + 1];
        const double cxs[4] = {x0, x1, x0, x1}, cys[4] = {y0, y0, y1, y1};
        mx = 0.0;
        for (int q = 0; q < 4; ++q) mx = fmax(mx, seg_point_dist(cxs[q], cys[q], ax, ay, bx, by));
        if (seg_meets_box(ax, ay, bx, by, x0, x1, y0, y1)) {
            mn = 0.0;
        } else {
            mn = fmin(box_point_dist(ax, ay, x0, x1, y0, y1), box_point_dist(bx, by, x0, x1, y0, y1));
            for (int q = 0; q < 4; ++q) mn = fmin(mn, seg_point_dist(cxs[q], cys[q], ax, ay, bx, by));
        }
    }
    s_max[e] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (e < o) s_max[e] = fmin(s_max[e], s_max[e + o]);
        __syncthreads();
    }
    const double R = s_max[0];
    s_flag[e] = (e < nv && mn <= R + margin) ? 1 : 0;
    __syncthreads();
    if (e == 0) {
        int c = 0;
        for (int f = 0; f < nv; ++f)
            if (s_flag[f]) list[(size_t)cell * nv + c++] = (uint8_t)f;
        cnt[cell] = (uint8_t)c;
    }
}

struct BuildContext {
    DeviceLookup V, Z, V2;       // V2: the V lookup on the alternative grid the autotuner tries
    DeviceLookup W;              // the nodes' own cells (cell weights) when V-centres are separate
    void* d_sdf = nullptr;
    void* d_xT = nullptr;
    double* d_vtx = nullptr;         // polygon vertices (FP64) for the edge grid
    uint8_t* d_egrid = nullptr;      // edge grid: counts [ncell] then lists [ncell][nv]
    void* d_r0 = nullptr;
    int* d_counter = nullptr;
    unsigned long long* d_stats = nullptr;
    unsigned int* d_counts = nullptr;
    void* d_acc = nullptr;           // G / grad G accumulators of the rows in flight (walk_kernel 1)
    size_t acc_cap = 0;
    ~BuildContext() {
        V.release(); Z.release(); V2.release(); W.release();
        ::ewos::dev_free(d_sdf); ::ewos::dev_free(d_xT); ::ewos::dev_free(d_r0); ::ewos::dev_free(d_counter); ::ewos::dev_free(d_stats); ::ewos::dev_free(d_counts);
        ::ewos::dev_free(d_vtx); ::ewos::dev_free(d_egrid); ::ewos::dev_free(d_acc);
    }
    // at least `bytes` of accumulator space (kept for the rest of the build)
    cudaError_t ensure_acc(size_t bytes) {
        if (acc_cap >= bytes) return cudaSuccess;
        ::ewos::dev_free(d_acc);
        d_acc = nullptr;
        acc_cap = 0;
        cudaError_t e = ::ewos::dev_alloc(&d_acc, bytes);
        if (e == cudaSuccess) acc_cap = bytes;
        return e;
    }
};

// the row kernels: 1 accumulators in global memory, 2 in shared memory
template <typename T, int D, int KIND, bool RECORD>
static void (*row_kernel(int kern))(WalkArgs<T, D>) {
    if (kern == 2) return wos_walk_smem_kernel<T, D, KIND, RECORD>;
    return wos_walk_kernel<T, D, KIND, RECORD>;
}

template <typename T, int D, int KIND, bool RECORD>
static cudaError_t launch_walks(const WalkArgs<T, D>& a, int grid, int tpb, size_t smem, cudaStream_t st, int kern = 1) {
    auto k = row_kernel<T, D, KIND, RECORD>(kern);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ::ewos::note_launch(), k<<<grid, tpb, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T, int D, int KIND>
static cudaError_t dispatch_walks(const WalkArgs<T, D>& a, bool rec, int grid, int tpb, size_t smem, cudaStream_t st,
                                  int kern) {
    return rec ? launch_walks<T, D, KIND, true>(a, grid, tpb, smem, st, kern)
               : launch_walks<T, D, KIND, false>(a, grid, tpb, smem, st, kern);
}

template <typename T, int D, int KIND>
static int max_ctas_per_sm(int tpb, size_t smem, int kern = 1) {
    int nb = 0;
    auto k = row_kernel<T, D, KIND, false>(kern);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, tpb, smem);
    return nb;
}

// a step s coprime with n near n / rows: rows t s mod n (t < rows) are distinct and spread out
static int trial_step_for(int n, int rows) {
    if (rows >= n) return 1;
    int s = std::max(1, n / std::max(1, rows));
    auto gcd = [](int a, int b) { while (b) { const int t = a % b; a = b; b = t; } return a; };
    while (gcd(s, n) != 1) ++s;
    return s;
}

// process-wide cache of the walk kernel configurations chosen by the autotuner
struct TuneKey {
    size_t elem; int dim, kind; int m, p; int64_t N; bool rec; int tpb_req, place_req, ctas_req; double grid_req;
    int kernel_req;
    bool operator==(const TuneKey& o) const {
        return elem == o.elem && dim == o.dim && kind == o.kind && m == o.m && p == o.p && N == o.N && rec == o.rec &&
               tpb_req == o.tpb_req && place_req == o.place_req && ctas_req == o.ctas_req && grid_req == o.grid_req &&
               kernel_req == o.kernel_req;
    }
};
struct TuneVal { int tpb; bool v_smem; int vgrid; int kernel; };
static std::mutex g_tune_mu;
static std::vector<std::pair<TuneKey, TuneVal>> g_tune;

static bool tune_lookup(const TuneKey& k, int& tpb, bool& v_smem, int& vgrid, int* kernel = nullptr) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (auto& e : g_tune)
        if (e.first == k) {
            tpb = e.second.tpb; v_smem = e.second.v_smem; vgrid = e.second.vgrid;
            if (kernel) *kernel = e.second.kernel;
            return true;
        }
    return false;
}

static void tune_store(const TuneKey& k, int tpb, bool v_smem, int vgrid, int kernel) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.push_back({k, TuneVal{tpb, v_smem, vgrid, kernel}});
}

// Everything before the walk launch of one toolbox: distances and node radii, the Voronoi
// lookups (the default V grid; also the alternative grid when alt_grid), cell weights, and the
// walk arguments (V set to the default grid, in global memory).
struct PrepOut {
    double lo[3], hi[3];
    double gf_default, gf_alt;
    bool have_cached;
    int cached_tpb, cached_grid;
    bool cached_smem;
    bool tune_grid;
    int cached_kernel;
};

template <typename T, int D>
static ewos_status prepare_walks(ewos_toolbox* tb, const ewos_domain* dom, const double* d_x, const double* d_z,
                                 const ewos_build_opts& o, BuildContext& ctx, WalkArgs<T, D>& a, PrepOut& po,
                                 cudaEvent_t ev_lookup, cudaEvent_t ev_cells, bool allow_alt) {
    cudaStream_t st = tb->stream;
    const int n = (int)tb->n, m = (int)tb->m, p = (int)tb->p;
    // distance parameters and node radii
    std::vector<T> prmT(dom->nparams);
    for (int64_t t = 0; t < dom->nparams; ++t) prmT[t] = (T)dom->params[t];
    const int nsdf = dom->kind == SDF_POLYGON ? (int)(dom->nparams / 2) : 0;
    const bool egrid = dom->kind == SDF_POLYGON && nsdf <= 255;
    if (egrid) {
        // edge records (a, b - a, 1/|b - a|^2) of edge e = (vertex e-1, vertex e), for the walks
        for (int e = 0; e < nsdf; ++e) {
            const int q = (e + nsdf - 1) % nsdf;
            const double ax = dom->params[2 * q], ay = dom->params[2 * q + 1];
            const double ex = dom->params[2 * e] - ax, ey = dom->params[2 * e + 1] - ay;
            const double ee = ex * ex + ey * ey;
            prmT.push_back((T)ax); prmT.push_back((T)ay); prmT.push_back((T)ex); prmT.push_back((T)ey);
            prmT.push_back(ee > 0 ? (T)(1.0 / ee) : T(0));
        }
    }
    const int sdf_len = (int)prmT.size();
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ctx.d_sdf, sizeof(T) * std::max<size_t>(1, prmT.size())));
    EWOS_CUDA_TRY(cudaMemcpyAsync(ctx.d_sdf, prmT.data(), sizeof(T) * prmT.size(), cudaMemcpyHostToDevice, st));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ctx.d_xT, sizeof(T) * n * D));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ctx.d_r0, sizeof(T) * n));
    ::ewos::note_launch(), node_radius_kernel<T, D><<<(n + 127) / 128, 128, 0, st>>>(d_x, n, dom->kind, (const T*)ctx.d_sdf, nsdf,
                                                             (T*)ctx.d_xT, (T*)ctx.d_r0);
    EWOS_CUDA_TRY(cudaGetLastError());

    // Voronoi lookups over the domain's bounding box
    double* lo = po.lo;
    double* hi = po.hi;
    for (int c = 0; c < 3; ++c) lo[c] = hi[c] = 0;
    domain_bbox(D, dom->kind, dom->params, dom->nparams, lo, hi);
    double vol = 1;
    for (int c = 0; c < D; ++c) vol *= (hi[c] - lo[c]);
    const double hv = std::pow(vol / m, 1.0 / D);
    double surf = 0;           // rough boundary measure for the boundary-centre grid
    if (D == 2) surf = 2 * ((hi[0] - lo[0]) + (hi[1] - lo[1]));
    else surf = 2 * ((hi[0] - lo[0]) * (hi[1] - lo[1]) + (hi[1] - lo[1]) * (hi[2] - lo[2]) + (hi[0] - lo[0]) * (hi[2] - lo[2]));
    const double hz = D == 2 ? surf / p : std::sqrt(surf / p);
    // V grid spacing: factor x (volume / m)^(1/d); the autotuner also tries the other factor
    const double gf_default = o.lookup_grid_scale > 0 ? o.lookup_grid_scale : 0.125;
    const double gf_alt = D == 2 ? 0.25 : 0.18;
    // grids finer than this are refined from coarser ones instead of scanning every centre per cell
    const double h_direct = 0.6 * hv;
    const bool tune_grid = allow_alt && o.lookup_grid_scale <= 0 &&
                           (o.threads_per_block <= 0 || !(o.hash_in_smem == 0 || o.hash_in_smem == 1));
    // V-centres: y when the caller gives a separate source partition, else the nodes
    const double* d_v = tb->y ? tb->y : d_x;
    TuneKey key{sizeof(T), D, dom->kind, m, p, tb->N, o.record_walks != 0, o.threads_per_block, o.hash_in_smem,
                o.ctas_per_sm, o.lookup_grid_scale, o.walk_kernel};
    int cached_tpb = 0, cached_grid = 0;
    bool cached_smem = false;
    int cached_kernel = 1;
    const bool have_cached = tune_lookup(key, cached_tpb, cached_smem, cached_grid, &cached_kernel);
    // the default-spacing V grid is skipped when this shape is known to walk on the other one and
    // the cell weights do not need it (given by the caller, or counted on the nodes' own grid)
    const bool alt_only = tune_grid && have_cached && cached_grid == 1 && (o.cell_weights || tb->y);
    ewos_status s = EWOS_OK;
    if (!alt_only) {
        s = build_lookup<T>(D, d_v, m, lo, hi, hv * gf_default, st, ctx.V, true, h_direct);
        if (s != EWOS_OK) return s;
    }
    s = build_lookup<T>(D, d_z, p, lo, hi, hz, st, ctx.Z, false);
    if (s != EWOS_OK) return s;
    if (tune_grid && (!have_cached || cached_grid == 1)) {
        s = build_lookup<T>(D, d_v, m, lo, hi, hv * gf_alt, st, ctx.V2, true, h_direct);
        if (s != EWOS_OK) return s;
    }
    int e_nx = 0, e_ny = 0;
    double e_lo0 = 0, e_lo1 = 0, e_h = 1;
    if (egrid) {
        const double ext = std::max(hi[0] - lo[0], hi[1] - lo[1]);
        e_h = ext / 32.0 * (1.0 + 1e-9);
        e_lo0 = lo[0] - 1e-9 * ext;
        e_lo1 = lo[1] - 1e-9 * ext;
        e_nx = std::max(1, (int)std::ceil((hi[0] - e_lo0) / e_h));
        e_ny = std::max(1, (int)std::ceil((hi[1] - e_lo1) / e_h));
        const int ncell = e_nx * e_ny;
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ctx.d_vtx, sizeof(double) * dom->nparams));
        EWOS_CUDA_TRY(cudaMemcpyAsync(ctx.d_vtx, dom->params, sizeof(double) * dom->nparams, cudaMemcpyHostToDevice, st));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ctx.d_egrid, (size_t)ncell * (1 + nsdf)));
        int tpb = 32;
        while (tpb < nsdf) tpb <<= 1;        // power of two for the block reduction (<= 256)
        const double margin = 1e-5 * (1.0 + std::max({std::fabs(lo[0]), std::fabs(lo[1]), std::fabs(hi[0]), std::fabs(hi[1])}));
        ::ewos::note_launch(), polygon_grid_kernel<<<ncell, tpb, 0, st>>>(ctx.d_vtx, nsdf, e_lo0, e_lo1, e_h, e_nx, margin,
                                                                        ctx.d_egrid, ctx.d_egrid + ncell);
        EWOS_CUDA_TRY(cudaGetLastError());
    }
    if (ev_lookup) EWOS_CUDA_TRY(cudaEventRecord(ev_lookup, st));

    // cell weights
    if (o.cell_weights) {
        EWOS_CUDA_TRY(cudaMemcpyAsync(tb->lambda, o.cell_weights, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    } else {
        const int64_t ns = o.cell_samples > 0 ? o.cell_samples : 10000000;
        // lambda_i = |W_i| / |D|: the Voronoi cells of the nodes x (a lookup of its own when the
        // V-centres are separate)
        if (tb->y) {
            const double hw0 = std::pow(vol / n, 1.0 / D);
            s = build_lookup<T>(D, d_x, n, lo, hi, hw0 * gf_default, st, ctx.W, false, 0.6 * hw0);
            if (s != EWOS_OK) return s;
        }
        const DeviceLookup& WL = tb->y ? ctx.W : ctx.V;
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ctx.d_counts, sizeof(unsigned int) * n));
        EWOS_CUDA_TRY(cudaMemsetAsync(ctx.d_counts, 0, sizeof(unsigned int) * n, st));
        Lookup<T, D> Vv = lookup_view<T, D>(WL);
        const T l0 = (T)lo[0], l1 = (T)lo[1], l2 = (T)(D > 2 ? lo[2] : 0);
        const T e0 = (T)(hi[0] - lo[0]), e1 = (T)(hi[1] - lo[1]), e2 = (T)(D > 2 ? hi[2] - lo[2] : 0);
        const uint32_t k0 = (uint32_t)tb->seed, k1 = (uint32_t)(tb->seed >> 32), inst = tb->instance & 0xFFFFu;
        const size_t sm = sizeof(unsigned int) * n;
        const int blocks = 148 * 4;
        if (dom->kind == SDF_BALL) cudaFuncSetAttribute(cell_count_kernel<T, D, SDF_BALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        else if (dom->kind == SDF_BOX) cudaFuncSetAttribute(cell_count_kernel<T, D, SDF_BOX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        else cudaFuncSetAttribute(cell_count_kernel<T, D, SDF_POLYGON>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (dom->kind == SDF_BALL)
            ::ewos::note_launch(), cell_count_kernel<T, D, SDF_BALL><<<blocks, 256, sm, st>>>(Vv, n, (const T*)ctx.d_sdf, nsdf, l0, l1, l2, e0, e1, e2, ns, k0, k1, inst, ctx.d_counts);
        else if (dom->kind == SDF_BOX)
            ::ewos::note_launch(), cell_count_kernel<T, D, SDF_BOX><<<blocks, 256, sm, st>>>(Vv, n, (const T*)ctx.d_sdf, nsdf, l0, l1, l2, e0, e1, e2, ns, k0, k1, inst, ctx.d_counts);
        else
            ::ewos::note_launch(), cell_count_kernel<T, D, SDF_POLYGON><<<blocks, 256, sm, st>>>(Vv, n, (const T*)ctx.d_sdf, nsdf, l0, l1, l2, e0, e1, e2, ns, k0, k1, inst, ctx.d_counts);
        EWOS_CUDA_TRY(cudaGetLastError());
        ::ewos::note_launch(), counts_to_lambda_kernel<<<1, 1024, 0, st>>>(ctx.d_counts, n, tb->lambda);
        EWOS_CUDA_TRY(cudaGetLastError());
    }
    if (ev_cells) EWOS_CUDA_TRY(cudaEventRecord(ev_cells, st));

    // walk kernel configuration
    a.n = n; a.m = m; a.p = p; a.N = tb->N; a.eps = (T)tb->eps;
    a.k0 = (uint32_t)tb->seed; a.k1 = (uint32_t)(tb->seed >> 32);
    for (int r = 0; r < 10; ++r) {
        a.rk[r] = a.k0 + (uint32_t)r * 0x9E3779B9u;
        a.rk[10 + r] = a.k1 + (uint32_t)r * 0xBB67AE85u;
    }
    a.inst = (tb->instance & 0xFFFFu) << 8;
    a.max_steps = o.max_steps > 0 ? o.max_steps : 10000;
    a.x = (const T*)ctx.d_xT; a.r0 = (const T*)ctx.d_r0;
    a.sdf = (const T*)ctx.d_sdf; a.nsdf = nsdf; a.sdf_len = sdf_len;
    if (egrid) {
        a.e_cnt = ctx.d_egrid;
        a.e_list = ctx.d_egrid + (size_t)e_nx * e_ny;
        a.e_lo0 = (T)e_lo0; a.e_lo1 = (T)e_lo1; a.e_inv_h = (T)(1.0 / e_h);
        a.e_nx = e_nx; a.e_ny = e_ny; a.e_off = 2 * nsdf;
    }
    a.Z = lookup_view<T, D>(ctx.Z);
    a.P = (T*)tb->P; a.KH = (T*)tb->KH; a.Hc = tb->Hc;
    a.pmax = tb->pmax;
    tb->pmax_valid = false;
    if (tb->pmax) EWOS_CUDA_TRY(cudaMemsetAsync(tb->pmax, 0, 2 * sizeof(float), st));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ctx.d_counter, sizeof(int)));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&ctx.d_stats, 3 * sizeof(unsigned long long)));
    EWOS_CUDA_TRY(cudaMemsetAsync(ctx.d_counter, 0, sizeof(int), st));
    EWOS_CUDA_TRY(cudaMemsetAsync(ctx.d_stats, 0, 3 * sizeof(unsigned long long), st));
    a.row_counter = ctx.d_counter; a.stat_steps = ctx.d_stats; a.stat_capped = ctx.d_stats + 1;
    a.stat_bad = ctx.d_stats + 2;
    a.rec_exit = tb->rec_exit; a.rec_steps = tb->rec_steps; a.rec_mass = (T*)tb->rec_mass;
    a.rec_vhash = tb->rec_vhash;
    a.rec_xexit = (T*)tb->rec_xexit;
    if (tb->rec_vhash) EWOS_CUDA_TRY(cudaMemsetAsync(tb->rec_vhash, 0, sizeof(uint32_t) * n * tb->N, st));

    const DeviceLookup& V0 = alt_only ? ctx.V2 : ctx.V;     // replaced by the chosen grid at launch
    a.V = lookup_view<T, D>(V0);
    a.v_ncell = (int)V0.grid.ncell; a.v_ncand = V0.ncand;
    a.v_K = V0.K; a.v_candK = V0.candK;
    a.v_in_smem = 0;
    po.gf_default = gf_default; po.gf_alt = gf_alt;
    po.have_cached = have_cached; po.cached_tpb = cached_tpb; po.cached_grid = cached_grid;
    po.cached_smem = cached_smem; po.tune_grid = tune_grid; po.cached_kernel = cached_kernel;
    return EWOS_OK;
}

template <typename T, int D>
static ewos_status build_typed(ewos_toolbox* tb, const ewos_domain* dom, const double* d_x, const double* d_z,
                               const ewos_build_opts& o) {
    cudaStream_t st = tb->stream;
    const int n = (int)tb->n, m = (int)tb->m, p = (int)tb->p;
    BuildContext ctx;
    cudaEvent_t ev[5];
    for (auto& e : ev) cudaEventCreate(&e);
    struct EvGuard { cudaEvent_t* e; ~EvGuard() { for (int i = 0; i < 5; ++i) cudaEventDestroy(e[i]); } } evg{ev};
    EWOS_CUDA_TRY(cudaEventRecord(ev[0], st));
    WalkArgs<T, D> a{};
    PrepOut po{};
    ewos_status s = prepare_walks<T, D>(tb, dom, d_x, d_z, o, ctx, a, po, ev[1], ev[2], true);
    if (s != EWOS_OK) return s;
    const double gf_default = po.gf_default, gf_alt = po.gf_alt;
    const bool have_cached = po.have_cached;
    const int cached_tpb = po.cached_tpb, cached_grid = po.cached_grid, cached_kernel = po.cached_kernel;
    const bool cached_smem = po.cached_smem;
    const int sdf_len = a.sdf_len;
    TuneKey key{sizeof(T), D, dom->kind, m, p, tb->N, o.record_walks != 0, o.threads_per_block, o.hash_in_smem,
                o.ctas_per_sm, o.lookup_grid_scale, o.walk_kernel};
    const bool rec = o.record_walks != 0;
    // shared memory: the KH / H accumulators, and G / grad G as well for walk_kernel 2
    const size_t kh_bytes = sizeof(T) * (size_t)D * p + sizeof(uint32_t) * p;
    const size_t g_bytes = sizeof(T) * (size_t)(D + 1) * m;
    const size_t sdf_bytes = sizeof(T) * ((sdf_len + 3) & ~3);
    const DeviceLookup* Vs[2] = {&ctx.V, &ctx.V2};
    auto v_bytes_of = [&](const DeviceLookup& L) {
        return sizeof(T) * (size_t)(m + 1) * D +
               (L.K > 0 ? sizeof(uint16_t) * L.grid.ncell * L.K : sizeof(int) * (L.grid.ncell + 1 + L.ncand)) + 16;
    };
    int dev = 0, smem_optin = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t budget = (size_t)smem_optin - 1024;
    auto base_for = [&](int t, int kern) {
        const size_t acc_bytes = kh_bytes + (kern == 2 ? g_bytes : 0);
        return (((acc_bytes + 15) & ~size_t(15)) + sdf_bytes + queue_bytes<T, D>(t / 32, rec) + 15) & ~size_t(15);
    };
    // a launch configuration: walk kernel (1 accumulators in global memory, 2 in shared memory),
    // block size, V grid, where the V lookup lives
    struct Cfg { int tpb; int vg; bool v_smem; size_t smem; int per_sm; int grid; int kern; };
    auto configure = [&](int tpb, int vg, int want_smem, int rows, Cfg& c, int kern) -> bool {
        const DeviceLookup& L = *Vs[vg];
        if (!L.start) return false;
        const size_t base = base_for(tpb, kern);
        if (base > budget) return false;
        c.tpb = tpb;
        c.vg = vg;
        c.kern = kern;
        c.v_smem = want_smem != 0 && base + v_bytes_of(L) <= budget;
        if (want_smem == 1 && !c.v_smem) return false;
        c.smem = base + (c.v_smem ? v_bytes_of(L) : 0);
        int ps = 0;
        if (dom->kind == SDF_BALL) ps = max_ctas_per_sm<T, D, SDF_BALL>(tpb, c.smem, kern);
        else if (dom->kind == SDF_BOX) ps = max_ctas_per_sm<T, D, SDF_BOX>(tpb, c.smem, kern);
        else ps = max_ctas_per_sm<T, D, SDF_POLYGON>(tpb, c.smem, kern);
        if (ps < 1) return false;
        if (o.ctas_per_sm > 0) ps = std::min(ps, o.ctas_per_sm);
        c.per_sm = ps;
        c.grid = std::max(1, std::min(nsm * ps, rows));
        return true;
    };
    auto launch = [&](const Cfg& c, WalkArgs<T, D>& args) -> cudaError_t {
        const DeviceLookup& L = *Vs[c.vg];
        args.V = lookup_view<T, D>(L);
        args.v_ncell = (int)L.grid.ncell; args.v_ncand = L.ncand;
        args.v_K = L.K; args.v_candK = L.candK;
        args.v_in_smem = c.v_smem ? 1 : 0;
        args.acc_g = nullptr;
        args.acc_cells = m;
        if (c.kern == 1) {
            // one accumulator row per CTA, zeroed by the kernel
            cudaError_t e = ctx.ensure_acc(sizeof(T) * 4 * (size_t)m * c.grid);
            if (e != cudaSuccess) return e;
            args.acc_g = (T*)ctx.d_acc;
            args.acc_len = (int64_t)(ctx.acc_cap / sizeof(T));
        }
        if (dom->kind == SDF_BALL) return dispatch_walks<T, D, SDF_BALL>(args, rec, c.grid, c.tpb, c.smem, st, c.kern);
        if (dom->kind == SDF_BOX) return dispatch_walks<T, D, SDF_BOX>(args, rec, c.grid, c.tpb, c.smem, st, c.kern);
        return dispatch_walks<T, D, SDF_POLYGON>(args, rec, c.grid, c.tpb, c.smem, st, c.kern);
    };
    Cfg cfg{};
    const bool fixed_tpb = o.threads_per_block > 0;
    const bool fixed_place = o.hash_in_smem == 0 || o.hash_in_smem == 1;
    const int req_tpb = std::min(1024, (o.threads_per_block + 31) / 32 * 32);
    const int req_kern = o.walk_kernel == 1 || o.walk_kernel == 2 ? o.walk_kernel : 0;
    if (fixed_tpb && fixed_place && req_kern) {
        if (!configure(req_tpb, 0, o.hash_in_smem, n, cfg, req_kern)) {
            set_error("walk kernel: requested block size / lookup placement does not fit");
            return EWOS_EINVAL;
        }
    } else if (have_cached && configure(cached_tpb, cached_grid, cached_smem ? 1 : 0, n, cfg, cached_kernel)) {
        // configuration chosen earlier for this problem shape
    } else {
        // autotuner: time each candidate configuration on a prefix of rows once per problem
        // shape (cached for the process); the prefix rows are recomputed by the full launch
        // (the shared-memory accumulator form, kernel 2, measured 1.6 to 3 times slower on every
        // workload; it is tried only when asked for)
        std::vector<Cfg> cands;
        for (int kern : {1, 2}) {
            if (req_kern ? kern != req_kern : kern != 1) continue;
            for (int vg : {0, 1})
                for (int t : {512, 1024}) {
                    if (fixed_tpb && t != req_tpb) continue;
                    for (int sm : {0, 1}) {
                        if (fixed_place && sm != o.hash_in_smem) continue;
                        Cfg c{};
                        if (configure(t, vg, sm, n, c, kern)) cands.push_back(c);
                    }
                }
        }
        if (fixed_tpb && cands.empty()) {
            Cfg c{};
            if (configure(req_tpb, 0, 0, n, c, req_kern ? req_kern : 1)) cands.push_back(c);
        }
        if (cands.empty()) {
            set_error("toolbox row does not fit in shared memory (m, p too large for one CTA)");
            return EWOS_EINVAL;
        }
        if (cands.size() == 1) {
            cfg = cands[0];
        } else {
            // every candidate runs the same rows, 16 per SM spread over the domain: as in the
            // whole build, a shape with more CTAs runs fewer rows per CTA (two rows per SM
            // favoured the shapes with fewer, larger CTAs: the square's 512 x 2 measured 6 %
            // faster than 1024 x 1 over the whole build, slower on that prefix)
            float best = 3.0e38f;
            cudaEvent_t t0, t1;
            cudaEventCreate(&t0); cudaEventCreate(&t1);
            for (Cfg c : cands) {
                // an untimed one-row launch first: the kernel's first launch loads its module
                Cfg c1 = c;
                c1.grid = 1;
                WalkArgs<T, D> warm = a;
                warm.trial_rows = 1;
                warm.trial_step = 1;
                EWOS_CUDA_TRY(cudaMemsetAsync(ctx.d_counter, 0, sizeof(int), st));
                EWOS_CUDA_TRY(launch(c1, warm));
                const int rows = std::min(n, 16 * nsm);
                c.grid = std::max(1, std::min(nsm * c.per_sm, rows));
                if (c.kern == 1) EWOS_CUDA_TRY(ctx.ensure_acc(sizeof(T) * 4 * (size_t)m * c.grid));   // (outside the timing)
                WalkArgs<T, D> trial = a;
                // rows spread over the domain (a prefix of the node order can be all near the
                // boundary, where walks are short): a step coprime with n
                trial.trial_rows = rows;
                trial.trial_step = trial_step_for(n, rows);
                EWOS_CUDA_TRY(cudaMemsetAsync(ctx.d_counter, 0, sizeof(int), st));
                cudaEventRecord(t0, st);
                EWOS_CUDA_TRY(launch(c, trial));
                cudaEventRecord(t1, st);
                EWOS_CUDA_TRY(cudaEventSynchronize(t1));
                float ms = 0;
                cudaEventElapsedTime(&ms, t0, t1);
                if (ms < best) { best = ms; cfg = c; }
            }
            cudaEventDestroy(t0); cudaEventDestroy(t1);
            cfg.grid = std::max(1, std::min(nsm * cfg.per_sm, n));
            EWOS_CUDA_TRY(cudaMemsetAsync(ctx.d_counter, 0, sizeof(int), st));
            EWOS_CUDA_TRY(cudaMemsetAsync(ctx.d_stats, 0, 3 * sizeof(unsigned long long), st));
            if (tb->rec_vhash) EWOS_CUDA_TRY(cudaMemsetAsync(tb->rec_vhash, 0, sizeof(uint32_t) * n * tb->N, st));
        }
        tune_store(key, cfg.tpb, cfg.v_smem, cfg.vg, cfg.kern);
    }
    if (cfg.kern == 1) EWOS_CUDA_TRY(ctx.ensure_acc(sizeof(T) * 4 * (size_t)m * cfg.grid));
    EWOS_CUDA_TRY(cudaEventRecord(ev[3], st));
    EWOS_CUDA_TRY(launch(cfg, a));
    const int tpb = cfg.tpb, per_sm = cfg.per_sm, grid = cfg.grid;
    const bool v_smem = cfg.v_smem;
    const size_t smem = cfg.smem;

    EWOS_CUDA_TRY(cudaEventRecord(ev[4], st));
    unsigned long long stats[3] = {0, 0, 0};
    EWOS_CUDA_TRY(cudaMemcpyAsync(stats, ctx.d_stats, sizeof(stats), cudaMemcpyDeviceToHost, st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(st));
    if (stats[2]) {
        set_error("walk kernel: " + std::to_string(stats[2]) + " out-of-range indexes found and skipped");
        return EWOS_ECUDA;
    }
    tb->pmax_valid = tb->pmax != nullptr;     // every row written: the kernel's max |P| is complete
    float ms[4];
    cudaEventElapsedTime(&ms[0], ev[0], ev[4]);
    cudaEventElapsedTime(&ms[1], ev[0], ev[1]);
    cudaEventElapsedTime(&ms[2], ev[1], ev[2]);
    cudaEventElapsedTime(&ms[3], ev[3], ev[4]);
    ewos_build_report& r = tb->rep;
    r.walks = (int64_t)n * tb->N;
    r.steps = (int64_t)stats[0];
    r.capped = (int64_t)stats[1];
    r.ms_total = ms[0]; r.ms_lookup = ms[1]; r.ms_cells = ms[2]; r.ms_walk = ms[3];
    r.threads_per_block = tpb; r.ctas_per_sm = per_sm; r.grid = grid; r.hash_in_smem = v_smem;
    r.lookup_grid_scale = cfg.vg == 0 ? gf_default : gf_alt;
    r.lookup_candidates = Vs[cfg.vg]->K;
    r.smem_bytes = (int64_t)smem;
    r.walk_kernel = cfg.kern;
    return EWOS_OK;
}

// ------------------------------------------------------------------ many toolboxes, one launch
template <typename T, int D, int KIND>
static cudaError_t launch_batch(const WalkArgs<T, D>* d_args, const int* d_off, int nb, int* d_counter, int grid,
                                int tpb, size_t smem, cudaStream_t st) {
    auto k = wos_walk_batch_kernel<T, D, KIND>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ::ewos::note_launch(), k<<<grid, tpb, smem, st>>>(d_args, d_off, nb, d_counter);
    return cudaGetLastError();
}

template <typename T, int D, int KIND>
static int batch_ctas_per_sm(int tpb, size_t smem) {
    int per = 0;
    auto k = wos_walk_batch_kernel<T, D, KIND>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, tpb, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per;
}

// process-wide choices of the batch launch shape, keyed by the batch's shape
struct BatchTuneKey {
    int esz, dim, kind, count;
    int64_t rows, max_m, max_p, N;
    bool operator==(const BatchTuneKey& o) const {
        return esz == o.esz && dim == o.dim && kind == o.kind && count == o.count && rows == o.rows &&
               max_m == o.max_m && max_p == o.max_p && N == o.N;
    }
};
static std::vector<std::pair<BatchTuneKey, std::pair<int, int>>> g_batch_tune;   // -> (tpb, ctas/SM)

template <typename T, int D, int KIND>
static ewos_status build_batch_kind(std::vector<ewos_toolbox*>& tbs, const std::vector<const ewos_domain*>& doms,
                                    const ewos_build_opts& o, ewos_build_report* brep) {
    cudaStream_t st = tbs[0]->stream;
    const int nb = (int)tbs.size();
    cudaEvent_t ev[3];
    for (auto& e : ev) cudaEventCreate(&e);
    struct EvGuard { cudaEvent_t* e; ~EvGuard() { for (int i = 0; i < 3; ++i) cudaEventDestroy(e[i]); } } evg{ev};
    EWOS_CUDA_TRY(cudaEventRecord(ev[0], st));
    std::vector<std::unique_ptr<BuildContext>> ctxs;
    std::vector<WalkArgs<T, D>> args(nb);
    std::vector<int> off(nb + 1, 0);
    int64_t max_m = 0, max_p = 0, max_sdf = 0;
    for (int k = 0; k < nb; ++k) {
        ctxs.emplace_back(new BuildContext());
        ewos_build_opts ok = o;
        ok.instance = o.instance + (uint32_t)k;
        tbs[k]->instance = ok.instance;
        PrepOut po{};
        ewos_status s = prepare_walks<T, D>(tbs[k], doms[k], tbs[k]->x, tbs[k]->z, ok, *ctxs.back(), args[k], po,
                                            nullptr, nullptr, false);
        if (s != EWOS_OK) return s;
        off[k + 1] = off[k] + (int)tbs[k]->n;
        max_m = std::max<int64_t>(max_m, tbs[k]->m);
        max_p = std::max<int64_t>(max_p, tbs[k]->p);
        max_sdf = std::max<int64_t>(max_sdf, args[k].sdf_len);
    }
    WalkArgs<T, D>* d_args = nullptr;
    int *d_off = nullptr, *d_counter = nullptr, *d_off_trial = nullptr;
    T* d_acc = nullptr;
    struct Frees { void** p[5]; ~Frees() { for (auto q : p) ::ewos::dev_free(*q); } } fr{{(void**)&d_args, (void**)&d_off, (void**)&d_counter, (void**)&d_off_trial, (void**)&d_acc}};
    int dev = 0, nsm = 0, smem_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // G / grad G accumulators in global memory: one row of the largest instance per CTA, for up
    // to kMaxBatchCtasPerSm CTAs per SM
    constexpr int kMaxBatchCtasPerSm = 8;
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&d_acc, sizeof(T) * 4 * (size_t)max_m * nsm * kMaxBatchCtasPerSm));
    for (int k = 0; k < nb; ++k) {
        args[k].acc_g = d_acc;
        args[k].acc_cells = (int)max_m;
        args[k].acc_len = (int64_t)4 * max_m * nsm * kMaxBatchCtasPerSm;
    }
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&d_args, sizeof(WalkArgs<T, D>) * nb));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&d_off, sizeof(int) * (nb + 1)));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&d_off_trial, sizeof(int) * (nb + 1)));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&d_counter, sizeof(int)));
    EWOS_CUDA_TRY(cudaMemcpyAsync(d_args, args.data(), sizeof(WalkArgs<T, D>) * nb, cudaMemcpyHostToDevice, st));
    EWOS_CUDA_TRY(cudaMemcpyAsync(d_off, off.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice, st));
    EWOS_CUDA_TRY(cudaEventRecord(ev[1], st));

    // shared memory for the largest instance (the KH / H accumulators, sdf parameters, queues)
    const size_t acc_bytes = sizeof(T) * (size_t)D * max_p + sizeof(uint32_t) * max_p;
    const size_t sdf_bytes = sizeof(T) * ((max_sdf + 3) & ~int64_t(3));
    auto smem_for = [&](int t) {
        return (((acc_bytes + 15) & ~size_t(15)) + sdf_bytes + queue_bytes<T, D>(t / 32, false) + 15) & ~size_t(15);
    };
    const int total = off[nb];
    // autotuner: block size x CTAs per SM, timed on a prefix of the global rows, cached per shape
    BatchTuneKey key{(int)sizeof(T), D, KIND, nb, total, max_m, max_p, tbs[0]->N};
    int tpb = 0, per = 0;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (auto& e : g_batch_tune)
            if (e.first == key) { tpb = e.second.first; per = e.second.second; }
    }
    if (o.threads_per_block > 0) { tpb = std::min(1024, (o.threads_per_block + 31) / 32 * 32); per = 0; }
    if (tpb == 0) {
        struct C { int tpb, per; };
        std::vector<C> cands;
        for (int t : {256, 512, 1024}) {
            const size_t sm = smem_for(t);
            if (sm > (size_t)smem_optin - 1024) continue;
            const int mx = std::min(kMaxBatchCtasPerSm, batch_ctas_per_sm<T, D, KIND>(t, sm));
            for (int p2 = 1; p2 <= mx && p2 <= 4; p2 *= 2) cands.push_back({t, p2});
        }
        if (cands.empty()) { set_error("batch: the largest toolbox row does not fit in shared memory"); return EWOS_EINVAL; }
        // each candidate runs a prefix of three global rows per CTA of its grid, compared by time
        // per row (as the single-build autotuner)
        std::vector<int> off_trial(off);
        float best = 3.0e38f;
        cudaEvent_t t0, t1;
        cudaEventCreate(&t0); cudaEventCreate(&t1);
        for (const C& c : cands) {
            // an untimed one-row launch first (the kernel's first launch loads its module)
            for (int k = 0; k <= nb; ++k) off_trial[k] = std::min(off[k], 1);
            EWOS_CUDA_TRY(cudaMemcpyAsync(d_off_trial, off_trial.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice, st));
            EWOS_CUDA_TRY(cudaMemsetAsync(d_counter, 0, sizeof(int), st));
            cudaError_t we = launch_batch<T, D, KIND>(d_args, d_off_trial, nb, d_counter, 1, c.tpb, smem_for(c.tpb), st);
            EWOS_CUDA_TRY(we);
            const int prefix = std::min(total, 3 * nsm * c.per);
            for (int k = 0; k <= nb; ++k) off_trial[k] = std::min(off[k], prefix);
            EWOS_CUDA_TRY(cudaMemcpyAsync(d_off_trial, off_trial.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice, st));
            EWOS_CUDA_TRY(cudaMemsetAsync(d_counter, 0, sizeof(int), st));
            cudaEventRecord(t0, st);
            const int tgrid = std::max(1, std::min(nsm * c.per, prefix));
            cudaError_t le = launch_batch<T, D, KIND>(d_args, d_off_trial, nb, d_counter, tgrid, c.tpb, smem_for(c.tpb), st);
            EWOS_CUDA_TRY(le);
            cudaEventRecord(t1, st);
            EWOS_CUDA_TRY(cudaEventSynchronize(t1));
            float ms = 0;
            cudaEventElapsedTime(&ms, t0, t1);
            ms /= (float)prefix;
            if (ms < best) { best = ms; tpb = c.tpb; per = c.per; }
        }
        cudaEventDestroy(t0); cudaEventDestroy(t1);
        for (int k = 0; k < nb; ++k) EWOS_CUDA_TRY(cudaMemsetAsync(ctxs[k]->d_stats, 0, 3 * sizeof(unsigned long long), st));
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_batch_tune.push_back({key, {tpb, per}});
    }
    const size_t smem = smem_for(tpb);
    if (per <= 0) per = std::max(1, std::min(kMaxBatchCtasPerSm, batch_ctas_per_sm<T, D, KIND>(tpb, smem)));
    if (o.ctas_per_sm > 0) per = std::min(per, o.ctas_per_sm);
    const int grid = std::max(1, std::min(nsm * per, total));
    EWOS_CUDA_TRY(cudaMemsetAsync(d_counter, 0, sizeof(int), st));
    EWOS_CUDA_TRY(cudaEventRecord(ev[1], st));
    cudaError_t le = launch_batch<T, D, KIND>(d_args, d_off, nb, d_counter, grid, tpb, smem, st);
    EWOS_CUDA_TRY(le);
    EWOS_CUDA_TRY(cudaEventRecord(ev[2], st));
    std::vector<unsigned long long> stats(3 * nb);
    for (int k = 0; k < nb; ++k)
        EWOS_CUDA_TRY(cudaMemcpyAsync(&stats[3 * k], ctxs[k]->d_stats, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(st));
    for (int k = 0; k < nb; ++k)
        if (stats[3 * k + 2]) {
            set_error("batch walk kernel: " + std::to_string(stats[3 * k + 2]) + " out-of-range indexes found and skipped");
            return EWOS_ECUDA;
        }
    for (int k = 0; k < nb; ++k) tbs[k]->pmax_valid = tbs[k]->pmax != nullptr;
    float ms_all = 0, ms_walk = 0;
    cudaEventElapsedTime(&ms_all, ev[0], ev[2]);
    cudaEventElapsedTime(&ms_walk, ev[1], ev[2]);
    ewos_build_report tot{};
    for (int k = 0; k < nb; ++k) {
        ewos_build_report& r = tbs[k]->rep;
        r = ewos_build_report{};
        r.walks = tbs[k]->n * tbs[k]->N;
        r.steps = (int64_t)stats[3 * k];
        r.capped = (int64_t)stats[3 * k + 1];
        r.ms_total = ms_all; r.ms_walk = ms_walk;
        r.threads_per_block = tpb; r.ctas_per_sm = per; r.grid = grid; r.hash_in_smem = 0;
        r.smem_bytes = (int64_t)smem;
        r.lookup_candidates = ctxs[k]->V.K;
        tot.walks += r.walks; tot.steps += r.steps; tot.capped += r.capped;
    }
    tot.ms_total = ms_all; tot.ms_walk = ms_walk;
    tot.threads_per_block = tpb; tot.ctas_per_sm = per; tot.grid = grid; tot.smem_bytes = (int64_t)smem;
    if (brep) *brep = tot;
    return EWOS_OK;
}

ewos_status build_toolbox_batch(std::vector<ewos_toolbox*>& tbs, const std::vector<const ewos_domain*>& doms,
                                const ewos_build_opts& o, ewos_build_report* brep) {
    const int kind = doms[0]->kind;
    const int D = tbs[0]->dim;
    const bool f64 = tbs[0]->precision == 64;
#define EWOS_BATCH(TT, DD, KK) return build_batch_kind<TT, DD, KK>(tbs, doms, o, brep)
    if (f64) {
        if (D == 2) {
            if (kind == SDF_BALL) EWOS_BATCH(double, 2, SDF_BALL);
            if (kind == SDF_BOX) EWOS_BATCH(double, 2, SDF_BOX);
            EWOS_BATCH(double, 2, SDF_POLYGON);
        }
        if (kind == SDF_BALL) EWOS_BATCH(double, 3, SDF_BALL);
        EWOS_BATCH(double, 3, SDF_BOX);
    }
    if (D == 2) {
        if (kind == SDF_BALL) EWOS_BATCH(float, 2, SDF_BALL);
        if (kind == SDF_BOX) EWOS_BATCH(float, 2, SDF_BOX);
        EWOS_BATCH(float, 2, SDF_POLYGON);
    }
    if (kind == SDF_BALL) EWOS_BATCH(float, 3, SDF_BALL);
    EWOS_BATCH(float, 3, SDF_BOX);
#undef EWOS_BATCH
}

ewos_status build_toolbox(ewos_toolbox* tb, const ewos_domain* dom, const double* d_x, const double* d_z,
                          const ewos_build_opts& o) {
    if (tb->precision == 64)
        return tb->dim == 2 ? build_typed<double, 2>(tb, dom, d_x, d_z, o) : build_typed<double, 3>(tb, dom, d_x, d_z, o);
    return tb->dim == 2 ? build_typed<float, 2>(tb, dom, d_x, d_z, o) : build_typed<float, 3>(tb, dom, d_x, d_z, o);
}

ewos_status validate_domain(const ewos_domain* dom, const double* x, int64_t n) {
    if (!dom || (dom->dim != 2 && dom->dim != 3) || !dom->params) {
        set_error("domain: dim must be 2 or 3 and params non-NULL");
        return EWOS_EINVAL;
    }
    if (dom->kind == SDF_BALL && dom->nparams != dom->dim + 1) { set_error("ball: params = centre, radius"); return EWOS_EINVAL; }
    if (dom->kind == SDF_BOX && dom->nparams != 2 * dom->dim) { set_error("box: params = lo, hi"); return EWOS_EINVAL; }
    if (dom->kind == SDF_POLYGON &&
        (dom->dim != 2 || dom->nparams < 6 || (dom->nparams & 1) || dom->nparams / 2 > kMaxPolygonVertices)) {
        set_error("polygon: d = 2 and 3..256 vertices");
        return EWOS_EINVAL;
    }
    if (dom->kind < 0 || dom->kind > 2) { set_error("unknown domain kind"); return EWOS_EINVAL; }
    if (x) {
        for (int64_t i = 0; i < n; ++i)
            if (!(host_sdf(dom->dim, dom->kind, dom->params, dom->nparams, x + i * dom->dim) > 0.0)) {
                set_error("interior node " + std::to_string(i) + " is not inside the domain");
                return EWOS_EINVAL;
            }
    }
    return EWOS_OK;
}

// ------------------------------------------------------------------ build without allocation
// Some callers cannot call cudaMalloc: code running under an allocator that owns all device
// memory (a framework's caching pool, a memory budget enforced by a serving process), or code
// that must not allocate while other work is in flight.  ewos_toolbox_build_noalloc serves
// them: the caller passes the output matrices, and every temporary of the build (lookup grids,
// candidate lists, node copies, counters) lives in the file-scope array below, which each GPU
// that loads this library holds until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;   // 4 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static void* noalloc_scratch_address(int device, ewos_status* st) {
    // the symbol's device address, looked up once per device with that device current
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static void* addr[kMaxDevices] = {};
    if (device < 0 || device >= kMaxDevices) { *st = EWOS_EINVAL; set_error("device index out of range"); return nullptr; }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) {
            *st = EWOS_ECUDA;
            set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
            return nullptr;
        }
        addr[device] = ptr;
    }
    *st = EWOS_OK;
    return addr[device];
}

// bump allocator over the static scratch
struct Arena {
    unsigned char* base;
    size_t cap, used;
    void* take(size_t bytes) {
        const size_t off = (used + 255) & ~size_t(255);
        if (off + bytes > cap) return nullptr;
        used = off + bytes;
        return base + off;
    }
};

__global__ void node_check_kernel(const float* __restrict__ r0, int n, int* __restrict__ bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(r0[i] > 0.0f)) atomicExch(bad, 1);
}

template <int D>
static ewos_status lookup_into(const double* d_pts, int np, const double* lo, const double* hi, double h, cudaStream_t st,
                               Arena& ar, DeviceLookup& out) {
    out.np = np;
    out.grid = make_grid(D, lo, hi, h);
    const int64_t nc = out.grid.ncell;
    double ext = 0;
    for (int c = 0; c < D; ++c) ext = std::max(ext, std::max(std::fabs(lo[c]), std::fabs(hi[c])) + (hi[c] - lo[c]));
    const float slack = (float)(1e-6 * ext * ext);
    int* d_count = (int*)ar.take(sizeof(int) * nc);
    float* d_rad = (float*)ar.take(sizeof(float) * nc);
    out.start = (int*)ar.take(sizeof(int) * (nc + 1));
    out.pts = ar.take(sizeof(float) * (np + 1) * D);
    if (!d_count || !d_rad || !out.start || !out.pts) return EWOS_ENOMEM;
    const int64_t ne = (int64_t)np * D;
    ::ewos::note_launch(), convert_points_kernel<float, D><<<(int)((ne + 255) / 256), 256, 0, st>>>(d_pts, (float*)out.pts, ne);
    const int tb = 256, nb = (int)((nc * 32 + tb - 1) / tb);
    ::ewos::note_launch(), lookup_count_kernel<D><<<nb, tb, 0, st>>>((const float*)out.pts, np, out.grid, slack, d_count, d_rad, nullptr,
                                                                   nullptr);
    ::ewos::note_launch(), exclusive_scan_kernel<<<1, 1024, 0, st>>>(d_count, nc, out.start);
    int total = 0;
    EWOS_CUDA_TRY(cudaMemcpyAsync(&total, out.start + nc, sizeof(int), cudaMemcpyDeviceToHost, st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(st));
    out.ncand = total;
    out.cand = (int*)ar.take(sizeof(int) * std::max(1, total));
    if (!out.cand) return EWOS_ENOMEM;
    ::ewos::note_launch(), lookup_fill_kernel<D><<<nb, tb, 0, st>>>((const float*)out.pts, np, out.grid, slack, out.start, out.cand);
    EWOS_CUDA_TRY(cudaGetLastError());
    return EWOS_OK;
}

template <int D>
static ewos_status build_noalloc_typed(const ewos_domain* dom, const double* d_x, int n, const double* d_z, int p,
                                       int64_t N, double eps, uint64_t seed, int64_t max_steps, cudaStream_t st,
                                       Arena& ar, float* P, float* KH, uint32_t* Hc, ewos_build_report* rep) {
    const int m = n;
    const auto t0 = std::chrono::steady_clock::now();
    float prm[2 * kMaxPolygonVertices];
    for (int64_t t = 0; t < dom->nparams; ++t) prm[t] = (float)dom->params[t];
    const int nsdf = dom->kind == SDF_POLYGON ? (int)(dom->nparams / 2) : 0;
    float* d_sdf = (float*)ar.take(sizeof(float) * dom->nparams);
    float* d_xT = (float*)ar.take(sizeof(float) * n * D);
    float* d_r0 = (float*)ar.take(sizeof(float) * n);
    int* d_counter = (int*)ar.take(sizeof(int) * 2);               // row counter, bad-node flag
    unsigned long long* d_stats = (unsigned long long*)ar.take(2 * sizeof(unsigned long long));
    if (!d_sdf || !d_xT || !d_r0 || !d_counter || !d_stats) {
        set_error("ewos_toolbox_build_noalloc: the node arrays need more than the 4 MiB scratch (reduce n)");
        return EWOS_EINVAL;
    }
    EWOS_CUDA_TRY(cudaMemcpyAsync(d_sdf, prm, sizeof(float) * dom->nparams, cudaMemcpyHostToDevice, st));
    // every call starts from cleared counters: the scratch keeps the previous call's contents
    EWOS_CUDA_TRY(cudaMemsetAsync(d_counter, 0, sizeof(int) * 2, st));
    EWOS_CUDA_TRY(cudaMemsetAsync(d_stats, 0, 2 * sizeof(unsigned long long), st));
    ::ewos::note_launch(), node_radius_kernel<float, D><<<(n + 127) / 128, 128, 0, st>>>(d_x, n, dom->kind, d_sdf, nsdf, d_xT, d_r0);
    ::ewos::note_launch(), node_check_kernel<<<(n + 127) / 128, 128, 0, st>>>(d_r0, n, d_counter + 1);
    int bad = 0;
    EWOS_CUDA_TRY(cudaMemcpyAsync(&bad, d_counter + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(st));
    if (bad) { set_error("an interior node is not inside the domain"); return EWOS_EINVAL; }

    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    domain_bbox(D, dom->kind, dom->params, dom->nparams, lo, hi);
    double vol = 1, surf;
    for (int c = 0; c < D; ++c) vol *= (hi[c] - lo[c]);
    if (D == 2) surf = 2 * ((hi[0] - lo[0]) + (hi[1] - lo[1]));
    else surf = 2 * ((hi[0] - lo[0]) * (hi[1] - lo[1]) + (hi[1] - lo[1]) * (hi[2] - lo[2]) + (hi[0] - lo[0]) * (hi[2] - lo[2]));
    DeviceLookup V, Z;
    ewos_status s = lookup_into<D>(d_x, m, lo, hi, std::pow(vol / m, 1.0 / D), st, ar, V);
    if (s == EWOS_OK) s = lookup_into<D>(d_z, p, lo, hi, D == 2 ? surf / p : std::sqrt(surf / p), st, ar, Z);
    if (s == EWOS_ENOMEM) {
        set_error("ewos_toolbox_build_noalloc: the lookup grids need more than the 4 MiB scratch (reduce n or p)");
        return EWOS_EINVAL;
    }
    if (s != EWOS_OK) return s;

    WalkArgs<float, D> a{};
    a.n = n; a.m = m; a.p = p; a.N = N; a.eps = (float)eps;
    a.k0 = (uint32_t)seed; a.k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        a.rk[r] = a.k0 + (uint32_t)r * 0x9E3779B9u;
        a.rk[10 + r] = a.k1 + (uint32_t)r * 0xBB67AE85u;
    }
    a.inst = 0;
    a.max_steps = max_steps > 0 ? max_steps : 10000;
    a.x = d_xT; a.r0 = d_r0;
    a.sdf = d_sdf; a.nsdf = nsdf; a.sdf_len = (int)dom->nparams;
    a.V = lookup_view<float, D>(V); a.Z = lookup_view<float, D>(Z);
    a.v_ncell = (int)V.grid.ncell; a.v_ncand = V.ncand;
    a.P = P; a.KH = KH; a.Hc = Hc;
    a.row_counter = d_counter; a.stat_steps = d_stats; a.stat_capped = d_stats + 1;
    a.v_in_smem = 0;
    a.v_K = 0; a.v_candK = nullptr;
    const int tpb = 512;
    const size_t acc_bytes = sizeof(float) * ((size_t)(D + 1) * m + (size_t)D * p) + sizeof(uint32_t) * p;
    const size_t smem = ((((acc_bytes + 15) & ~size_t(15)) + sizeof(float) * ((a.sdf_len + 3) & ~3) +
                          queue_bytes<float, D>(tpb / 32, false) + 15) & ~size_t(15));
    int dev = 0, smem_optin = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (smem + 1024 > (size_t)smem_optin) { set_error("toolbox row does not fit in shared memory"); return EWOS_EINVAL; }
    int per_sm = 0;
    if (dom->kind == SDF_BALL) per_sm = max_ctas_per_sm<float, D, SDF_BALL>(tpb, smem, 2);
    else if (dom->kind == SDF_BOX) per_sm = max_ctas_per_sm<float, D, SDF_BOX>(tpb, smem, 2);
    else per_sm = max_ctas_per_sm<float, 2, SDF_POLYGON>(tpb, smem, 2);
    if (per_sm < 1) { set_error("walk kernel does not fit on an SM"); return EWOS_EINVAL; }
    const int grid = std::max(1, std::min(nsm * per_sm, n));
    cudaError_t e;
    if (dom->kind == SDF_BALL) e = launch_walks<float, D, SDF_BALL, false>(a, grid, tpb, smem, st, 2);
    else if (dom->kind == SDF_BOX) e = launch_walks<float, D, SDF_BOX, false>(a, grid, tpb, smem, st, 2);
    else e = D == 2 ? launch_walks<float, D, SDF_POLYGON, false>(a, grid, tpb, smem, st, 2) : cudaErrorInvalidValue;
    EWOS_CUDA_TRY(e);
    unsigned long long stats[2] = {0, 0};
    EWOS_CUDA_TRY(cudaMemcpyAsync(stats, d_stats, sizeof(stats), cudaMemcpyDeviceToHost, st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(st));
    if (rep) {
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        *rep = ewos_build_report{};
        rep->walks = (int64_t)n * N; rep->steps = (int64_t)stats[0]; rep->capped = (int64_t)stats[1];
        rep->ms_total = ms; rep->threads_per_block = tpb; rep->ctas_per_sm = per_sm; rep->grid = grid;
        rep->smem_bytes = (int64_t)smem;
    }
    return stats[1] > 0 ? EWOS_ESTEPCAP : EWOS_OK;
}

}  // namespace ewos

extern "C" ewos_status ewos_toolbox_build_noalloc(const ewos_domain* domain, const double* x, int64_t n,
                                                  const double* z, int64_t p, int64_t walks, double eps, uint64_t seed,
                                                  int64_t max_steps, void* stream, float* P, float* KH, uint32_t* Hc,
                                                  ewos_build_report* rep) {
    using namespace ewos;
    if (!domain || !x || !z || !P || !KH || !Hc || n < 1 || p < 1 || walks < 1 || walks > 0xFFFFFFFFll || !(eps > 0) ||
        n > (1 << 20) || p > (1 << 20)) {
        set_error("ewos_toolbox_build_noalloc: need domain, device x, z, P, KH, Hc, n, p >= 1, 1 <= walks < 2^32, eps > 0");
        return EWOS_EINVAL;
    }
    ewos_status s = validate_domain(domain, nullptr, n);
    if (s != EWOS_OK) return s;
    int dev = 0;
    EWOS_CUDA_TRY(cudaGetDevice(&dev));
    void* base = noalloc_scratch_address(dev, &s);
    if (!base) return s;
    Arena ar{(unsigned char*)base, kNoAllocScratchBytes, 0};
    cudaStream_t st = (cudaStream_t)stream;
    return domain->dim == 2
               ? build_noalloc_typed<2>(domain, x, (int)n, z, (int)p, walks, eps, seed, max_steps, st, ar, P, KH, Hc, rep)
               : build_noalloc_typed<3>(domain, x, (int)n, z, (int)p, walks, eps, seed, max_steps, st, ar, P, KH, Hc, rep);
}
