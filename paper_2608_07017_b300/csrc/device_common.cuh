// device_common.cuh -- device building blocks of the walk kernel: counter-based random
// numbers, the samplers of Prop. 2.6, distances to the boundary (eq. r) and the
// nearest-centre lookup of the Voronoi binning (Sec. 2.3).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ewos {

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
// ten rounds of two 32x32->64 multiplies; the key advances by the Weyl constants between
// rounds.  ctr = (walk, step, node, tag<<24 | instance<<8 | slot), key = (seed_lo, seed_hi).
struct u32x4 { uint32_t a, b, c, d; };

__host__ __device__ __forceinline__ u32x4 philox4x32_10(u32x4 x, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        const uint32_t lo0 = 0xD2511F53u * x.a, hi0 = __umulhi(0xD2511F53u, x.a);
        const uint32_t lo1 = 0xCD9E8D57u * x.c, hi1 = __umulhi(0xCD9E8D57u, x.c);
#else
        const uint64_t p0 = (uint64_t)0xD2511F53u * x.a, p1 = (uint64_t)0xCD9E8D57u * x.c;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
#endif
        x = u32x4{hi1 ^ x.b ^ k0, lo1, hi0 ^ x.d ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return x;
}

// The same rounds with the key schedule precomputed: rk[r] = k0 + r 0x9E3779B9, rk[10 + r] =
// k1 + r 0xBB67AE85 (r < 10).  Read from the kernel's parameter space the keys are operands of the
// XORs themselves, which saves the schedule's two additions per round.
__device__ __forceinline__ u32x4 philox4x32_10_rk(u32x4 x, const uint32_t* rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * x.a, hi0 = __umulhi(0xD2511F53u, x.a);
        const uint32_t lo1 = 0xCD9E8D57u * x.c, hi1 = __umulhi(0xCD9E8D57u, x.c);
        x = u32x4{hi1 ^ x.b ^ rk[r], lo1, hi0 ^ x.d ^ rk[10 + r], lo0};
    }
    return x;
}

// uniform in (0,1): ((x >> 9) + 1/2) / 2^23 -- exact in FP32 and FP64 alike
template <typename T> __device__ __forceinline__ T u01(uint32_t x) {
    return (T)((float)(x >> 9) * 1.1920928955078125e-07f + 5.9604644775390625e-08f);
}

// ------------------------------------------------------------------ math wrappers
__device__ __forceinline__ float  m_sqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double m_sqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float  m_log(float v) { return logf(v); }
__device__ __forceinline__ double m_log(double v) { return log(v); }
__device__ __forceinline__ float  m_log1p(float v) { return log1pf(v); }
__device__ __forceinline__ double m_log1p(double v) { return log1p(v); }
__device__ __forceinline__ float  m_exp(float v) { return expf(v); }
__device__ __forceinline__ double m_exp(double v) { return exp(v); }
__device__ __forceinline__ float  m_newton_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double m_newton_div(double a, double b) { return a / b; }
__device__ __forceinline__ void m_sincos2pi(float u, float* s, float* c) { sincospif(2.0f * u, s, c); }
__device__ __forceinline__ void m_sincos2pi(double u, double* s, double* c) { sincospi(2.0 * u, s, c); }

// ------------------------------------------------------------------ samplers (Prop. 2.6)
// d = 2 Green density: radius with CDF F(t) = t^2 - t^2 ln t^2.  With t^2 = e^{-L},
// (1 + L) e^{-L} = u; g(L) = log1p(L) - L + a (a = -ln u) is concave and decreasing, and
// L0 = a + sqrt(2a) is an upper bound of the root (1 + s + s^2/2 <= e^s), so Newton's method
// from L0 decreases monotonically onto the root (two steps reach FP32 rounding, seven FP64).
template <typename T> struct GreenIters;
template <> struct GreenIters<float> { static constexpr int value = 2; };
template <> struct GreenIters<double> { static constexpr int value = 7; };

template <typename T> __device__ __forceinline__ T green_radius_2d(T u) {
    const T a = -m_log(u);
    T L = a + m_sqrt(T(2) * a);
#pragma unroll
    for (int it = 0; it < GreenIters<T>::value; ++it) {
        const T g = m_log1p(L) - L + a;
        L = L + m_newton_div(g * (T(1) + L), L);
    }
    return m_exp(T(-0.5) * L);
}

template <typename T> __device__ __forceinline__ T med3(T a, T b, T c) {
    return fmax(fmin(a, b), fmin(fmax(a, b), c));
}
__device__ __forceinline__ float med3(float a, float b, float c) {
    return fmaxf(fminf(a, b), fminf(fmaxf(a, b), c));
}

template <typename T> struct Vec { T v[3]; };

template <typename T> __device__ __forceinline__ void dir2(T u, T* o) {
    T s, c;
    m_sincos2pi(u, &s, &c);
    o[0] = c; o[1] = s;
}

// uniform direction on S^2: z = 1 - 2u, rho = sqrt(1 - z^2) = 2 sqrt(u (1 - u)), phi = 2 pi v
template <typename T> __device__ __forceinline__ void dir3(T uz, T uphi, T* o) {
    T s, c;
    m_sincos2pi(uphi, &s, &c);
    const T z = T(1) - T(2) * uz;
    const T rho = T(2) * m_sqrt(uz * (T(1) - uz));
    o[0] = rho * c; o[1] = rho * s; o[2] = z;
}

// ------------------------------------------------------------------ distance to the boundary
enum SdfKind { SDF_BALL = 0, SDF_BOX = 1, SDF_POLYGON = 2 };

template <typename T, int D, int KIND> struct Sdf;

template <typename T, int D> struct Sdf<T, D, SDF_BALL> {
    __device__ __forceinline__ static T eval(const T* prm, int, const T* x) {
        T s = 0;
#pragma unroll
        for (int c = 0; c < D; ++c) { const T t = x[c] - prm[c]; s += t * t; }
        return prm[D] - m_sqrt(s);
    }
};

template <typename T, int D> struct Sdf<T, D, SDF_BOX> {
    __device__ __forceinline__ static T eval(const T* prm, int, const T* x) {
        T r = x[0] - prm[0];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            r = fmin(r, x[c] - prm[c]);
            r = fmin(r, prm[D + c] - x[c]);
        }
        return r;
    }
};

// polygon (d = 2): distance to the nearest edge; signed by the even-odd crossing rule
template <typename T, int D> struct Sdf<T, D, SDF_POLYGON> {
    __device__ __forceinline__ static T eval(const T* prm, int nv, const T* x) {
        T best = T(3.0e38f);
        bool inside = false;
        const T px0 = x[0], py0 = x[1];
        T ax = prm[2 * (nv - 1)], ay = prm[2 * (nv - 1) + 1];
        for (int e = 0; e < nv; ++e) {
            const T bx = prm[2 * e], by = prm[2 * e + 1];
            const T ex = bx - ax, ey = by - ay, px = px0 - ax, py = py0 - ay;
            const T ee = ex * ex + ey * ey;
            T t = (px * ex + py * ey) / ee;
            t = fmin(fmax(t, T(0)), T(1));
            const T dx = px - t * ex, dy = py - t * ey;
            best = fmin(best, dx * dx + dy * dy);
            if ((ay > py0) != (by > py0)) {
                const T xc = ax + (py0 - ay) / (by - ay) * ex;
                if (px0 < xc) inside = !inside;
            }
            ax = bx; ay = by;
        }
        const T r = m_sqrt(best);
        return inside ? r : -r;
    }
};

// ------------------------------------------------------------------ nearest-centre lookup
// Uniform grid over the domain's bounding box.  Each grid cell Q lists every centre c with
// mindist(c, Q) <= R_Q, R_Q = min_c maxdist(c, Q): a superset of the centres that are nearest
// to some point of Q, so scanning the list gives the exact nearest centre; lists are in
// increasing centre index, so a strict '<' keeps the lowest index on ties.
template <typename T, int D> struct Lookup {
    const T* pts;          // [count][D]
    const int* start;      // [ncell + 1]
    const int* cand;       // [start[ncell]]
    T lo[D];
    T inv_h;
    int dims[D];
};

template <typename T, int D>
__device__ __forceinline__ int lookup_cell(const Lookup<T, D>& L, const T* q) {
    int cell = 0;
#pragma unroll
    for (int c = D - 1; c >= 0; --c) {
        int k = (int)floor((q[c] - L.lo[c]) * L.inv_h);
        k = k < 0 ? 0 : (k >= L.dims[c] ? L.dims[c] - 1 : k);
        cell = cell * L.dims[c] + k;
    }
    return cell;
}

template <typename T, int D>
__device__ __forceinline__ int nearest(const Lookup<T, D>& L, const T* q) {
    const int cell = lookup_cell(L, q);
    const int s = L.start[cell], e = L.start[cell + 1];
    T best = T(3.0e38f);
    int bi = 0;
    for (int t = s; t < e; ++t) {
        const int j = L.cand[t];
        T d2 = 0;
#pragma unroll
        for (int c = 0; c < D; ++c) { const T dd = q[c] - L.pts[j * D + c]; d2 += dd * dd; }
        if (d2 < best) { best = d2; bi = j; }
    }
    return bi;
}

}  // namespace ewos
