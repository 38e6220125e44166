// api.cu -- the C ABI (include/ewos.h): argument checks, device buffers owned by the toolbox,
// copies in and out, and the test hooks.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "device_common.cuh"
#include "toolbox.hpp"

namespace ewos {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void unnote_launches(unsigned long long k) { g_launches.fetch_sub(k, std::memory_order_relaxed); }
static std::atomic<uint64_t> g_toolbox_serial{0};
uint64_t next_toolbox_serial() { return g_toolbox_serial.fetch_add(1, std::memory_order_relaxed) + 1; }

static thread_local cudaStream_t g_alloc_stream = nullptr;
void set_alloc_stream(cudaStream_t s) { g_alloc_stream = s; }

// test hook: the allocation after this many more successful ones fails once (-1: never)
static std::atomic<long long> g_fail_alloc_after{-1};

cudaError_t dev_alloc(void** p, size_t bytes) {
    for (long long v = g_fail_alloc_after.load(); v >= 0;) {
        if (g_fail_alloc_after.compare_exchange_weak(v, v - 1)) {
            if (v == 0) { *p = nullptr; return cudaErrorMemoryAllocation; }
            break;
        }
    }
    constexpr int kMaxDevices = 64;
    static std::atomic<int> pool_ready[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevices && !pool_ready[dev].exchange(1)) {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;      // keep freed blocks in this process's pool
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    return cudaMallocAsync(p, bytes ? bytes : 1, g_alloc_stream);
}

cudaError_t dev_free(void* p) { return p ? cudaFreeAsync(p, g_alloc_stream) : cudaSuccess; }

ewos_status build_toolbox(ewos_toolbox* tb, const ewos_domain* dom, const double* d_x, const double* d_z,
                          const ewos_build_opts& o);
ewos_status validate_domain(const ewos_domain* dom, const double* x, int64_t n);
ewos_status build_toolbox_batch(std::vector<ewos_toolbox*>& tbs, const std::vector<const ewos_domain*>& doms,
                                const ewos_build_opts& o, ewos_build_report* brep);

static void release(ewos_toolbox* tb) {
    if (!tb) return;
    AllocStream as(tb->stream);
    ::ewos::dev_free(tb->P); ::ewos::dev_free(tb->KH); ::ewos::dev_free(tb->Hc); ::ewos::dev_free(tb->lambda);
    ::ewos::dev_free(tb->pmax);
    ::ewos::dev_free(tb->x); ::ewos::dev_free(tb->z); ::ewos::dev_free(tb->y);
    ::ewos::dev_free(tb->rec_exit); ::ewos::dev_free(tb->rec_steps); ::ewos::dev_free(tb->rec_mass); ::ewos::dev_free(tb->rec_vhash);
    ::ewos::dev_free(tb->rec_xexit);
    free_workspace(tb->ws);
    delete tb;
}

static ewos_status alloc_matrices(ewos_toolbox* tb, bool counts) {
    const size_t e = tb->elem();
    const int64_t d1 = tb->dim + 1;
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&tb->P, e * d1 * tb->n * tb->m));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&tb->KH, e * d1 * tb->n * tb->p));
    if (counts) {
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&tb->Hc, sizeof(uint32_t) * tb->n * tb->p));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&tb->pmax, 2 * sizeof(float)));
    }
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&tb->lambda, sizeof(double) * tb->n));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&tb->x, sizeof(double) * tb->n * tb->dim));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&tb->z, sizeof(double) * tb->p * tb->dim));
    return EWOS_OK;
}

template <typename T>
__global__ void widen_kernel(const T* __restrict__ in, double* __restrict__ out, int64_t count) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = (double)in[t];
}

template <typename T>
__global__ void narrow_kernel(const double* __restrict__ in, T* __restrict__ out, int64_t count) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = (T)in[t];
}

__global__ void philox_debug_kernel(const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1,
                                    uint32_t* __restrict__ out, int64_t count) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
        const u32x4 r = philox4x32_10(u32x4{ctr[4 * t], ctr[4 * t + 1], ctr[4 * t + 2], ctr[4 * t + 3]}, k0, k1);
        out[4 * t] = r.a; out[4 * t + 1] = r.b; out[4 * t + 2] = r.c; out[4 * t + 3] = r.d;
    }
}

template <typename T>
__global__ void green_debug_kernel(const T* __restrict__ u, T* __restrict__ R, int64_t count) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
        R[t] = green_radius_2d<T>(u[t]);
}

}  // namespace ewos

using namespace ewos;

extern "C" {

const char* ewos_status_string(ewos_status s) {
    switch (s) {
        case EWOS_OK: return "ok";
        case EWOS_EINVAL: return "invalid argument";
        case EWOS_ENOMEM: return "out of memory";
        case EWOS_ECUDA: return "CUDA error";
        case EWOS_ESINGULAR: return "singular matrix";
        case EWOS_ENOCONV: return "no convergence";
        case EWOS_ETIMEOUT: return "device wait timed out";
        case EWOS_ESTEPCAP: return "some walks hit max_steps";
        case EWOS_EIO: return "toolbox file error";
    }
    return "unknown status";
}

const char* ewos_last_error(void) { return g_last_error.c_str(); }

unsigned long long ewos_launch_count(void) { return g_launches.load(); }

ewos_status ewos_toolbox_build(const ewos_domain* domain, const double* x, int64_t n, const double* z, int64_t p,
                               int64_t walks, double eps, uint64_t seed, const ewos_build_opts* opts,
                               ewos_toolbox** out) {
    if (!out || !x || !z || n < 1 || p < 1 || walks < 1 || !(eps > 0) || n > (1 << 30) || p > (1 << 30) ||
        walks > 0xFFFFFFFFll) {
        set_error("ewos_toolbox_build: need out, x, z, n >= 1, p >= 1, 1 <= walks < 2^32, eps > 0");
        return EWOS_EINVAL;
    }
    *out = nullptr;
    ewos_build_opts o{};
    o.precision = 32;
    o.hash_in_smem = -1;
    if (opts) o = *opts;
    if (o.precision != 32 && o.precision != 64) { set_error("precision must be 32 or 64"); return EWOS_EINVAL; }
    const double* hx = x;
    std::vector<double> xh;
    if (o.inputs_on_device) {
        xh.resize((size_t)n * domain->dim);
        if (cudaMemcpy(xh.data(), x, sizeof(double) * xh.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
            set_error("cannot read device x");
            return EWOS_ECUDA;
        }
        hx = xh.data();
    }
    ewos_status s = validate_domain(domain, hx, n);
    if (s != EWOS_OK) return s;
    int64_t m = n;
    if (o.v_nodes) {
        if (o.m < 1 || o.m > (1 << 30)) { set_error("ewos_toolbox_build: v_nodes needs 1 <= m < 2^30"); return EWOS_EINVAL; }
        std::vector<double> yh;
        const double* hy = o.v_nodes;
        if (o.inputs_on_device) {
            yh.resize((size_t)o.m * domain->dim);
            if (cudaMemcpy(yh.data(), o.v_nodes, sizeof(double) * yh.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
                set_error("cannot read device v_nodes");
                return EWOS_ECUDA;
            }
            hy = yh.data();
        }
        s = validate_domain(domain, hy, o.m);
        if (s != EWOS_OK) return s;
        m = o.m;
    }
    AllocStream as((cudaStream_t)o.stream);
    ewos_toolbox* tb = new ewos_toolbox();
    tb->dim = domain->dim; tb->precision = o.precision;
    tb->n = n; tb->m = m; tb->p = p; tb->N = walks; tb->eps = eps; tb->seed = seed; tb->instance = o.instance;
    tb->stream = (cudaStream_t)o.stream;
    cudaGetDevice(&tb->device);
    s = alloc_matrices(tb, true);
    if (s == EWOS_OK && o.record_walks) {
        cudaError_t e1 = ::ewos::dev_alloc((void**)&tb->rec_exit, sizeof(int32_t) * n * walks);
        cudaError_t e2 = ::ewos::dev_alloc((void**)&tb->rec_steps, sizeof(int32_t) * n * walks);
        cudaError_t e3 = ::ewos::dev_alloc((void**)&tb->rec_mass, tb->elem() * n * walks);
        cudaError_t e4 = ::ewos::dev_alloc((void**)&tb->rec_vhash, sizeof(uint32_t) * n * walks);
        cudaError_t e5 = ::ewos::dev_alloc((void**)&tb->rec_xexit, tb->elem() * n * walks * domain->dim);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess || e5 != cudaSuccess) {
            set_error("records: out of memory");
            s = EWOS_ENOMEM;
        }
    }
    if (s == EWOS_OK) {
        const cudaMemcpyKind kind = o.inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        cudaError_t e1 = cudaMemcpyAsync(tb->x, x, sizeof(double) * n * tb->dim, kind, tb->stream);
        cudaError_t e2 = cudaMemcpyAsync(tb->z, z, sizeof(double) * p * tb->dim, kind, tb->stream);
        cudaError_t e3 = cudaSuccess;
        if (o.v_nodes) {
            e3 = ::ewos::dev_alloc((void**)&tb->y, sizeof(double) * m * tb->dim);
            if (e3 == cudaSuccess) e3 = cudaMemcpyAsync(tb->y, o.v_nodes, sizeof(double) * m * tb->dim, kind, tb->stream);
        }
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) { set_error("copy of nodes failed"); s = EWOS_ECUDA; }
    }
    if (s == EWOS_OK) s = build_toolbox(tb, domain, tb->x, tb->z, o);
    if (s != EWOS_OK) { release(tb); return s; }
    *out = tb;
    return tb->rep.capped > 0 ? EWOS_ESTEPCAP : EWOS_OK;
}

ewos_status ewos_toolbox_build_batch(int count, const ewos_domain* domains, const double* const* x, const int64_t* n,
                                     const double* const* z, const int64_t* p, int64_t walks, double eps, uint64_t seed,
                                     const ewos_build_opts* opts, ewos_toolbox** out, ewos_build_report* batch_report) {
    if (count < 1 || !domains || !x || !n || !z || !p || !out || walks < 1 || !(eps > 0) || walks > 0xFFFFFFFFll) {
        set_error("ewos_toolbox_build_batch: need count >= 1, domains, x, n, z, p, out, 1 <= walks < 2^32, eps > 0");
        return EWOS_EINVAL;
    }
    ewos_build_opts o{};
    o.precision = 32;
    o.hash_in_smem = -1;
    if (opts) o = *opts;
    if (o.precision != 32 && o.precision != 64) { set_error("precision must be 32 or 64"); return EWOS_EINVAL; }
    if (o.record_walks || o.cell_weights || o.inputs_on_device || o.v_nodes) {
        set_error("ewos_toolbox_build_batch: record_walks, cell_weights, v_nodes and device inputs are not supported");
        return EWOS_EINVAL;
    }
    int64_t rows = 0;
    for (int k = 0; k < count; ++k) {
        if (!x[k] || !z[k] || n[k] < 1 || p[k] < 1 || n[k] > (1 << 30) || p[k] > (1 << 30)) {
            set_error("ewos_toolbox_build_batch: every instance needs x, z, n >= 1, p >= 1");
            return EWOS_EINVAL;
        }
        if (domains[k].dim != domains[0].dim || domains[k].kind != domains[0].kind) {
            set_error("ewos_toolbox_build_batch: all domains must have the same dimension and distance kind");
            return EWOS_EINVAL;
        }
        ewos_status s = validate_domain(&domains[k], x[k], n[k]);
        if (s != EWOS_OK) return s;
        rows += n[k];
    }
    if (rows >= (1ll << 31)) { set_error("ewos_toolbox_build_batch: more than 2^31 rows"); return EWOS_EINVAL; }
    for (int k = 0; k < count; ++k) out[k] = nullptr;
    AllocStream as((cudaStream_t)o.stream);
    std::vector<ewos_toolbox*> tbs;
    std::vector<const ewos_domain*> doms;
    ewos_status s = EWOS_OK;
    for (int k = 0; k < count && s == EWOS_OK; ++k) {
        ewos_toolbox* tb = new ewos_toolbox();
        tb->dim = domains[k].dim; tb->precision = o.precision;
        tb->n = n[k]; tb->m = n[k]; tb->p = p[k]; tb->N = walks; tb->eps = eps; tb->seed = seed;
        tb->instance = o.instance + (uint32_t)k;
        tb->stream = (cudaStream_t)o.stream;
        cudaGetDevice(&tb->device);
        tbs.push_back(tb);
        doms.push_back(&domains[k]);
        s = alloc_matrices(tb, true);
        if (s == EWOS_OK) {
            cudaError_t e1 = cudaMemcpyAsync(tb->x, x[k], sizeof(double) * n[k] * tb->dim, cudaMemcpyHostToDevice, tb->stream);
            cudaError_t e2 = cudaMemcpyAsync(tb->z, z[k], sizeof(double) * p[k] * tb->dim, cudaMemcpyHostToDevice, tb->stream);
            if (e1 != cudaSuccess || e2 != cudaSuccess) { set_error("copy of nodes failed"); s = EWOS_ECUDA; }
        }
    }
    if (s == EWOS_OK) s = build_toolbox_batch(tbs, doms, o, batch_report);
    if (s != EWOS_OK) {
        for (ewos_toolbox* tb : tbs) release(tb);
        return s;
    }
    int64_t capped = 0;
    for (int k = 0; k < count; ++k) {
        out[k] = tbs[k];
        capped += tbs[k]->rep.capped;
    }
    return capped > 0 ? EWOS_ESTEPCAP : EWOS_OK;
}

ewos_status ewos_toolbox_from_host(int dim, int64_t n, int64_t p, const double* x, const double* z, const double* G,
                                   const double* gradG, const double* H, const double* gradH, const double* lambda,
                                   int precision, void* stream, ewos_toolbox** out) {
    if (!out || (dim != 2 && dim != 3) || n < 1 || p < 1 || !x || !z || !G || !gradG || !H || !gradH || !lambda ||
        (precision != 32 && precision != 64)) {
        set_error("ewos_toolbox_from_host: bad arguments");
        return EWOS_EINVAL;
    }
    *out = nullptr;
    AllocStream as((cudaStream_t)stream);
    ewos_toolbox* tb = new ewos_toolbox();
    tb->dim = dim; tb->precision = precision; tb->n = n; tb->m = n; tb->p = p; tb->N = 0;
    tb->stream = (cudaStream_t)stream;
    cudaGetDevice(&tb->device);
    ewos_status s = alloc_matrices(tb, false);
    if (s != EWOS_OK) { release(tb); return s; }
    const int64_t nm = n * n, np = n * p;
    std::vector<double> stage((size_t)(dim + 1) * std::max(nm, np));
    double* dstage = nullptr;
    if (::ewos::dev_alloc((void**)&dstage, sizeof(double) * stage.size()) != cudaSuccess) { release(tb); set_error("oom"); return EWOS_ENOMEM; }
    std::memcpy(stage.data(), gradG, sizeof(double) * dim * nm);
    std::memcpy(stage.data() + dim * nm, G, sizeof(double) * nm);
    cudaMemcpy(dstage, stage.data(), sizeof(double) * (dim + 1) * nm, cudaMemcpyHostToDevice);
    if (precision == 64) cudaMemcpy(tb->P, dstage, sizeof(double) * (dim + 1) * nm, cudaMemcpyDeviceToDevice);
    else ::ewos::note_launch(), narrow_kernel<float><<<1024, 256>>>(dstage, (float*)tb->P, (dim + 1) * nm);
    std::memcpy(stage.data(), gradH, sizeof(double) * dim * np);
    std::memcpy(stage.data() + dim * np, H, sizeof(double) * np);
    cudaMemcpy(dstage, stage.data(), sizeof(double) * (dim + 1) * np, cudaMemcpyHostToDevice);
    if (precision == 64) cudaMemcpy(tb->KH, dstage, sizeof(double) * (dim + 1) * np, cudaMemcpyDeviceToDevice);
    else ::ewos::note_launch(), narrow_kernel<float><<<1024, 256>>>(dstage, (float*)tb->KH, (dim + 1) * np);
    cudaMemcpy(tb->lambda, lambda, sizeof(double) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(tb->x, x, sizeof(double) * n * dim, cudaMemcpyHostToDevice);
    cudaMemcpy(tb->z, z, sizeof(double) * p * dim, cudaMemcpyHostToDevice);
    cudaError_t e = cudaDeviceSynchronize();
    ::ewos::dev_free(dstage);
    if (e != cudaSuccess) { release(tb); set_error(cudaGetErrorString(e)); return EWOS_ECUDA; }
    *out = tb;
    return EWOS_OK;
}

ewos_status ewos_toolbox_get(const ewos_toolbox* tb, int which, void* dst, size_t dst_bytes, int dst_on_device) {
    if (!tb || !dst) { set_error("ewos_toolbox_get: NULL argument"); return EWOS_EINVAL; }
    const int64_t d = tb->dim, nm = tb->n * tb->m, np = tb->n * tb->p;
    const void* src = nullptr;
    int64_t count = 0;
    bool widen = false;
    size_t raw_elem = 0;
    switch (which) {
        case EWOS_G: src = (const char*)tb->P + tb->elem() * d * nm; count = nm; widen = true; break;
        case EWOS_GRAD_G: src = tb->P; count = d * nm; widen = true; break;
        case EWOS_H: src = (const char*)tb->KH + tb->elem() * d * np; count = np; widen = true; break;
        case EWOS_GRAD_H: src = tb->KH; count = d * np; widen = true; break;
        case EWOS_H_COUNTS: src = tb->Hc; count = np; raw_elem = 4; break;
        case EWOS_LAMBDA: src = tb->lambda; count = tb->n; raw_elem = 8; break;
        case EWOS_WALK_EXIT: src = tb->rec_exit; count = tb->n * tb->N; raw_elem = 4; break;
        case EWOS_WALK_STEPS: src = tb->rec_steps; count = tb->n * tb->N; raw_elem = 4; break;
        case EWOS_WALK_MASS: src = tb->rec_mass; count = tb->n * tb->N; widen = true; break;
        case EWOS_WALK_VHASH: src = tb->rec_vhash; count = tb->n * tb->N; raw_elem = 4; break;
        case EWOS_WALK_XEXIT: src = tb->rec_xexit; count = tb->n * tb->N * d; widen = true; break;
        default: set_error("ewos_toolbox_get: unknown array"); return EWOS_EINVAL;
    }
    if (!src) { set_error("ewos_toolbox_get: array not available for this toolbox"); return EWOS_EINVAL; }
    const size_t need = widen ? sizeof(double) * count : raw_elem * count;
    if (dst_bytes < need) { set_error("ewos_toolbox_get: destination too small"); return EWOS_EINVAL; }
    const cudaMemcpyKind k = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    AllocStream as(tb->stream);
    if (!widen || tb->precision == 64) {
        EWOS_CUDA_TRY(cudaMemcpyAsync(dst, src, need, k, tb->stream));
        EWOS_CUDA_TRY(cudaStreamSynchronize(tb->stream));
        return EWOS_OK;
    }
    double* tmp = nullptr;
    if (dst_on_device) tmp = (double*)dst;
    else EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&tmp, need));
    ::ewos::note_launch(), widen_kernel<float><<<1024, 256, 0, tb->stream>>>((const float*)src, tmp, count);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !dst_on_device) e = cudaMemcpyAsync(dst, tmp, need, cudaMemcpyDeviceToHost, tb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(tb->stream);
    if (!dst_on_device) ::ewos::dev_free(tmp);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return EWOS_ECUDA; }
    return EWOS_OK;
}

ewos_status ewos_toolbox_report(const ewos_toolbox* tb, ewos_build_report* rep) {
    if (!tb || !rep) { set_error("ewos_toolbox_report: NULL argument"); return EWOS_EINVAL; }
    *rep = tb->rep;
    return EWOS_OK;
}

ewos_status ewos_toolbox_shape(const ewos_toolbox* tb, int* dim, int64_t* n, int64_t* m, int64_t* p, int* precision) {
    if (!tb) { set_error("ewos_toolbox_shape: NULL toolbox"); return EWOS_EINVAL; }
    if (dim) *dim = tb->dim;
    if (n) *n = tb->n;
    if (m) *m = tb->m;
    if (p) *p = tb->p;
    if (precision) *precision = tb->precision;
    return EWOS_OK;
}

void ewos_toolbox_free(ewos_toolbox* tb) { release(tb); }

// ------------------------------------------------------------------ toolbox files
namespace {

constexpr char kTbMagic[8] = {'E', 'W', 'O', 'S', 'T', 'B', 'X', '\0'};
constexpr uint32_t kTbVersion = 1;

struct TbFileHeader {
    char magic[8];
    uint32_t version;
    int32_t dim, precision;
    int32_t flags;            // bit 0: exit counts Hc present; bit 1: separate V-centres y present
    int64_t n, m, p, N;
    double eps;
    uint64_t seed;
    uint32_t instance, reserved;
    ewos_build_report rep;
};

// bytes of every array after the header, in file order
struct TbLayout {
    int64_t x, z, y, lambda, P, KH, Hc;
    int64_t total() const { return x + z + y + lambda + P + KH + Hc; }
};

TbLayout layout_of(const TbFileHeader& h) {
    const int64_t e = h.precision == 64 ? 8 : 4, d = h.dim;
    TbLayout L;
    L.x = 8 * h.n * d;
    L.z = 8 * h.p * d;
    L.y = (h.flags & 2) ? 8 * h.m * d : 0;
    L.lambda = 8 * h.n;
    L.P = e * (d + 1) * h.n * h.m;
    L.KH = e * (d + 1) * h.n * h.p;
    L.Hc = (h.flags & 1) ? 4 * h.n * h.p : 0;
    return L;
}

struct FileCloser {
    FILE* f;
    ~FileCloser() { if (f) std::fclose(f); }
};

constexpr size_t kChunk = size_t(64) << 20;    // host staging of the device copies

// device -> file (stream already synchronised by the caller)
ewos_status write_device(FILE* f, const void* dsrc, int64_t bytes, std::vector<char>& buf) {
    for (int64_t off = 0; off < bytes; off += (int64_t)buf.size()) {
        const size_t len = (size_t)std::min<int64_t>((int64_t)buf.size(), bytes - off);
        EWOS_CUDA_TRY(cudaMemcpy(buf.data(), (const char*)dsrc + off, len, cudaMemcpyDeviceToHost));
        if (std::fwrite(buf.data(), 1, len, f) != len) { set_error("toolbox file: write failed"); return EWOS_EIO; }
    }
    return EWOS_OK;
}

// file -> device
ewos_status read_device(FILE* f, void* ddst, int64_t bytes, std::vector<char>& buf) {
    for (int64_t off = 0; off < bytes; off += (int64_t)buf.size()) {
        const size_t len = (size_t)std::min<int64_t>((int64_t)buf.size(), bytes - off);
        if (std::fread(buf.data(), 1, len, f) != len) { set_error("toolbox file: read failed"); return EWOS_EIO; }
        EWOS_CUDA_TRY(cudaMemcpy((char*)ddst + off, buf.data(), len, cudaMemcpyHostToDevice));
    }
    return EWOS_OK;
}

}  // namespace

ewos_status ewos_toolbox_save(const ewos_toolbox* tb, const char* path) {
    if (!tb || !path) { set_error("ewos_toolbox_save: NULL argument"); return EWOS_EINVAL; }
    TbFileHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kTbMagic, sizeof(kTbMagic));
    h.version = kTbVersion;
    h.dim = tb->dim; h.precision = tb->precision;
    h.flags = (tb->Hc ? 1 : 0) | (tb->y ? 2 : 0);
    h.n = tb->n; h.m = tb->m; h.p = tb->p; h.N = tb->N;
    h.eps = tb->eps; h.seed = tb->seed; h.instance = tb->instance;
    h.rep = tb->rep;
    EWOS_CUDA_TRY(cudaStreamSynchronize(tb->stream));
    FileCloser fc{std::fopen(path, "wb")};
    if (!fc.f) { set_error(std::string("toolbox file: cannot open for writing: ") + path); return EWOS_EIO; }
    if (std::fwrite(&h, sizeof(h), 1, fc.f) != 1) { set_error("toolbox file: write failed"); return EWOS_EIO; }
    const TbLayout L = layout_of(h);
    std::vector<char> buf((size_t)std::min<int64_t>((int64_t)kChunk, std::max<int64_t>(1, L.total())));
    const std::pair<const void*, int64_t> parts[] = {{tb->x, L.x}, {tb->z, L.z}, {tb->y, L.y}, {tb->lambda, L.lambda},
                                                     {tb->P, L.P}, {tb->KH, L.KH}, {tb->Hc, L.Hc}};
    for (const auto& pt : parts) {
        if (pt.second == 0) continue;
        ewos_status s = write_device(fc.f, pt.first, pt.second, buf);
        if (s != EWOS_OK) return s;
    }
    if (std::fflush(fc.f) != 0) { set_error("toolbox file: write failed"); return EWOS_EIO; }
    return EWOS_OK;
}

ewos_status ewos_toolbox_load(const char* path, void* stream, ewos_toolbox** out) {
    if (!path || !out) { set_error("ewos_toolbox_load: NULL argument"); return EWOS_EINVAL; }
    *out = nullptr;
    FileCloser fc{std::fopen(path, "rb")};
    if (!fc.f) { set_error(std::string("toolbox file: cannot open: ") + path); return EWOS_EIO; }
    TbFileHeader h;
    if (std::fread(&h, sizeof(h), 1, fc.f) != 1 || std::memcmp(h.magic, kTbMagic, sizeof(kTbMagic)) != 0) {
        set_error("toolbox file: not a toolbox file");
        return EWOS_EIO;
    }
    if (h.version != kTbVersion || (h.dim != 2 && h.dim != 3) || (h.precision != 32 && h.precision != 64) ||
        h.n < 1 || h.m < 1 || h.p < 1 || h.N < 0 || (h.flags & ~3) != 0 || (!(h.flags & 2) && h.m != h.n) ||
        h.n > (int64_t(1) << 31) || h.m > (int64_t(1) << 31) || h.p > (int64_t(1) << 31)) {
        set_error("toolbox file: unsupported version or inconsistent header");
        return EWOS_EIO;
    }
    const TbLayout L = layout_of(h);
    if (std::fseek(fc.f, 0, SEEK_END) != 0) { set_error("toolbox file: cannot seek"); return EWOS_EIO; }
    const long long size = std::ftell(fc.f);
    if (size != (long long)sizeof(h) + L.total()) {
        set_error("toolbox file: size does not match its header");
        return EWOS_EIO;
    }
    std::fseek(fc.f, (long)sizeof(h), SEEK_SET);
    AllocStream as((cudaStream_t)stream);
    ewos_toolbox* tb = new ewos_toolbox();
    tb->dim = h.dim; tb->precision = h.precision; tb->n = h.n; tb->m = h.m; tb->p = h.p; tb->N = h.N;
    tb->eps = h.eps; tb->seed = h.seed; tb->instance = h.instance; tb->rep = h.rep;
    tb->stream = (cudaStream_t)stream;
    cudaGetDevice(&tb->device);
    ewos_status s = alloc_matrices(tb, (h.flags & 1) != 0);
    if (s == EWOS_OK && (h.flags & 2) && ::ewos::dev_alloc((void**)&tb->y, sizeof(double) * h.m * h.dim) != cudaSuccess) {
        set_error("toolbox file: out of device memory");
        s = EWOS_ENOMEM;
    }
    if (s == EWOS_OK) s = cudaStreamSynchronize(tb->stream) == cudaSuccess ? EWOS_OK : EWOS_ECUDA;
    std::vector<char> buf((size_t)std::min<int64_t>((int64_t)kChunk, std::max<int64_t>(1, L.total())));
    const std::pair<void*, int64_t> parts[] = {{tb->x, L.x}, {tb->z, L.z}, {tb->y, L.y}, {tb->lambda, L.lambda},
                                               {tb->P, L.P}, {tb->KH, L.KH}, {tb->Hc, L.Hc}};
    for (const auto& pt : parts) {
        if (s != EWOS_OK) break;
        if (pt.second == 0) continue;
        s = read_device(fc.f, pt.first, pt.second, buf);
    }
    if (s != EWOS_OK) { release(tb); return s; }
    *out = tb;
    return EWOS_OK;
}

ewos_status ewos_debug_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t count) {
    if (!ctr || !key || !out || count < 0) { set_error("ewos_debug_philox: bad arguments"); return EWOS_EINVAL; }
    if (count == 0) return EWOS_OK;
    uint32_t *dc = nullptr, *dout = nullptr;
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&dc, 16 * count));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&dout, 16 * count));
    cudaMemcpy(dc, ctr, 16 * count, cudaMemcpyHostToDevice);
    ::ewos::note_launch(), philox_debug_kernel<<<256, 256>>>(dc, key[0], key[1], dout, count);
    cudaError_t e = cudaMemcpy(out, dout, 16 * count, cudaMemcpyDeviceToHost);
    ::ewos::dev_free(dc); ::ewos::dev_free(dout);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return EWOS_ECUDA; }
    return EWOS_OK;
}

ewos_status ewos_debug_green_radius(const void* u, void* R, int64_t count, int precision) {
    if (!u || !R || count < 0 || (precision != 32 && precision != 64)) {
        set_error("ewos_debug_green_radius: bad arguments");
        return EWOS_EINVAL;
    }
    if (count == 0) return EWOS_OK;
    const size_t e = precision == 64 ? 8 : 4;
    void *du = nullptr, *dR = nullptr;
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&du, e * count));
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&dR, e * count));
    cudaMemcpy(du, u, e * count, cudaMemcpyHostToDevice);
    if (precision == 64) ::ewos::note_launch(), green_debug_kernel<double><<<256, 256>>>((const double*)du, (double*)dR, count);
    else ::ewos::note_launch(), green_debug_kernel<float><<<256, 256>>>((const float*)du, (float*)dR, count);
    cudaError_t err = cudaMemcpy(R, dR, e * count, cudaMemcpyDeviceToHost);
    ::ewos::dev_free(du); ::ewos::dev_free(dR);
    if (err != cudaSuccess) { set_error(cudaGetErrorString(err)); return EWOS_ECUDA; }
    return EWOS_OK;
}

}  // extern "C"

extern "C" void ewos_debug_fail_allocations(int64_t after) {
    ewos::g_fail_alloc_after.store(after < 0 ? -1 : (long long)after);
}
