// toolbox.hpp -- internal definition of the opaque ewos_toolbox and shared host helpers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ewos.h"

namespace ewos {

void set_error(const std::string& msg);
void note_launch();            // counts every kernel launch of the library (ewos_launch_count)
void unnote_launches(unsigned long long k);   // takes back launches recorded into a graph capture
uint64_t next_toolbox_serial();  // process-wide serial of a new toolbox (never reused)

// Device memory of the library comes from the device's stream-ordered pool (cudaMallocAsync),
// on the stream the current entry point runs on; freed blocks stay in the pool for reuse.
cudaError_t dev_alloc(void** p, size_t bytes);
cudaError_t dev_free(void* p);
void set_alloc_stream(cudaStream_t s);
struct AllocStream {
    explicit AllocStream(cudaStream_t s) { set_alloc_stream(s); }
    ~AllocStream() { set_alloc_stream(nullptr); }
};

#define EWOS_CUDA_TRY(expr)                                                              \
    do {                                                                                 \
        cudaError_t e__ = (expr);                                                        \
        if (e__ != cudaSuccess) {                                                        \
            ::ewos::set_error(std::string(#expr) + ": " + cudaGetErrorString(e__));      \
            return e__ == cudaErrorMemoryAllocation ? EWOS_ENOMEM : EWOS_ECUDA;          \
        }                                                                                \
    } while (0)

struct SolveWorkspace;   // solve.cu
void free_workspace(SolveWorkspace* ws);

}  // namespace ewos

struct ewos_toolbox {
    int dim = 0, precision = 32;
    int64_t n = 0, m = 0, p = 0, N = 0;
    double eps = 0;
    uint64_t seed = 0;
    uint32_t instance = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    // P = [d_1 G, ..., d_d G, G] of shape [(d+1)][n][m]; KH = [d_1 H, ..., d_d H, H] [(d+1)][n][p]
    void* P = nullptr;
    void* KH = nullptr;
    uint32_t* Hc = nullptr;          // [n][p] exit counts (empty for toolboxes made from matrices)
    // max |P| and max |G| (FP32, device [2]) as the build wrote P: the scales of the FP16 assembly and
    // Jacobian products without a pass over P; valid after a build (not for toolboxes made from
    // matrices or read from files)
    float* pmax = nullptr;
    bool pmax_valid = false;
    double* lambda = nullptr;        // [n]
    double* x = nullptr;             // [n][d]
    double* z = nullptr;             // [p][d]
    double* y = nullptr;             // [m][d] V-centres (NULL: y = x)
    int32_t* rec_exit = nullptr;     // [n][N] optional
    int32_t* rec_steps = nullptr;
    void* rec_mass = nullptr;        // T [n][N]
    uint32_t* rec_vhash = nullptr;   // [n][N]
    void* rec_xexit = nullptr;       // T [n][N][d]
    ewos_build_report rep{};
    ewos::SolveWorkspace* ws = nullptr;
    // Identity of this toolbox for caches that outlive it (the sweep graphs of a server slot's
    // workspace): a host address can be reused by a later toolbox, a serial is not.
    uint64_t serial = ewos::next_toolbox_serial();
    size_t elem() const { return precision == 64 ? 8 : 4; }
};
