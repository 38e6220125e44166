// mixed.cu -- tensor-core assembly of the Galerkin matrix, Lambda = P^T Q (eq. linear_q), on the
// 5th-generation tensor cores: tcgen05.mma kind::tf32 with FP32 accumulation in TMEM.
//
// Both operands are staged K-major (A = P^T as [M][Kp], B = Q^T as [N][Kp], Kp = K padded to a
// multiple of 32 with zeros) by a tiled transpose, then
//   * TMA (cp.async.bulk.tensor, 128-byte swizzle) loads 128 x 32 (A) and 256 x 32 (B) tiles
//     into a 4-stage shared-memory ring guarded by mbarriers (3xTF32: hi and lo tiles of both,
//     N = 128, 3 stages);
//   * one thread issues tcgen05.mma (M = 128, N = 256, K = 8 per instruction, four per stage; 3xTF32:
//     three per step) into a 128-lane FP32 accumulator in tensor memory, and tcgen05.commit
//     releases each stage back to the producer;
//   * four warps read the accumulator with tcgen05.ld (32 lanes each) and store the tile.
// Every mbarrier wait is bounded; on a timeout the kernel records an error, frees its tensor
// memory and returns (the call then reports EWOS_ETIMEOUT).
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include "pdl.cuh"
#include "tf32.cuh"
#include "toolbox.hpp"

namespace ewos {

namespace tc {

constexpr int BM = 128, BK = 32;
constexpr long long kWaitLimit = 1ll << 22;

// plain TF32: tiles A (128 x 32) and B (256 x 32) per stage, 4 stages.
// split TF32 (3xTF32): A = A_hi + A_lo, B = B_hi + B_lo, products hi.hi + hi.lo + lo.hi into the
// same accumulator; tiles A_hi, A_lo (128 x 32) and B_hi, B_lo (128 x 32) per stage, 3 stages.
// ST > 0 sets the ring depth instead (the LU's trailing updates, K = 64, use two stages).
// F16: the operands are FP16 (the split of a scaled FP32 value into an FP16 part and an FP16
// remainder) and each stage holds 64 of them per row (the same 128 bytes); kind::f16 runs at twice
// the TF32 rate.
template <bool SPLIT, int ST = 0, bool F16 = false>
struct Cfg {
    static constexpr int BN = SPLIT ? 128 : 256;
    static constexpr int STAGES = ST > 0 ? ST : (SPLIT ? 3 : 4);
    static constexpr int A_BYTES = BM * BK * 4;
    static constexpr int B_BYTES = BN * BK * 4;
    static constexpr int STAGE_BYTES = (SPLIT ? 2 : 1) * (A_BYTES + B_BYTES);
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
    static constexpr int KSTAGE = F16 ? 2 * BK : BK;      // operand elements per row and stage
    static constexpr uint32_t IDESC = (1u << 4) | ((F16 ? 0u : 2u) << 7) | ((F16 ? 0u : 2u) << 10) |
                                      ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bounded wait for the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// as mbar_wait, sleeping `ns` nanoseconds between polls: for warps that wait long and share their
// SM sub-partition with the TMA and MMA threads (a hot poll takes issue slots from them)
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* bar, uint32_t parity, int ns) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        __nanosleep(ns);
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row atoms 1024 B apart
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
    const uint64_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;             // start address
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: next 8-row atom
    d |= (uint64_t)1 << 46;                    // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                    // swizzle: 128 B
    return d;
}

// instruction descriptor (Cfg::IDESC): kind::tf32 -- D format F32 (bits 4-5 = 1), A and B format
// TF32 (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

// C tile of the subtracting update staged in shared memory (CSM): 128 rows of BN floats, rows
// padded to BN + 4 floats so that the row-per-thread float4 reads of the epilogue are free of
// bank conflicts; filled with cp.async by all threads at kernel start, under the main loop.
constexpr int kCsmLd = 128 + 4;
constexpr int kCsmBytes = BM * kCsmLd * 4;

template <bool SPLIT, int ST = 0, bool CSM = false, bool F16 = false>
__global__ void __launch_bounds__(128, 1) gemm_tf32_kernel(const __grid_constant__ CUtensorMap mapA,
                                                           const __grid_constant__ CUtensorMap mapB,
                                                           const __grid_constant__ CUtensorMap mapAl,
                                                           const __grid_constant__ CUtensorMap mapBl, int M, int N,
                                                           int Kp, float* __restrict__ C, int64_t ldc,
                                                           int* __restrict__ err, int sub, int tri = 0,
                                                           const int* __restrict__ tiles = nullptr,
                                                           const float* __restrict__ cscale = nullptr, int lband = -1) {
    using CF = Cfg<SPLIT, ST, F16>;
    constexpr int BN = CF::BN, STAGES = CF::STAGES, A_BYTES = CF::A_BYTES, B_BYTES = CF::B_BYTES;
    constexpr int STAGE_BYTES = CF::STAGE_BYTES;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tri: a symmetric result; the 1D grid runs over the tiles on and below the diagonal (ty >= tx)
    // and each off-diagonal tile is also stored transposed
    int tile_y = blockIdx.y, tile_x = blockIdx.x;
    if (tiles) {
        // blocked order (CTAs that run together share row and column panels in L2)
        tile_y = tiles[2 * blockIdx.x];
        tile_x = tiles[2 * blockIdx.x + 1];
    } else if (tri) {
        const int t = blockIdx.x;
        int ty = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while ((ty + 1) * (ty + 2) / 2 <= t) ++ty;
        while (ty * (ty + 1) / 2 > t) --ty;
        tile_y = ty;
        tile_x = t - ty * (ty + 1) / 2;
    }
    int m0 = tile_y * BM, n0 = tile_x * BN;
    if (lband >= 0) {
        // L-shaped update (1D grid): rows [0, lband) x columns [0, N), then rows [lband, M) x
        // columns [0, lband); each tile's bounds are those of its part
        const int ntx1 = (N + BN - 1) / BN, t1 = ((lband + BM - 1) / BM) * ntx1;
        const int t = blockIdx.x;
        if (t < t1) {
            m0 = (t / ntx1) * BM;
            n0 = (t % ntx1) * BN;
            M = lband;
        } else {
            const int ntx2 = (lband + BN - 1) / BN, t2 = t - t1;
            m0 = lband + (t2 / ntx2) * BM;
            n0 = (t2 % ntx2) * BN;
            N = lband;
        }
    }
    const bool mirror = tri && tile_x != tile_y;
    const int nk = Kp / CF::KSTAGE;                // (Kp counts operand elements)
    ::ewos::pdl_trigger();

    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    ::ewos::pdl_wait();                       // operands and C come from the preceding launches
    float* Cs = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES + 256);
    if constexpr (CSM) {
        static_assert(BN == 128, "the staged C tile is 128 columns wide");
        // 16-byte pieces e = thread + 128 k: row e / 32, columns 4 (e % 32) .. + 3 (the host
        // checked that C rows start on 16-byte boundaries)
        for (int e = threadIdx.x; e < BM * BN / 4; e += 128) {
            const int r = e >> 5, c4 = (e & 31) * 4;
            if (m0 + r < M && n0 + c4 + 3 < N) {
                const float* g = C + (int64_t)(m0 + r) * ldc + n0 + c4;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(Cs + r * kCsmLd + c4)),
                             "l"(g)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }

    if (threadIdx.x == 0) {
        // producer: TMA loads into the ring
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (uint32_t)((kb / STAGES) & 1);
            if (!mbar_wait(&empty[s], ph ^ 1u)) { s_fail = 1; break; }
            unsigned char* st = smem + s * STAGE_BYTES;
            mbar_expect_tx(&full[s], STAGE_BYTES);
            tma_load_2d(st, &mapA, &full[s], kb * CF::KSTAGE, m0);
            tma_load_2d(st + A_BYTES, &mapB, &full[s], kb * CF::KSTAGE, n0);
            if (SPLIT) {
                tma_load_2d(st + A_BYTES + B_BYTES, &mapAl, &full[s], kb * CF::KSTAGE, m0);
                tma_load_2d(st + 2 * A_BYTES + B_BYTES, &mapBl, &full[s], kb * CF::KSTAGE, n0);
            }
        }
    } else if (threadIdx.x == 32) {
        // MMA issuer
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (uint32_t)((kb / STAGES) & 1);
            if (!mbar_wait(&full[s], ph)) { s_fail = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            unsigned char* st = smem + s * STAGE_BYTES;
#pragma unroll
            for (int k = 0; k < BK / 8; ++k) {      // 32-byte steps: K = 8 TF32 or 16 FP16 per MMA
                const uint64_t da = smem_desc(st + k * 32);
                const uint64_t db = smem_desc(st + A_BYTES + k * 32);
                const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                if constexpr (F16) mma_f16(tmem, da, db, CF::IDESC, acc);
                else mma_tf32(tmem, da, db, CF::IDESC, acc);
                if (SPLIT) {
                    const uint64_t dal = smem_desc(st + A_BYTES + B_BYTES + k * 32);
                    const uint64_t dbl = smem_desc(st + 2 * A_BYTES + B_BYTES + k * 32);
                    if constexpr (F16) {
                        mma_f16(tmem, da, dbl, CF::IDESC, 1u);
                        mma_f16(tmem, dal, db, CF::IDESC, 1u);
                    } else {
                        mma_tf32(tmem, da, dbl, CF::IDESC, 1u);
                        mma_tf32(tmem, dal, db, CF::IDESC, 1u);
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(done))
                     : "memory");
    }
    __syncwarp();
    // epilogue: wait for the accumulator, read 32 lanes per warp in 32-column chunks.  For the
    // subtracting update the thread's row of C is fetched a chunk ahead: the first chunk while
    // the MMAs still run, each next one while the current chunk is written.
    const int row = m0 + warp * 32 + lane;
    auto c_fast = [&](int c) {
        const int col0 = n0 + c * 32;
        return row < M && col0 + 32 <= N && (ldc & 3) == 0 &&
               ((reinterpret_cast<uintptr_t>(C + (int64_t)row * ldc + col0) & 15) == 0);
    };
    float4 cpre[8];
    auto c_fetch = [&](int c) {
        if (sub && c_fast(c)) {
            const float4* cp4 = reinterpret_cast<const float4*>(C + (int64_t)row * ldc + n0 + c * 32);
#pragma unroll
            for (int q = 0; q < 8; ++q) cpre[q] = cp4[q];
        }
    };
    if (!CSM) c_fetch(0);
    bool ok = mbar_wait(done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if constexpr (CSM) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();                      // every thread's pieces of the C tile have landed
    }
    if (ok && !s_fail) {
        for (int c = 0; c < BN / 32; ++c) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int col0 = n0 + c * 32;
            if constexpr (F16) {
                // the operands were scaled by powers of two: undo it (exact)
                const float sc = cscale ? *cscale : 1.0f;
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] = __float_as_uint(__uint_as_float(v[q]) * sc);
            }
            float4 ccur[8];
            if constexpr (CSM) {
                const float4* cs4 = reinterpret_cast<const float4*>(Cs + (warp * 32 + lane) * kCsmLd + c * 32);
#pragma unroll
                for (int q = 0; q < 8; ++q) ccur[q] = cs4[q];
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) ccur[q] = cpre[q];
                if (c + 1 < BN / 32) c_fetch(c + 1);
            }
            if (row < M) {
                float* cp = C + (int64_t)row * ldc + col0;
                if (c_fast(c)) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float4 o = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                               __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
                        if (sub) {
                            const float4 c4 = ccur[q];
                            o = make_float4(c4.x - o.x, c4.y - o.y, c4.z - o.z, c4.w - o.w);
                        }
                        if constexpr (CSM)      // written back to the tile; stored row-contiguously below
                            reinterpret_cast<float4*>(Cs + (warp * 32 + lane) * kCsmLd + c * 32)[q] = o;
                        else
                            reinterpret_cast<float4*>(cp)[q] = o;
                    }
                } else {
                    for (int q = 0; q < 32; ++q)
                        if (col0 + q < N) cp[q] = sub ? cp[q] - __uint_as_float(v[q]) : __uint_as_float(v[q]);
                }
                if (mirror) {
                    // C[col][row]: for each column the warp's 32 rows are 32 consecutive floats
                    for (int q = 0; q < 32; ++q)
                        if (col0 + q < N) C[(int64_t)(col0 + q) * ldc + row] = __uint_as_float(v[q]);
                }
            }
        }
    }
    if constexpr (CSM) {
        // every thread reaches this barrier; the tile is stored only when no wait gave up
        if (__syncthreads_and(ok && !s_fail)) {
            // the 16-byte pieces of every full 32-column chunk of a row, as they were staged
            for (int e = threadIdx.x; e < BM * BN / 4; e += 128) {
                const int r = e >> 5, c4 = (e & 31) * 4, chunk0 = n0 + (c4 & ~31);
                if (m0 + r < M && chunk0 + 32 <= N)
                    *reinterpret_cast<float4*>(C + (int64_t)(m0 + r) * ldc + n0 + c4) =
                        *reinterpret_cast<const float4*>(Cs + r * kCsmLd + c4);
            }
        }
    }
    if (!ok || s_fail) {
        if (threadIdx.x == 0) atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

#ifndef EWOS_DRAIN_SLEEP
#define EWOS_DRAIN_SLEEP 128
#endif

// The long-K products of the assembly (Lambda = P^T Q and the Jacobian's G^T D G, K up to 4 n)
// with two-level accumulation.  The tensor cores round the FP32 accumulation of each MMA toward
// zero, so one accumulator run over all of K loses about 5e-9 K of every entry's magnitude (a bias,
// not noise: 6e-5 at K = 12288).  Here the MMAs accumulate chunks of `dk` k-blocks (256 operand
// elements by default) into one of two TMEM accumulators in turn, while four drain warps add the
// finished chunks into FP32 registers (round to nearest): the bias is then that of one chunk,
// about 1e-6 (measured: 6.5e-7 for chunks of 128, 2e-6 for 512).  Each drain reads 64 KB of TMEM
// and costs the MMAs about 125 ns (more accumulators, to give the drains slack, did not change
// that), so the chunk stays long: 4 % over one accumulator for all of K at 256.  Warp roles: warps 0-3 drain (warp w reads TMEM lanes 32 w .. 32 w + 31, its 32 rows of
// the 128-row tile) and store the tile; warp 4 loads operands by TMA; warp 5 issues the MMAs.
template <bool F16>
__global__ void __launch_bounds__(192, 1) gemm_drain_kernel(const __grid_constant__ CUtensorMap mapA,
                                                            const __grid_constant__ CUtensorMap mapB,
                                                            const __grid_constant__ CUtensorMap mapAl,
                                                            const __grid_constant__ CUtensorMap mapBl, int M, int N,
                                                            int Kp, float* __restrict__ C, int64_t ldc,
                                                            int* __restrict__ err, int tri,
                                                            const int* __restrict__ tiles,
                                                            const float* __restrict__ cscale, int dk) {
    using CF = Cfg<true, 0, F16>;
    constexpr int BN = CF::BN, STAGES = CF::STAGES, A_BYTES = CF::A_BYTES, B_BYTES = CF::B_BYTES;
    constexpr int STAGE_BYTES = CF::STAGE_BYTES;
    constexpr int NACC = 2;
    static_assert(BN == 128, "128-column accumulators");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;        // [NACC]: a chunk's MMAs have completed into accumulator b
    uint64_t* tempty = tfull + NACC;         // [NACC]: the drain warps have read accumulator b
    uint64_t* done = tempty + NACC;          // every MMA of the CTA has completed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int tile_y = blockIdx.y, tile_x = blockIdx.x;
    if (tiles) {
        tile_y = tiles[2 * blockIdx.x];
        tile_x = tiles[2 * blockIdx.x + 1];
    }
    const int m0 = tile_y * BM, n0 = tile_x * BN;
    const bool mirror = tri && tile_x != tile_y;
    const int nk = Kp / CF::KSTAGE;
    const int nchunk = (nk + dk - 1) / dk;
    ::ewos::pdl_trigger();

    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < NACC; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], 4); }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(NACC * BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    ::ewos::pdl_wait();

    if (warp == 4) {
        if (lane == 0) {
            int issued = 0;
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)((kb / STAGES) & 1);
                if (!mbar_wait(&empty[s], ph ^ 1u)) { s_fail = 1; break; }
                unsigned char* st = smem + s * STAGE_BYTES;
                mbar_expect_tx(&full[s], STAGE_BYTES);
                tma_load_2d(st, &mapA, &full[s], kb * CF::KSTAGE, m0);
                tma_load_2d(st + A_BYTES, &mapB, &full[s], kb * CF::KSTAGE, n0);
                tma_load_2d(st + A_BYTES + B_BYTES, &mapAl, &full[s], kb * CF::KSTAGE, m0);
                tma_load_2d(st + 2 * A_BYTES + B_BYTES, &mapBl, &full[s], kb * CF::KSTAGE, n0);
                issued = kb + 1;
            }
            // after a failed wait, let the loads still in flight land before the CTA exits
            if (issued < nk)
                for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
                    mbar_wait(&full[kb % STAGES], (uint32_t)((kb / STAGES) & 1));
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // the issue loop is on the critical path (the tensor pipe waits for it whenever the
            // ring runs dry): no divisions, descriptors of stage 0 computed once (a stage, and a
            // 32-byte step inside one, move the descriptor's address field by bytes / 16)
            const uint64_t d0a = smem_desc(smem), d0b = smem_desc(smem + A_BYTES);
            const uint64_t d0al = smem_desc(smem + A_BYTES + B_BYTES), d0bl = smem_desc(smem + 2 * A_BYTES + B_BYTES);
            int chunk = 0, kin = 0, s = 0;
            uint32_t ph = 0;
            for (int kb = 0; kb < nk; ++kb) {
                const int b = chunk & (NACC - 1);
                const bool first = kin == 0, last = kin == dk - 1 || kb == nk - 1;
                // accumulator b is free again once the chunk NACC back has been drained
                if (first && chunk >= NACC && !mbar_wait(&tempty[b], (uint32_t)(((chunk >> 1) - 1) & 1))) {
                    s_fail = 1;
                    break;
                }
                if (!mbar_wait(&full[s], ph)) { s_fail = 1; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t so = (uint64_t)(s * (STAGE_BYTES >> 4));
                const uint32_t d = tmem + (uint32_t)(b * BN);
#pragma unroll
                for (int k = 0; k < BK / 8; ++k) {
                    const uint64_t ko = so + (uint64_t)(k * 2);
                    const uint32_t acc = (!first || k > 0) ? 1u : 0u;
                    if constexpr (F16) {
                        mma_f16(d, d0a + ko, d0b + ko, CF::IDESC, acc);
                        mma_f16(d, d0a + ko, d0bl + ko, CF::IDESC, 1u);
                        mma_f16(d, d0al + ko, d0b + ko, CF::IDESC, 1u);
                    } else {
                        mma_tf32(d, d0a + ko, d0b + ko, CF::IDESC, acc);
                        mma_tf32(d, d0a + ko, d0bl + ko, CF::IDESC, 1u);
                        mma_tf32(d, d0al + ko, d0b + ko, CF::IDESC, 1u);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&empty[s]))
                             : "memory");
                if (last)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&tfull[b]))
                                 : "memory");
                if (++kin == dk) { kin = 0; ++chunk; }
                if (++s == STAGES) { s = 0; ph ^= 1u; }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(done))
                         : "memory");
        }
    } else {
        float acc[BN];
#pragma unroll
        for (int q = 0; q < BN; ++q) acc[q] = 0.f;
        bool ok = true;
        for (int chunk = 0; chunk < nchunk; ++chunk) {
            const int b = chunk & (NACC - 1);
            if (!mbar_wait_sleep(&tfull[b], (uint32_t)((chunk >> 1) & 1), EWOS_DRAIN_SLEEP) || s_fail) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int c = 0; c < BN / 32; ++c) {
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * BN + c * 32);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                    "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                      "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int q = 0; q < 32; ++q) acc[c * 32 + q] += __uint_as_float(v[q]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[b])) : "memory");
        }
        // every MMA has completed (also after a failed wait) before TMEM is released
        if (!mbar_wait_sleep(done, 0, EWOS_DRAIN_SLEEP)) ok = false;
        if (ok && !s_fail) {
            const float sc = (F16 && cscale) ? *cscale : 1.0f;
            const int row = m0 + warp * 32 + lane;
            if (row < M) {
#pragma unroll
                for (int c = 0; c < BN / 32; ++c) {
                    const int col0 = n0 + c * 32;
                    float* cp = C + (int64_t)row * ldc + col0;
                    const bool fast = col0 + 32 <= N && (ldc & 3) == 0 && ((reinterpret_cast<uintptr_t>(cp) & 15) == 0);
                    if (fast) {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            reinterpret_cast<float4*>(cp)[q] = make_float4(acc[c * 32 + 4 * q] * sc, acc[c * 32 + 4 * q + 1] * sc,
                                                                           acc[c * 32 + 4 * q + 2] * sc, acc[c * 32 + 4 * q + 3] * sc);
                    } else {
#pragma unroll
                        for (int q = 0; q < 32; ++q)
                            if (col0 + q < N) cp[q] = acc[c * 32 + q] * sc;
                    }
                    if (mirror) {
#pragma unroll
                        for (int q = 0; q < 32; ++q)
                            if (col0 + q < N) C[(int64_t)(col0 + q) * ldc + row] = acc[c * 32 + q] * sc;
                    }
                }
            }
        } else {
            s_fail = 1;
        }
    }
    __syncwarp();
    __syncthreads();
    if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NACC * BN));
}

// The LU's subtracting update C -= diag(1/s) (A_h B_h + A_h B_l + A_l B_h) diag(1/t) on FP16 halves
// (the rank-512 updates), persistent: a CTA per SM takes output tiles b, b + G, .. (G CTAs) in
// bands of kUpdBand tile rows, column by column inside a band (the CTAs that run together share
// kUpdBand row panels of A and a run of column panels of B in L2).  Two TMEM accumulators: the
// MMAs of a tile run into one while the four epilogue warps read the other's tile, subtract it
// from C (read and written in HBM) and release it, so that the C traffic of one tile hides under
// the next tile's MMAs instead of following them.  Warp roles: warps 0-3 epilogue (warp w reads
// TMEM lanes 32 w .. 32 w + 31: a row of the tile per thread), warp 4 the TMA loads, warp 5 the
// MMA issue.
constexpr int kUpdBand = 8;

__global__ void __launch_bounds__(192, 1) gemm_upd16_kernel(const __grid_constant__ CUtensorMap mapA,
                                                            const __grid_constant__ CUtensorMap mapB,
                                                            const __grid_constant__ CUtensorMap mapAl,
                                                            const __grid_constant__ CUtensorMap mapBl, int M, int N,
                                                            int Kp, float* __restrict__ C, int64_t ldc,
                                                            int* __restrict__ err, const float* __restrict__ rinv,
                                                            const float* __restrict__ cinv) {
    using CF = Cfg<true, 0, true>;
    constexpr int BN = CF::BN, STAGES = CF::STAGES, A_BYTES = CF::A_BYTES, B_BYTES = CF::B_BYTES;
    constexpr int STAGE_BYTES = CF::STAGE_BYTES;
    constexpr int NACC = 2;
    static_assert(BN == 128 && BM == 128, "128 x 128 tiles");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;        // [NACC]: a tile's MMAs have completed into accumulator b
    uint64_t* tempty = tfull + NACC;         // [NACC]: the epilogue warps have read accumulator b
    uint64_t* done = tempty + NACC;          // every MMA of the CTA has completed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = (M + BM - 1) / BM, ntx = (N + BN - 1) / BN;
    const int ntiles = mt * ntx;
    const int nk = Kp / CF::KSTAGE;
    // tile t of the order: band of kUpdBand tile rows, columns in turn inside the band
    auto tile_of = [&](int t, int& m0, int& n0) {
        const int by = (t / (kUpdBand * ntx)) * kUpdBand;
        const int h = min(kUpdBand, mt - by);
        const int r = t - by * ntx;
        m0 = (by + r % h) * BM;
        n0 = (r / h) * BN;
    };
    ::ewos::pdl_trigger();

    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < NACC; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], 4); }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(NACC * BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    ::ewos::pdl_wait();                       // operands and C come from the preceding launches

    if (warp == 4) {
        if (lane == 0) {
            int s = 0, issued = 0;
            uint32_t ph = 0;
            for (int t = blockIdx.x; t < ntiles && !s_fail; t += gridDim.x) {
                int m0, n0;
                tile_of(t, m0, n0);
                for (int kb = 0; kb < nk; ++kb) {
                    if (!mbar_wait(&empty[s], ph ^ 1u)) { s_fail = 1; break; }
                    unsigned char* st = smem + s * STAGE_BYTES;
                    mbar_expect_tx(&full[s], STAGE_BYTES);
                    tma_load_2d(st, &mapA, &full[s], kb * CF::KSTAGE, m0);
                    tma_load_2d(st + A_BYTES, &mapB, &full[s], kb * CF::KSTAGE, n0);
                    tma_load_2d(st + A_BYTES + B_BYTES, &mapAl, &full[s], kb * CF::KSTAGE, m0);
                    tma_load_2d(st + 2 * A_BYTES + B_BYTES, &mapBl, &full[s], kb * CF::KSTAGE, n0);
                    ++issued;
                    if (++s == STAGES) { s = 0; ph ^= 1u; }
                }
            }
            // after a failed wait, let the loads still in flight land before the CTA exits
            if (s_fail)
                for (int g = issued > STAGES ? issued - STAGES : 0; g < issued; ++g)
                    mbar_wait(&full[g % STAGES], (uint32_t)((g / STAGES) & 1));
        }
    } else if (warp == 5) {
        if (lane == 0) {
            const uint64_t d0a = smem_desc(smem), d0b = smem_desc(smem + A_BYTES);
            const uint64_t d0al = smem_desc(smem + A_BYTES + B_BYTES), d0bl = smem_desc(smem + 2 * A_BYTES + B_BYTES);
            int s = 0, j = 0;
            uint32_t ph = 0;
            bool bad = false;
            for (int t = blockIdx.x; t < ntiles && !bad; t += gridDim.x, ++j) {
                const int b = j & (NACC - 1);
                // accumulator b is free again once tile j - NACC has been read by the epilogue
                if (j >= NACC && !mbar_wait(&tempty[b], (uint32_t)(((j >> 1) - 1) & 1))) { bad = true; break; }
                const uint32_t d = tmem + (uint32_t)(b * BN);
                for (int kb = 0; kb < nk; ++kb) {
                    if (!mbar_wait(&full[s], ph)) { bad = true; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t so = (uint64_t)(s * (STAGE_BYTES >> 4));
#pragma unroll
                    for (int k = 0; k < BK / 8; ++k) {
                        const uint64_t ko = so + (uint64_t)(k * 2);
                        const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                        mma_f16(d, d0a + ko, d0b + ko, CF::IDESC, acc);
                        mma_f16(d, d0a + ko, d0bl + ko, CF::IDESC, 1u);
                        mma_f16(d, d0al + ko, d0b + ko, CF::IDESC, 1u);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&empty[s]))
                                 : "memory");
                    if (++s == STAGES) { s = 0; ph ^= 1u; }
                }
                if (bad) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&tfull[b]))
                             : "memory");
            }
            if (bad) s_fail = 1;
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(done))
                         : "memory");
        }
    } else {
        bool ok = true;
        int j = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
            int m0, n0;
            tile_of(t, m0, n0);
            const int b = j & (NACC - 1);
            const int row = m0 + warp * 32 + lane;
            // the thread's row of C, a 32-column chunk ahead: the first one under the MMAs
            auto fast = [&](int c) {
                const int col0 = n0 + c * 32;
                return row < M && col0 + 32 <= N && (ldc & 3) == 0 &&
                       ((reinterpret_cast<uintptr_t>(C + (int64_t)row * ldc + col0) & 15) == 0);
            };
            float4 cpre[8];
            auto fetch = [&](int c) {
                if (fast(c)) {
                    const float4* cp4 = reinterpret_cast<const float4*>(C + (int64_t)row * ldc + n0 + c * 32);
#pragma unroll
                    for (int q = 0; q < 8; ++q) cpre[q] = cp4[q];
                }
            };
            fetch(0);
            if (!mbar_wait_sleep(&tfull[b], (uint32_t)((j >> 1) & 1), EWOS_DRAIN_SLEEP) || s_fail) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float acc[BN];
#pragma unroll
            for (int c = 0; c < BN / 32; ++c) {
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * BN + c * 32);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                    "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                      "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int q = 0; q < 32; ++q) acc[c * 32 + q] = __uint_as_float(v[q]);
            }
            // the accumulator is free for tile j + NACC once the four warps have read it
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[b])) : "memory");
            const float rs = row < M ? rinv[row] : 0.f;
#pragma unroll
            for (int c = 0; c < BN / 32; ++c) {
                const int col0 = n0 + c * 32;
                const float cl = col0 + lane < N ? cinv[col0 + lane] : 0.f;
#pragma unroll
                for (int q = 0; q < 32; ++q) acc[c * 32 + q] = acc[c * 32 + q] * rs * __shfl_sync(0xffffffffu, cl, q);
                const bool f = fast(c);
                float4 ccur[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) ccur[q] = cpre[q];
                if (c + 1 < BN / 32) fetch(c + 1);
                if (row < M) {
                    float* cp = C + (int64_t)row * ldc + col0;
                    if (f) {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            reinterpret_cast<float4*>(cp)[q] =
                                make_float4(ccur[q].x - acc[c * 32 + 4 * q], ccur[q].y - acc[c * 32 + 4 * q + 1],
                                            ccur[q].z - acc[c * 32 + 4 * q + 2], ccur[q].w - acc[c * 32 + 4 * q + 3]);
                    } else {
                        for (int q = 0; q < 32; ++q)
                            if (col0 + q < N) cp[q] = cp[q] - acc[c * 32 + q];
                    }
                }
            }
        }
        // every MMA has completed (also after a failed wait) before TMEM is released
        if (!mbar_wait_sleep(done, 0, EWOS_DRAIN_SLEEP)) ok = false;
        if (!ok) s_fail = 1;
    }
    __syncwarp();
    __syncthreads();
    if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NACC * BN));
}

// out[c][k] = in[k][c] for in [K][C] (row-major), out [C][Kp] with zero padding k in [K, Kp)
__global__ void transpose_pad_kernel(const float* __restrict__ in, int K, int Ccols, float* __restrict__ out, int Kp) {
    __shared__ float tile[32][33];
    ::ewos::pdl_trigger();
    ::ewos::pdl_wait();
    const int c0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int k = k0 + r, c = c0 + threadIdx.x;
        tile[r][threadIdx.x] = (k < K && c < Ccols) ? in[(int64_t)k * Ccols + c] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int c = c0 + r, k = k0 + threadIdx.x;
        if (c < Ccols && k < Kp) out[(int64_t)c * Kp + k] = tile[threadIdx.x][r];
    }
}

// as transpose_pad_kernel, also splitting each value into a TF32 part (round to nearest, 10
// explicit mantissa bits) and the FP32 remainder: v = hi + lo exactly
__global__ void transpose_split_kernel(const float* __restrict__ in, int K, int Ccols, float* __restrict__ hi,
                                       float* __restrict__ lo, int Kp) {
    __shared__ float tile[32][33];
    ::ewos::pdl_trigger();
    ::ewos::pdl_wait();
    const int c0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int k = k0 + r, c = c0 + threadIdx.x;
        tile[r][threadIdx.x] = (k < K && c < Ccols) ? in[(int64_t)k * Ccols + c] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int c = c0 + r, k = k0 + threadIdx.x;
        if (c < Ccols && k < Kp) {
            const float v = tile[threadIdx.x][r];
            const uint32_t b = __float_as_uint(v);
            const uint32_t hb = (b + 0x0FFFu + ((b >> 13) & 1u)) & 0xFFFFE000u;
            const float h = isfinite(v) ? __uint_as_float(hb) : v;
            hi[(int64_t)c * Kp + k] = h;
            lo[(int64_t)c * Kp + k] = v - h;
        }
    }
}

// hi/lo [M][Kp] from a row-major [M][K] operand with row stride ld (K contiguous), zero padding
__global__ void rows_split_kernel(const float* __restrict__ in, int64_t ld, int M, int K, float* __restrict__ hi,
                                  float* __restrict__ lo, int Kp) {
    ::ewos::pdl_trigger();
    ::ewos::pdl_wait();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)M * Kp) return;
    const int64_t i = t / Kp;
    const int k = (int)(t % Kp);
    float h = 0.f, l = 0.f;
    if (k < K) tf32_split(in[i * ld + k], h, l);
    hi[t] = h;
    lo[t] = l;
}

// hi/lo [N][Kp] = transpose of a row-major [K][N] operand with row stride ld
__global__ void cols_split_kernel(const float* __restrict__ in, int64_t ld, int K, int N, float* __restrict__ hi,
                                  float* __restrict__ lo, int Kp) {
    __shared__ float tile[32][33];
    ::ewos::pdl_trigger();
    ::ewos::pdl_wait();
    const int c0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int k = k0 + r, c = c0 + threadIdx.x;
        tile[r][threadIdx.x] = (k < K && c < N) ? in[(int64_t)k * ld + c] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int c = c0 + r, k = k0 + threadIdx.x;
        if (c < N && k < Kp) {
            float h, l;
            tf32_split(tile[threadIdx.x][r], h, l);
            hi[(int64_t)c * Kp + k] = h;
            lo[(int64_t)c * Kp + k] = l;
        }
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

static bool make_map(CUtensorMap* map, const float* base, int rows, int Kp, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 4};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// FP16 operand: [rows][Kp] halves, box of 64 halves (128 bytes) by box_rows
static bool make_map16(CUtensorMap* map, const void* base, int rows, int Kp, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * BK), (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// scratch for the K-major operands and the error word (stream-ordered pool)
struct Scratch {
    float* At = nullptr;
    float* Bt = nullptr;
    float* Atl = nullptr;
    float* Btl = nullptr;
    int* err = nullptr;
    size_t cap = 0;
    float* scale = nullptr;        // FP16 forms: [0], [1] the maxima that set [2] s_A (s_P), [3] s_B (s_Q); [4] 1/(s_A s_B);
                                   // [5] max |P|, [6] max |A| kept for the operand of key pkey, akey
    uint64_t pkey = 0, akey = 0;   // (a toolbox's serial: its P, and the G plane of P, never change)
    float* rcinv = nullptr;        // the FP16 update: 1 / s_i per row of A, 1 / t_j and max_k |B_kj| per column of B
    size_t rccap = 0;
    int* tiles = nullptr;          // (tile row, tile column) per CTA, blocked order
    long long tiles_key = -1;      // shape the table was made for
    int tiles_count = 0;
};
static Scratch g_scratch[64];

// Output tiles in blocks of kTileBlock x kTileBlock (about one wave of one-CTA-per-SM tiles), block
// rows in order: the CTAs that run together read kTileBlock row panels and kTileBlock column
// panels, which L2 then serves to the other CTAs of the block.  tri: only tiles with tx <= ty.
constexpr int kTileBlock = 12;
static ewos_status tile_table(Scratch& S, int mt, int nt, bool tri, cudaStream_t st, int* count) {
    const long long key = ((long long)mt << 32) ^ ((long long)nt << 1) ^ (tri ? 1 : 0);
    if (S.tiles && S.tiles_key == key) { *count = S.tiles_count; return EWOS_OK; }
    std::vector<int> t;
    for (int by = 0; by < mt; by += kTileBlock)
        for (int bx = 0; bx < nt; bx += kTileBlock) {
            if (tri && bx > by) break;
            for (int ty = by; ty < std::min(mt, by + kTileBlock); ++ty)
                for (int tx = bx; tx < std::min(nt, bx + kTileBlock); ++tx) {
                    if (tri && tx > ty) break;
                    t.push_back(ty);
                    t.push_back(tx);
                }
        }
    ::ewos::dev_free(S.tiles);
    S.tiles = nullptr;
    S.tiles_key = -1;
    EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.tiles, sizeof(int) * t.size()));
    EWOS_CUDA_TRY(cudaMemcpyAsync(S.tiles, t.data(), sizeof(int) * t.size(), cudaMemcpyHostToDevice, st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(st));
    S.tiles_key = key;
    S.tiles_count = (int)(t.size() / 2);
    *count = S.tiles_count;
    return EWOS_OK;
}
static std::mutex g_mu;

// operand elements per chunk of the two-level accumulation (gemm_drain_kernel)
#ifndef EWOS_DRAIN_ELEMS
#define EWOS_DRAIN_ELEMS 256
#endif

template <bool F16>
static ewos_status launch_drain(Scratch& S, const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mal,
                                const CUtensorMap& mbl, int M, int N, int Kp, float* C, int64_t ldc, bool tri,
                                int ntiles, const float* cscale, cudaStream_t st) {
    using CF = Cfg<true, 0, F16>;
    auto k = gemm_drain_kernel<F16>;
    EWOS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM_BYTES));
    const int dk = EWOS_DRAIN_ELEMS / CF::KSTAGE > 0 ? EWOS_DRAIN_ELEMS / CF::KSTAGE : 1;
    ::ewos::note_launch(), k<<<ntiles, 192, CF::SMEM_BYTES, st>>>(ma, mb, mal, mbl, M, N, Kp, C, ldc, S.err, tri ? 1 : 0,
                                                                  S.tiles, cscale, dk);
    EWOS_CUDA_TRY(cudaGetLastError());
    return EWOS_OK;
}

}  // namespace tc

bool tc_assemble_available() {
    static int avail = -1;
    if (avail < 0) {
        int dev = 0, major = 0, minor = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        avail = (major == 10 && tc::encode_fn() != nullptr) ? 1 : 0;
    }
    return avail == 1;
}

// C [M][N] = A^T B for A = P [K][M] and B = Q [K][N], both FP32 row-major, on the tensor cores:
// split = false: TF32 inputs (relative error about 2^-11 per product); split = true: 3xTF32
// (about 2^-21), three MMAs per step.
// Scratch of one caller (a solve workspace): operand transposes and the error word.
struct TcScratch {
    tc::Scratch s;
};

void tc_scratch_free(TcScratch* t) {
    if (!t) return;
    ::ewos::dev_free(t->s.At); ::ewos::dev_free(t->s.Bt); ::ewos::dev_free(t->s.Atl); ::ewos::dev_free(t->s.Btl);
    ::ewos::dev_free(t->s.err); ::ewos::dev_free(t->s.tiles); ::ewos::dev_free(t->s.scale); ::ewos::dev_free(t->s.rcinv);
    delete t;
}

// Enqueues the transposes and the GEMM on st; the pipeline-timeout word is left in *err_dev
// for the caller to check after the stream has run (no host synchronisation here).
// scale[0] = max |A|, scale[1] = max |B| over na and nb values (the FP16 form of tc_enqueue)
__global__ void absmax2_kernel(const float* __restrict__ A, int64_t na, const float* __restrict__ B, int64_t nb,
                               float* __restrict__ scale) {
    float ma = 0.f, mb = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < na; t += stride) ma = fmaxf(ma, fabsf(A[t]));
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nb; t += stride) mb = fmaxf(mb, fabsf(B[t]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
        mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(reinterpret_cast<unsigned int*>(scale), __float_as_uint(ma));       // (non-negative floats)
        atomicMax(reinterpret_cast<unsigned int*>(scale + 1), __float_as_uint(mb));
    }
}

// powers of two s_A, s_B with max |A| s_A and max |B| s_B in [2^13, 2^14), and 1 / (s_A s_B);
// max |A| from scale[0], or from the kept scale[6] (cached), and kept there (keep).  With bprod,
// B = diag(d) A and scale[1] holds max |d|: max |B| is bounded by max |A| max |d| (a bound keeps
// every scaled value below 2^14)
__global__ void ab_scale_kernel(float* scale, int cached, int keep, int bprod = 0) {
    if (threadIdx.x != 0) return;
    if (cached) scale[0] = scale[6];
    else if (keep) scale[6] = scale[0];
    if (bprod) scale[1] = scale[0] * scale[1] * 1.0001f;
    auto pw = [](float mxv) {
        if (!(mxv > 0.f) || !isfinite(mxv)) return 1.0f;
        int e;
        frexpf(mxv, &e);
        return ldexpf(1.0f, 14 - e);
    };
    const float sa = pw(scale[0]), sb = pw(scale[1]);
    scale[2] = sa;
    scale[3] = sb;
    scale[4] = 1.0f / (sa * sb);
}

__device__ __forceinline__ void f16_split_tc(float v, __half& h, __half& l) {
    h = __float2half_rn(v);
    l = __float2half_rn(v - __half2float(h));
}

// hi/lo [C][Kp] halves of both s_A in^T and s_B (diag(d) in)^T for in [K][C] FP32 (row-major),
// d [K]: the operands of G^T diag(d) G from one read of G (the product d_k g in FP32, as a
// scaled copy of G would hold it); zero padding k in [K, Kp)
__global__ void transpose_split16_ab_kernel(const float* __restrict__ in, const float* __restrict__ d, int K, int Ccols,
                                            __half* __restrict__ ahi, __half* __restrict__ alo, __half* __restrict__ bhi,
                                            __half* __restrict__ blo, int Kp, const float* __restrict__ scale) {
    __shared__ float tile[32][33];
    __shared__ float dk[32];
    const float sa = scale[2], sb = scale[3];
    const int c0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int k = k0 + r, c = c0 + threadIdx.x;
        tile[r][threadIdx.x] = (k < K && c < Ccols) ? in[(int64_t)k * Ccols + c] : 0.f;
    }
    if (threadIdx.y == 0) dk[threadIdx.x] = k0 + (int)threadIdx.x < K ? d[k0 + threadIdx.x] : 0.f;
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int c = c0 + r, k = k0 + threadIdx.x;
        if (c < Ccols && k < Kp) {
            const float v = tile[threadIdx.x][r];
            __half h, l;
            f16_split_tc(v * sa, h, l);
            ahi[(int64_t)c * Kp + k] = h;
            alo[(int64_t)c * Kp + k] = l;
            f16_split_tc((dk[threadIdx.x] * v) * sb, h, l);
            bhi[(int64_t)c * Kp + k] = h;
            blo[(int64_t)c * Kp + k] = l;
        }
    }
}

// hi/lo [C][Kp] halves of s * in^T for in [K][C] FP32 (row-major), zero padding k in [K, Kp);
// s = scale[which]
__global__ void transpose_split16_kernel(const float* __restrict__ in, int K, int Ccols, __half* __restrict__ hi,
                                         __half* __restrict__ lo, int Kp, const float* __restrict__ scale, int which) {
    __shared__ float tile[32][33];
    const float sc = scale[which];
    const int c0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int k = k0 + r, c = c0 + threadIdx.x;
        tile[r][threadIdx.x] = (k < K && c < Ccols) ? in[(int64_t)k * Ccols + c] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int c = c0 + r, k = k0 + threadIdx.x;
        if (c < Ccols && k < Kp) {
            __half h, l;
            f16_split_tc(tile[threadIdx.x][r] * sc, h, l);
            hi[(int64_t)c * Kp + k] = h;
            lo[(int64_t)c * Kp + k] = l;
        }
    }
}

// the power of two s with mx s in [2^13, 2^14) (1 for a zero or non-finite mx; at most 2^127)
__device__ __forceinline__ float pow2_scale(float mx) {
    if (!(mx > 0.f) || !isfinite(mx)) return 1.0f;
    int e;
    frexpf(mx, &e);
    return ldexpf(1.0f, min(14 - e, 127));
}

// FP16 halves [M][Kp] of s_i A_i for a row-major A [M][K] (row stride ld), s_i the power of two
// that puts max_k |A_ik| in [2^13, 2^14); rinv[i] = 1 / s_i; zero padding k in [K, Kp).  One warp
// per row (the LU's update operand: rows of the L block, K = the update's rank).
__global__ void rows_split16_kernel(const float* __restrict__ in, int64_t ld, int M, int K, __half* __restrict__ hi,
                                    __half* __restrict__ lo, int Kp, float* __restrict__ rinv) {
    ::ewos::pdl_trigger();
    ::ewos::pdl_wait();
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= M) return;
    const float* a = in + (int64_t)i * ld;
    float mx = 0.f;
    for (int k = lane; k < K; k += 32) mx = fmaxf(mx, fabsf(a[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float s = pow2_scale(mx);
    __half2* h2 = reinterpret_cast<__half2*>(hi + (int64_t)i * Kp);
    __half2* l2 = reinterpret_cast<__half2*>(lo + (int64_t)i * Kp);
    for (int k = 2 * lane; k < Kp; k += 64) {       // (Kp is even: 4-byte pairs)
        __half h0, l0, h1, l1;
        f16_split_tc(k < K ? a[k] * s : 0.f, h0, l0);
        f16_split_tc(k + 1 < K ? a[k + 1] * s : 0.f, h1, l1);
        h2[k >> 1] = __halves2half2(h0, h1);
        l2[k >> 1] = __halves2half2(l0, l1);
    }
    if (lane == 0) rinv[i] = 1.0f / s;
}

// cmax[j] = max_k |B_kj| for a row-major B [K][N] (row stride ld), as the bits of non-negative
// floats (cmax zeroed first); 32 x 32 tiles, one atomic per column and tile
__global__ void cols_absmax_kernel(const float* __restrict__ in, int64_t ld, int K, int N, float* __restrict__ cmax) {
    __shared__ float red[8][32];
    ::ewos::pdl_trigger();
    ::ewos::pdl_wait();
    const int c = blockIdx.x * 32 + threadIdx.x, k0 = blockIdx.y * 32;
    float mx = 0.f;
    if (c < N)
        for (int r = threadIdx.y; r < 32; r += blockDim.y)
            if (k0 + r < K) mx = fmaxf(mx, fabsf(in[(int64_t)(k0 + r) * ld + c]));
    red[threadIdx.y][threadIdx.x] = mx;
    __syncthreads();
    if (threadIdx.y == 0 && c < N) {
        for (int r = 1; r < (int)blockDim.y; ++r) mx = fmaxf(mx, red[r][threadIdx.x]);
        atomicMax(reinterpret_cast<unsigned int*>(cmax + c), __float_as_uint(mx));
    }
}

// FP16 halves [N][Kp] of t_j B_j for the columns of a row-major B [K][N] (row stride ld), t_j the
// power of two that puts cmax[j] = max_k |B_kj| in [2^13, 2^14); cinv[j] = 1 / t_j; zero padding
// k in [K, Kp).  32 x 32 tiles transposed through shared memory.
__global__ void cols_split16_kernel(const float* __restrict__ in, int64_t ld, int K, int N, __half* __restrict__ hi,
                                    __half* __restrict__ lo, int Kp, const float* __restrict__ cmax,
                                    float* __restrict__ cinv) {
    __shared__ float tile[32][33];
    __shared__ float sc[32];
    ::ewos::pdl_trigger();
    ::ewos::pdl_wait();
    const int c0 = blockIdx.x * 32, k0 = blockIdx.y * 32, c = c0 + threadIdx.x;
    if (threadIdx.y == 0) {
        const float t = pow2_scale(c < N ? cmax[c] : 0.f);
        sc[threadIdx.x] = t;
        if (blockIdx.y == 0 && c < N) cinv[c] = 1.0f / t;
    }
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int k = k0 + r;
        tile[r][threadIdx.x] = (k < K && c < N) ? in[(int64_t)k * ld + c] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int cc = c0 + r, k = k0 + threadIdx.x;
        if (cc < N && k < Kp) {
            __half h, l;
            f16_split_tc(tile[threadIdx.x][r] * sc[r], h, l);
            hi[(int64_t)cc * Kp + k] = h;
            lo[(int64_t)cc * Kp + k] = l;
        }
    }
}

static ewos_status tc_enqueue(tc::Scratch& S, const float* Akm, const float* Bkm, float* C, int M, int N, int K,
                              cudaStream_t st, bool split, bool sym = false) {
    using namespace tc;
    const int Kp = (K + BK - 1) / BK * BK;
    const size_t need = (size_t)std::max(M, N) * Kp;
    if (S.cap < need || (split && !S.Atl)) {
        ::ewos::dev_free(S.At); ::ewos::dev_free(S.Bt); ::ewos::dev_free(S.Atl); ::ewos::dev_free(S.Btl);
        S.At = S.Bt = S.Atl = S.Btl = nullptr;
        S.cap = 0;
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.At, sizeof(float) * need));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Bt, sizeof(float) * need));
        if (split) {
            EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Atl, sizeof(float) * need));
            EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Btl, sizeof(float) * need));
        }
        S.cap = need;
    }
    if (!S.err) EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.err, sizeof(int)));
    dim3 tb(32, 8);
    if (split) {
        ::ewos::note_launch(), transpose_split_kernel<<<dim3((M + 31) / 32, (Kp + 31) / 32), tb, 0, st>>>(Akm, K, M, S.At, S.Atl, Kp);
        ::ewos::note_launch(), transpose_split_kernel<<<dim3((N + 31) / 32, (Kp + 31) / 32), tb, 0, st>>>(Bkm, K, N, S.Bt, S.Btl, Kp);
    } else {
        ::ewos::note_launch(), transpose_pad_kernel<<<dim3((M + 31) / 32, (Kp + 31) / 32), tb, 0, st>>>(Akm, K, M, S.At, Kp);
        ::ewos::note_launch(), transpose_pad_kernel<<<dim3((N + 31) / 32, (Kp + 31) / 32), tb, 0, st>>>(Bkm, K, N, S.Bt, Kp);
    }
    const int bn = split ? Cfg<true>::BN : Cfg<false>::BN;
    CUtensorMap ma, mb, mal, mbl;
    bool ok = make_map(&ma, S.At, M, Kp, BM) && make_map(&mb, S.Bt, N, Kp, bn);
    if (split) ok = ok && make_map(&mal, S.Atl, M, Kp, BM) && make_map(&mbl, S.Btl, N, Kp, bn);
    else { mal = ma; mbl = mb; }
    if (!ok) {
        set_error("tensor-core assembly: cuTensorMapEncodeTiled failed");
        return EWOS_ECUDA;
    }
    EWOS_CUDA_TRY(cudaMemsetAsync(S.err, 0, sizeof(int), st));
    dim3 grid((N + bn - 1) / bn, (M + BM - 1) / BM);
    if (split) {
        const bool tri = sym && M == N;
        int ntiles = 0;
        if (ewos_status ts = tile_table(S, (M + BM - 1) / BM, (N + bn - 1) / bn, tri, st, &ntiles); ts != EWOS_OK)
            return ts;
        if (ewos_status ls = launch_drain<false>(S, ma, mb, mal, mbl, M, N, Kp, C, N, tri, ntiles, nullptr, st);
            ls != EWOS_OK)
            return ls;
    } else {
        EWOS_CUDA_TRY(cudaFuncSetAttribute(gemm_tf32_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<false>::SMEM_BYTES));
        ::ewos::note_launch(), gemm_tf32_kernel<false><<<grid, 128, Cfg<false>::SMEM_BYTES, st>>>(ma, mb, mal, mbl, M, N, Kp, C, N, S.err, 0);
    }
    EWOS_CUDA_TRY(cudaGetLastError());
    return EWOS_OK;
}

// The FP16 form of tc_enqueue's split product (C = A^T B, FP32 operands scaled by powers of two
// and split into FP16 halves, three kind::f16 products, unscaled in the epilogue): twice the TF32
// rate; as accurate as the TF32 split while max |A| and max |B| do not exceed the other entries
// by more than about 2^17 (below that an entry keeps an absolute error of 2^-39 of the largest).
// dscale: B = diag(dscale) A (K values; Bkm unused, N = M): both operands from one pass over A
static ewos_status tc_enqueue16(tc::Scratch& S, const float* Akm, const float* Bkm, float* C, int M, int N, int K,
                                cudaStream_t st, bool sym, uint64_t akey = 0, const float* dscale = nullptr,
                                const float* amax = nullptr) {
    using namespace tc;
    using CF = Cfg<true, 0, true>;
    const int Kp = (K + 2 * BK - 1) / (2 * BK) * (2 * BK);
    const size_t need_f = ((size_t)std::max(M, N) * Kp + 1) / 2;
    if (S.cap < need_f || !S.Atl) {
        ::ewos::dev_free(S.At); ::ewos::dev_free(S.Bt); ::ewos::dev_free(S.Atl); ::ewos::dev_free(S.Btl);
        S.At = S.Bt = S.Atl = S.Btl = nullptr;
        S.cap = 0;
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.At, sizeof(float) * need_f));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Bt, sizeof(float) * need_f));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Atl, sizeof(float) * need_f));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Btl, sizeof(float) * need_f));
        S.cap = need_f;
    }
    if (!S.err) EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.err, sizeof(int)));
    if (!S.scale) EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.scale, sizeof(float) * 8));
    __half* at = reinterpret_cast<__half*>(S.At);
    __half* atl = reinterpret_cast<__half*>(S.Atl);
    __half* bt = reinterpret_cast<__half*>(S.Bt);
    __half* btl = reinterpret_cast<__half*>(S.Btl);
    // max |A| is kept between calls for the same operand (akey: the toolbox's serial), or given
    // (amax, on the device)
    if (amax) {
        EWOS_CUDA_TRY(cudaMemcpyAsync(S.scale + 6, amax, sizeof(float), cudaMemcpyDeviceToDevice, st));
        S.akey = akey;
    }
    const bool acached = amax != nullptr || (akey != 0 && S.akey == akey);
    EWOS_CUDA_TRY(cudaMemsetAsync(S.scale, 0, sizeof(float) * 5, st));
    ::ewos::note_launch(), absmax2_kernel<<<4 * 148, 256, 0, st>>>(Akm, acached ? 0 : (int64_t)K * M,
                                                                  dscale ? dscale : Bkm, dscale ? (int64_t)K : (int64_t)K * N,
                                                                  S.scale);
    ::ewos::note_launch(), ab_scale_kernel<<<1, 32, 0, st>>>(S.scale, acached ? 1 : 0, akey != 0 ? 1 : 0, dscale ? 1 : 0);
    if (akey != 0) S.akey = akey;
    const dim3 tb(32, 8);
    if (dscale) {
        ::ewos::note_launch(), transpose_split16_ab_kernel<<<dim3((M + 31) / 32, (Kp + 31) / 32), tb, 0, st>>>(
                                   Akm, dscale, K, M, at, atl, bt, btl, Kp, S.scale);
    } else {
        ::ewos::note_launch(), transpose_split16_kernel<<<dim3((M + 31) / 32, (Kp + 31) / 32), tb, 0, st>>>(Akm, K, M, at, atl,
                                                                                                         Kp, S.scale, 2);
        ::ewos::note_launch(), transpose_split16_kernel<<<dim3((N + 31) / 32, (Kp + 31) / 32), tb, 0, st>>>(Bkm, K, N, bt, btl,
                                                                                                         Kp, S.scale, 3);
    }
    EWOS_CUDA_TRY(cudaGetLastError());
    CUtensorMap ma, mb, mal, mbl;
    if (!(make_map16(&ma, at, M, Kp, BM) && make_map16(&mb, bt, N, Kp, CF::BN) && make_map16(&mal, atl, M, Kp, BM) &&
          make_map16(&mbl, btl, N, Kp, CF::BN))) {
        set_error("tensor-core assembly: cuTensorMapEncodeTiled failed");
        return EWOS_ECUDA;
    }
    EWOS_CUDA_TRY(cudaMemsetAsync(S.err, 0, sizeof(int), st));
    const bool tri = sym && M == N;
    int ntiles = 0;
    if (ewos_status ts = tile_table(S, (M + BM - 1) / BM, (N + CF::BN - 1) / CF::BN, tri, st, &ntiles); ts != EWOS_OK)
        return ts;
    return launch_drain<true>(S, ma, mb, mal, mbl, M, N, Kp, C, N, tri, ntiles, S.scale + 4, st);
}

static ewos_status tc_check(tc::Scratch& S, cudaStream_t st) {
    int herr = 0;
    cudaError_t e = cudaMemcpyAsync(&herr, S.err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess || herr) S.pkey = S.akey = 0;      // the kept maxima may not have been written
    EWOS_CUDA_TRY(e);
    if (herr) {
        set_error("tensor-core assembly: a pipeline wait timed out");
        return EWOS_ETIMEOUT;
    }
    return EWOS_OK;
}

// Operands of Lambda = P^T Q, Q = M P, in one pass over P: P is [(d+1)][n][m] (row k = l n + i
// of the K x m operand is P[l][i][:]), M [n][d+1][d+1] the per-node coefficient blocks.  A tile
// of 32 nodes x 32 columns of every P[l] is read once into shared memory; the kernel writes the
// K-major split operands At/Atl [m][Kp] (from P) and Bt/Btl [m][Kp] (from Q, formed in FP32 as
// Q[j][i][c] = sum_l M_i[j][l] P[l][i][c]), k = l n + i.
template <int E>
__global__ void pq_split_kernel(const float* __restrict__ P, const double* __restrict__ M, int n, int m,
                                float* __restrict__ at, float* __restrict__ atl, float* __restrict__ bt,
                                float* __restrict__ btl, int Kp) {
    __shared__ float Pt[E][32][33];
    __shared__ float Ms[32][E * E];
    ::ewos::pdl_trigger();
    ::ewos::pdl_wait();
    const int c0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const size_t nm = (size_t)n * m;
    for (int r = ty; r < 32; r += blockDim.y) {
        const int i = i0 + r, c = c0 + tx;
#pragma unroll
        for (int l = 0; l < E; ++l) Pt[l][r][tx] = (i < n && c < m) ? P[l * nm + (size_t)i * m + c] : 0.f;
    }
    for (int t = ty * 32 + tx; t < 32 * E * E; t += 32 * blockDim.y) {
        const int r = t / (E * E), q = t % (E * E);
        Ms[r][q] = i0 + r < n ? (float)M[(size_t)(i0 + r) * E * E + q] : 0.f;
    }
    __syncthreads();
    const int i = i0 + tx;
    if (i >= n) return;
    for (int cc = ty; cc < 32; cc += blockDim.y) {
        const int c = c0 + cc;
        if (c >= m) break;
        float pv[E];
#pragma unroll
        for (int l = 0; l < E; ++l) pv[l] = Pt[l][tx][cc];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            float qv = 0.f;
#pragma unroll
            for (int l = 0; l < E; ++l) qv = fmaf(Ms[tx][j * E + l], pv[l], qv);
            const size_t k = (size_t)j * n + i, o = (size_t)c * Kp + k;
            float h, lo;
            tf32_split(pv[j], h, lo);
            at[o] = h;
            atl[o] = lo;
            tf32_split(qv, h, lo);
            bt[o] = h;
            btl[o] = lo;
        }
    }
}

// The FP16 form of the assembly.  FP16 has the 11-bit significand of TF32 and twice its tensor-core
// rate, but a narrow exponent range, so P and Q enter scaled by powers of two s_P, s_Q that put
// their largest magnitudes in [2^13, 2^14); v s = h + l with h = fp16(v s) and l = fp16(v s - h),
// and the three products hi.hi + hi.lo + lo.hi are unscaled by 1 / (s_P s_Q) in the epilogue
// (exact).  Entries below 2^-3 after scaling keep an absolute error of 2^-25 (the low part is an
// FP16 subnormal there), 2^-39 of the largest entry.
__device__ __forceinline__ void f16_split(float v, __half& h, __half& l) {
    h = __float2half_rn(v);
    l = __float2half_rn(v - __half2float(h));
}

// scale[0] = max |P| over `count` values, scale[1] = max over the nodes of the largest row sum of |M_i|
__global__ void pq_absmax_kernel(const float* __restrict__ P, int64_t count, const double* __restrict__ M, int n,
                                 int E, float* __restrict__ scale) {
    float mx = 0.f;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
        mx = fmaxf(mx, fabsf(P[t]));
    float mm = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int j = 0; j < E; ++j) {
            double r = 0.0;
            for (int l = 0; l < E; ++l) r += fabs(M[(size_t)i * E * E + j * E + l]);
            mm = fmaxf(mm, (float)r);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(reinterpret_cast<unsigned int*>(scale), __float_as_uint(mx));       // (non-negative floats)
        atomicMax(reinterpret_cast<unsigned int*>(scale + 1), __float_as_uint(mm));
    }
}

// powers of two s_P, s_Q with max |P| s_P and max |Q| s_Q in [2^13, 2^14) (|Q| <= max |P| times the
// largest row sum of |M|, with a little room for the rounding of Q), and their inverse product;
// max |P| from scale[0], or from the kept scale[5] (cached), and kept there (keep)
__global__ void pq_scale_kernel(float* scale, int cached, int keep) {
    if (threadIdx.x != 0) return;
    if (cached) scale[0] = scale[5];
    else if (keep) scale[5] = scale[0];
    const float mp = scale[0], mq = scale[0] * scale[1] * 1.0001f;
    auto pw = [](float mxv) {
        if (!(mxv > 0.f) || !isfinite(mxv)) return 1.0f;
        int e;
        frexpf(mxv, &e);               // mxv in [2^(e-1), 2^e)
        return ldexpf(1.0f, 14 - e);
    };
    const float sp = pw(mp), sq = pw(mq);
    scale[2] = sp;
    scale[3] = sq;
    scale[4] = 1.0f / (sp * sq);
}

template <int E>
__global__ void pq_split16_kernel(const float* __restrict__ P, const double* __restrict__ M, int n, int m,
                                  __half* __restrict__ at, __half* __restrict__ atl, __half* __restrict__ bt,
                                  __half* __restrict__ btl, int Kp, const float* __restrict__ scale) {
    __shared__ float Pt[E][32][33];
    __shared__ float Ms[32][E * E];
    ::ewos::pdl_trigger();
    ::ewos::pdl_wait();
    const float sp = scale[2], sq = scale[3];
    const int c0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const size_t nm = (size_t)n * m;
    for (int r = ty; r < 32; r += blockDim.y) {
        const int i = i0 + r, c = c0 + tx;
#pragma unroll
        for (int l = 0; l < E; ++l) Pt[l][r][tx] = (i < n && c < m) ? P[l * nm + (size_t)i * m + c] : 0.f;
    }
    for (int t = ty * 32 + tx; t < 32 * E * E; t += 32 * blockDim.y) {
        const int r = t / (E * E), q = t % (E * E);
        Ms[r][q] = i0 + r < n ? (float)M[(size_t)(i0 + r) * E * E + q] : 0.f;
    }
    __syncthreads();
    const int i = i0 + tx;
    if (i >= n) return;
    for (int cc = ty; cc < 32; cc += blockDim.y) {
        const int c = c0 + cc;
        if (c >= m) break;
        float pv[E];
#pragma unroll
        for (int l = 0; l < E; ++l) pv[l] = Pt[l][tx][cc];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            float qv = 0.f;
#pragma unroll
            for (int l = 0; l < E; ++l) qv = fmaf(Ms[tx][j * E + l], pv[l], qv);
            const size_t k = (size_t)j * n + i, o = (size_t)c * Kp + k;
            __half h, lo;
            f16_split(pv[j] * sp, h, lo);
            at[o] = h;
            atl[o] = lo;
            f16_split(qv * sq, h, lo);
            bt[o] = h;
            btl[o] = lo;
        }
    }
}

// Lambda [m][m] = P^T Q with Q = M P, both operands prepared by pq_split_kernel, then the
// three-product TF32 GEMM; waits for the launch (pipeline timeouts are reported)
// The FP16 form of tc_assemble_pq (same operands in FP16 halves, twice the tensor-core rate)
static ewos_status tc_assemble_pq16(tc::Scratch& S, const float* P, const double* Mc, int n, int m, int D, float* C,
                                    cudaStream_t st, bool sym, uint64_t pkey = 0, const float* pmax = nullptr) {
    using namespace tc;
    const int E = D + 1, K = E * n;
    const int Kp = (K + 2 * BK - 1) / (2 * BK) * (2 * BK);          // halves, 128-byte rows
    const size_t need_f = ((size_t)m * Kp + 1) / 2;                   // floats of scratch per operand
    if (S.cap < need_f || !S.Atl) {
        ::ewos::dev_free(S.At); ::ewos::dev_free(S.Bt); ::ewos::dev_free(S.Atl); ::ewos::dev_free(S.Btl);
        S.At = S.Bt = S.Atl = S.Btl = nullptr;
        S.cap = 0;
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.At, sizeof(float) * need_f));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Bt, sizeof(float) * need_f));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Atl, sizeof(float) * need_f));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Btl, sizeof(float) * need_f));
        S.cap = need_f;
    }
    if (!S.err) EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.err, sizeof(int)));
    if (!S.scale) EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.scale, sizeof(float) * 8));
    __half* at = reinterpret_cast<__half*>(S.At);
    __half* atl = reinterpret_cast<__half*>(S.Atl);
    __half* bt = reinterpret_cast<__half*>(S.Bt);
    __half* btl = reinterpret_cast<__half*>(S.Btl);
    if (Kp > K) {   // zero padding of the reduction dimension
        for (__half* b : {at, atl, bt, btl})
            EWOS_CUDA_TRY(cudaMemset2DAsync(b + K, sizeof(__half) * Kp, 0, sizeof(__half) * (Kp - K), m, st));
    }
    // max |P| is kept between calls for the same toolbox (pkey: its serial), or given by the build
    // that wrote P (pmax, on the device)
    if (pmax) {
        EWOS_CUDA_TRY(cudaMemcpyAsync(S.scale + 5, pmax, sizeof(float), cudaMemcpyDeviceToDevice, st));
        S.pkey = pkey;
    }
    const bool pcached = pmax != nullptr || (pkey != 0 && S.pkey == pkey);
    EWOS_CUDA_TRY(cudaMemsetAsync(S.scale, 0, sizeof(float) * 5, st));
    if (E != 3 && E != 4) {
        set_error("tensor-core assembly: dimension must be 2 or 3");
        return EWOS_EINVAL;
    }
    ::ewos::note_launch(), pq_absmax_kernel<<<4 * 148, 256, 0, st>>>(P, pcached ? 0 : (int64_t)E * n * m, Mc, n, E, S.scale);
    ::ewos::note_launch(), pq_scale_kernel<<<1, 32, 0, st>>>(S.scale, pcached ? 1 : 0, pkey != 0 ? 1 : 0);
    if (pkey != 0) S.pkey = pkey;
    const dim3 grid((unsigned)((m + 31) / 32), (unsigned)((n + 31) / 32)), tb(32, 8);
    ::ewos::note_launch();
    if (E == 3) pq_split16_kernel<3><<<grid, tb, 0, st>>>(P, Mc, n, m, at, atl, bt, btl, Kp, S.scale);
    else if (E == 4) pq_split16_kernel<4><<<grid, tb, 0, st>>>(P, Mc, n, m, at, atl, bt, btl, Kp, S.scale);
    else {
        set_error("tensor-core assembly: dimension must be 2 or 3");
        return EWOS_EINVAL;
    }
    EWOS_CUDA_TRY(cudaGetLastError());
    using CF = Cfg<true, 0, true>;
    CUtensorMap ma, mb, mal, mbl;
    if (!(make_map16(&ma, at, m, Kp, BM) && make_map16(&mb, bt, m, Kp, CF::BN) && make_map16(&mal, atl, m, Kp, BM) &&
          make_map16(&mbl, btl, m, Kp, CF::BN))) {
        set_error("tensor-core assembly: cuTensorMapEncodeTiled failed");
        return EWOS_ECUDA;
    }
    EWOS_CUDA_TRY(cudaMemsetAsync(S.err, 0, sizeof(int), st));
    const int nt = (m + BM - 1) / BM;
    int ntiles = 0;
    if (ewos_status ts = tile_table(S, nt, (m + CF::BN - 1) / CF::BN, sym, st, &ntiles); ts != EWOS_OK) return ts;
    if (ewos_status ls = launch_drain<true>(S, ma, mb, mal, mbl, m, m, Kp, C, m, sym, ntiles, S.scale + 4, st); ls != EWOS_OK)
        return ls;
    return tc_check(S, st);
}

ewos_status tc_assemble_pq(const float* P, const double* Mc, int n, int m, int D, float* C, cudaStream_t st,
                           TcScratch** owned, bool sym = false, bool f16 = true, uint64_t pkey = 0,
                           const float* pmax = nullptr) {
    using namespace tc;
    if (!*owned) *owned = new TcScratch();
    Scratch& S = (*owned)->s;
    if (f16) return tc_assemble_pq16(S, P, Mc, n, m, D, C, st, sym, pkey, pmax);
    const int E = D + 1, K = E * n;
    const int Kp = (K + BK - 1) / BK * BK;
    const size_t need = (size_t)m * Kp;
    if (S.cap < need || !S.Atl) {
        ::ewos::dev_free(S.At); ::ewos::dev_free(S.Bt); ::ewos::dev_free(S.Atl); ::ewos::dev_free(S.Btl);
        S.At = S.Bt = S.Atl = S.Btl = nullptr;
        S.cap = 0;
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.At, sizeof(float) * need));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Bt, sizeof(float) * need));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Atl, sizeof(float) * need));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Btl, sizeof(float) * need));
        S.cap = need;
    }
    if (!S.err) EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.err, sizeof(int)));
    if (Kp > K) {   // zero padding of the reduction dimension
        for (float* b : {S.At, S.Atl, S.Bt, S.Btl})
            EWOS_CUDA_TRY(cudaMemset2DAsync(b + K, sizeof(float) * Kp, 0, sizeof(float) * (Kp - K), m, st));
    }
    const dim3 grid((unsigned)((m + 31) / 32), (unsigned)((n + 31) / 32)), tb(32, 8);
    ::ewos::note_launch();
    if (E == 3) pq_split_kernel<3><<<grid, tb, 0, st>>>(P, Mc, n, m, S.At, S.Atl, S.Bt, S.Btl, Kp);
    else if (E == 4) pq_split_kernel<4><<<grid, tb, 0, st>>>(P, Mc, n, m, S.At, S.Atl, S.Bt, S.Btl, Kp);
    else {
        set_error("tensor-core assembly: dimension must be 2 or 3");
        return EWOS_EINVAL;
    }
    EWOS_CUDA_TRY(cudaGetLastError());
    CUtensorMap ma, mb, mal, mbl;
    if (!(make_map(&ma, S.At, m, Kp, BM) && make_map(&mb, S.Bt, m, Kp, Cfg<true>::BN) && make_map(&mal, S.Atl, m, Kp, BM) &&
          make_map(&mbl, S.Btl, m, Kp, Cfg<true>::BN))) {
        set_error("tensor-core assembly: cuTensorMapEncodeTiled failed");
        return EWOS_ECUDA;
    }
    EWOS_CUDA_TRY(cudaMemsetAsync(S.err, 0, sizeof(int), st));
    const int nt = (m + BM - 1) / BM;
    static_assert(Cfg<true>::BN == BM, "square tiles for the symmetric launch");
    int ntiles = 0;
    if (ewos_status ts = tile_table(S, nt, (m + Cfg<true>::BN - 1) / Cfg<true>::BN, sym, st, &ntiles); ts != EWOS_OK)
        return ts;
    if (ewos_status ls = launch_drain<false>(S, ma, mb, mal, mbl, m, m, Kp, C, m, sym, ntiles, nullptr, st); ls != EWOS_OK)
        return ls;
    return tc_check(S, st);
}


// Allocates the update scratch for operands of up to max_mn rows and K = k on the calling
// thread's allocation stream (so a producer kernel can write the split operands into it).
ewos_status tc_update_reserve(int max_mn, int k, cudaStream_t st, TcScratch** owned) {
    using namespace tc;
    if (!*owned) *owned = new TcScratch();
    Scratch& S = (*owned)->s;
    const int Kp = (k + BK - 1) / BK * BK;
    const size_t need = (size_t)max_mn * Kp;
    if (S.cap < need || !S.Atl) {
        ::ewos::dev_free(S.At); ::ewos::dev_free(S.Bt); ::ewos::dev_free(S.Atl); ::ewos::dev_free(S.Btl);
        S.At = S.Bt = S.Atl = S.Btl = nullptr;
        S.cap = 0;
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.At, sizeof(float) * need));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Bt, sizeof(float) * need));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Atl, sizeof(float) * need));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Btl, sizeof(float) * need));
        S.cap = need;
    }
    if (!S.err) {
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.err, sizeof(int)));
        EWOS_CUDA_TRY(cudaMemsetAsync(S.err, 0, sizeof(int), st));
    }
    return EWOS_OK;
}

// The operand buffers of the update, in the layout tc_update_enqueue reads with presplit set:
// A hi/lo [M][Kp] (row i of A), B hi/lo [N][Kp] (column j of B), Kp = K rounded up to 32.
void tc_update_operands(TcScratch* t, float** a_hi, float** a_lo, float** b_hi, float** b_lo) {
    *a_hi = t->s.At; *a_lo = t->s.Atl; *b_hi = t->s.Bt; *b_lo = t->s.Btl;
}

// The FP16 form of tc_update_enqueue (operands split here, one scale per row of A and column of B;
// the persistent gemm_upd16_kernel)
static ewos_status tc_update_enqueue16(tc::Scratch& S, const float* A, int64_t lda, const float* B, int64_t ldb,
                                       float* C, int64_t ldc, int M, int N, int K, cudaStream_t st) {
    using namespace tc;
    using CF = Cfg<true, 0, true>;
    const int Kp = (K + 2 * BK - 1) / (2 * BK) * (2 * BK);
    const size_t need_f = ((size_t)std::max(M, N) * Kp + 1) / 2;     // halves, in floats
    if (S.cap < need_f || !S.Atl) {
        ::ewos::dev_free(S.At); ::ewos::dev_free(S.Bt); ::ewos::dev_free(S.Atl); ::ewos::dev_free(S.Btl);
        S.At = S.Bt = S.Atl = S.Btl = nullptr;
        S.cap = 0;
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.At, sizeof(float) * need_f));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Bt, sizeof(float) * need_f));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Atl, sizeof(float) * need_f));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Btl, sizeof(float) * need_f));
        S.cap = need_f;
    }
    if (S.rccap < (size_t)M + 2 * (size_t)N) {
        ::ewos::dev_free(S.rcinv);
        S.rcinv = nullptr;
        S.rccap = 0;
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.rcinv, sizeof(float) * ((size_t)M + 2 * (size_t)N)));
        S.rccap = (size_t)M + 2 * (size_t)N;
    }
    if (!S.err) {
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.err, sizeof(int)));
        EWOS_CUDA_TRY(cudaMemsetAsync(S.err, 0, sizeof(int), st));
    }
    __half* at = reinterpret_cast<__half*>(S.At);
    __half* atl = reinterpret_cast<__half*>(S.Atl);
    __half* bt = reinterpret_cast<__half*>(S.Bt);
    __half* btl = reinterpret_cast<__half*>(S.Btl);
    float* rinv = S.rcinv;
    float* cinv = S.rcinv + M;
    float* cmax = S.rcinv + M + N;
    EWOS_CUDA_TRY(cudaMemsetAsync(cmax, 0, sizeof(float) * N, st));
    ::ewos::note_launch();
    EWOS_CUDA_TRY(::ewos::launch_pdl(rows_split16_kernel, dim3((unsigned)((M + 7) / 8)), dim3(256), 0, st, A, lda, M, K, at,
                                     atl, Kp, rinv));
    ::ewos::note_launch();
    EWOS_CUDA_TRY(::ewos::launch_pdl(cols_absmax_kernel, dim3((unsigned)((N + 31) / 32), (unsigned)((K + 31) / 32)),
                                     dim3(32, 8), 0, st, B, ldb, K, N, cmax));
    ::ewos::note_launch();
    EWOS_CUDA_TRY(::ewos::launch_pdl(cols_split16_kernel, dim3((unsigned)((N + 31) / 32), (unsigned)(Kp / 32)), dim3(32, 8),
                                     0, st, B, ldb, K, N, bt, btl, Kp, (const float*)cmax, cinv));
    CUtensorMap ma, mb, mal, mbl;
    if (!(make_map16(&ma, at, M, Kp, BM) && make_map16(&mb, bt, N, Kp, CF::BN) && make_map16(&mal, atl, M, Kp, BM) &&
          make_map16(&mbl, btl, N, Kp, CF::BN))) {
        set_error("tensor-core update: cuTensorMapEncodeTiled failed");
        return EWOS_ECUDA;
    }
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    static int nsm = 0;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(gemm_upd16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM_BYTES);
        int dev = 0;
        if (attr == cudaSuccess) attr = cudaGetDevice(&dev);
        if (attr == cudaSuccess) attr = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    });
    EWOS_CUDA_TRY(attr);
    const int ntiles = ((M + BM - 1) / BM) * ((N + CF::BN - 1) / CF::BN);
    const int grid = std::max(1, std::min(ntiles, nsm));
    ::ewos::note_launch();
    EWOS_CUDA_TRY(::ewos::launch_pdl(gemm_upd16_kernel, dim3(grid), dim3(192), (size_t)CF::SMEM_BYTES, st, ma, mb, mal, mbl,
                                     M, N, Kp, C, ldc, S.err, (const float*)rinv, (const float*)cinv));
    return EWOS_OK;
}

// C [M][N] (row stride ldc) -= A B for a row-major A [M][K] (stride lda) and B [K][N] (stride
// ldb): the LU's trailing update on the tensor cores (three TF32 products).  With presplit the
// operands are already in the scratch (tc_update_operands; A and B are not read), starting at
// operand row a_off of A and b_off of B.  Otherwise, with f16, the rows of A and the columns of B
// are scaled by powers of two (s_i, t_j: the largest entry of each in [2^13, 2^14)) and split into
// FP16 halves, three kind::f16 products at twice the TF32 rate, unscaled by 1 / (s_i t_j) in the
// epilogue: an entry x keeps about 22 bits, or an absolute error of 2^-38 of its row's (column's)
// largest, like the TF32 halves.  Enqueued only; a pipeline timeout sets the scratch's error
// word, which tc_update_check reads (and clears).
ewos_status tc_update_enqueue(const float* A, int64_t lda, const float* B, int64_t ldb, float* C, int64_t ldc, int M,
                              int N, int K, cudaStream_t st, TcScratch** owned, bool presplit, int a_off, int b_off,
                              bool f16) {
    using namespace tc;
    if (!*owned) *owned = new TcScratch();
    Scratch& S = (*owned)->s;
    if (!presplit && f16) return tc_update_enqueue16(S, A, lda, B, ldb, C, ldc, M, N, K, st);
    const int Kp = (K + BK - 1) / BK * BK;
    const size_t need = (size_t)std::max(M, N) * Kp;
    if (!presplit) a_off = b_off = 0;
    if (presplit && (S.cap < (size_t)std::max(a_off + M, b_off + N) * Kp || !S.Atl || !S.err || a_off < 0 || b_off < 0)) {
        set_error("tensor-core update: split operands expected in a scratch that is too small");
        return EWOS_EINVAL;
    }
    if (S.cap < need || !S.Atl) {
        ::ewos::dev_free(S.At); ::ewos::dev_free(S.Bt); ::ewos::dev_free(S.Atl); ::ewos::dev_free(S.Btl);
        S.At = S.Bt = S.Atl = S.Btl = nullptr;
        S.cap = 0;
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.At, sizeof(float) * need));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Bt, sizeof(float) * need));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Atl, sizeof(float) * need));
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.Btl, sizeof(float) * need));
        S.cap = need;
    }
    if (!S.err) {
        EWOS_CUDA_TRY(::ewos::dev_alloc((void**)&S.err, sizeof(int)));
        EWOS_CUDA_TRY(cudaMemsetAsync(S.err, 0, sizeof(int), st));
    }
    if (!presplit) {
        const int64_t na = (int64_t)M * Kp;
        ::ewos::note_launch();
        EWOS_CUDA_TRY(::ewos::launch_pdl(rows_split_kernel, dim3((unsigned)((na + 255) / 256)), dim3(256), 0, st, A, lda,
                                         M, K, S.At, S.Atl, Kp));
        ::ewos::note_launch();
        EWOS_CUDA_TRY(::ewos::launch_pdl(cols_split_kernel, dim3((N + 31) / 32, (Kp + 31) / 32), dim3(32, 8), 0, st, B,
                                         ldb, K, N, S.Bt, S.Btl, Kp));
    }
    constexpr int bn = Cfg<true>::BN;
    CUtensorMap ma, mb, mal, mbl;
    const size_t ao = (size_t)a_off * Kp, bo = (size_t)b_off * Kp;
    if (!(make_map(&ma, S.At + ao, M, Kp, BM) && make_map(&mb, S.Bt + bo, N, Kp, bn) &&
          make_map(&mal, S.Atl + ao, M, Kp, BM) && make_map(&mbl, S.Btl + bo, N, Kp, bn))) {
        set_error("tensor-core update: cuTensorMapEncodeTiled failed");
        return EWOS_ECUDA;
    }
    // K = 64 needs two ring stages; the shared memory left holds the C tile (when C's rows start
    // on 16-byte boundaries), fetched under the main loop instead of by the epilogue
    constexpr int kUpd = 2;
    constexpr size_t kCsmSmem = (size_t)Cfg<true, kUpd>::SMEM_BYTES + kCsmBytes;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(gemm_tf32_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<true>::SMEM_BYTES);
        if (attr == cudaSuccess)
            attr = cudaFuncSetAttribute(gemm_tf32_kernel<true, kUpd, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kCsmSmem);
    });
    EWOS_CUDA_TRY(attr);
    dim3 grid((N + bn - 1) / bn, (M + BM - 1) / BM);
    const bool csm = Kp <= kUpd * BK && (ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0;
    ::ewos::note_launch();
    if (csm)
        EWOS_CUDA_TRY(::ewos::launch_pdl(gemm_tf32_kernel<true, kUpd, true>, grid, dim3(128), kCsmSmem, st, ma, mb, mal, mbl,
                                         M, N, Kp, C, ldc, S.err, 1, 0, (const int*)nullptr, (const float*)nullptr, -1));
    else
        EWOS_CUDA_TRY(::ewos::launch_pdl(gemm_tf32_kernel<true>, grid, dim3(128), (size_t)Cfg<true>::SMEM_BYTES, st, ma, mb,
                                         mal, mbl, M, N, Kp, C, ldc, S.err, 1, 0, (const int*)nullptr, (const float*)nullptr, -1));
    return EWOS_OK;
}

// The two rank-64 updates of a panel in one launch, on the operands the panel kernel split
// (tc_update_operands, rows from 0): with C the block right of and below the diagonal block (rest
// x rest, row stride ldc), C[0, band) x [0, rest) and C[band, rest) x [0, band) -= A B, the rows
// of the super panel's later panels across every column and the rows below it across the super
// panel's later columns (the rest of C waits for the super panel's rank-512 update).
ewos_status tc_update_lshape_enqueue(float* C, int64_t ldc, int rest, int band, int K, cudaStream_t st,
                                     TcScratch** owned) {
    using namespace tc;
    if (!*owned) *owned = new TcScratch();
    Scratch& S = (*owned)->s;
    const int Kp = (K + BK - 1) / BK * BK;
    constexpr int kUpd = 2;
    constexpr int bn = Cfg<true>::BN;
    if (rest <= 0 || band <= 0 || band > rest || S.cap < (size_t)rest * Kp || !S.Atl || !S.err || Kp > kUpd * BK ||
        (ldc & 3) != 0 || (reinterpret_cast<uintptr_t>(C) & 15) != 0) {
        set_error("tensor-core update: L-shaped update outside its preconditions");
        return EWOS_EINVAL;
    }
    CUtensorMap ma, mb, mal, mbl;
    if (!(make_map(&ma, S.At, rest, Kp, BM) && make_map(&mb, S.Bt, rest, Kp, bn) && make_map(&mal, S.Atl, rest, Kp, BM) &&
          make_map(&mbl, S.Btl, rest, Kp, bn))) {
        set_error("tensor-core update: cuTensorMapEncodeTiled failed");
        return EWOS_ECUDA;
    }
    constexpr size_t kCsmSmem = (size_t)Cfg<true, kUpd>::SMEM_BYTES + kCsmBytes;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(gemm_tf32_kernel<true, kUpd, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kCsmSmem);
    });
    EWOS_CUDA_TRY(attr);
    const int t1 = ((band + BM - 1) / BM) * ((rest + bn - 1) / bn);
    const int t2 = ((rest - band + BM - 1) / BM) * ((band + bn - 1) / bn);
    ::ewos::note_launch();
    EWOS_CUDA_TRY(::ewos::launch_pdl(gemm_tf32_kernel<true, kUpd, true>, dim3((unsigned)(t1 + t2)), dim3(128), kCsmSmem, st,
                                     ma, mb, mal, mbl, rest, rest, Kp, C, ldc, S.err, 1, 0, (const int*)nullptr,
                                     (const float*)nullptr, band));
    return EWOS_OK;
}

ewos_status tc_update_check(TcScratch* t, cudaStream_t st) {
    if (!t || !t->s.err) return EWOS_OK;
    int herr = 0;
    EWOS_CUDA_TRY(cudaMemcpyAsync(&herr, t->s.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    EWOS_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr) {
        cudaMemsetAsync(t->s.err, 0, sizeof(int), st);
        set_error("tensor-core update: a pipeline wait timed out");
        return EWOS_ETIMEOUT;
    }
    return EWOS_OK;
}

// C [M][N] = A^T B for K-major FP32 operands A [K][M], B [K][N].  With a caller scratch the
// call is reentrant across workspaces; without one the per-device scratch is used under a lock.
ewos_status tc_assemble(const float* Akm, const float* Bkm, float* C, int M, int N, int K, cudaStream_t st,
                        bool split, TcScratch** owned, bool sym = false, bool f16 = false, uint64_t akey = 0,
                        const float* dscale = nullptr, const float* amax = nullptr) {
    if (dscale && (!f16 || M != N)) {
        set_error("tensor-core product: the row-scaled form needs the FP16 split and a square result");
        return EWOS_EINVAL;
    }
    int dev = 0;
    EWOS_CUDA_TRY(cudaGetDevice(&dev));
    if (owned) {
        if (!*owned) *owned = new TcScratch();
        ewos_status s = f16 ? tc_enqueue16((*owned)->s, Akm, Bkm, C, M, N, K, st, sym, akey, dscale, amax)
                            : tc_enqueue((*owned)->s, Akm, Bkm, C, M, N, K, st, split, sym);
        if (s != EWOS_OK) return s;
        return tc_check((*owned)->s, st);
    }
    std::lock_guard<std::mutex> lock(tc::g_mu);
    tc::Scratch& S = tc::g_scratch[dev & 63];
    ewos_status s = f16 ? tc_enqueue16(S, Akm, Bkm, C, M, N, K, st, sym, akey, dscale, amax)
                        : tc_enqueue(S, Akm, Bkm, C, M, N, K, st, split, sym);
    if (s != EWOS_OK) return s;
    return tc_check(S, st);
}

}  // namespace ewos

// Test hook (no counterpart in the paper): C [M][N] = A^T B with A [K][M], B [K][N] host FP32
// arrays, through the tensor-core path used by the mixed-precision assembly; split = 2 takes the
// symmetric launch (tiles on and below the diagonal, mirrored; for a symmetric A^T B).
extern "C" ewos_status ewos_debug_tc_gemm(const float* A, const float* B, float* C, int M, int N, int K, int split) {
    using namespace ewos;
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || split < 0 || split > 4) {
        set_error("ewos_debug_tc_gemm: bad arguments");
        return EWOS_EINVAL;
    }
    if (!tc_assemble_available()) { set_error("tensor cores (sm_100 family) not available"); return EWOS_EINVAL; }
    AllocStream as(nullptr);
    float *dA = nullptr, *dB = nullptr, *dC = nullptr;
    EWOS_CUDA_TRY(dev_alloc((void**)&dA, sizeof(float) * (size_t)K * M));
    EWOS_CUDA_TRY(dev_alloc((void**)&dB, sizeof(float) * (size_t)K * N));
    EWOS_CUDA_TRY(dev_alloc((void**)&dC, sizeof(float) * (size_t)M * N));
    cudaMemcpy(dA, A, sizeof(float) * (size_t)K * M, cudaMemcpyHostToDevice);
    cudaMemcpy(dB, B, sizeof(float) * (size_t)K * N, cudaMemcpyHostToDevice);
    ewos_status s = tc_assemble(dA, dB, dC, M, N, K, nullptr, split != 0, nullptr, split == 2 || split == 4, split >= 3);
    if (s == EWOS_OK && cudaMemcpy(C, dC, sizeof(float) * (size_t)M * N, cudaMemcpyDeviceToHost) != cudaSuccess) s = EWOS_ECUDA;
    dev_free(dA); dev_free(dB); dev_free(dC);
    cudaDeviceSynchronize();
    return s;
}

extern "C" ewos_status ewos_debug_tc_update(const float* A, const float* B, float* C, int M, int N, int K, int f16) {
    using namespace ewos;
    if (!A || !B || !C || M < 1 || N < 1 || K < 1) {
        set_error("ewos_debug_tc_update: bad arguments");
        return EWOS_EINVAL;
    }
    if (!tc_assemble_available()) { set_error("tensor cores (sm_100 family) not available"); return EWOS_EINVAL; }
    AllocStream as(nullptr);
    float *dA = nullptr, *dB = nullptr, *dC = nullptr;
    TcScratch* owned = nullptr;
    ewos_status s = EWOS_OK;
    if (dev_alloc((void**)&dA, sizeof(float) * (size_t)M * K) != cudaSuccess ||
        dev_alloc((void**)&dB, sizeof(float) * (size_t)K * N) != cudaSuccess ||
        dev_alloc((void**)&dC, sizeof(float) * (size_t)M * N) != cudaSuccess) {
        set_error("ewos_debug_tc_update: out of device memory");
        s = EWOS_ENOMEM;
    }
    if (s == EWOS_OK && (cudaMemcpy(dA, A, sizeof(float) * (size_t)M * K, cudaMemcpyHostToDevice) != cudaSuccess ||
                         cudaMemcpy(dB, B, sizeof(float) * (size_t)K * N, cudaMemcpyHostToDevice) != cudaSuccess ||
                         cudaMemcpy(dC, C, sizeof(float) * (size_t)M * N, cudaMemcpyHostToDevice) != cudaSuccess))
        s = EWOS_ECUDA;
    if (s == EWOS_OK) s = tc_update_enqueue(dA, K, dB, N, dC, N, M, N, K, nullptr, &owned, false, 0, 0, f16 != 0);
    if (s == EWOS_OK) s = tc_update_check(owned, nullptr);
    if (s == EWOS_OK && cudaMemcpy(C, dC, sizeof(float) * (size_t)M * N, cudaMemcpyDeviceToHost) != cudaSuccess) s = EWOS_ECUDA;
    cudaDeviceSynchronize();
    tc_scratch_free(owned);
    dev_free(dA); dev_free(dB); dev_free(dC);
    return s;
}

extern "C" ewos_status ewos_debug_tc_assemble(const float* P, const double* M, int n, int m, int D, float* C, int sym,
                                              int f16) {
    using namespace ewos;
    if (!P || !M || !C || n < 1 || m < 1 || (D != 2 && D != 3)) {
        set_error("ewos_debug_tc_assemble: bad arguments");
        return EWOS_EINVAL;
    }
    if (!tc_assemble_available()) { set_error("tensor cores (sm_100 family) not available"); return EWOS_EINVAL; }
    const size_t E = (size_t)D + 1, np_ = E * (size_t)n * m, nm_ = (size_t)n * E * E, nc = (size_t)m * m;
    AllocStream as(nullptr);
    float *dP = nullptr, *dC = nullptr;
    double* dM = nullptr;
    TcScratch* owned = nullptr;
    ewos_status s = EWOS_OK;
    if (dev_alloc((void**)&dP, sizeof(float) * np_) != cudaSuccess || dev_alloc((void**)&dM, sizeof(double) * nm_) != cudaSuccess ||
        dev_alloc((void**)&dC, sizeof(float) * nc) != cudaSuccess) {
        set_error("ewos_debug_tc_assemble: out of device memory");
        s = EWOS_ENOMEM;
    }
    if (s == EWOS_OK && (cudaMemcpy(dP, P, sizeof(float) * np_, cudaMemcpyHostToDevice) != cudaSuccess ||
                         cudaMemcpy(dM, M, sizeof(double) * nm_, cudaMemcpyHostToDevice) != cudaSuccess ||
                         cudaMemset(dC, 0, sizeof(float) * nc) != cudaSuccess))
        s = EWOS_ECUDA;
    if (s == EWOS_OK) s = tc_assemble_pq(dP, dM, n, m, D, dC, nullptr, &owned, sym != 0, f16 != 0);
    if (s == EWOS_OK && cudaMemcpy(C, dC, sizeof(float) * nc, cudaMemcpyDeviceToHost) != cudaSuccess) s = EWOS_ECUDA;
    cudaDeviceSynchronize();
    tc_scratch_free(owned);
    dev_free(dP); dev_free(dM); dev_free(dC);
    return s;
}
