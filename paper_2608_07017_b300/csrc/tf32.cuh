// tf32.cuh -- the split of an FP32 value into a TF32 part and the FP32 remainder, used wherever
// an operand of the three-product tensor-core GEMM is prepared.
#pragma once
#include <cstdint>

namespace ewos {

// v = h + l exactly: h is v rounded to nearest (ties to even) at 10 explicit mantissa bits, the
// TF32 input format of the tensor cores; non-finite values pass through in h
__device__ __forceinline__ void tf32_split(float v, float& h, float& l) {
    const uint32_t b = __float_as_uint(v);
    const uint32_t hb = (b + 0x0FFFu + ((b >> 13) & 1u)) & 0xFFFFE000u;
    h = isfinite(v) ? __uint_as_float(hb) : v;
    l = v - h;
}

}  // namespace ewos
