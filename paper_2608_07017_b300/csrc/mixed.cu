// mixed.cu -- tensor-core assembly of the Galerkin matrix (placeholder: the FP32 SIMT GEMM of
// solve.cu is used while no tensor-core kernel is compiled in).
#include "toolbox.hpp"

namespace ewos {
bool tc_assemble_available() { return false; }
ewos_status tc_assemble(const float*, const float*, float*, int, int, int, cudaStream_t) {
    set_error("tensor-core assembly is not available in this build");
    return EWOS_EINVAL;
}
}  // namespace ewos
