// mixed.cu -- mixed-precision solve path (tensor-core assembly, low-precision LU, FP64
// refinement).  Placeholder until the tensor-core kernels land.
#include "toolbox.hpp"

namespace ewos {
ewos_status solve_mixed(ewos_toolbox*, const ewos_problem*, double, double, int, ewos_solve_report*) {
    set_error("mixed-precision solve is not available in this build");
    return EWOS_EINVAL;
}
}  // namespace ewos
