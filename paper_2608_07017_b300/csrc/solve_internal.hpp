// solve_internal.hpp -- the solve entry on an explicit workspace, shared by ewos_solve and the
// request server.
#pragma once
#include "toolbox.hpp"

namespace ewos {

struct SolveOptions {
    // Mixed mode: refine all right-hand sides of the request together, one CUDA-graph launch per
    // sweep; semilinear problems by the chord iteration s <- s - (Lambda + alpha I)^-1 (R(s) +
    // alpha s) on the same factors (exact Newton per right-hand side when it does not converge).
    bool batched = false;
    // Linear problems only: take Lambda + alpha I's factors (and alpha) from the previous solve on
    // this workspace, for the same toolbox and coefficients, instead of assembling and factoring
    // again (the operator estimates solve their unit right-hand sides in chunks this way).
    bool reuse_factors = false;
    // Semilinear mixed solves: keep the FP32 factors of an earlier Newton step's Jacobian as
    // the refinement's preconditioner while the refinement still converges (refactor otherwise).
    bool newton_reuse = true;
};

struct SolveWorkspace;
ewos_status solve_on(ewos_toolbox* tb, SolveWorkspace*& ws, const ewos_problem* pb, double* u_out, double* s_out,
                     int outputs_on_device, ewos_solve_report* rep, const SolveOptions& opt);
// Device bytes a workspace for this toolbox needs (mixed or FP64 mode, nrhs right-hand sides).
size_t workspace_bytes(const ewos_toolbox* tb, int64_t nrhs, bool mixed);

}  // namespace ewos
