// Learned preconditioner entry points used inside a solver iteration.
#pragma once
#include "ok_launch.cuh"

namespace okgb {

// out = P in, as net_apply, except that every layer launch does nothing when *halt (device memory,
// read by the kernels at launch) is nonzero: the preconditioner application of a BiCGStab iteration
// that the host enqueued ahead of its convergence check and that the solver state has since halted.
// `halt` may be null (always apply).
int net_apply_unless_halted(ok_net* N, const ok_W* W, const cx<float>* in, cx<float>* out, const int* halt,
                            cudaStream_t st);

}  // namespace okgb
