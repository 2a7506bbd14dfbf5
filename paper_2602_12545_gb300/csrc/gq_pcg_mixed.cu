// Mixed-precision single-problem solve kernel, k_pcg<true> (FP32 Krylov vectors inside
// FP64 refinement); the solver is in gq_pcg.cuh.
#include "gq_pcg.cuh"

namespace gq {

const void* solve_kernel_mixed() { return reinterpret_cast<const void*>(k_pcg<true>); }

}  // namespace gq
