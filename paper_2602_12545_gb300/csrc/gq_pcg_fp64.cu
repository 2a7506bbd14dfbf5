// FP64 single-problem solve kernel, k_pcg<false>, and the host launchers of the
// single-problem solve; the solver is in gq_pcg.cuh.
#include "gq_pcg.cuh"

namespace gq {

const void* solve_kernel_fp64() { return reinterpret_cast<const void*>(k_pcg<false>); }

int solve_max_blocks_per_sm() {
    int a = 0, b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, solve_kernel_mixed(), kSolveThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, solve_kernel_fp64(), kSolveThreads, 0);
    return a < b ? a : b;
}

cudaError_t launch_solve(const SolveParams& p, const Workspace& w, int grid, cudaStream_t st) {
    SolveParams pc = p;
    Workspace wc = w;
    void* args[] = {&pc, &wc};
    const void* fn = p.mixed ? solve_kernel_mixed() : solve_kernel_fp64();
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kSolveThreads), args, 0, st);
}

}  // namespace gq
