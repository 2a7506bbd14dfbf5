// FP64 single-problem solve kernel, k_pcg<false>, and the host launchers of the
// single-problem solve; the solver is in gq_pcg.cuh.
#include "gq_pcg.cuh"

namespace gq {

const void* solve_kernel_fp64() { return reinterpret_cast<const void*>(k_pcg<false>); }

// the tiled kernel's dynamic shared memory is opted in once per device
static bool tiled_ready(int dev) {
    static int done[64] = {0};
    if (dev < 0 || dev >= 64) return false;
    if (!done[dev]) {
        if (cudaFuncSetAttribute(solve_kernel_tiled(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(tiled_smem_bytes())) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        done[dev] = 1;
    }
    return true;
}

int solve_max_blocks_per_sm() {
    int a = 0, b = 0, c = 0, dev = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, solve_kernel_mixed(), kSolveThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, solve_kernel_fp64(), kSolveThreads, 0);
    int m = a < b ? a : b;
    if (cudaGetDevice(&dev) == cudaSuccess && tiled_ready(dev) &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, solve_kernel_tiled(), tiled_threads(), tiled_smem_bytes()) ==
            cudaSuccess &&
        c >= 1)
        m = m < c ? m : c;
    cudaGetLastError();
    return m;
}

cudaError_t launch_solve(const SolveParams& p, const Workspace& w, int grid, cudaStream_t st, int* kernel) {
    SolveParams pc = p;
    Workspace wc = w;
    void* args[] = {&pc, &wc};
    int dev = 0;
    if (kernel) *kernel = 0;
    if (p.tiled && tiled_eligible(p, w) && cudaGetDevice(&dev) == cudaSuccess && tiled_ready(dev)) {
        const cudaError_t e = launch_tiled(p, w, grid, st);
        if (e != cudaErrorInvalidValue) {
            if (kernel) *kernel = 1;
            return e;
        }
        cudaGetLastError();     // the tensor maps could not be built: the untiled kernel
    }
    const void* fn = p.mixed ? solve_kernel_mixed() : solve_kernel_fp64();
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kSolveThreads), args, 0, st);
}

}  // namespace gq
