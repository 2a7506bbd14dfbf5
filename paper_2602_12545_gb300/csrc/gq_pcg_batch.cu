// Batched persistent solve kernel, kb_pcg, and its host launchers; the solver is in
// gq_pcg.cuh.
#include "gq_pcg.cuh"

namespace gq {

namespace {

// Batched persistent solve: the co-resident grid is split into teams; the leader block
// of a team takes the next problem of the team's class from the class queue, the team
// solves it, and repeats until the queue is empty.  Teams synchronise only among
// themselves, so small problems (one-block teams) never touch an inter-block barrier.
__global__ void __launch_bounds__(kSolveThreads, 1) kb_pcg(BatchArgs a) {
    __shared__ RedShared sh;
    __shared__ MGShared msh;
    __shared__ int s_idx;
    const int tm = a.block_team[blockIdx.x];
    const Team team{static_cast<int>(blockIdx.x) - a.team_first[tm], a.team_size[tm]};
    const int c = a.team_class[tm];
    const int qlen = a.class_start[c + 1] - a.class_start[c];
    unsigned* tbar = a.team_bar + tm;
    while (true) {
        if (team.rank == 0 && threadIdx.x == 0) a.team_slot[tm] = atomicAdd(a.queue_head + c, 1);
        if (!team_barrier(tbar, team, a.spin_limit, a.abort_flag)) return;
        if (threadIdx.x == 0) s_idx = __ldcg(a.team_slot + tm);
        // every block of the team has read the slot before the leader may overwrite it
        if (!team_barrier(tbar, team, a.spin_limit, a.abort_flag)) return;
        const int idx = s_idx;
        if (idx >= qlen) return;
        const ProbDesc& d = a.desc[a.queue[a.class_start[c] + idx]];
        const bool ok = d.sp.mixed ? pcg_solve_outlined<true>(d.solve, d.w, team, sh, msh)
                                   : pcg_solve_outlined<false>(d.solve, d.w, team, sh, msh);
        if (!ok) return;
    }
}

}  // namespace

int batch_solve_max_blocks_per_sm() {
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, kb_pcg, kSolveThreads, 0);
    return a;
}

cudaError_t launch_batch_solve(const BatchArgs& a, int grid, cudaStream_t st) {
    BatchArgs ac = a;
    void* args[] = {&ac};
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kSolveThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(kb_pcg), args);
}

}  // namespace gq
