// Internal structures of the GB300 FLD library (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gq_fld.h"

namespace gq {

// Device-resident control block of one solve.  Written by the kernels, copied to the
// host once per step.
struct SolveCtl {
    int status;          // gq_status
    int iterations;
    int refinements;
    int input_flags;     // bit 0: a field value <= 0, bit 1: a non-finite field value
    double crit;         // cell-wise relative residual of the last FP64 residual
    double l2;           // |b - A x|_2 / |b|_2 of the reduced system
    double energy0;      // sum V (E + e_g) before
    double energy1;      // and after
    int abort;           // set by a block whose inter-block wait timed out
    int pad[3];
};

// Geometry of a plan in device memory (FP64).  Face arrays:
//   gx [ny][nx+1]  A_f / d_f of x-face i (between cells i-1, i); boundary faces hold A_f / h
//   gy [ny+1][nx]  the same for y-faces
// 1-D arrays: dxf[nx+1] centre distance (boundary: half-cell distance h) of x-face i,
//   thx[nx+1] interpolation weight (x_f - x_{i-1}) / (x_i - x_{i-1}),
//   ymet[nx] metric of the y direction (1, or r_c for spherical-polar),
//   dyf[ny+1], thy[ny+1] the y-face analogues (distance in y or theta, before the metric).
struct DeviceGeometry {
    const double *V, *gx, *gy, *dxf, *thx, *ymet, *dyf, *thy;
};

// Aggregation multigrid hierarchy (preconditioner of the Krylov solve).  Level 0 is the
// Jacobi-scaled fine system itself; level l+1 aggregates 2 x 2 cells of level l.  Every
// level is stored Jacobi-scaled (unit diagonal): c_W, c_S are its scaled couplings and
// t[k] = s_{l+1}[parent(k)] / s_l[k] the transfer weight of cell k to its parent, so that
// restriction is r_{l+1}[I] = sum_{k in I} t[k] r_l[k] and prolongation its transpose.
// The FP64 arrays hold the unscaled Galerkin operator (mass m and face weights) from
// which the next level is built.
constexpr int kMaxLevels = 32;
constexpr int kCoarseMax = 32;       // the coarsest level is solved densely (<= 32 cells)
constexpr int kBlockLevelMax = 8192; // levels at most this large run inside one block

struct MGLevel {
    int nx, ny, N;
    double *m, *wW, *wS, *s;    // unscaled Galerkin operator and diag^{-1/2} (levels >= 1)
    float *cW, *cS;             // scaled couplings (level 0: the workspace's FP32 copies)
    float *t;                   // transfer weight to the parent (all but the coarsest level)
    float *xa, *xb, *r;         // smoother buffers and right-hand side (level 0: r is the CG residual)
};

struct MGHierarchy {
    int nlev;                   // levels including level 0 (1 = no coarse levels)
    MGLevel L[kMaxLevels];
    double* dense;              // FP64 scratch for the coarsest inverse [nc][2 nc]
    float* inv;                 // inverse of the coarsest scaled operator [nc][nc]
    float* z;                   // FP32 preconditioned residual of level 0 (two buffers)
    float* zold;
    float* r32;                 // FP32 residual for the V-cycle of the FP64 path
    double* p64s;               // FP64 path: second direction buffer unused (reserved)
};

// Workspace of one step in device memory.
struct Workspace {
    // setup outputs (FP64); the scaled system overwrites some in place
    double *sig;     // sigma = kappa_R rho
    double *dloc;    // V (1 + beta~), later s = diag^{-1/2}
    double *rhs;     // b, later b^ = s b
    double *tA, *tB; // T^{n+1} = tA + tB E^{n+1}
    double *wW, *wS; // interior face weights (west, south), later the scaled c = w s_k s_m
    double *wB;      // Milne boundary weights of the cell (diagonal only)
    // solve (FP64 path and the outer FP64 iterate / residual of the mixed path)
    double *y, *r64, *p64[2], *q64;
    // solve (FP32 inner path)
    float *cW32, *cS32, *d32, *r32, *p32[2], *q32;
    // reductions, barrier, control
    MGHierarchy mg;
    double *partials;    // [2][max_blocks][kSlots]
    double *epart;       // [2][max_setup_blocks] energy partial sums (before, after)
    unsigned *bar;       // [2]
    SolveCtl *ctl;
};

constexpr int kSlots = 6;
constexpr int kSolveThreads = 512;
constexpr int kSetupThreads = 256;

struct StepParams {
    int nx, ny, N;
    int precond;
    int bc[4];
    int limiter;
    int mixed;
    double kR[4], kP[4];
    double cvfac;        // C_V / rho = k_B / ((gamma - 1) mu m_H)
    double dt;
    const double *rho, *eg;
    double *E;           // in E^n, out E^{n+1}
    double *eg_out;
    double *T_out;
};

struct SolveParams {
    int nx, N;
    int mixed;
    int restart;
    int max_iter, max_refine;
    double rtol, drop;
    long long spin_limit;
    int precond;         // GQ_PRECOND_JACOBI or GQ_PRECOND_MG
    float mg_omega;      // Jacobi smoothing weight of the V-cycle
    float mg_over;       // coarse-correction over-relaxation
    int pad;
};

// status of a problem of a batch that no team has solved yet
constexpr int kPending = 100;

// One problem of a batched step: its per-step parameters, geometry, workspace and
// solver settings (device-resident table, one entry per problem).
struct ProbDesc {
    StepParams sp;
    DeviceGeometry g;
    Workspace w;
    SolveParams solve;
    int setup_blocks;    // blocks of the batched set-up launches for this problem
    int pad;
};

// Arguments of the batched kernels.  Set-up kernels map block b to problem p with
// setup_prefix[p] <= b < setup_prefix[p+1].  The solve kernel partitions its blocks
// into teams; team t (team_first[t] .. + team_size[t]) takes problems of its class
// from the class queue (largest estimated work first) until the queue is empty.
struct BatchArgs {
    const ProbDesc* desc;
    int n;
    int nclass;
    const int* setup_prefix;   // [n+1]
    const int* block_team;     // [G]
    const int* team_first;     // [T]
    const int* team_size;      // [T]
    const int* team_class;     // [T]
    const int* queue;          // [n]
    const int* class_start;    // [nclass+1]
    int* queue_head;           // [nclass]
    int* team_slot;            // [T]
    unsigned* team_bar;        // [2T]
    int* abort_flag;
    long long spin_limit;
    SolveCtl* ctl_out;         // [n] gathered control blocks
};

// launchers (stream-ordered)
cudaError_t launch_setup(const StepParams& sp, const DeviceGeometry& g, const Workspace& w,
                         int setup_blocks, cudaStream_t st);
cudaError_t launch_solve(const SolveParams& p, const Workspace& w, int grid, cudaStream_t st);
cudaError_t launch_backsub(const StepParams& sp, const DeviceGeometry& g, const Workspace& w,
                           int setup_blocks, cudaStream_t st);
int solve_max_blocks_per_sm();
int batch_solve_max_blocks_per_sm();
cudaError_t launch_batch_setup(const BatchArgs& a, int total_setup_blocks, cudaStream_t st);
cudaError_t launch_batch_solve(const BatchArgs& a, int grid, cudaStream_t st);
cudaError_t launch_batch_finish(const BatchArgs& a, int total_setup_blocks, cudaStream_t st);

constexpr long long kDefaultSpin = 1ll << 24;

// argument validation and parameter blocks shared by the single and batched steps
gq_status make_step_params(const gq_fld_plan* P, const double* rho, double* e_g, double* E_r, double* T_g_out,
                           const gq_opacity_law* op, const gq_eos* eos, double dt, const gq_bc* bc,
                           const gq_solver_opts* opts, StepParams* sp, SolveParams* pp, int* timing);
gq_status status_of(const SolveCtl& c);
// lays out a plan's arrays from base (nullptr: sizing only); returns the bytes used.
// P->nx, ny, N, solve_grid_max and setup_blocks must be set.  Used by the
// allocation-free step, which places the plan in its static array.
size_t plan_layout(gq_fld_plan* P, char* base);
gq_status batch_create_capacity(int device, int num_sms, int cap, const gq_batch_opts* opts, gq_batch** out);
gq_status batch_rebind(gq_batch* B, gq_fld_plan* const* plans, int n);
void fill_info(const SolveCtl& c, gq_status status, gq_step_info* info);

}  // namespace gq

// A plan: one grid's geometry and the device workspace of its step.
struct gq_fld_plan {
    int nx, ny, N, coord;
    int device;
    int num_sms;
    int solve_grid_max;      // co-resident blocks of the solve kernel (also the partials capacity)
    int setup_blocks;
    void* arena;
    size_t arena_bytes;
    gq::DeviceGeometry geo;
    gq::Workspace ws;
    gq::SolveCtl* ctl_host;  // pinned
    cudaEvent_t ev[4];       // phase timing
};
