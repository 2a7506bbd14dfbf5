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
    int levels;          // levels of the multigrid hierarchy of this solve
    long long t_start;   // device clock (ns): solve entry, preconditioner built, solve end
    long long t_built;
    long long t_end;
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
constexpr int kBlockLevelMax = 1024; // multigrid levels at most this large run inside one block

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

// Classical algebraic multigrid (preconditioner GQ_PRECOND_AMG).  Level 0 is the fine
// system; level l+1 consists of the C-points of a PMIS splitting of level l (strength
// measured on the unscaled operator), P_l is direct interpolation truncated to kAmgPmax
// coarse points per row, and A_{l+1} = P_l^T A_l P_l (FP64, unscaled).  The cycle runs
// on the Jacobi-scaled levels in FP32.  All sizes are decided on the device during the
// set-up and written to AMGInfo; the arrays come from pools of fixed capacity (rows over
// all levels, off-diagonal entries over all levels), and coarsening stops early when a
// pool would overflow.
constexpr int kAmgMaxLevels = 24;
// largest grid (cells) of one plan: the multigrid entry pools (12 per cell) are int-indexed
constexpr long long kMaxCells = 1ll << 27;
constexpr int kAmgPmax = 4;          // interpolation entries per row (ELL layout)
constexpr int kAmgRowMax = 64;       // distinct entries of one coarse row during the product

struct AMGInfo {
    int nlev;                        // levels built (1: level 0 only)
    int stop;                        // why coarsening stopped (diagnostic)
    int n[kAmgMaxLevels];            // rows of level l
    int nnz[kAmgMaxLevels];          // off-diagonal entries of level l
    int rnz[kAmgMaxLevels];          // entries of the restriction of level l -> l+1
    int row_off[kAmgMaxLevels];      // first row of level l in the per-row pools
    int nnz_off[kAmgMaxLevels];      // first entry of level l in the per-entry pools
    int rnz_off[kAmgMaxLevels];      // first entry of R_l in the restriction pool
    long long tns[kAmgMaxLevels + 2];  // device clock: start, fine copy done, level l coarsened
    long long bph[8];                  // build time per phase, summed over the levels (ns)
    long long cyc[kAmgMaxLevels];      // time per level over all cycles of the solve; last: the rest
    int ctr, rctr;                     // tail reservations of the Galerkin product (entries, restriction)
};

struct AMGData {
    int n0;
    int cap_rows;        // rows of all levels (level 0 included)
    int cap_nnz;         // off-diagonal entries of all levels
    AMGInfo* info;
    int* rowptr;         // [cap_rows + kAmgMaxLevels]: level l at row_off[l] + l, entries relative to nnz_off[l]
    int* col;            // [cap_nnz] column (row index within the level)
    double* a64;         // [cap_nnz] unscaled off-diagonal entries
    float* a32;          // [cap_nnz] Jacobi-scaled entries (levels >= 1)
    unsigned char* sfl;  // [cap_nnz] strength: bit 0 row depends on column, bit 1 column depends on row
    double* diag;        // [cap_rows] unscaled diagonal
    double* s;           // [cap_rows] diag^{-1/2} (level 0: the workspace's dloc)
    int* pc;             // [kAmgPmax cap_rows] P of level l -> l+1 (ELL): coarse column or -1
    float* pv32;         // [kAmgPmax cap_rows] scaled interpolation weights
    int* rrow;           // [cap_rows + kAmgMaxLevels] restriction rows (one per coarse row)
    int* rent;           // [kAmgPmax cap_rows] restriction entries: index into the P pool
    float *x, *b, *t;    // [cap_rows] cycle vectors (level 0 uses the Krylov buffers for b, x)
    // set-up temporaries over the largest level (n0 rows)
    double* pv64;        // [kAmgPmax n0] unscaled interpolation weights of the current level
    double* rowmax;      // [n0]
    double* wgt;         // [n0] PMIS weights
    signed char *stA, *stB;  // [n0] C/F states
    int *cidx, *cf, *cnt, *cnt2;  // [n0] coarse index, fine index of a coarse row, counts
    int *toff, *troff;   // [n0] staged places of a coarse row's entries and restriction entries
    double* dense;       // [kCoarseMax][2 kCoarseMax] Gauss-Jordan scratch
    float* inv;          // [kCoarseMax][kCoarseMax] inverse of the coarsest level
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
    float *r32b;     // second FP32 residual (the fused update writes the new one beside the old)
    // reductions, barrier, control
    MGHierarchy mg;
    AMGData amg;
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
    double cvfac;        // C_V / rho = k_B / ((gamma - 1) mu m_H) (ideal gas)
    int eos_n;           // tabulated EoS: number of points (0: ideal gas)
    const double *eos_T, *eos_u;  // its temperatures and specific internal energies
    double dt;
    const double *rho, *eg;
    double *E;           // in E^n, out E^{n+1}
    double *eg_out;
    double *T_out;
    const double *sadv;  // explicit radiation source S_adv per cell (Eq. adv), or null
    const double *sig_n, *E_n;  // sigma and E the face coefficients are formed from when
                                // they are held over sub-steps, or null (this step's)
};

struct SolveParams {
    int nx, N;
    int mixed;
    int restart;
    int max_iter, max_refine;
    double rtol, drop;
    long long spin_limit;
    int precond;         // GQ_PRECOND_JACOBI, GQ_PRECOND_MG or GQ_PRECOND_AMG
    float mg_omega;      // Jacobi smoothing weight of the V-cycle
    float mg_over;       // coarse-correction over-relaxation
    int block_cells;     // multigrid levels up to this size run in one block
    int tiled;           // 1: the tiled solve kernel where the problem allows it
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
// *kernel (may be null) receives the kernel launched: 0 k_pcg, 1 k_pcg_tiled
cudaError_t launch_solve(const SolveParams& p, const Workspace& w, int grid, cudaStream_t st, int* kernel = nullptr);
cudaError_t launch_backsub(const StepParams& sp, const DeviceGeometry& g, const Workspace& w,
                           int setup_blocks, cudaStream_t st);
// the per-cell pass of the set-up alone (C_V, T^n, opacities, the mass term and right-hand
// side of the reduced system, input checks, energy before the step): the multilevel step
// forms its faces and operator itself
cudaError_t launch_cells(const StepParams& sp, const DeviceGeometry& g, const Workspace& w, int setup_blocks,
                         cudaStream_t st);
cudaError_t launch_adv_source(int nx, int ny, const DeviceGeometry& g, const double* rho, const double* E,
                              const double* fx, const double* fy, double* S, int nblk, cudaStream_t st);
cudaError_t launch_face_flux(const StepParams& sp, const DeviceGeometry& g, const Workspace& w, double weight,
                             bool accumulate, double* Fx, double* Fy, int nblk, cudaStream_t st);
int solve_max_blocks_per_sm();
// the tiled solve (gq_pcg_tiled.cu): its kernel, dynamic shared memory and eligibility
const void* solve_kernel_tiled();
size_t tiled_smem_bytes();
int tiled_threads();
bool tiled_eligible(const SolveParams& p, const Workspace& w);
cudaError_t launch_tiled(const SolveParams& p, const Workspace& w, int grid, cudaStream_t st);
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
    int last_precond;        // preconditioner of the last step (-1: none yet)
    const double* S_adv;     // attached explicit radiation source (caller's device array) or null
    double* frz;             // 2 N doubles: sigma^n, E^n of a sub-cycled step (allocated on first use)
    int frz_on;              // 1 while a sub-cycled step forms its faces from frz
};
