/*
 * gq_fld.h -- C ABI of the GB300 implicit flux-limited-diffusion (FLD) radiation step.
 *
 * The operation is the radiation / gas-thermodynamics sub-step of Chen & Bai, "Guangqi:
 * a two-dimensional radiation hydrodynamic code with realistic equations of state"
 * (arXiv 2602.12545), Sec. 3.2: one backward-Euler step of
 *     dE/dt - div(D grad E) = -G0,   C_V dT/dt = G0,   G0 = rho c kappa_P E - eta,
 * eta = kappa_P rho c a T^4 (Sec. 2), with the flux-limited diffusion coefficient
 * D = c lambda(R) / (kappa_R rho) (Sec. 2, Eqs. limiter and reducer; face values per
 * Eq. diffcoeff), the linearisation (T^{n+1})^4 ~ 4 T^3 T^{n+1} - 3 T^4 (Sec. 3.2.1), the
 * coefficients phi_1..phi_11, psi_5, psi_6, psi_11 (Eqs. phi1-psi7, alpha, fldg) and the
 * coupled linear system of Eqs. linearsys1-2, which is reduced exactly to a symmetric
 * positive-definite 5-point system in E and solved by a preconditioned Krylov method to a
 * relative residual (Eq. linearsystem).
 *
 * Conventions shared by every entry point
 *   - Cell arrays are row-major [ny][nx], x (or r) fastest, float64, in DEVICE memory
 *     owned by the caller, unless a parameter says "host".
 *   - Units are CGS.  Boundary sides are ordered -x, +x, -y, +y (r-, r+, theta-, theta+).
 *   - Every call returns a gq_status and never aborts.  Work is enqueued on the given CUDA
 *     stream (a cudaStream_t passed as void*, NULL = legacy default stream); where a call
 *     fills a host result struct, it has synchronised with that stream before returning.
 *   - A plan is used by one host thread at a time.
 */
#ifndef GQ_FLD_H
#define GQ_FLD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GQ_OK = 0,
    GQ_ERR_INVALID_ARG = 1,     /* bad pointer, size, option or non-positive field value */
    GQ_ERR_CUDA = 2,            /* a CUDA runtime call failed */
    GQ_ERR_OOM = 3,             /* device allocation failed */
    GQ_ERR_NOT_CONVERGED = 4,   /* max_iter reached; the best iterate is written */
    GQ_ERR_NONFINITE = 5,       /* NaN / Inf in the inputs or in a solver reduction */
    GQ_ERR_TIMEOUT = 6,         /* an inter-block wait exceeded its spin limit */
    GQ_ERR_BUDGET = 7           /* serving: request does not fit the memory budget */
} gq_status;

enum { GQ_CARTESIAN = 0, GQ_SPHERICAL_POLAR = 1 };
enum { GQ_BC_REFLECT = 0, GQ_BC_OUTFLOW_MILNE = 1 };
enum { GQ_LIMITER_LP = 0, GQ_LIMITER_MINERBO = 1, GQ_LIMITER_NONE = 2 };
enum { GQ_PREC_FP64 = 0, GQ_PREC_MIXED = 1 };
enum { GQ_PRECOND_JACOBI = 0, GQ_PRECOND_MG = 1, GQ_PRECOND_AMG = 2 };

/* Grid geometry (Sec. 3.2.1 and Eq. fldg).  Cartesian (x, y) per unit depth, or
 * axisymmetric spherical-polar (r, theta) with the common factor 2 pi dropped.
 * x_faces: host, nx+1 strictly increasing face coordinates (x or r > 0).
 * y_faces: host, ny+1 strictly increasing (y, or theta in [0, pi]).
 * area_x [ny][nx+1], area_y [ny+1][nx], volume [ny][nx]: optional host arrays that
 * replace the derived face areas dS and volumes dV; NULL derives them from the faces. */
typedef struct {
    int nx, ny;
    int coord;                       /* GQ_CARTESIAN or GQ_SPHERICAL_POLAR */
    const double *x_faces, *y_faces;
    const double *area_x, *area_y, *volume;
} gq_grid_desc;

/* Mean opacities as power laws kappa = k0 + k1 rho^a T^b (cm^2/g) at T = T_g^n
 * (Sec. 2 defines kappa_R and kappa_P; the paper tabulates them, a power law stands in). */
typedef struct { double k0_R, k1_R, a_R, b_R, k0_P, k1_P, a_P, b_P; } gq_opacity_law;

/* Equation of state.
 * table_n = 0: ideal gas, e_g = C_V T with C_V = rho k_B / ((gamma - 1) mu m_H) (Sec. 3.2,
 *   C_V = de/dT).
 * table_n >= 2: a tabulated EoS for the non-linear C_V of Sec. 3.2.1.  table_T (K) and
 *   table_u (specific internal energy, erg/g) are DEVICE arrays of table_n increasing
 *   values, owned by the caller.  u(T) is piecewise linear and extended linearly past both
 *   ends.  Per cell, T^n solves u(T) = e_g / rho on the last segment whose lower end is at
 *   or below e_g / rho, and C_V = rho du/dT on that segment; e_g^{n+1} = e_g^n +
 *   C_V (T^{n+1} - T^n).  gamma and mu must still be valid but are not used.  A segment
 *   that does not increase makes the step return GQ_ERR_NONFINITE.  Single and
 *   sub-cycled steps only: batched steps and server requests with a table return
 *   GQ_ERR_INVALID_ARG.
 * Other table_n, or a table with a NULL array: GQ_ERR_INVALID_ARG. */
typedef struct {
    double gamma, mu;
    int table_n;
    const double *table_T, *table_u;
} gq_eos;

/* Per-side boundary kind: GQ_BC_REFLECT (no flux) or GQ_BC_OUTFLOW_MILNE (Eq. milne). */
typedef struct { int side[4]; } gq_bc;

/* Solver options.
 *   prec        GQ_PREC_FP64: FP64 PCG.  GQ_PREC_MIXED: FP32 PCG inside FP64 iterative
 *               refinement (the FP64 residual b - A x is recomputed whenever the FP32
 *               residual has fallen by inner_rtol, keeping the search direction).  The
 *               multigrid preconditioners run in FP32 for both.
 *   limiter     GQ_LIMITER_LP (Levermore-Pomraning rational form), _MINERBO (Eq. limiter),
 *               _NONE (lambda = 1/3).
 *   rtol        stop when max_k |b - A x|_k / (A_kk |x_k|) <= rtol (the cell-wise relative
 *               residual of the reduced system; the paper's 2-norm form of Eq. linearsystem
 *               is reported in gq_step_info.rel_residual_l2).
 *   max_iter    cap on Krylov iterations (> 0).
 *   inner_rtol  mixed only: FP32 residual drop that triggers an FP64 refinement, in (0, 1).
 *   max_refine  cap on FP64 residual evaluations after the first (> 0).  Independently,
 *               the solve ends with GQ_ERR_NOT_CONVERGED when six consecutive FP64
 *               residuals, spanning at least 32 Krylov iterations, fail to improve the
 *               best one by 10% (rtol below the FP64 rounding floor of the cell-wise
 *               residual).
 *   spin_limit  cap on the polling iterations of any inter-block wait (0 = default, about
 *               a second); exceeding it ends the solve with GQ_ERR_TIMEOUT.
 *   restart     mixed only: 1 restarts the Krylov space at every refinement (classical
 *               iterative refinement), 0 keeps the search direction (default).
 *   timing      1 records CUDA events around the set-up, solve and finish phases on the
 *               stream and reports their durations in gq_step_info (0 = off).
 *   precond     GQ_PRECOND_AMG (default): CG preconditioned by one V-cycle of classical
 *               algebraic multigrid, built on the device every step (PMIS coarsening with
 *               strength taken on the unscaled operator, direct interpolation truncated
 *               to 4 entries, Galerkin coarse operators), robust where the face weights
 *               jump by orders of magnitude from cell to cell; FP32 cycle for both
 *               precisions, Polak-Ribiere directions.
 *               GQ_PRECOND_MG: one V-cycle of aggregation multigrid (2 x 2 Galerkin
 *               coarsening of the Jacobi-scaled operator, two weighted-Jacobi sweeps
 *               before and after, exact solve of the coarsest <= 32 cells); cheapest per
 *               step on smooth fields.
 *               GQ_PRECOND_JACOBI: diagonal (Jacobi) preconditioning only.
 *   mg_omega    Jacobi smoothing weight of the V-cycle, in (0, 1] (0 = default 0.8).
 *   mg_over     coarse-correction factor, in (0, 2) (0 = default 1.5; the AMG cycle
 *               applies no factor).
 *   mg_block_cells  multigrid levels of at most this many cells are processed by one
 *               block of the solve (the others wait), larger ones by all blocks with
 *               grid-wide barriers between passes (0 = default 1024; >= 0).
 *   subcycle_freeze_D  gq_fld_step_subcycled only.  1 (default): every sub-step forms its
 *               face coefficients (kappa_R rho, the limiter, Milne faces) from the hydro
 *               step's start state E^n, T^n, with its own dt: the order of the radiation
 *               algorithm of Sec. 3.2.1, which updates alpha and keeps D between sub-steps.
 *               0: each sub-step re-forms them from the state it starts from.
 *               Other values: GQ_ERR_INVALID_ARG.
 *   untiled     0 (default): the mixed path with GQ_PRECOND_MG runs the tiled solve
 *               kernel (each multigrid level the whole grid works on in two fused passes
 *               over shared-memory tiles) where every such level has a width divisible by
 *               8 and an even height; 1: always the untiled kernel.  Both compute the same
 *               cycle; other values: GQ_ERR_INVALID_ARG. */
typedef struct {
    int prec;
    int limiter;
    double rtol;
    int max_iter;
    double inner_rtol;
    int max_refine;
    int64_t spin_limit;
    int restart;
    int timing;
    int precond;
    int mg_block_cells;
    double mg_omega;
    double mg_over;
    int subcycle_freeze_D;
    int untiled;
} gq_solver_opts;

/* Result of one step (host struct). */
typedef struct {
    int iterations;             /* Krylov iterations (FP32 ones for the mixed path) */
    int refinements;            /* FP64 residual evaluations after the initial one */
    double rel_residual;        /* final cell-wise relative residual (see rtol) */
    double rel_residual_l2;     /* |b - A x|_2 / |b|_2 of the reduced system (Eq. linearsystem) */
    double energy_before;       /* sum_k V_k (E_k + e_g,k) at time n (axisymmetric: / 2 pi) */
    double energy_after;        /* the same at time n+1 */
    int status;                 /* gq_status of the step */
    int solve_blocks;           /* blocks of the cooperative solve launch */
    double t_setup_ms;          /* with opts.timing: set-up kernels (coefficients, scaling) */
    double t_solve_ms;          /* with opts.timing: the Krylov solve kernel */
    double t_finish_ms;         /* with opts.timing: back-substitution and energy sums */
    float t_precond_ms;         /* device clock: build of the preconditioner inside the solve */
    float t_iter_us;            /* device clock: solve time after that build per Krylov iteration */
    int precond_levels;         /* levels of the multigrid hierarchy (1 for Jacobi) */
    int solve_kernel;           /* the solve kernel that ran: 0 untiled, 1 tiled (see opts.untiled) */
} gq_step_info;

typedef struct gq_fld_plan gq_fld_plan;

/* Build a plan for one grid: validates the geometry, computes volumes, face areas,
 * volume centres and centre distances in FP64 on the host (Eqs. fldg and alpha), uploads
 * them and allocates the device workspace of one step.  The plan owns that memory until
 * gq_fld_destroy.  Errors: GQ_ERR_INVALID_ARG (nx or ny < 1, NULL faces, non-increasing
 * faces, theta outside [0, pi], r <= 0), GQ_ERR_OOM, GQ_ERR_CUDA.  *out is NULL on error. */
gq_status gq_fld_setup(const gq_grid_desc *grid, gq_fld_plan **out);

/* Device bytes held by a plan (geometry and workspace). */
size_t gq_fld_plan_bytes(const gq_fld_plan *plan);

/* Device bytes gq_fld_setup would allocate for an nx x ny grid on the current device
 * (0 for invalid sizes or when no device is available).  Allocates nothing. */
size_t gq_fld_plan_bytes_for(int nx, int ny);

/* One implicit FLD step (Sec. 3.2.1, a single sub-cycle, n_sub = 1): face coefficients,
 * C_V, the phi / psi coefficients, the reduced system, its Krylov solve and T^{n+1}.
 *   rho      [ny][nx] device, g/cm^3, > 0, read only.
 *   e_g      [ny][nx] device, erg/cm^3, > 0, in: e_g^n, out: e_g^{n+1}.
 *   E_r      [ny][nx] device, erg/cm^3, > 0, in: E^n, out: E^{n+1}.
 *   T_g_out  [ny][nx] device, K, out: T_g^{n+1} (may be NULL).
 *   opacity, eos, bc, opts: host structs.  dt > 0 (s).
 *   info     host, filled on return (may be NULL).
 * e_g and E_r are written only when the step returns GQ_OK or GQ_ERR_NOT_CONVERGED.
 * Errors: GQ_ERR_INVALID_ARG (arguments, or a field value <= 0), GQ_ERR_NONFINITE,
 * GQ_ERR_NOT_CONVERGED, GQ_ERR_TIMEOUT, GQ_ERR_CUDA. */
gq_status gq_fld_step(gq_fld_plan *plan, const double *rho, double *e_g, double *E_r, double *T_g_out,
                      const gq_opacity_law *opacity, const gq_eos *eos, double dt, const gq_bc *bc,
                      const gq_solver_opts *opts, void *stream, gq_step_info *info);

/* The hydro step dt_total split into n_sub implicit FLD steps of geometrically growing
 * length (Sec. 3.2, Eq. subtimesteps): dt_i = dt_0 q_t^(i-1), i = 1..n_sub, with
 * dt_0 = dt_total (1 - q_t) / (1 - q_t^n_sub), so that they add up to dt_total (q_t = 1:
 * equal sub-steps).  Each sub-step is gq_fld_step from the state the previous one left,
 * so C_V, the Planck opacity and the linearisation are re-evaluated; the face
 * coefficients (kappa_R rho, the limiter, D) are held from the hydro step's start
 * (opts->subcycle_freeze_D = 1, the default: the order of the radiation algorithm of
 * Sec. 3.2.1) or re-formed per sub-step (0).  Arguments as gq_fld_step;
 * n_sub >= 1, q_t > 0 (the paper uses 1 < q_t < 2), dt_total > 0.  info: iterations and
 * refinements summed, residuals the largest of the sub-steps, energy_before of the first
 * and energy_after of the last sub-step, timings summed.  A sub-step that ends with
 * GQ_ERR_NOT_CONVERGED does not stop the series (the call then returns that status);
 * any other error stops it and is returned.
 *   Fx, Fy   [ny][nx+1], [ny+1][nx] device (each may be NULL): the radiative flux of the
 *            hydro step through every face, erg cm^-2 s^-1, positive along +x / +y: the
 *            sub-steps' fluxes -D grad E (the D they were solved with, and E after the sub-step) weighted
 *            by dt_i / dt_total, so that dt_total times it is the energy the face carried
 *            (the accumulation of Sec. 3.2.1).  Reflecting faces carry 0; Milne faces
 *            D_b E / (h (1 + k)) outward. */
gq_status gq_fld_step_subcycled(gq_fld_plan *plan, const double *rho, double *e_g, double *E_r,
                                double *T_g_out, const gq_opacity_law *opacity, const gq_eos *eos,
                                double dt_total, int n_sub, double q_t, const gq_bc *bc,
                                const gq_solver_opts *opts, double *Fx, double *Fy, void *stream,
                                gq_step_info *info);

/* Release a plan and its device memory (NULL is ignored). */
void gq_fld_destroy(gq_fld_plan *plan);

/* Multigrid hierarchy of a plan's last step (diagnostics; the paper's solver builds no
 * hierarchy).  For GQ_PRECOND_AMG: rows and off-diagonal entries of every level as built
 * on the device, why coarsening stopped (1 coarsest small enough, 2 level cap, 3 a level
 * did not shrink, 4 row pool, 5 entry pool, 6 a coarse row too long), and the device time
 * of each part of the build.  For GQ_PRECOND_MG: the fixed 2 x 2 hierarchy's rows, and the
 * cycle time with the levels run by one block summed in the slot of the first of them.
 * Synchronises with the device.  GQ_ERR_INVALID_ARG before any step or for Jacobi. */
typedef struct {
    int precond;
    int levels;
    int stop_reason;
    int rows[24];
    int entries[24];
    float build_ms[24];         /* AMG: coarsening level l into level l + 1 */
    float fine_copy_ms;         /* AMG: copy of the fine operator into the hierarchy */
    float coarsest_ms;          /* AMG: inverse of the coarsest level */
    float build_phase_ms[8];    /* AMG: build time per phase summed over the levels (strength,
                                   splitting rounds, numbering, interpolation, product count,
                                   scans, product fill, scaling) */
    float cycle_ms[24];         /* multigrid: time per level summed over the solve's cycles
                                   (levels 0..19); [20] the direction pass and its reduction,
                                   [21] the update pass, its reduction and the stop test,
                                   [22] the FP64 residual evaluations, [23] the reduction after
                                   the cycle (device clock of the first block) */
} gq_precond_info;

gq_status gq_fld_precond_info(const gq_fld_plan *plan, gq_precond_info *out);

/* Explicit radiation advection, Sec. 3.2.1 (Eq. adv, with g = dS / dV of Eq. fldg).
 *
 * gq_fld_adv_source writes S_adv [ny][nx] (device, erg cm^-3 s^-1) for the plan's grid:
 * for each cell, the sum over its four faces of (A_face / V) f e_r, added on its lower
 * faces (-x, -y) and subtracted on its upper ones, where
 *   fx [ny][nx+1], fy [ny+1][nx]  device face mass fluxes (rho v from the hydro Riemann
 *                                 solution), g cm^-2 s^-1, positive along +x / +y;
 *   e_r = E_r / rho               of the upwind cell; a boundary face takes its one cell's.
 * rho and E_r are device [ny][nx].  Enqueued on stream; nothing is checked on the device.
 * Errors: GQ_ERR_INVALID_ARG (NULL pointer), GQ_ERR_CUDA (launch failed).
 *
 * gq_fld_set_source attaches S_adv (device [ny][nx], owned by the caller, which keeps it
 * valid while attached; NULL detaches) to the plan.  Every later gq_fld_step and
 * gq_fld_step_subcycled of this plan then adds S_adv dt to phi_11 (each sub-step adds
 * S_adv times its own dt, so the hydro step receives S_adv dt_total, S_adv being
 * computed once per hydro step from E^n as the paper's algorithm does).  A step whose
 * E^n + S_adv dt is not positive in some cell returns GQ_ERR_INVALID_ARG (not finite:
 * GQ_ERR_NONFINITE), fields unchanged; in a sub-cycled step the test is made on each
 * sub-step's E, which strong gas coupling can drop far below E^n within a sub-step.
 * Batched, serving and allocation-free steps take no source. */
gq_status gq_fld_adv_source(gq_fld_plan *plan, const double *rho, const double *E_r, const double *fx,
                            const double *fy, double *S_adv, void *stream);
gq_status gq_fld_set_source(gq_fld_plan *plan, const double *S_adv);

/* Allocation-free single step (the paper has no counterpart).  For callers that cannot
 * allocate device memory: hosts whose device memory is fixed at start-up, plug-ins inside
 * another application's memory manager, loops that cannot afford the device
 * synchronisation of cudaMalloc / cudaFree.  The step is gq_fld_step's, but every piece of device scratch (geometry,
 * workspace, reductions, control) lives in one static array of gq_fld_step_noalloc_max_bytes()
 * bytes (32 MiB) that each GPU loading the library holds until the process exits; the call
 * makes no cudaMalloc / cudaFree / allocating call.  The caller passes inputs and outputs:
 * x_faces (nx+1) and y_faces (ny+1) as DEVICE arrays, the fields as in gq_fld_step (no
 * explicit areas or volumes).  Grids whose footprint exceeds the array (about 50 000 cells)
 * return GQ_ERR_INVALID_ARG before any work.  The faces are checked on the device as
 * gq_fld_setup checks them on the host (finite, strictly increasing, r > 0 and theta in
 * [0, pi] for spherical-polar grids, positive volumes): a violation returns
 * GQ_ERR_INVALID_ARG with the fields untouched.  All calls on a device share the array and
 * it keeps the previous call's contents; the call resets what must start at zero, and calls
 * that overlap on the GPU (other streams or host threads) race: serialise them.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture.  Every call synchronises with its stream before
 * returning (it reads the step's status back).  info->t_*_ms are not filled. */
gq_status gq_fld_step_noalloc(int nx, int ny, int coord, const double *x_faces, const double *y_faces,
                              const double *rho, double *e_g, double *E_r, double *T_g_out,
                              const gq_opacity_law *opacity, const gq_eos *eos, double dt, const gq_bc *bc,
                              const gq_solver_opts *opts, void *stream, gq_step_info *info);

/* Size in bytes of the static scratch array behind gq_fld_step_noalloc. */
size_t gq_fld_step_noalloc_max_bytes(void);

/* ---------------------------------------------------------------------------------------
 * Batched steps: many independent problems (each with its own plan, i.e. its own grid,
 * Cartesian or spherical-polar, and its own dt, opacity law, boundaries and options) in
 * one persistent cooperative launch.  Each problem is exactly the step of gq_fld_step;
 * batching changes only how the GPU is shared: a problem is solved by a team of blocks
 * sized to it, teams pull problems from per-size queues (largest work first), and the
 * whole step (set-up, solve, back-substitution, result gather) is captured once in a
 * CUDA graph and replayed.  Not in the paper: its code solves one grid per MPI job.
 * --------------------------------------------------------------------------------------- */

/* One problem of a batched step: the arguments of gq_fld_step, by value. */
typedef struct {
    const double *rho;
    double *e_g;
    double *E_r;
    double *T_g_out;              /* may be NULL */
    gq_opacity_law opacity;
    gq_eos eos;
    double dt;
    gq_bc bc;
    gq_solver_opts opts;
} gq_batch_item;

/* Batch schedule options.
 *   cells_per_block  a problem's team has about N / cells_per_block blocks (power of two)
 *   max_team         largest team, in blocks
 *   use_graph        1: capture the batched step in a CUDA graph on first use and replay it
 * Zero fields take the value the autotuner cached for the batch's shape class, else
 * 32768 cells per block and teams of at most 16 blocks. */
typedef struct {
    int cells_per_block;
    int max_team;
    int use_graph;
    int reserved[5];
} gq_batch_opts;

typedef struct gq_batch gq_batch;

/* Defaults: cells_per_block 0, max_team 0 (autotuned or built-in), use_graph 1. */
void gq_batch_opts_default(gq_batch_opts *opts);

/* Create a batch over n >= 1 plans on one device (host array of plan pointers, copied;
 * the plans must outlive the batch).  Allocates the schedule tables, a private stream
 * and pinned staging.  Errors: GQ_ERR_INVALID_ARG, GQ_ERR_OOM, GQ_ERR_CUDA. */
gq_status gq_batch_create(gq_fld_plan *const *plans, int n, const gq_batch_opts *opts, gq_batch **out);

/* One step of every problem: items is a host array of n items (device field pointers
 * as in gq_fld_step), infos a host array of n results (may be NULL).  The step is
 * ordered after prior work on `stream` and later work on `stream` waits for it; the
 * call returns when it has completed.  Returns GQ_OK, or the first non-OK per-problem
 * status (each problem's own status is in infos[p].status); GQ_ERR_INVALID_ARG for a
 * bad item before anything runs.  infos[p].t_solve_ms is the whole batch's device time. */
gq_status gq_batch_step(gq_batch *batch, const gq_batch_item *items, void *stream, gq_step_info *infos);

/* Rebuild the schedule with new options (NULL keeps them) from the latest per-problem
 * iteration counts; drops the captured graph. */
gq_status gq_batch_reschedule(gq_batch *batch, const gq_batch_opts *opts);

/* Autotune cells_per_block x max_team by timing full batched steps on the given items
 * (their e_g and E_r are restored afterwards; a temporary device copy of them is
 * allocated).  Keeps the fastest schedule, caches it for the batch's shape class, and
 * reports it (best and best_ms may be NULL). */
gq_status gq_batch_autotune(gq_batch *batch, const gq_batch_item *items, void *stream, gq_batch_opts *best,
                            double *best_ms);

/* Device time of the last gq_batch_step, in ms. */
double gq_batch_last_step_ms(const gq_batch *batch);

/* 1 if the batch replays a captured CUDA graph, 0 if it launches eagerly. */
int gq_batch_uses_graph(const gq_batch *batch);

/* Release a batch (not its plans; NULL is ignored). */
void gq_batch_destroy(gq_batch *batch);

/* One batched step without keeping a batch (no graph): create, step, destroy. */
gq_status gq_fld_step_batched(gq_fld_plan *const *plans, int n, const gq_batch_item *items, void *stream,
                              gq_step_info *infos);

/* ---------------------------------------------------------------------------------------
 * Serving: a continuous-batching request loop.  Requests (a grid, initial fields and a
 * number of consecutive implicit steps) are queued with host copies of their inputs.
 * Each engine tick (gq_server_poll) admits queued requests in arrival order while their
 * device footprint fits the memory budget, keeps admitted requests' state resident on
 * the device, steps every resident request once (the smaller ones together in one
 * batched launch, the large ones each on the whole GPU right after it), and retires the
 * finished ones (results copied to the caller's host buffers, memory returned).  Not in
 * the paper.
 * --------------------------------------------------------------------------------------- */

typedef struct {
    size_t budget_bytes;   /* device bytes resident requests may hold (plans + fields), > 0 */
    int max_active;        /* most requests resident and stepped together (0 = 256) */
    int use_graph;         /* 1: replay a captured graph while the resident set is unchanged */
    int solo_cells;        /* requests of at least this many cells step alone on the whole GPU
                              (gq_fld_step) after the batched launch of the smaller ones;
                              0 = 524288 (the size at which a batch team reaches its cap);
                              < 0: every request in the batched launch */
    int reserved[5];
} gq_server_opts;

typedef struct {
    gq_grid_desc grid;                      /* host geometry, copied at submit */
    const double *rho, *e_g, *E_r;          /* host initial fields [ny][nx], copied at submit */
    gq_opacity_law opacity;
    gq_eos eos;
    double dt;                              /* per step */
    gq_bc bc;
    gq_solver_opts opts;
    int n_steps;                            /* consecutive implicit steps, >= 1 */
    double *E_r_out, *e_g_out, *T_g_out;    /* host buffers [ny][nx] filled at completion (may be NULL) */
} gq_request;

typedef struct {
    int state;                 /* 0 queued, 1 resident, 2 done */
    int status;                /* gq_status (GQ_OK until a step fails) */
    int steps_done;
    int iterations;            /* Krylov iterations summed over the request's steps */
    double submit_s, admit_s, done_s;   /* host steady-clock seconds */
    double energy_before;      /* sum V (E + e_g) before the first step */
    double energy_after;       /* and after the last */
    size_t device_bytes;       /* resident footprint */
    int reserved[4];
} gq_request_info;

typedef struct gq_server gq_server;

/* Create a server on the current device.  Errors: GQ_ERR_INVALID_ARG, GQ_ERR_OOM, GQ_ERR_CUDA. */
gq_status gq_server_create(const gq_server_opts *opts, gq_server **out);

/* Device bytes a request of an nx x ny grid holds while resident (plan arena + fields). */
size_t gq_server_request_bytes(int nx, int ny);

/* Queue a request (inputs copied; output buffers must stay valid until it is done).
 * Errors: GQ_ERR_INVALID_ARG, GQ_ERR_BUDGET (the request alone exceeds the budget). */
gq_status gq_server_submit(gq_server *server, const gq_request *request, int64_t *id);

/* One engine tick: admit, step every resident request once, retire finished ones.
 * *completed (may be NULL) receives the number of requests finished in this tick.
 * A request whose step fails finishes with that status; GQ_ERR_CUDA if nothing ran. */
gq_status gq_server_poll(gq_server *server, int *completed);

/* State and timings of a request (until released). */
gq_status gq_server_info(gq_server *server, int64_t id, gq_request_info *info);

/* Forget a finished request. */
gq_status gq_server_release(gq_server *server, int64_t id);

/* Requests queued or resident. */
int gq_server_pending(gq_server *server);

/* Device bytes held by resident requests. */
size_t gq_server_used_bytes(gq_server *server);

/* Destroy the server and everything it holds (NULL is ignored). */
void gq_server_destroy(gq_server *server);

/* ---------------------------------------------------------------------------------------
 * Multilevel (statically refined) grids, Sec. 3.2.2 (Eq. linearsys1_amr and the figure of
 * the interpolation at a level jump): one implicit FLD step over a two-level Cartesian grid
 * whose base cells in one rectangle are replaced by 2 x 2 fine cells.  All composite cells
 * enter one linear system: across a level jump, a coarse cell couples directly to each of
 * the two fine cells beside its side, so it has five neighbours, and each such face is a
 * fine face (half a coarse side) whose weight dt A D / d both cells share.  Face values of
 * E and kappa_R rho are linear in the normal coordinate between the two centres (3/4 of a
 * coarse width apart across the jump), R uses their normal difference over that distance,
 * and the coarse centre's tangential offset is not used.  Everything else is the
 * single-level step (C_V, opacities at T_g^n, the limiter, Milne and reflecting sides, T
 * eliminated from the psi row, the cell-wise stop rule).
 * --------------------------------------------------------------------------------------- */

/* Two-level grid: nx x ny base cells of widths dx, dy (cm) from the origin; base cells
 * i0 <= i < i1, j0 <= j < j1 are refined (i0 == i1 or j0 == j1: no refinement; otherwise
 * 0 <= i0 < i1 <= nx, 0 <= j0 < j1 <= ny).  Composite cell order, for every field array:
 * the base cells outside the rectangle in row-major order, then the 2 (i1 - i0) x
 * 2 (j1 - j0) fine cells in row-major order (x fastest). */
typedef struct {
    int nx, ny;
    double dx, dy;
    int i0, i1, j0, j1;
} gq_smr_grid;

typedef struct gq_smr_plan gq_smr_plan;

/* Build a plan: the composite cell list, its faces (interior, with the neighbour pair,
 * A / d and the interpolation weight; boundary, with A / h) and the workspace of one step,
 * computed on the host and uploaded.  Errors: GQ_ERR_INVALID_ARG (sizes, widths not
 * positive and finite, a rectangle outside the grid), GQ_ERR_OOM, GQ_ERR_CUDA. */
gq_status gq_smr_setup(const gq_smr_grid *grid, gq_smr_plan **out);

/* Composite cells of a plan (0 for NULL). */
int gq_smr_cells(const gq_smr_plan *plan);

/* One implicit step on the composite grid.  rho, e_g, E_r, T_g_out: DEVICE arrays of
 * gq_smr_cells(plan) doubles in composite order, with the meaning and ownership of
 * gq_fld_step's.  The composite system is solved by Jacobi-preconditioned conjugate
 * gradients (opts->precond and the multigrid options are not used), FP64 or FP32 inner
 * iterations inside FP64 iterative refinement (opts->prec), to the cell-wise relative
 * residual opts->rtol; eos must be the ideal gas (table_n = 0).  Errors as gq_fld_step. */
gq_status gq_smr_step(gq_smr_plan *plan, const double *rho, double *e_g, double *E_r, double *T_g_out,
                      const gq_opacity_law *opacity, const gq_eos *eos, double dt, const gq_bc *bc,
                      const gq_solver_opts *opts, void *stream, gq_step_info *info);

/* Release a plan (NULL is ignored). */
void gq_smr_destroy(gq_smr_plan *plan);

/* Default solver options: FP64, LP limiter, rtol 1e-10, max_iter 200000, inner_rtol 0.1,
 * max_refine 200, default spin limit, keep the search direction, algebraic multigrid
 * preconditioning (omega 0.8; coarse factor 1.5 for the aggregation cycle), sub-cycled
 * steps in the paper's order (subcycle_freeze_D = 1). */
void gq_solver_opts_default(gq_solver_opts *opts);

/* Static description of a status code. */
const char *gq_status_string(gq_status status);

/* Library version "major.minor.patch". */
const char *gq_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GQ_FLD_H */
