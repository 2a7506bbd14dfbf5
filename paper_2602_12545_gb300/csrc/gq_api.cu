// C ABI of the GB300 implicit FLD step: plans (geometry + workspace) and the step call.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "gq_device.cuh"
#include "gq_geometry.cuh"
#include "gq_internal.h"

namespace {


// ---------------------------------------------------------------------------
// host geometry (FP64): volumes, face areas, volume centres, centre distances
// ---------------------------------------------------------------------------

struct HostGeometry {
    std::vector<double> V, gx, gy, dxf, thx, ymet, dyf, thy;
};

gq_status build_geometry(const gq_grid_desc* gd, HostGeometry& H) {
    const int nx = gd->nx, ny = gd->ny;
    const double* xf = gd->x_faces;
    const double* yf = gd->y_faces;
    for (int i = 0; i <= nx; i++)
        if (!std::isfinite(xf[i]) || (i > 0 && !(xf[i] > xf[i - 1]))) return GQ_ERR_INVALID_ARG;
    for (int j = 0; j <= ny; j++)
        if (!std::isfinite(yf[j]) || (j > 0 && !(yf[j] > yf[j - 1]))) return GQ_ERR_INVALID_ARG;
    const bool sph = gd->coord == GQ_SPHERICAL_POLAR;
    if (sph && (!(xf[0] > 0.0) || yf[0] < 0.0 || yf[ny] > M_PI + 1e-12)) return GQ_ERR_INVALID_ARG;

    std::vector<double> xc(nx), yc(ny), dcos(ny);
    for (int i = 0; i < nx; i++) xc[i] = gq::geom::x_centre(xf[i], xf[i + 1], sph);
    for (int j = 0; j < ny; j++) yc[j] = gq::geom::y_centre(yf[j], yf[j + 1], sph, &dcos[j]);
    const size_t N = (size_t)nx * ny;
    H.V.assign(N, 0.0);
    std::vector<double> Ax((size_t)ny * (nx + 1)), Ay((size_t)(ny + 1) * nx);
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++)
            H.V[(size_t)j * nx + i] = gq::geom::cell_volume(xf[i], xf[i + 1], yf[j], yf[j + 1], sph, dcos[j]);
    for (int j = 0; j < ny; j++)
        for (int i = 0; i <= nx; i++)
            Ax[(size_t)j * (nx + 1) + i] = gq::geom::x_face_area(xf[i], yf[j], yf[j + 1], sph, dcos[j]);
    for (int j = 0; j <= ny; j++)
        for (int i = 0; i < nx; i++)
            Ay[(size_t)j * nx + i] = gq::geom::y_face_area(yf[j], xf[i], xf[i + 1], sph);
    if (gd->volume) std::memcpy(H.V.data(), gd->volume, sizeof(double) * N);
    if (gd->area_x) std::memcpy(Ax.data(), gd->area_x, sizeof(double) * Ax.size());
    if (gd->area_y) std::memcpy(Ay.data(), gd->area_y, sizeof(double) * Ay.size());
    for (double v : H.V)
        if (!(v > 0.0) || !std::isfinite(v)) return GQ_ERR_INVALID_ARG;

    H.dxf.assign(nx + 1, 0.0);
    H.thx.assign(nx + 1, 0.0);
    H.dyf.assign(ny + 1, 0.0);
    H.thy.assign(ny + 1, 0.0);
    H.ymet.assign(nx, 1.0);
    if (sph)
        for (int i = 0; i < nx; i++) H.ymet[i] = xc[i];
    for (int i = 1; i < nx; i++) {
        H.dxf[i] = xc[i] - xc[i - 1];
        H.thx[i] = (xf[i] - xc[i - 1]) / (xc[i] - xc[i - 1]);
    }
    H.dxf[0] = xc[0] - xf[0];
    H.dxf[nx] = xf[nx] - xc[nx - 1];
    for (int j = 1; j < ny; j++) {
        H.dyf[j] = yc[j] - yc[j - 1];
        H.thy[j] = (yf[j] - yc[j - 1]) / (yc[j] - yc[j - 1]);
    }
    H.dyf[0] = yc[0] - yf[0];
    H.dyf[ny] = yf[ny] - yc[ny - 1];
    H.gx.assign(Ax.size(), 0.0);
    H.gy.assign(Ay.size(), 0.0);
    for (int j = 0; j < ny; j++)
        for (int i = 0; i <= nx; i++) H.gx[(size_t)j * (nx + 1) + i] = Ax[(size_t)j * (nx + 1) + i] / H.dxf[i];
    for (int j = 0; j <= ny; j++)
        for (int i = 0; i < nx; i++)
            H.gy[(size_t)j * nx + i] = Ay[(size_t)j * nx + i] / (H.ymet[i] * H.dyf[j]);
    return GQ_OK;
}

// bump allocator over one device allocation
struct Bump {
    char* base;
    size_t off;
    template <class T>
    T* take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off += n * sizeof(T);
        return p;
    }
};

void layout(gq_fld_plan* P, Bump& b) {
    const size_t N = P->N, nx = P->nx, ny = P->ny;
    auto& g = P->geo;
    auto& w = P->ws;
    g.V = b.take<double>(N);
    g.gx = b.take<double>(ny * (nx + 1));
    g.gy = b.take<double>((ny + 1) * nx);
    g.dxf = b.take<double>(nx + 1);
    g.thx = b.take<double>(nx + 1);
    g.ymet = b.take<double>(nx);
    g.dyf = b.take<double>(ny + 1);
    g.thy = b.take<double>(ny + 1);
    w.sig = b.take<double>(N);
    w.dloc = b.take<double>(N);
    w.rhs = b.take<double>(N);
    w.tA = b.take<double>(N);
    w.tB = b.take<double>(N);
    w.wW = b.take<double>(N);
    w.wS = b.take<double>(N);
    w.wB = b.take<double>(N);
    w.y = b.take<double>(N);
    w.r64 = b.take<double>(N);
    w.p64[0] = b.take<double>(N);
    w.p64[1] = b.take<double>(N);
    w.q64 = b.take<double>(N);
    w.cW32 = b.take<float>(N);
    w.cS32 = b.take<float>(N);
    w.d32 = b.take<float>(N);
    w.r32 = b.take<float>(N);
    w.p32[0] = b.take<float>(N);
    w.p32[1] = b.take<float>(N);
    w.q32 = b.take<float>(N);
    w.r32b = b.take<float>(N);
    // multigrid hierarchy: level l has ceil(nx / 2^l) x ceil(ny / 2^l) cells; coarsen until
    // the level has at most kCoarseMax cells
    {
        auto& mg = w.mg;
        int lx = P->nx, ly = P->ny, nl = 0;
        while (true) {
            gq::MGLevel& L = mg.L[nl];
            L.nx = lx;
            L.ny = ly;
            L.N = lx * ly;
            const size_t n = (size_t)L.N;
            if (nl == 0) {
                L.m = L.wW = L.wS = L.s = nullptr;        // level 0 lives in the workspace
                L.cW = w.cW32;
                L.cS = w.cS32;
            } else {
                L.m = b.take<double>(n);
                L.wW = b.take<double>(n);
                L.wS = b.take<double>(n);
                L.s = b.take<double>(n);
                L.cW = b.take<float>(n);
                L.cS = b.take<float>(n);
            }
            L.t = b.take<float>(n);
            L.xa = b.take<float>(n);
            L.xb = b.take<float>(n);
            L.r = nl == 0 ? nullptr : b.take<float>(n);
            nl++;
            if (L.N <= gq::kCoarseMax || nl == gq::kMaxLevels || (lx == 1 && ly == 1)) break;
            lx = (lx + 1) / 2;
            ly = (ly + 1) / 2;
        }
        mg.nlev = nl;
        const int nc = mg.L[nl - 1].N;
        mg.dense = b.take<double>((size_t)nc * 2 * nc);
        mg.inv = b.take<float>((size_t)nc * nc);
        mg.z = b.take<float>(N);
        mg.zold = b.take<float>(N);
        mg.r32 = b.take<float>(N);
        mg.p64s = nullptr;
    }
    // algebraic multigrid pools: rows of all levels (coarse levels hold at most about half
    // of their fine level's rows), off-diagonal entries (4 per fine row, about 8 per fine
    // row over the coarse levels)
    {
        auto& a = w.amg;
        a.n0 = (int)N;
        a.cap_rows = (int)(2 * N + 64);
        a.cap_nnz = (int)(12 * N + 1024);
        const size_t R = (size_t)a.cap_rows, E = (size_t)a.cap_nnz, K = gq::kAmgPmax;
        a.info = b.take<gq::AMGInfo>(1);
        a.rowptr = b.take<int>(R + gq::kAmgMaxLevels);
        a.col = b.take<int>(E);
        a.a64 = b.take<double>(E);
        a.a32 = b.take<float>(E);
        a.sfl = b.take<unsigned char>(E);
        a.diag = b.take<double>(R);
        a.s = b.take<double>(R);
        a.pc = b.take<int>(K * R);
        a.pv32 = b.take<float>(K * R);
        a.rrow = b.take<int>(R + gq::kAmgMaxLevels);
        a.rent = b.take<int>(K * R);
        a.x = b.take<float>(R);
        a.b = b.take<float>(R);
        a.t = b.take<float>(R);
        a.pv64 = b.take<double>(K * N);
        a.rowmax = b.take<double>(N);
        a.wgt = b.take<double>(N);
        a.stA = b.take<signed char>(N);
        a.stB = b.take<signed char>(N);
        a.cidx = b.take<int>(N);
        a.cf = b.take<int>(N);
        a.cnt = b.take<int>(N + 1);
        a.cnt2 = b.take<int>(N + 1);
        a.toff = b.take<int>(N);
        a.troff = b.take<int>(N);
        a.dense = b.take<double>((size_t)gq::kCoarseMax * 2 * gq::kCoarseMax);
        a.inv = b.take<float>((size_t)gq::kCoarseMax * gq::kCoarseMax);
    }
    w.partials = b.take<double>(2 * (size_t)P->solve_grid_max * gq::kSlots);
    w.epart = b.take<double>(2 * (size_t)P->setup_blocks);
    w.bar = b.take<unsigned>(2);
    w.ctl = b.take<gq::SolveCtl>(1);
}

// device, launch geometry and arena size of a plan whose nx, ny, N are set
bool size_plan(gq_fld_plan* P) {
    if (cudaGetDevice(&P->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int per_sm = gq::solve_max_blocks_per_sm();
    if (per_sm < 1) return false;
    const int need = (P->N + gq::kSolveThreads - 1) / gq::kSolveThreads;
    P->solve_grid_max = std::max(1, std::min(per_sm * P->num_sms, need));
    P->setup_blocks = std::max(1, std::min(P->num_sms * 8, (P->N + gq::kSetupThreads - 1) / gq::kSetupThreads));
    Bump sizing{nullptr, 0};
    layout(P, sizing);
    P->arena_bytes = sizing.off + 256;
    return true;
}

}  // namespace

size_t gq::plan_layout(gq_fld_plan* P, char* base) {
    Bump b{base, 0};
    layout(P, b);
    return b.off;
}

namespace {

bool finite_all(const double* v, int n) {
    for (int i = 0; i < n; i++)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace

namespace gq {

gq_status make_step_params(const gq_fld_plan* P, const double* rho, double* e_g, double* E_r, double* T_g_out,
                           const gq_opacity_law* op, const gq_eos* eos, double dt, const gq_bc* bc,
                           const gq_solver_opts* opts_in, StepParams* sp_out, SolveParams* pp_out,
                           int* timing) {
    if (!P || !rho || !e_g || !E_r || !op || !eos || !bc) return GQ_ERR_INVALID_ARG;
    gq_solver_opts opts;
    if (opts_in) opts = *opts_in;
    else gq_solver_opts_default(&opts);
    const double kR[4] = {op->k0_R, op->k1_R, op->a_R, op->b_R};
    const double kP[4] = {op->k0_P, op->k1_P, op->a_P, op->b_P};
    if (!finite_all(kR, 4) || !finite_all(kP, 4)) return GQ_ERR_INVALID_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt)) return GQ_ERR_INVALID_ARG;
    if (eos->table_n < 0 || eos->table_n == 1 || (eos->table_n >= 2 && (!eos->table_T || !eos->table_u)))
        return GQ_ERR_INVALID_ARG;
    if (!(eos->gamma > 1.0) || !(eos->mu > 0.0) || !std::isfinite(eos->gamma) || !std::isfinite(eos->mu))
        return GQ_ERR_INVALID_ARG;
    for (int s = 0; s < 4; s++)
        if (bc->side[s] != GQ_BC_REFLECT && bc->side[s] != GQ_BC_OUTFLOW_MILNE) return GQ_ERR_INVALID_ARG;
    if (opts.prec != GQ_PREC_FP64 && opts.prec != GQ_PREC_MIXED) return GQ_ERR_INVALID_ARG;
    if (opts.limiter < GQ_LIMITER_LP || opts.limiter > GQ_LIMITER_NONE) return GQ_ERR_INVALID_ARG;
    if (!(opts.rtol > 0.0) || !(opts.rtol < 1.0) || opts.max_iter < 1) return GQ_ERR_INVALID_ARG;
    if (opts.prec == GQ_PREC_MIXED && (!(opts.inner_rtol > 0.0) || !(opts.inner_rtol < 1.0)))
        return GQ_ERR_INVALID_ARG;
    if (opts.max_refine < 1 || opts.spin_limit < 0) return GQ_ERR_INVALID_ARG;
    if (opts.precond != GQ_PRECOND_JACOBI && opts.precond != GQ_PRECOND_MG && opts.precond != GQ_PRECOND_AMG)
        return GQ_ERR_INVALID_ARG;
    const double omega = opts.mg_omega == 0.0 ? 0.8 : opts.mg_omega;
    const double over = opts.mg_over == 0.0 ? 1.5 : opts.mg_over;
    if (!(omega > 0.0 && omega <= 1.0) || !(over > 0.0 && over < 2.0)) return GQ_ERR_INVALID_ARG;
    if (opts.mg_block_cells < 0) return GQ_ERR_INVALID_ARG;
    if (opts.subcycle_freeze_D != 0 && opts.subcycle_freeze_D != 1) return GQ_ERR_INVALID_ARG;
    if (opts.untiled != 0 && opts.untiled != 1) return GQ_ERR_INVALID_ARG;

    StepParams sp{};
    sp.nx = P->nx;
    sp.ny = P->ny;
    sp.N = P->N;
    for (int s = 0; s < 4; s++) sp.bc[s] = bc->side[s];
    sp.limiter = opts.limiter;
    sp.mixed = opts.prec == GQ_PREC_MIXED;
    sp.precond = opts.precond;
    for (int t = 0; t < 4; t++) {
        sp.kR[t] = kR[t];
        sp.kP[t] = kP[t];
    }
    sp.cvfac = kKB / ((eos->gamma - 1.0) * eos->mu * kMH);
    sp.eos_n = eos->table_n;
    sp.eos_T = eos->table_T;
    sp.eos_u = eos->table_u;
    sp.dt = dt;
    sp.rho = rho;
    sp.eg = e_g;
    sp.E = E_r;
    sp.eg_out = e_g;
    sp.T_out = T_g_out;
    sp.sadv = P->S_adv;
    if (P->frz_on) {
        sp.sig_n = P->frz;
        sp.E_n = P->frz + P->N;
    }

    SolveParams pp{};
    pp.nx = P->nx;
    pp.N = P->N;
    pp.mixed = sp.mixed;
    pp.restart = opts.restart;
    pp.max_iter = opts.max_iter;
    pp.max_refine = opts.max_refine;
    pp.rtol = opts.rtol;
    pp.drop = opts.inner_rtol;
    pp.spin_limit = opts.spin_limit > 0 ? opts.spin_limit : kDefaultSpin;
    pp.precond = opts.precond;
    pp.mg_omega = (float)omega;
    pp.mg_over = (float)over;
    pp.block_cells = opts.mg_block_cells > 0 ? opts.mg_block_cells : gq::kBlockLevelMax;
    pp.tiled = opts.untiled ? 0 : 1;
    *sp_out = sp;
    *pp_out = pp;
    if (timing) *timing = opts.timing;
    return GQ_OK;
}

gq_status status_of(const SolveCtl& c) {
    if (c.input_flags & 2) return GQ_ERR_NONFINITE;
    if (c.input_flags & 1) return GQ_ERR_INVALID_ARG;
    if (c.abort || c.status == kPending) return GQ_ERR_TIMEOUT;
    return static_cast<gq_status>(c.status);
}

void fill_info(const SolveCtl& c, gq_status status, gq_step_info* info) {
    info->iterations = c.iterations;
    info->refinements = c.refinements;
    info->rel_residual = c.crit;
    info->rel_residual_l2 = c.l2;
    info->energy_before = c.energy0;
    info->energy_after = c.energy1;
    info->status = status;
    info->t_precond_ms = c.t_built > c.t_start && c.t_start > 0 ? (float)((c.t_built - c.t_start) * 1e-6) : 0.f;
    info->t_iter_us = c.iterations > 0 && c.t_end > c.t_built && c.t_built > 0
                          ? (float)((double)(c.t_end - c.t_built) * 1e-3 / c.iterations)
                          : 0.f;
    info->precond_levels = c.levels;
}

}  // namespace gq

extern "C" {

const char* gq_version(void) { return "0.1.0"; }

const char* gq_status_string(gq_status s) {
    switch (s) {
        case GQ_OK: return "ok";
        case GQ_ERR_INVALID_ARG: return "invalid argument";
        case GQ_ERR_CUDA: return "CUDA error";
        case GQ_ERR_OOM: return "out of device memory";
        case GQ_ERR_NOT_CONVERGED: return "solver did not converge";
        case GQ_ERR_NONFINITE: return "non-finite value";
        case GQ_ERR_TIMEOUT: return "inter-block wait timed out";
        case GQ_ERR_BUDGET: return "memory budget exceeded";
    }
    return "unknown status";
}

void gq_solver_opts_default(gq_solver_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->prec = GQ_PREC_FP64;
    o->limiter = GQ_LIMITER_LP;
    o->rtol = 1e-10;
    o->max_iter = 200000;
    o->inner_rtol = 0.1;
    o->max_refine = 200;
    o->spin_limit = 0;
    o->restart = 0;
    o->timing = 0;
    o->precond = GQ_PRECOND_AMG;
    o->mg_omega = 0.8;
    o->mg_over = 1.5;
    o->subcycle_freeze_D = 1;
}

gq_status gq_fld_setup(const gq_grid_desc* gd, gq_fld_plan** out) {
    if (!out) return GQ_ERR_INVALID_ARG;
    *out = nullptr;
    if (!gd || !gd->x_faces || !gd->y_faces || gd->nx < 1 || gd->ny < 1) return GQ_ERR_INVALID_ARG;
    if (gd->coord != GQ_CARTESIAN && gd->coord != GQ_SPHERICAL_POLAR) return GQ_ERR_INVALID_ARG;
    if ((long long)gd->nx * gd->ny > gq::kMaxCells) return GQ_ERR_INVALID_ARG;
    HostGeometry H;
    gq_status st = build_geometry(gd, H);
    if (st != GQ_OK) return st;

    gq_fld_plan* P = new (std::nothrow) gq_fld_plan();
    if (!P) return GQ_ERR_OOM;
    P->last_precond = -1;
    P->nx = gd->nx;
    P->ny = gd->ny;
    P->N = gd->nx * gd->ny;
    P->coord = gd->coord;
    if (!size_plan(P)) {
        delete P;
        return GQ_ERR_CUDA;
    }
    if (cudaMalloc(&P->arena, P->arena_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete P;
        return GQ_ERR_OOM;
    }
    Bump real{static_cast<char*>(P->arena), 0};
    layout(P, real);
    if (cudaMallocHost(reinterpret_cast<void**>(&P->ctl_host), sizeof(gq::SolveCtl)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(P->arena);
        delete P;
        return GQ_ERR_OOM;
    }
    for (int t = 0; t < 4; t++) {
        if (cudaEventCreate(&P->ev[t]) != cudaSuccess) {
            cudaGetLastError();
            gq_fld_destroy(P);
            return GQ_ERR_CUDA;
        }
    }
    auto up = [](const double* dst, const std::vector<double>& v) {
        return cudaMemcpy(const_cast<double*>(dst), v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice);
    };
    cudaError_t e = cudaSuccess;
    const auto& g = P->geo;
    if (e == cudaSuccess) e = up(g.V, H.V);
    if (e == cudaSuccess) e = up(g.gx, H.gx);
    if (e == cudaSuccess) e = up(g.gy, H.gy);
    if (e == cudaSuccess) e = up(g.dxf, H.dxf);
    if (e == cudaSuccess) e = up(g.thx, H.thx);
    if (e == cudaSuccess) e = up(g.ymet, H.ymet);
    if (e == cudaSuccess) e = up(g.dyf, H.dyf);
    if (e == cudaSuccess) e = up(g.thy, H.thy);
    if (e != cudaSuccess) {
        gq_fld_destroy(P);
        return GQ_ERR_CUDA;
    }
    *out = P;
    return GQ_OK;
}

size_t gq_fld_plan_bytes(const gq_fld_plan* P) { return P ? P->arena_bytes : 0; }

size_t gq_fld_plan_bytes_for(int nx, int ny) {
    if (nx < 1 || ny < 1 || (long long)nx * ny > gq::kMaxCells) return 0;
    gq_fld_plan tmp{};
    tmp.nx = nx;
    tmp.ny = ny;
    tmp.N = nx * ny;
    return size_plan(&tmp) ? tmp.arena_bytes : 0;
}

void gq_fld_destroy(gq_fld_plan* P) {
    if (!P) return;
    if (P->arena) cudaFree(P->arena);
    if (P->frz) cudaFree(P->frz);
    if (P->ctl_host) cudaFreeHost(P->ctl_host);
    for (int t = 0; t < 4; t++)
        if (P->ev[t]) cudaEventDestroy(P->ev[t]);
    delete P;
}

gq_status gq_fld_set_source(gq_fld_plan* P, const double* S_adv) {
    if (!P) return GQ_ERR_INVALID_ARG;
    P->S_adv = S_adv;
    return GQ_OK;
}

gq_status gq_fld_adv_source(gq_fld_plan* P, const double* rho, const double* E_r, const double* fx,
                            const double* fy, double* S_adv, void* stream) {
    if (!P || !rho || !E_r || !fx || !fy || !S_adv) return GQ_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(P->device);
    if (e == cudaSuccess)
        e = gq::launch_adv_source(P->nx, P->ny, P->geo, rho, E_r, fx, fy, S_adv, P->setup_blocks,
                                  static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GQ_ERR_CUDA;
    }
    return GQ_OK;
}

gq_status gq_fld_precond_info(const gq_fld_plan* P, gq_precond_info* out) {
    if (!P || !out) return GQ_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->precond = P->last_precond;
    if (P->last_precond != GQ_PRECOND_AMG && P->last_precond != GQ_PRECOND_MG) return GQ_ERR_INVALID_ARG;
    gq::AMGInfo I{};
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return GQ_ERR_CUDA;
    if (cur != P->device && cudaSetDevice(P->device) != cudaSuccess) return GQ_ERR_CUDA;
    cudaError_t e = cudaMemcpy(&I, P->ws.amg.info, sizeof(I), cudaMemcpyDeviceToHost);
    if (cur != P->device) cudaSetDevice(cur);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GQ_ERR_CUDA;
    }
    for (int k = 0; k < gq::kAmgMaxLevels && k < 24; k++) out->cycle_ms[k] = (float)(I.cyc[k] * 1e-6);
    if (P->last_precond == GQ_PRECOND_MG) {
        // the fixed 2 x 2 hierarchy; its cycle time: team levels one by one, the levels
        // run by block 0 together in the slot of the first of them
        const gq::MGHierarchy& mg = P->ws.mg;
        out->levels = mg.nlev;
        out->stop_reason = 1;
        for (int l = 0; l < mg.nlev && l < 24; l++) {
            const gq::MGLevel& L = mg.L[l];
            out->rows[l] = L.N;
            out->entries[l] = 2 * ((L.nx - 1) * L.ny + L.nx * (L.ny - 1));
        }
        return GQ_OK;
    }
    const int nl = std::min(std::max(I.nlev, 0), std::min(gq::kAmgMaxLevels, 24));
    out->levels = nl;
    out->stop_reason = I.stop;
    for (int l = 0; l < nl; l++) {
        out->rows[l] = I.n[l];
        out->entries[l] = I.nnz[l];
        if (l + 1 < nl) out->build_ms[l] = (float)((I.tns[2 + l] - I.tns[1 + l]) * 1e-6);
    }
    if (nl > 0) {
        out->fine_copy_ms = (float)((I.tns[1] - I.tns[0]) * 1e-6);
        out->coarsest_ms = (float)((I.tns[nl + 1] - I.tns[nl]) * 1e-6);
    }
    for (int k = 0; k < 8; k++) out->build_phase_ms[k] = (float)(I.bph[k] * 1e-6);
    return GQ_OK;
}

gq_status gq_fld_step(gq_fld_plan* P, const double* rho, double* e_g, double* E_r, double* T_g_out,
                      const gq_opacity_law* op, const gq_eos* eos, double dt, const gq_bc* bc,
                      const gq_solver_opts* opts_in, void* stream, gq_step_info* info) {
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->status = GQ_ERR_INVALID_ARG;
    }
    gq::StepParams sp{};
    gq::SolveParams pp{};
    int timing_flag = 0;
    gq_status vs = gq::make_step_params(P, rho, e_g, E_r, T_g_out, op, eos, dt, bc, opts_in, &sp, &pp, &timing_flag);
    if (vs != GQ_OK) return vs;

    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return GQ_ERR_CUDA;
    if (cur != P->device && cudaSetDevice(P->device) != cudaSuccess) return GQ_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    const bool timing = timing_flag != 0;
    P->last_precond = pp.precond;
    cudaError_t e = cudaMemsetAsync(P->ws.ctl, 0, sizeof(gq::SolveCtl), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->ws.bar, 0, 2 * sizeof(unsigned), st);
    if (e == cudaSuccess && timing) e = cudaEventRecord(P->ev[0], st);
    if (e == cudaSuccess) e = gq::launch_setup(sp, P->geo, P->ws, P->setup_blocks, st);
    if (e == cudaSuccess && timing) e = cudaEventRecord(P->ev[1], st);
    int kernel = 0;
    if (e == cudaSuccess) e = gq::launch_solve(pp, P->ws, P->solve_grid_max, st, &kernel);
    if (e == cudaSuccess && timing) e = cudaEventRecord(P->ev[2], st);
    if (e == cudaSuccess) e = gq::launch_backsub(sp, P->geo, P->ws, P->setup_blocks, st);
    if (e == cudaSuccess && timing) e = cudaEventRecord(P->ev[3], st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->ctl_host, P->ws.ctl, sizeof(gq::SolveCtl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (cur != P->device) cudaSetDevice(cur);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (info) info->status = GQ_ERR_CUDA;
        return GQ_ERR_CUDA;
    }
    const gq::SolveCtl& c = *P->ctl_host;
    const gq_status status = gq::status_of(c);
    if (info) {
        gq::fill_info(c, status, info);
        info->solve_blocks = P->solve_grid_max;
        info->solve_kernel = kernel;
        if (timing) {
            float t0 = 0.f, t1 = 0.f, t2 = 0.f;
            cudaEventElapsedTime(&t0, P->ev[0], P->ev[1]);
            cudaEventElapsedTime(&t1, P->ev[1], P->ev[2]);
            cudaEventElapsedTime(&t2, P->ev[2], P->ev[3]);
            info->t_setup_ms = t0;
            info->t_solve_ms = t1;
            info->t_finish_ms = t2;
        }
    }
    return status;
}

gq_status gq_fld_step_subcycled(gq_fld_plan* P, const double* rho, double* e_g, double* E_r, double* T_g_out,
                                const gq_opacity_law* op, const gq_eos* eos, double dt_total, int n_sub, double q_t,
                                const gq_bc* bc, const gq_solver_opts* opts, double* Fx, double* Fy, void* stream,
                                gq_step_info* info) {
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->status = GQ_ERR_INVALID_ARG;
    }
    if (!P || n_sub < 1 || !(q_t > 0.0) || !std::isfinite(q_t) || !(dt_total > 0.0) || !std::isfinite(dt_total))
        return GQ_ERR_INVALID_ARG;
    // Eq. subtimesteps; q_t = 1 is the limit of the formula (equal sub-steps)
    const double dt0 = q_t == 1.0 ? dt_total / n_sub : dt_total * (1.0 - q_t) / (1.0 - std::pow(q_t, n_sub));
    if (!(dt0 > 0.0) || !std::isfinite(dt0)) return GQ_ERR_INVALID_ARG;
    const int freeze_D = opts ? opts->subcycle_freeze_D : 1;      // NULL options: the defaults
    if (freeze_D != 0 && freeze_D != 1) return GQ_ERR_INVALID_ARG;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    // the order of the radiation algorithm: sigma^n and E^n of the hydro step's start form
    // every sub-step's face coefficients (sub-step 1 forms them itself)
    const bool freeze = freeze_D == 1 && n_sub > 1;
    if (freeze) {
        if (!E_r) return GQ_ERR_INVALID_ARG;
        if (!P->frz) {
            if (cudaSetDevice(P->device) != cudaSuccess) return GQ_ERR_CUDA;
            if (cudaMalloc(&P->frz, 2 * sizeof(double) * (size_t)P->N) != cudaSuccess) {
                cudaGetLastError();
                P->frz = nullptr;
                return GQ_ERR_OOM;
            }
        }
        if (cudaMemcpyAsync(P->frz + P->N, E_r, sizeof(double) * (size_t)P->N, cudaMemcpyDeviceToDevice, cs) !=
            cudaSuccess) {
            cudaGetLastError();
            return GQ_ERR_CUDA;
        }
    }
    gq_step_info acc{};
    gq_status result = GQ_OK;
    for (int i = 0; i < n_sub; i++) {
        const double dt = q_t == 1.0 ? dt0 : dt0 * std::pow(q_t, i);
        gq_step_info si{};
        P->frz_on = freeze && i > 0 ? 1 : 0;
        const gq_status s = gq_fld_step(P, rho, e_g, E_r, T_g_out, op, eos, dt, bc, opts, stream, &si);
        if (freeze && i == 0 && (s == GQ_OK || s == GQ_ERR_NOT_CONVERGED)) {
            // sigma^n as sub-step 1's set-up formed it
            if (cudaMemcpyAsync(P->frz, P->ws.sig, sizeof(double) * (size_t)P->N, cudaMemcpyDeviceToDevice, cs) !=
                cudaSuccess) {
                cudaGetLastError();
                result = GQ_ERR_CUDA;
                break;
            }
        }
        if ((Fx || Fy) && (s == GQ_OK || s == GQ_ERR_NOT_CONVERGED)) {
            // this sub-step's flux, weighted by its share of the hydro step (the workspace
            // still holds its coefficients)
            gq::StepParams sp{};
            gq::SolveParams pp{};
            gq_status vs = gq::make_step_params(P, rho, e_g, E_r, T_g_out, op, eos, dt, bc, opts, &sp, &pp, nullptr);
            cudaError_t e = vs == GQ_OK ? cudaSuccess : cudaErrorInvalidValue;
            if (e == cudaSuccess)
                e = gq::launch_face_flux(sp, P->geo, P->ws, dt / dt_total, i > 0, Fx, Fy, P->setup_blocks,
                                         static_cast<cudaStream_t>(stream));
            if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
            if (e != cudaSuccess) {
                cudaGetLastError();
                result = vs == GQ_OK ? GQ_ERR_CUDA : vs;
                break;
            }
        }
        if (i == 0) acc.energy_before = si.energy_before;
        acc.iterations += si.iterations;
        acc.refinements += si.refinements;
        acc.rel_residual = std::max(acc.rel_residual, si.rel_residual);
        acc.rel_residual_l2 = std::max(acc.rel_residual_l2, si.rel_residual_l2);
        acc.energy_after = si.energy_after;
        acc.solve_blocks = si.solve_blocks;
        acc.t_setup_ms += si.t_setup_ms;
        acc.t_solve_ms += si.t_solve_ms;
        acc.t_finish_ms += si.t_finish_ms;
        acc.t_precond_ms += si.t_precond_ms;
        acc.precond_levels = si.precond_levels;
        acc.solve_kernel = si.solve_kernel;
        if (s == GQ_ERR_NOT_CONVERGED) {
            result = s;
        } else if (s != GQ_OK) {
            result = s;
            break;
        }
    }
    P->frz_on = 0;
    acc.t_iter_us = acc.iterations > 0 ? (float)(1e3 * (acc.t_solve_ms - acc.t_precond_ms) / acc.iterations) : 0.f;
    acc.status = result;
    if (info) *info = acc;
    return result;
}

}  // extern "C"
