// Set-up and back-substitution kernels of the implicit FLD step (FP64).
//
// Per cell (Sec. 3.2.1): C_V = rho k_B / ((gamma-1) mu m_H), T = e_g / C_V, power-law
// kappa_R and kappa_P at T^n, sigma = kappa_R rho, beta = kappa_P rho c dt (kappa_e =
// kappa_P), q = 4 beta a T^3.  Eliminating T^{n+1} from the psi row (Eqs. phi1-psi7)
// gives, per unit volume,
//     diag = 1 + sum_f alpha g D + beta C_V / (C_V + q),
//     rhs  = E^n + beta a T^4 C_V / (C_V + q),
//     T^{n+1} = (C_V T^n + 3 beta a T^4 + beta E^{n+1}) / (C_V + q),
// which are the exact Schur complement of the coupled system written without the
// subtraction of beta-sized terms.  Rows are multiplied by V, so the off-diagonals are
// -w_f with w_f = dt A_f D_f / d_f shared by both cells of a face (Eqs. alpha, fldg),
// and the system is symmetric positive definite.
#include "gq_device.cuh"
#include "gq_internal.h"
#include "gq_physics.cuh"

namespace gq {

namespace {

template <int NT>
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[NT / 32];
    v = warp_reduce<false>(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < NT / 32 ? sh[lane] : 0.0;
        t = warp_reduce<false>(t);
    }
    __syncthreads();
    return t;   // valid in thread 0
}

// T^n and C_V of a cell: the ideal gas (C_V = rho cvfac, T = e / C_V), or the tabulated
// u(T) inverted on the last segment whose lower end is at or below u = e / rho
// (C_V = rho du/dT there; the end segments extend the table)
__device__ __forceinline__ void cell_eos(const StepParams& sp, double rho, double e, double& cv, double& T) {
    if (sp.eos_n >= 2) {
        const double u = e / rho;
        int s = 0, a = 1, b = sp.eos_n - 2;
        while (a <= b) {
            const int m = (a + b) >> 1;
            if (sp.eos_u[m] <= u) {
                s = m;
                a = m + 1;
            } else {
                b = m - 1;
            }
        }
        const double slope = (sp.eos_u[s + 1] - sp.eos_u[s]) / (sp.eos_T[s + 1] - sp.eos_T[s]);
        T = sp.eos_T[s] + (u - sp.eos_u[s]) / slope;
        cv = rho * slope;
    } else {
        cv = rho * sp.cvfac;
        T = e / cv;
    }
}

}  // namespace

// Each body below processes one problem with nblk blocks, this block being number blk;
// the single-problem kernels pass (blockIdx.x, gridDim.x), the batched kernels the
// block's rank within its problem.

// K1a: per-cell coupling coefficients, input validation, energy before the step
__device__ void cells_body(const StepParams& sp, const DeviceGeometry& g, const Workspace& w, int blk, int nblk) {
    double eloc = 0.0;
    int flags = 0;
    for (int k = blk * blockDim.x + threadIdx.x; k < sp.N; k += nblk * blockDim.x) {
        const double rho = sp.rho[k], e = sp.eg[k], E = sp.E[k];
        // E^n + S_adv dt: the explicit part of phi_11 (S_g = 0)
        const double Ea = sp.sadv ? E + sp.dt * sp.sadv[k] : E;
        if (!(isfinite(rho) && isfinite(e) && isfinite(E) && isfinite(Ea))) flags |= 2;
        else if (!(rho > 0.0 && e > 0.0 && E > 0.0 && Ea > 0.0)) flags |= 1;
        const double V = g.V[k];
        double cv, T;
        cell_eos(sp, rho, e, cv, T);
        if (sp.eos_n >= 2 && !(cv > 0.0 && isfinite(cv) && isfinite(T))) flags |= 2;
        const double kR = opacity(sp.kR, rho, T);
        const bool same = sp.kP[0] == sp.kR[0] && sp.kP[1] == sp.kR[1] && sp.kP[2] == sp.kR[2] &&
                          sp.kP[3] == sp.kR[3];
        const double kP = same ? kR : opacity(sp.kP, rho, T);
        const double beta = kP * rho * kC * sp.dt;
        const double aT3 = kARad * T * T * T;
        const double aT4 = aT3 * T;
        const double psi6 = cv + 4.0 * beta * aT3;
        const double ipsi = 1.0 / psi6;
        const double f = cv * ipsi;
        w.sig[k] = kR * rho;
        w.dloc[k] = V * (1.0 + beta * f);
        w.rhs[k] = V * (Ea + beta * aT4 * f);
        // psi_11 = C_V T^n + 3 beta a T^4 (C_V T^n is e_g only for the ideal gas)
        w.tA[k] = (cv * T + 3.0 * beta * aT4) * ipsi;
        w.tB[k] = beta * ipsi;
        eloc += V * (E + e);
    }
    if (flags) atomicOr(&w.ctl->input_flags, flags);
    const double t = block_sum<kSetupThreads>(eloc);
    if (threadIdx.x == 0) w.epart[blk] = t;
}

// K1b: face weights (each cell owns its west and south faces; boundary faces are
// folded into the cell's diagonal)
__device__ void faces_body(const StepParams& sp, const DeviceGeometry& g, const Workspace& w, int blk, int nblk) {
    const int nx = sp.nx, ny = sp.ny;
    // sigma and E of the face coefficients: this step's, or those held from the start of
    // a sub-cycled hydro step
    const double* sg = sp.sig_n ? sp.sig_n : w.sig;
    const double* Eh = sp.E_n ? sp.E_n : sp.E;
    for (int k = blk * blockDim.x + threadIdx.x; k < sp.N; k += nblk * blockDim.x) {
        const int j = k / nx, i = k - j * nx;
        const double sk = sg[k], Ek = Eh[k];
        double ww = 0.0, ws = 0.0, wb = 0.0;
        if (i > 0)
            ww = face_weight(sg[k - 1], sk, Eh[k - 1], Ek, g.thx[i], g.dxf[i],
                             g.gx[j * (nx + 1) + i], sp.limiter, sp.dt);
        if (j > 0)
            ws = face_weight(sg[k - nx], sk, Eh[k - nx], Ek, g.thy[j], g.ymet[i] * g.dyf[j],
                             g.gy[j * nx + i], sp.limiter, sp.dt);
        if (i == 0 && sp.bc[0] == 1) wb += milne_weight(sk, g.dxf[0], g.gx[j * (nx + 1)], sp.limiter, sp.dt);
        if (i == nx - 1 && sp.bc[1] == 1)
            wb += milne_weight(sk, g.dxf[nx], g.gx[j * (nx + 1) + nx], sp.limiter, sp.dt);
        if (j == 0 && sp.bc[2] == 1) wb += milne_weight(sk, g.ymet[i] * g.dyf[0], g.gy[i], sp.limiter, sp.dt);
        if (j == ny - 1 && sp.bc[3] == 1)
            wb += milne_weight(sk, g.ymet[i] * g.dyf[ny], g.gy[ny * nx + i], sp.limiter, sp.dt);
        w.wW[k] = ww;
        w.wS[k] = ws;
        w.wB[k] = wb;
    }
}

// Galerkin coarsening of level 0 to level 1 (aggregation multigrid): for each 2 x 2
// aggregate the mass sum(V (1 + beta~) + Milne term) and the summed weights of the fine
// faces on the aggregate's west and south sides.  Runs before the diagonal pass, while
// dloc and the face weights are still unscaled.
__device__ void coarsen0_body(const StepParams& sp, const Workspace& w, int blk, int nblk) {
    if (sp.precond != GQ_PRECOND_MG || w.mg.nlev < 2) return;
    const MGLevel& C = w.mg.L[1];
    const int nx = sp.nx, ny = sp.ny;
    for (int c = blk * blockDim.x + threadIdx.x; c < C.N; c += nblk * blockDim.x) {
        const int jc = c / C.nx, ic = c - jc * C.nx;
        const int i0 = 2 * ic, j0 = 2 * jc;
        const int i1 = min(i0 + 1, nx - 1), j1 = min(j0 + 1, ny - 1);
        double m = 0.0, ww = 0.0, ws = 0.0;
        for (int j = j0; j <= j1; j++) {
            for (int i = i0; i <= i1; i++) {
                const int k = j * nx + i;
                m += w.dloc[k] + w.wB[k];
            }
            ww += w.wW[j * nx + i0];
        }
        for (int i = i0; i <= i1; i++) ws += w.wS[j0 * nx + i];
        C.m[c] = m;
        C.wW[c] = ww;
        C.wS[c] = ws;
    }
}

// K1c: diagonal of the reduced system and its Jacobi scale s = diag^{-1/2} (in place of dloc)
__device__ void diag_body(const StepParams& sp, const Workspace& w, int blk, int nblk) {
    const int nx = sp.nx, ny = sp.ny;
    for (int k = blk * blockDim.x + threadIdx.x; k < sp.N; k += nblk * blockDim.x) {
        const int j = k / nx, i = k - j * nx;
        double d = w.dloc[k] + w.wB[k] + w.wW[k] + w.wS[k];
        if (i < nx - 1) d += w.wW[k + 1];
        if (j < ny - 1) d += w.wS[k + nx];
        w.dloc[k] = 1.0 / sqrt(d);
    }
}

// K1d: scaled system  A^ = S A S (unit diagonal), b^ = S b, y0 = E^n / s; FP32 copies
__device__ void scale_body(const StepParams& sp, const Workspace& w, int blk, int nblk) {
    const int nx = sp.nx;
    const double* s = w.dloc;
    for (int k = blk * blockDim.x + threadIdx.x; k < sp.N; k += nblk * blockDim.x) {
        const int j = k / nx, i = k - j * nx;
        const double sk = s[k];
        const double cw = i > 0 ? w.wW[k] * sk * s[k - 1] : 0.0;
        const double cs = j > 0 ? w.wS[k] * sk * s[k - nx] : 0.0;
        w.wW[k] = cw;
        w.wS[k] = cs;
        w.rhs[k] *= sk;
        w.y[k] = sp.E[k] / sk;
        if (sp.mixed || sp.precond != GQ_PRECOND_JACOBI) {
            w.cW32[k] = static_cast<float>(cw);
            w.cS32[k] = static_cast<float>(cs);
        }
    }
}

// K6: back-substitution T^{n+1} = tA + tB E^{n+1}, e_g^{n+1} = e_g + C_V (T^{n+1} - T^n),
// energy after the step
__device__ void backsub_body(const StepParams& sp, const DeviceGeometry& g, const Workspace& w, int blk,
                             int nblk) {
    const SolveCtl* ctl = w.ctl;
    const int st = __ldcg(&ctl->status);
    const bool write = (st == kOk || st == kErrNotConverged) && __ldcg(&ctl->abort) == 0 &&
                       __ldcg(&ctl->input_flags) == 0;
    double eloc = 0.0;
    if (write) {
        for (int k = blk * blockDim.x + threadIdx.x; k < sp.N; k += nblk * blockDim.x) {
            const double En = w.dloc[k] * w.y[k];
            const double Tn = w.tA[k] + w.tB[k] * En;
            const double e = sp.eg[k];
            double cv, T0;
            cell_eos(sp, sp.rho[k], e, cv, T0);
            const double en = e + cv * (Tn - T0);
            sp.E[k] = En;
            sp.eg_out[k] = en;
            if (sp.T_out) sp.T_out[k] = Tn;
            eloc += g.V[k] * (En + en);
        }
    }
    const double t = block_sum<kSetupThreads>(eloc);
    if (threadIdx.x == 0) w.epart[nblk + blk] = t;
}

// deterministic final sums of the energy partials (one block per problem)
__device__ void finalize_body(const Workspace& w, int nblk) {
    double a = 0.0, b = 0.0;
    for (int t = threadIdx.x; t < nblk; t += blockDim.x) {
        a += w.epart[t];
        b += w.epart[nblk + t];
    }
    a = block_sum<kSetupThreads>(a);
    b = block_sum<kSetupThreads>(b);
    if (threadIdx.x == 0) {
        w.ctl->energy0 = a;
        w.ctl->energy1 = b;
    }
}

namespace {

__global__ void __launch_bounds__(kSetupThreads) k_cells(StepParams sp, DeviceGeometry g, Workspace w) {
    cells_body(sp, g, w, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kSetupThreads) k_faces(StepParams sp, DeviceGeometry g, Workspace w) {
    faces_body(sp, g, w, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kSetupThreads) k_diag(StepParams sp, Workspace w) {
    diag_body(sp, w, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kSetupThreads) k_coarsen0(StepParams sp, Workspace w) {
    coarsen0_body(sp, w, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kSetupThreads) k_scale(StepParams sp, Workspace w) {
    scale_body(sp, w, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kSetupThreads) k_backsub(StepParams sp, DeviceGeometry g, Workspace w) {
    backsub_body(sp, g, w, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kSetupThreads) k_finalize(Workspace w, int nblk) { finalize_body(w, nblk); }

// ---- batched variants: one launch covers every problem of a batch ---------------------

// problem p of block b: setup_prefix[p] <= b < setup_prefix[p+1] (binary search)
__device__ __forceinline__ int problem_of_block(const int* prefix, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// reset every problem's control block and barrier (status: not solved yet)
__global__ void kb_init(BatchArgs a) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += gridDim.x * blockDim.x) {
        const Workspace& w = a.desc[p].w;
        SolveCtl c{};
        c.status = kPending;
        *w.ctl = c;
        w.bar[0] = 0u;
        w.bar[1] = 0u;
    }
}

__global__ void __launch_bounds__(kSetupThreads) kb_cells(BatchArgs a) {
    const int p = problem_of_block(a.setup_prefix, a.n, blockIdx.x);
    const ProbDesc& d = a.desc[p];
    cells_body(d.sp, d.g, d.w, blockIdx.x - a.setup_prefix[p], d.setup_blocks);
}
__global__ void __launch_bounds__(kSetupThreads) kb_faces(BatchArgs a) {
    const int p = problem_of_block(a.setup_prefix, a.n, blockIdx.x);
    const ProbDesc& d = a.desc[p];
    faces_body(d.sp, d.g, d.w, blockIdx.x - a.setup_prefix[p], d.setup_blocks);
}
__global__ void __launch_bounds__(kSetupThreads) kb_coarsen0(BatchArgs a) {
    const int p = problem_of_block(a.setup_prefix, a.n, blockIdx.x);
    const ProbDesc& d = a.desc[p];
    coarsen0_body(d.sp, d.w, blockIdx.x - a.setup_prefix[p], d.setup_blocks);
}
__global__ void __launch_bounds__(kSetupThreads) kb_diag(BatchArgs a) {
    const int p = problem_of_block(a.setup_prefix, a.n, blockIdx.x);
    const ProbDesc& d = a.desc[p];
    diag_body(d.sp, d.w, blockIdx.x - a.setup_prefix[p], d.setup_blocks);
}
__global__ void __launch_bounds__(kSetupThreads) kb_scale(BatchArgs a) {
    const int p = problem_of_block(a.setup_prefix, a.n, blockIdx.x);
    const ProbDesc& d = a.desc[p];
    scale_body(d.sp, d.w, blockIdx.x - a.setup_prefix[p], d.setup_blocks);
}
__global__ void __launch_bounds__(kSetupThreads) kb_backsub(BatchArgs a) {
    const int p = problem_of_block(a.setup_prefix, a.n, blockIdx.x);
    const ProbDesc& d = a.desc[p];
    backsub_body(d.sp, d.g, d.w, blockIdx.x - a.setup_prefix[p], d.setup_blocks);
}
// one block per problem: energy sums, then gather the control block
__global__ void __launch_bounds__(kSetupThreads) kb_finalize(BatchArgs a) {
    const ProbDesc& d = a.desc[blockIdx.x];
    finalize_body(d.w, d.setup_blocks);
    __syncthreads();
    if (threadIdx.x == 0) a.ctl_out[blockIdx.x] = *d.w.ctl;
}

}  // namespace

cudaError_t launch_setup(const StepParams& sp, const DeviceGeometry& g, const Workspace& w, int nblk,
                         cudaStream_t st) {
    k_cells<<<nblk, kSetupThreads, 0, st>>>(sp, g, w);
    k_faces<<<nblk, kSetupThreads, 0, st>>>(sp, g, w);
    if (sp.precond == GQ_PRECOND_MG && w.mg.nlev > 1) k_coarsen0<<<nblk, kSetupThreads, 0, st>>>(sp, w);
    k_diag<<<nblk, kSetupThreads, 0, st>>>(sp, w);
    k_scale<<<nblk, kSetupThreads, 0, st>>>(sp, w);
    return cudaGetLastError();
}

cudaError_t launch_cells(const StepParams& sp, const DeviceGeometry& g, const Workspace& w, int nblk,
                         cudaStream_t st) {
    k_cells<<<nblk, kSetupThreads, 0, st>>>(sp, g, w);
    return cudaGetLastError();
}

cudaError_t launch_batch_setup(const BatchArgs& a, int total, cudaStream_t st) {
    kb_init<<<(a.n + 127) / 128, 128, 0, st>>>(a);
    kb_cells<<<total, kSetupThreads, 0, st>>>(a);
    kb_faces<<<total, kSetupThreads, 0, st>>>(a);
    kb_coarsen0<<<total, kSetupThreads, 0, st>>>(a);
    kb_diag<<<total, kSetupThreads, 0, st>>>(a);
    kb_scale<<<total, kSetupThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_batch_finish(const BatchArgs& a, int total, cudaStream_t st) {
    kb_backsub<<<total, kSetupThreads, 0, st>>>(a);
    kb_finalize<<<a.n, kSetupThreads, 0, st>>>(a);
    return cudaGetLastError();
}

// Eq. adv: S_adv of each cell, sum over its four faces of +-(A / V) f e_r (lower faces
// add, upper faces subtract) with e_r = E / rho of the upwind cell; a boundary face takes
// its one cell's e_r.  A face's area is its geometric factor times its normal distance
// (gx = A / dxf, gy = A / (ymet dyf)).
__global__ void k_adv_source(int nx, int ny, DeviceGeometry g, const double* __restrict__ rho,
                             const double* __restrict__ E, const double* __restrict__ fx,
                             const double* __restrict__ fy, double* __restrict__ S) {
    const int N = nx * ny;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        const int j = k / nx, i = k - j * nx;
        const double ek = E[k] / rho[k];
        const int fw = j * (nx + 1) + i, fs = j * nx + i;
        const double yw = g.ymet[i];
        double s = 0.0;
        {   // west (lower x)
            const double f = fx[fw];
            const double er = (f > 0.0 && i > 0) ? E[k - 1] / rho[k - 1] : ek;
            s += g.gx[fw] * g.dxf[i] * f * er;
        }
        {   // east (upper x)
            const double f = fx[fw + 1];
            const double er = (f < 0.0 && i < nx - 1) ? E[k + 1] / rho[k + 1] : ek;
            s -= g.gx[fw + 1] * g.dxf[i + 1] * f * er;
        }
        {   // south (lower y)
            const double f = fy[fs];
            const double er = (f > 0.0 && j > 0) ? E[k - nx] / rho[k - nx] : ek;
            s += g.gy[fs] * (yw * g.dyf[j]) * f * er;
        }
        {   // north (upper y)
            const double f = fy[fs + nx];
            const double er = (f < 0.0 && j < ny - 1) ? E[k + nx] / rho[k + nx] : ek;
            s -= g.gy[fs + nx] * (yw * g.dyf[j + 1]) * f * er;
        }
        S[k] = s / g.V[k];
    }
}

cudaError_t launch_adv_source(int nx, int ny, const DeviceGeometry& g, const double* rho, const double* E,
                              const double* fx, const double* fy, double* S, int nblk, cudaStream_t st) {
    k_adv_source<<<nblk, kSetupThreads, 0, st>>>(nx, ny, g, rho, E, fx, fy, S);
    return cudaGetLastError();
}

// Radiative face flux of a finished step (F = -D grad E with the step's D and E^{n+1},
// positive along +x / +y), times weight, written (accumulate = 0) or added to Fx
// [ny][nx+1] and Fy [ny+1][nx].  Interior faces: D / d from the face weight w = dt A D / d
// (recovered as c / (s_k s_m) from the scaled coupling); Milne faces: D_b E / (h (1 + k)),
// outward; reflecting faces: 0.
__global__ void k_face_flux(StepParams sp, DeviceGeometry g, Workspace w, double weight, int accumulate, double* Fx,
                            double* Fy) {
    const int nx = sp.nx, ny = sp.ny;
    const long long nfx = (long long)ny * (nx + 1), nfy = (long long)(ny + 1) * nx;
    const double* E = sp.E;
    const double* s = w.dloc;
    const double* sg = sp.sig_n ? sp.sig_n : w.sig;   // the sigma the Milne faces were formed with
    auto milne = [&](double sig, double h, double Ek) {
        const double kk = 2.0 / (3.0 * sig * h);
        return kC * limiter(sp.limiter, 1.5) / sig * Ek / (h * (1.0 + kk));
    };
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nfx + nfy;
         t += (long long)gridDim.x * blockDim.x) {
        double F = 0.0;
        if (t < nfx) {
            const int j = (int)(t / (nx + 1)), i = (int)(t - (long long)j * (nx + 1));
            if (i > 0 && i < nx) {
                const int k = j * nx + i;
                const double gA = g.gx[t];
                if (gA > 0.0) F = w.wW[k] / (s[k] * s[k - 1]) / (sp.dt * gA) * (E[k - 1] - E[k]) / g.dxf[i];
            } else if (sp.bc[i == 0 ? 0 : 1] == GQ_BC_OUTFLOW_MILNE) {
                const int k = j * nx + (i == 0 ? 0 : nx - 1);
                F = (i == 0 ? -1.0 : 1.0) * milne(sg[k], g.dxf[i], E[k]);
            }
            if (Fx) Fx[t] = (accumulate ? Fx[t] : 0.0) + weight * F;
        } else {
            const long long f = t - nfx;
            const int j = (int)(f / nx), i = (int)(f - (long long)j * nx);
            if (j > 0 && j < ny) {
                const int k = j * nx + i;
                const double gA = g.gy[f];
                if (gA > 0.0)
                    F = w.wS[k] / (s[k] * s[k - nx]) / (sp.dt * gA) * (E[k - nx] - E[k]) / (g.ymet[i] * g.dyf[j]);
            } else if (sp.bc[j == 0 ? 2 : 3] == GQ_BC_OUTFLOW_MILNE) {
                const int k = j == 0 ? i : (ny - 1) * nx + i;
                F = (j == 0 ? -1.0 : 1.0) * milne(sg[k], g.ymet[i] * g.dyf[j], E[k]);
            }
            if (Fy) Fy[f] = (accumulate ? Fy[f] : 0.0) + weight * F;
        }
    }
}

cudaError_t launch_face_flux(const StepParams& sp, const DeviceGeometry& g, const Workspace& w, double weight,
                             bool accumulate, double* Fx, double* Fy, int nblk, cudaStream_t st) {
    k_face_flux<<<nblk, kSetupThreads, 0, st>>>(sp, g, w, weight, accumulate ? 1 : 0, Fx, Fy);
    return cudaGetLastError();
}

cudaError_t launch_backsub(const StepParams& sp, const DeviceGeometry& g, const Workspace& w, int nblk,
                           cudaStream_t st) {
    k_backsub<<<nblk, kSetupThreads, 0, st>>>(sp, g, w);
    k_finalize<<<1, kSetupThreads, 0, st>>>(w, nblk);
    return cudaGetLastError();
}

}  // namespace gq
