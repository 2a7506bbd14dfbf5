// Implicit FLD step on a two-level (statically refined) Cartesian grid: the multilevel
// matrix of Sec. 3.2.2 (Eq. linearsys1_amr).
//
// The composite cell list is the base cells outside one refined rectangle followed by the
// fine cells that replace it (2 x 2 per base cell).  Every face of the composite grid is a
// pair of cells with A / d and the interpolation weight of its position between the two
// volume centres; across a level jump a coarse side splits into two fine faces, so the
// coarse cell has up to five neighbours and shares each face weight dt A D / d with the
// fine cell across it (the flux leaving one equals the flux entering the other).
//
// Device path: the per-cell pass of the single-level set-up (C_V, T^n, opacities, mass
// term and right-hand side, input checks, energy before the step; launch_cells), then
//   k_smr_faces   face weights w_f = dt (A / d) c lambda(R_f) / sigma_f, one thread a face;
//   k_smr_diag    diagonal V (1 + beta~) + sum of the cell's face weights + Milne terms,
//                 Jacobi scale s = diag^{-1/2};
//   k_smr_scale   scaled couplings c = w s_k s_m in a slot-major ELL layout ([5][N], FP64 and
//                 FP32), b^ = s b, y0 = E^n / s;
//   k_smr_pcg     one persistent cooperative launch: conjugate gradients on the scaled
//                 system (unit diagonal, i.e. Jacobi preconditioning) in FP64 or in FP32
//                 inside FP64 iterative refinement, with the cell-wise stop rule
//                 max_k |b^ - A^ y|_k / |y_k| <= rtol;
// and the single-level back-substitution (T^{n+1}, e_g^{n+1}, energy after the step).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "gq_device.cuh"
#include "gq_internal.h"
#include "gq_physics.cuh"

namespace gq {
namespace {

constexpr int kSmrSlots = 5;          // neighbours of a composite cell (a coarse cell beside the patch)
constexpr int kSmrThreads = 512;      // threads of a solve block
constexpr int kSmrRed = 4;            // reduction slots

// geometry of the composite grid in device memory
struct SmrGeometry {
    int N, nf;
    const double* V;       // [N]
    const int* fk;         // [nf] cell on the lower side of face f
    const int* fm;         // [nf] cell on the upper side
    const double* fgeo;    // [nf] A / d
    const double* fth;     // [nf] (x_f - x_k) / (x_m - x_k)
    const double* fd;      // [nf] d = x_m - x_k
    const int* nb;         // [kSmrSlots][N] neighbour in slot s (the cell itself when empty)
    const int* nf_of;      // [kSmrSlots][N] face in slot s (-1 when empty)
    const double* bgeo;    // [4][N] A / h of the cell's boundary face on side s (0: none)
    const double* bh;      // [4][N] h of that face (half the cell width)
};

struct SmrWork {
    double* w;             // [nf] face weights
    double* c64;           // [kSmrSlots][N] scaled couplings
    float* c32;            // [kSmrSlots][N]
    double *r64, *p64[2], *q64, *d64;   // FP64 inner vectors
    float *r32, *p32[2], *q32, *d32;    // FP32 inner vectors
};

struct SmrSolve {
    int N;
    int max_iter, max_refine;
    double rtol, drop;
    long long spin;
    SmrGeometry g;
    SmrWork v;
    Workspace w;           // s (dloc), b^ (rhs), y, partials, barrier, control block
};

__global__ void __launch_bounds__(kSetupThreads) k_smr_faces(SmrGeometry g, const double* sig, const double* E,
                                                             int lim, double dt, double* w) {
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < g.nf; f += gridDim.x * blockDim.x) {
        const int k = g.fk[f], m = g.fm[f];
        w[f] = face_weight(sig[k], sig[m], E[k], E[m], g.fth[f], g.fd[f], g.fgeo[f], lim, dt);
    }
}

__global__ void __launch_bounds__(kSetupThreads) k_smr_diag(SmrGeometry g, Workspace ws, const double* w,
                                                            gq_bc bc, int lim, double dt) {
    const int N = g.N;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        double d = ws.dloc[k];
        for (int s = 0; s < kSmrSlots; s++) {
            const int f = g.nf_of[s * N + k];
            if (f >= 0) d += w[f];
        }
        for (int side = 0; side < 4; side++) {
            const double geo = g.bgeo[side * N + k];
            if (geo > 0.0 && bc.side[side] == GQ_BC_OUTFLOW_MILNE)
                d += milne_weight(ws.sig[k], g.bh[side * N + k], geo, lim, dt);
        }
        ws.dloc[k] = 1.0 / sqrt(d);
    }
}

__global__ void __launch_bounds__(kSetupThreads) k_smr_scale(SmrGeometry g, Workspace ws, SmrWork v,
                                                             const double* E) {
    const int N = g.N;
    const double* s = ws.dloc;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        const double sk = s[k];
        for (int t = 0; t < kSmrSlots; t++) {
            const int f = g.nf_of[t * N + k];
            const double c = f >= 0 ? v.w[f] * sk * s[g.nb[t * N + k]] : 0.0;
            v.c64[t * N + k] = c;
            v.c32[t * N + k] = static_cast<float>(c);
        }
        ws.rhs[k] *= sk;
        ws.y[k] = E[k] / sk;
    }
}

struct SmrShared {
    double warp[kSmrThreads / 32][kSmrRed];
    double tot[kSmrRed];
};

// block-reduce NS values (sums, except a max in slot MAXSLOT if >= 0), publish the block
// partials, wait for the grid, reduce the partials in one order in every block
template <int NS, int MAXSLOT>
__device__ bool smr_allreduce(double (&v)[NS], const SmrSolve& P, int& parity, SmrShared& sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int G = gridDim.x;
#pragma unroll
    for (int s = 0; s < NS; s++) {
        v[s] = s == MAXSLOT ? warp_reduce<true>(v[s]) : warp_reduce<false>(v[s]);
        if (lane == 0) sh.warp[warp][s] = v[s];
    }
    __syncthreads();
    double* mine = P.w.partials + (size_t)parity * G * kSlots;
    if (warp == 0) {
#pragma unroll
        for (int s = 0; s < NS; s++) {
            double a = lane < nw ? sh.warp[lane][s] : 0.0;
            a = s == MAXSLOT ? warp_reduce<true>(a) : warp_reduce<false>(a);
            if (lane == 0) mine[blockIdx.x * kSlots + s] = a;
        }
    }
    if (!team_barrier(P.w.bar, Team{static_cast<int>(blockIdx.x), G}, P.spin, &P.w.ctl->abort)) return false;
    if (warp == 0) {
#pragma unroll
        for (int s = 0; s < NS; s++) {
            double a = 0.0;
            for (int b = lane; b < G; b += 32) {
                const double z = __ldcg(mine + b * kSlots + s);
                a = s == MAXSLOT ? nanmax(a, z) : a + z;
            }
            a = s == MAXSLOT ? warp_reduce<true>(a) : warp_reduce<false>(a);
            if (lane == 0) sh.tot[s] = a;
        }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < NS; s++) v[s] = sh.tot[s];
    parity ^= 1;
    return true;
}

// (A^ x)_k with unit diagonal and the ELL couplings (R = float or double)
template <class R>
__device__ __forceinline__ R smr_apply(const R* __restrict__ c, const int* __restrict__ nb, const R* x, int k,
                                       int N) {
    R a = __ldcg(x + k);
#pragma unroll
    for (int t = 0; t < kSmrSlots; t++) a -= c[t * N + k] * __ldcg(x + nb[t * N + k]);
    return a;
}

// Conjugate gradients on A^ d = r in precision R inside FP64 iterative refinement of
// A^ y = b^.  The inner residual is carried with a power-of-two scale that keeps its
// entries O(1); the refinement (y += d / scale, FP64 residual, stop tests) happens when
// the inner residual has fallen by `drop`, and the search direction is kept across it.
template <bool MIXED>
__global__ void __launch_bounds__(kSmrThreads, 1) k_smr_pcg(SmrSolve P) {
    using R = std::conditional_t<MIXED, float, double>;
    __shared__ SmrShared sh;
    const int N = P.N;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    SolveCtl* ctl = P.w.ctl;
    const double* __restrict__ bh = P.w.rhs;
    const double* __restrict__ s = P.w.dloc;
    double* y = P.w.y;
    const int* nb = P.g.nb;
    const double* c64 = P.v.c64;
    const R* c;
    R *r, *pb[2], *q, *d;
    if constexpr (MIXED) {
        c = P.v.c32; r = P.v.r32; pb[0] = P.v.p32[0]; pb[1] = P.v.p32[1]; q = P.v.q32; d = P.v.d32;
    } else {
        c = P.v.c64; r = P.v.r64; pb[0] = P.v.p64[0]; pb[1] = P.v.p64[1]; q = P.v.q64; d = P.v.d64;
    }
    double* r64 = P.v.r64;
    int parity = 0;
    const int flags = __ldcg(&ctl->input_flags);
    if (flags) {
        if (tid == 0) ctl->status = (flags & 2) ? kErrNonfinite : kErrInvalid;
        return;
    }
    if (tid == 0) ctl->t_start = ctl->t_built = global_ns();

    int it = 0, nref = -1, status = kErrNotConverged, stall = 0, it_best = 0, cur = 0;
    double crit = 0.0, l2 = 0.0, bb = 1.0, best = 0.0, rr = 0.0, rr_ref = 0.0, scale = 1.0;
    bool use_p = false;
    while (true) {
        // ---- refinement: y += d / scale; FP64 residual r64 = b^ - A^ y; norms --------
        double t4[4] = {0.0, 0.0, 0.0, 0.0};   // |r|^2, |r / s|^2, |b / s|^2, max |r_k / y_k|
        const double inv = 1.0 / scale;
        if (nref >= 0) {
            for (int k = tid; k < N; k += stride) {
                y[k] += static_cast<double>(d[k]) * inv;
                d[k] = R(0);
            }
            if (!team_barrier(P.w.bar, Team{static_cast<int>(blockIdx.x), static_cast<int>(gridDim.x)}, P.spin,
                              &ctl->abort))
                goto timeout;
        }
        for (int k = tid; k < N; k += stride) {
            const double rk = bh[k] - smr_apply<double>(c64, nb, y, k, N);
            r64[k] = rk;
            if (nref < 0) d[k] = R(0);
            const double ru = rk / s[k], bu = bh[k] / s[k];
            t4[0] += rk * rk;
            t4[1] += ru * ru;
            t4[2] += bu * bu;
            t4[3] = nanmax(t4[3], fabs(rk / __ldcg(y + k)));
        }
        if (!smr_allreduce<4, 3>(t4, P, parity, sh)) goto timeout;
        nref++;
        if (nref == 0) bb = t4[2];
        crit = t4[3];
        l2 = sqrt(t4[1] / bb);
        if (!isfinite(t4[0]) || !(crit == crit)) { status = kErrNonfinite; break; }
        if (crit <= P.rtol) { status = kOk; break; }
        if (nref == 0 || crit < 0.9 * best) {
            best = crit;
            it_best = it;
            stall = 0;
        } else {
            stall++;
        }
        if (it >= P.max_iter || nref >= P.max_refine || (stall >= 6 && it - it_best >= 32)) {
            status = kErrNotConverged;
            break;
        }
        {
            // new inner residual: r = scale * r64, with the power-of-two scale fixed at the
            // first residual so that FP32 entries start O(1) (the kept direction and the
            // correction d stay in one unit throughout)
            if (nref == 0) {
                double mx[1] = {0.0};
                for (int k = tid; k < N; k += stride) mx[0] = nanmax(mx[0], fabs(r64[k]));
                if (!smr_allreduce<1, 0>(mx, P, parity, sh)) goto timeout;
                scale = MIXED ? exp2(-(double)ilogb(mx[0] > 0.0 ? mx[0] : 1.0)) : 1.0;
            }
            for (int k = tid; k < N; k += stride) r[k] = static_cast<R>(r64[k] * scale);
            const double rr_true = t4[0] * scale * scale;
            // keep the direction: the new residual continues the old Krylov recurrence
            const double beta0 = (use_p && rr > 0.0) ? rr_true / rr : 0.0;
            rr = rr_true;
            rr_ref = rr_true;
            if (!team_barrier(P.w.bar, Team{static_cast<int>(blockIdx.x), static_cast<int>(gridDim.x)}, P.spin,
                              &ctl->abort))
                goto timeout;
            double beta = beta0;
            // ---- inner CG ------------------------------------------------------------
            while (true) {
                // S: p = r + beta p_old (own cell and neighbours), q = A^ p, p.q
                const R* __restrict__ pold = pb[cur];
                R* __restrict__ pnew = pb[cur ^ 1];
                const R rb = static_cast<R>(beta);
                double pq[1] = {0.0};
                for (int k = tid; k < N; k += stride) {
                    const R pk = use_p ? __ldcg(r + k) + rb * __ldcg(pold + k) : __ldcg(r + k);
                    R a = pk;
#pragma unroll
                    for (int t = 0; t < kSmrSlots; t++) {
                        const int m = nb[t * N + k];
                        const R pm = use_p ? __ldcg(r + m) + rb * __ldcg(pold + m) : __ldcg(r + m);
                        a -= c[t * N + k] * pm;
                    }
                    pnew[k] = pk;
                    q[k] = a;
                    pq[0] += static_cast<double>(pk) * static_cast<double>(a);
                }
                if (!smr_allreduce<1, -1>(pq, P, parity, sh)) goto timeout;
                if (!isfinite(pq[0])) { status = kErrNonfinite; goto done; }
                if (!(pq[0] > 0.0)) break;          // rounding noise: go to the FP64 check
                const R ra = static_cast<R>(rr / pq[0]);
                cur ^= 1;
                use_p = true;
                // U: d += alpha p, r -= alpha q, r.r
                double rn[1] = {0.0};
                for (int k = tid; k < N; k += stride) {
                    const R rk = r[k] - ra * q[k];
                    d[k] += ra * pnew[k];
                    r[k] = rk;
                    rn[0] += static_cast<double>(rk) * static_cast<double>(rk);
                }
                if (!smr_allreduce<1, -1>(rn, P, parity, sh)) goto timeout;
                it++;
                if (!isfinite(rn[0])) { status = kErrNonfinite; goto done; }
                beta = rn[0] / rr;
                rr = rn[0];
                if (sqrt(rr) <= P.drop * sqrt(rr_ref) || it >= P.max_iter) break;
            }
        }
    }
done:
    if (tid == 0) {
        ctl->t_end = global_ns();
        ctl->status = status;
        ctl->iterations = it;
        ctl->refinements = nref;
        ctl->crit = crit;
        ctl->l2 = l2;
        ctl->levels = 1;
    }
    return;
timeout:
    if (threadIdx.x == 0) atomicExch(&ctl->status, kErrTimeout);
}

int smr_blocks_per_sm(bool mixed) {
    int nb = 0;
    const cudaError_t e = mixed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_smr_pcg<true>, kSmrThreads, 0)
                                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_smr_pcg<false>, kSmrThreads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

// ---- host: the composite grid -----------------------------------------------------------

struct HostFace {
    int k, m;
    double geo, th, d;
};

struct HostComposite {
    int N = 0;
    std::vector<double> V, x, y, hx, hy;
    std::vector<HostFace> faces;
    std::vector<int> nb, nf_of;          // [kSmrSlots][N]
    std::vector<double> bgeo, bh;        // [4][N]
};

gq_status build_composite(const gq_smr_grid& G, HostComposite& H) {
    const bool patch = G.i0 < G.i1 && G.j0 < G.j1;
    const int pw = patch ? G.i1 - G.i0 : 0, ph = patch ? G.j1 - G.j0 : 0;
    const int nfx = 2 * pw, nfy = 2 * ph;
    auto refined = [&](int i, int j) { return patch && i >= G.i0 && i < G.i1 && j >= G.j0 && j < G.j1; };
    std::vector<int> cidx((size_t)G.nx * G.ny, -1), fidx((size_t)nfx * nfy, -1);
    const double dx = G.dx, dy = G.dy;
    for (int j = 0; j < G.ny; j++)
        for (int i = 0; i < G.nx; i++)
            if (!refined(i, j)) {
                cidx[(size_t)j * G.nx + i] = (int)H.x.size();
                H.x.push_back((i + 0.5) * dx);
                H.y.push_back((j + 0.5) * dy);
                H.hx.push_back(dx);
                H.hy.push_back(dy);
            }
    for (int J = 0; J < nfy; J++)
        for (int I = 0; I < nfx; I++) {
            fidx[(size_t)J * nfx + I] = (int)H.x.size();
            H.x.push_back(G.i0 * dx + (I + 0.5) * 0.5 * dx);
            H.y.push_back(G.j0 * dy + (J + 0.5) * 0.5 * dy);
            H.hx.push_back(0.5 * dx);
            H.hy.push_back(0.5 * dy);
        }
    const int N = (int)H.x.size();
    H.N = N;
    H.V.resize(N);
    for (int k = 0; k < N; k++) H.V[k] = H.hx[k] * H.hy[k];
    H.nb.assign((size_t)kSmrSlots * N, 0);
    H.nf_of.assign((size_t)kSmrSlots * N, -1);
    for (int t = 0; t < kSmrSlots; t++)
        for (int k = 0; k < N; k++) H.nb[(size_t)t * N + k] = k;
    H.bgeo.assign((size_t)4 * N, 0.0);
    H.bh.assign((size_t)4 * N, 0.0);
    std::vector<int> used(N, 0);
    bool overflow = false;
    // face between k (lower) and m (upper) along axis (0: x, 1: y) with area A at normal
    // coordinate pos
    auto add_face = [&](int k, int m, int axis, double A, double pos) {
        const double pk = axis == 0 ? H.x[k] : H.y[k], pm = axis == 0 ? H.x[m] : H.y[m];
        const double d = pm - pk;
        const int f = (int)H.faces.size();
        H.faces.push_back(HostFace{k, m, A / d, (pos - pk) / d, d});
        for (int c : {k, m}) {
            if (used[c] >= kSmrSlots) {
                overflow = true;
                continue;
            }
            H.nb[(size_t)used[c] * N + c] = c == k ? m : k;
            H.nf_of[(size_t)used[c] * N + c] = f;
            used[c]++;
        }
    };
    auto add_boundary = [&](int k, int side, double A, double h) {
        H.bgeo[(size_t)side * N + k] = A / h;
        H.bh[(size_t)side * N + k] = h;
    };
    auto fine_at = [&](int I, int J) { return fidx[(size_t)J * nfx + I]; };
    auto coarse_at = [&](int i, int j) { return cidx[(size_t)j * G.nx + i]; };
    // base cells outside the patch: their +x and +y sides, and domain boundaries
    for (int j = 0; j < G.ny; j++)
        for (int i = 0; i < G.nx; i++) {
            if (refined(i, j)) continue;
            const int k = coarse_at(i, j);
            if (i == 0) add_boundary(k, 0, dy, 0.5 * dx);
            if (j == 0) add_boundary(k, 2, dx, 0.5 * dy);
            if (i == G.nx - 1) add_boundary(k, 1, dy, 0.5 * dx);
            else if (!refined(i + 1, j)) add_face(k, coarse_at(i + 1, j), 0, dy, (i + 1) * dx);
            else {
                const int I = 2 * (i + 1 - G.i0), J = 2 * (j - G.j0);
                add_face(k, fine_at(I, J), 0, 0.5 * dy, (i + 1) * dx);
                add_face(k, fine_at(I, J + 1), 0, 0.5 * dy, (i + 1) * dx);
            }
            if (j == G.ny - 1) add_boundary(k, 3, dx, 0.5 * dy);
            else if (!refined(i, j + 1)) add_face(k, coarse_at(i, j + 1), 1, dx, (j + 1) * dy);
            else {
                const int I = 2 * (i - G.i0), J = 2 * (j + 1 - G.j0);
                add_face(k, fine_at(I, J), 1, 0.5 * dx, (j + 1) * dy);
                add_face(k, fine_at(I + 1, J), 1, 0.5 * dx, (j + 1) * dy);
            }
        }
    // fine cells: their +x and +y sides (to a fine cell, to a coarse cell across the
    // patch edge, or the domain boundary), and domain boundaries on their -x / -y sides
    for (int J = 0; J < nfy; J++)
        for (int I = 0; I < nfx; I++) {
            const int k = fine_at(I, J);
            const double xe = G.i0 * dx + (I + 1) * 0.5 * dx, yn = G.j0 * dy + (J + 1) * 0.5 * dy;
            if (I == 0 && G.i0 == 0) add_boundary(k, 0, 0.5 * dy, 0.25 * dx);
            if (J == 0 && G.j0 == 0) add_boundary(k, 2, 0.5 * dx, 0.25 * dy);
            if (I + 1 < nfx) add_face(k, fine_at(I + 1, J), 0, 0.5 * dy, xe);
            else if (G.i1 == G.nx) add_boundary(k, 1, 0.5 * dy, 0.25 * dx);
            else add_face(k, coarse_at(G.i1, G.j0 + J / 2), 0, 0.5 * dy, xe);
            if (J + 1 < nfy) add_face(k, fine_at(I, J + 1), 1, 0.5 * dx, yn);
            else if (G.j1 == G.ny) add_boundary(k, 3, 0.5 * dx, 0.25 * dy);
            else add_face(k, coarse_at(G.i0 + I / 2, G.j1), 1, 0.5 * dx, yn);
        }
    // the coarse cells on the patch's lower sides: their +x / +y faces into the patch were
    // added from the coarse side above; the fine cells' -x / -y faces into coarse cells are
    // those same faces
    return overflow ? GQ_ERR_INVALID_ARG : GQ_OK;
}

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

}  // namespace
}  // namespace gq

struct gq_smr_plan {
    int N, nf;
    int device, num_sms, grid_max, setup_blocks;
    void* arena;
    size_t arena_bytes;
    gq::SmrGeometry g;
    gq::SmrWork v;
    gq::Workspace w;
    gq::DeviceGeometry geo;      // V only (for the shared cell pass and back-substitution)
    gq::SolveCtl* ctl_host;
};

namespace {

void smr_layout(gq_smr_plan* P, gq::Bump& b) {
    const size_t N = P->N, nf = std::max(P->nf, 1);
    auto& g = P->g;
    auto& v = P->v;
    auto& w = P->w;
    g.N = P->N;
    g.nf = P->nf;
    g.V = b.take<double>(N);
    g.fk = b.take<int>(nf);
    g.fm = b.take<int>(nf);
    g.fgeo = b.take<double>(nf);
    g.fth = b.take<double>(nf);
    g.fd = b.take<double>(nf);
    g.nb = b.take<int>(gq::kSmrSlots * N);
    g.nf_of = b.take<int>(gq::kSmrSlots * N);
    g.bgeo = b.take<double>(4 * N);
    g.bh = b.take<double>(4 * N);
    v.w = b.take<double>(nf);
    v.c64 = b.take<double>(gq::kSmrSlots * N);
    v.c32 = b.take<float>(gq::kSmrSlots * N);
    v.r64 = b.take<double>(N);
    v.p64[0] = b.take<double>(N);
    v.p64[1] = b.take<double>(N);
    v.q64 = b.take<double>(N);
    v.d64 = b.take<double>(N);
    v.r32 = b.take<float>(N);
    v.p32[0] = b.take<float>(N);
    v.p32[1] = b.take<float>(N);
    v.q32 = b.take<float>(N);
    v.d32 = b.take<float>(N);
    std::memset(&w, 0, sizeof(w));
    w.sig = b.take<double>(N);
    w.dloc = b.take<double>(N);
    w.rhs = b.take<double>(N);
    w.tA = b.take<double>(N);
    w.tB = b.take<double>(N);
    w.y = b.take<double>(N);
    w.partials = b.take<double>(2 * (size_t)P->grid_max * gq::kSlots);
    w.epart = b.take<double>(2 * (size_t)P->setup_blocks);
    w.bar = b.take<unsigned>(2);
    w.ctl = b.take<gq::SolveCtl>(1);
    std::memset(&P->geo, 0, sizeof(P->geo));
    P->geo.V = g.V;
}

}  // namespace

extern "C" {

gq_status gq_smr_setup(const gq_smr_grid* G, gq_smr_plan** out) {
    if (!out) return GQ_ERR_INVALID_ARG;
    *out = nullptr;
    if (!G || G->nx < 1 || G->ny < 1) return GQ_ERR_INVALID_ARG;
    if (!(G->dx > 0.0) || !(G->dy > 0.0) || !std::isfinite(G->dx) || !std::isfinite(G->dy)) return GQ_ERR_INVALID_ARG;
    const bool patch = G->i0 != G->i1 && G->j0 != G->j1;
    if (patch && !(G->i0 >= 0 && G->i0 < G->i1 && G->i1 <= G->nx && G->j0 >= 0 && G->j0 < G->j1 && G->j1 <= G->ny))
        return GQ_ERR_INVALID_ARG;
    const long long n_est = (long long)G->nx * G->ny + (patch ? 3ll * (G->i1 - G->i0) * (G->j1 - G->j0) : 0);
    if (n_est > gq::kMaxCells) return GQ_ERR_INVALID_ARG;
    gq_smr_grid g = *G;
    if (!patch) g.i0 = g.i1 = g.j0 = g.j1 = 0;
    gq::HostComposite H;
    gq_status st = gq::build_composite(g, H);
    if (st != GQ_OK) return st;

    gq_smr_plan* P = new (std::nothrow) gq_smr_plan();
    if (!P) return GQ_ERR_OOM;
    P->N = H.N;
    P->nf = (int)H.faces.size();
    if (cudaGetDevice(&P->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device) != cudaSuccess) {
        cudaGetLastError();
        delete P;
        return GQ_ERR_CUDA;
    }
    const int per_sm = std::min(gq::smr_blocks_per_sm(true), gq::smr_blocks_per_sm(false));
    if (per_sm < 1) {
        delete P;
        return GQ_ERR_CUDA;
    }
    P->grid_max = std::max(1, std::min(per_sm * P->num_sms, (P->N + gq::kSmrThreads - 1) / gq::kSmrThreads));
    P->setup_blocks = std::max(1, std::min(P->num_sms * 8, (P->N + gq::kSetupThreads - 1) / gq::kSetupThreads));
    gq::Bump sizing{nullptr, 0};
    smr_layout(P, sizing);
    P->arena_bytes = sizing.off + 256;
    if (cudaMalloc(&P->arena, P->arena_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete P;
        return GQ_ERR_OOM;
    }
    gq::Bump real{static_cast<char*>(P->arena), 0};
    smr_layout(P, real);
    if (cudaMallocHost(reinterpret_cast<void**>(&P->ctl_host), sizeof(gq::SolveCtl)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(P->arena);
        delete P;
        return GQ_ERR_OOM;
    }
    std::vector<int> fk(P->nf), fm(P->nf);
    std::vector<double> fgeo(P->nf), fth(P->nf), fd(P->nf);
    for (int f = 0; f < P->nf; f++) {
        fk[f] = H.faces[f].k;
        fm[f] = H.faces[f].m;
        fgeo[f] = H.faces[f].geo;
        fth[f] = H.faces[f].th;
        fd[f] = H.faces[f].d;
    }
    auto up = [](const void* dst, const void* src, size_t bytes) {
        return bytes ? cudaMemcpy(const_cast<void*>(dst), src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
    };
    cudaError_t e = up(P->g.V, H.V.data(), sizeof(double) * H.N);
    if (e == cudaSuccess) e = up(P->g.fk, fk.data(), sizeof(int) * P->nf);
    if (e == cudaSuccess) e = up(P->g.fm, fm.data(), sizeof(int) * P->nf);
    if (e == cudaSuccess) e = up(P->g.fgeo, fgeo.data(), sizeof(double) * P->nf);
    if (e == cudaSuccess) e = up(P->g.fth, fth.data(), sizeof(double) * P->nf);
    if (e == cudaSuccess) e = up(P->g.fd, fd.data(), sizeof(double) * P->nf);
    if (e == cudaSuccess) e = up(P->g.nb, H.nb.data(), sizeof(int) * H.nb.size());
    if (e == cudaSuccess) e = up(P->g.nf_of, H.nf_of.data(), sizeof(int) * H.nf_of.size());
    if (e == cudaSuccess) e = up(P->g.bgeo, H.bgeo.data(), sizeof(double) * H.bgeo.size());
    if (e == cudaSuccess) e = up(P->g.bh, H.bh.data(), sizeof(double) * H.bh.size());
    if (e != cudaSuccess) {
        cudaGetLastError();
        gq_smr_destroy(P);
        return GQ_ERR_CUDA;
    }
    *out = P;
    return GQ_OK;
}

int gq_smr_cells(const gq_smr_plan* P) { return P ? P->N : 0; }

void gq_smr_destroy(gq_smr_plan* P) {
    if (!P) return;
    if (P->arena) cudaFree(P->arena);
    if (P->ctl_host) cudaFreeHost(P->ctl_host);
    delete P;
}

gq_status gq_smr_step(gq_smr_plan* P, const double* rho, double* e_g, double* E_r, double* T_g_out,
                      const gq_opacity_law* op, const gq_eos* eos, double dt, const gq_bc* bc,
                      const gq_solver_opts* opts_in, void* stream, gq_step_info* info) {
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->status = GQ_ERR_INVALID_ARG;
    }
    if (!P || !eos || eos->table_n != 0) return GQ_ERR_INVALID_ARG;
    // argument checks and the physical parameters, shared with the single-level step (a
    // plan-shaped view: one row of N cells)
    gq_fld_plan view{};
    view.nx = P->N;
    view.ny = 1;
    view.N = P->N;
    gq::StepParams sp{};
    gq::SolveParams pp{};
    gq_status vs = gq::make_step_params(&view, rho, e_g, E_r, T_g_out, op, eos, dt, bc, opts_in, &sp, &pp, nullptr);
    if (vs != GQ_OK) return vs;
    sp.precond = GQ_PRECOND_JACOBI;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return GQ_ERR_CUDA;
    if (cur != P->device && cudaSetDevice(P->device) != cudaSuccess) return GQ_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    gq::SmrSolve S{};
    S.N = P->N;
    S.max_iter = pp.max_iter;
    S.max_refine = pp.max_refine;
    S.rtol = pp.rtol;
    S.drop = pp.mixed ? pp.drop : 1e-2;
    S.spin = pp.spin_limit;
    S.g = P->g;
    S.v = P->v;
    S.w = P->w;
    const int nblk = P->setup_blocks;
    const int fblk = std::max(1, std::min(P->num_sms * 8, (P->nf + gq::kSetupThreads - 1) / gq::kSetupThreads));
    cudaError_t e = cudaMemsetAsync(P->w.ctl, 0, sizeof(gq::SolveCtl), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->w.bar, 0, 2 * sizeof(unsigned), st);
    if (e == cudaSuccess) e = gq::launch_cells(sp, P->geo, P->w, nblk, st);
    if (e == cudaSuccess && P->nf > 0) {
        gq::k_smr_faces<<<fblk, gq::kSetupThreads, 0, st>>>(P->g, P->w.sig, E_r, sp.limiter, dt, P->v.w);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        gq::k_smr_diag<<<nblk, gq::kSetupThreads, 0, st>>>(P->g, P->w, P->v.w, *bc, sp.limiter, dt);
        gq::k_smr_scale<<<nblk, gq::kSetupThreads, 0, st>>>(P->g, P->w, P->v, E_r);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        void* args[] = {&S};
        const void* fn = pp.mixed ? reinterpret_cast<const void*>(gq::k_smr_pcg<true>)
                                  : reinterpret_cast<const void*>(gq::k_smr_pcg<false>);
        e = cudaLaunchCooperativeKernel(fn, dim3(P->grid_max), dim3(gq::kSmrThreads), args, 0, st);
    }
    if (e == cudaSuccess) e = gq::launch_backsub(sp, P->geo, P->w, nblk, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->ctl_host, P->w.ctl, sizeof(gq::SolveCtl), cudaMemcpyDeviceToHost, st);
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
        info->solve_blocks = P->grid_max;
    }
    return status;
}

}  // extern "C"
