// Persistent preconditioned conjugate-gradient solve of the reduced FLD system (the
// Krylov step of Sec. 3.2.1, with a residual-based stop in the spirit of
// Eq. linearsystem).
//
// The system is solved in Jacobi-scaled form A^ y = b^ with A^ = S A S (unit diagonal,
// off-diagonals -c_f = -w_f s_k s_m); the matrix-free 5-point product reads two
// coefficient arrays per cell: c_W (face to the west neighbour) and c_S (face to the
// south neighbour); the east and north coefficients of cell k are c_W[k+1] and
// c_S[k+nx] (zero across the boundary).  The preconditioner is Jacobi (plain CG on A^),
// one V-cycle of 2 x 2 aggregation multigrid (gq_mg.cuh) or one V-cycle of classical
// algebraic multigrid built in the kernel's prologue (gq_amg.cuh); with multigrid the
// directions use the Polak-Ribiere beta.
//
// One cooperative launch runs the whole solve.  Each iteration is the preconditioner
// and two passes separated by team-wide reductions:
//   S: p = z + beta p_old (p double-buffered), q = A^ p, partial p.q
//   U: x += alpha p, r -= alpha q, partial r.r (FP64 path: also max |r_k / y_k|)
// In the mixed multigrid paths with a vectorised level 0, U is fused with the next
// cycle's first level-0 sweep (the residual alternates between two buffers).
// A thread handles W consecutive cells of one row with 16-byte loads (W = 4 in FP32,
// 2 in FP64) when nx is a multiple of W, one cell otherwise.  All blocks reduce the
// per-block partials in the same order, so every block takes bitwise-identical control
// decisions without a broadcast, and results are reproducible run to run.
//
// FP64 path: x is the FP64 iterate y.  When the recursive cell-wise residual
// max |r_k / y_k| reaches its target (rtol, halved after every disagreeing check), the
// true residual b^ - A^ y is recomputed (in place of r) and the stop test applied to it.
// Mixed path: the Krylov vectors, the coefficients and the correction d are FP32.  When
// |r|_2 has fallen by inner_rtol since the last FP64 residual, y += d (FP64), d = 0, the
// FP64 residual is recomputed and, unless converged, becomes the new FP32 residual; the
// search direction is kept (reliable update) unless `restart` is set.  The FP32 residual
// is carried with a fixed power-of-two scale so that its entries stay O(1).
// Both paths end with GQ_ERR_NOT_CONVERGED (best iterate kept) when the true residual
// has not improved by 10% in 6 consecutive checks spanning at least 32 iterations: the
// FP64 rounding floor of the cell-wise criterion lies above rtol.
// The solver is compiled in three translation units that each instantiate one kernel:
// gq_pcg_mixed.cu (k_pcg<true>), gq_pcg_fp64.cu (k_pcg<false>, and the host launchers of
// the single-problem solve) and gq_pcg_batch.cu (kb_pcg).
#pragma once

#include <type_traits>

#include "gq_device.cuh"
#include "gq_internal.h"

namespace gq {

namespace {

constexpr double kStallGain = 0.9;   // a true residual must improve by 10% ...
constexpr int kStallChecks = 6;      // ... within this many consecutive checks
constexpr int kStallIters = 32;      // ... spanning at least this many Krylov iterations

struct RedShared {
    double warp[32][kSlots];           // up to 1024 threads a block
    double tot[kSlots];
};

// ---- 16-byte vector access ------------------------------------------------------------

template <class R, int W>
__device__ __forceinline__ void ldv(const R* p, R (&o)[W]) {
    if constexpr (W == 1) {
        o[0] = __ldcg(p);
    } else if constexpr (std::is_same_v<R, float> && W == 4) {
        const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else {
        static_assert(std::is_same_v<R, double> && W == 2, "unsupported vector");
        const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
        o[0] = v.x; o[1] = v.y;
    }
}

template <class R, int W>
__device__ __forceinline__ void stv(R* p, const R (&o)[W]) {
    if constexpr (W == 1) {
        p[0] = o[0];
    } else if constexpr (std::is_same_v<R, float> && W == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    }
}

// W doubles (W = 1, 2 or 4) from an address aligned to 16 bytes when W > 1
template <int W>
__device__ __forceinline__ void ld64(const double* p, double (&o)[W]) {
    if constexpr (W == 1) {
        o[0] = __ldcg(p);
    } else {
#pragma unroll
        for (int h = 0; h < W / 2; h++) {
            const double2 v = __ldcg(reinterpret_cast<const double2*>(p) + h);
            o[2 * h] = v.x;
            o[2 * h + 1] = v.y;
        }
    }
}

template <int W>
__device__ __forceinline__ void st64(double* p, const double (&o)[W]) {
    if constexpr (W == 1) {
        p[0] = o[0];
    } else {
#pragma unroll
        for (int h = 0; h < W / 2; h++)
            reinterpret_cast<double2*>(p)[h] = make_double2(o[2 * h], o[2 * h + 1]);
    }
}

// W floats (W = 1, 2 or 4) at an address aligned to 4 W bytes
template <int W>
__device__ __forceinline__ void ldf(const float* p, float (&o)[W]) {
    if constexpr (W == 1) {
        o[0] = __ldcg(p);
    } else if constexpr (W == 2) {
        const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
        o[0] = v.x; o[1] = v.y;
    } else {
        const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
}

template <int W>
__device__ __forceinline__ void stf(float* p, const float (&o)[W]) {
    if constexpr (W == 1) {
        p[0] = o[0];
    } else if constexpr (W == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
    } else {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
}

// Block-reduce NSUM sums and NMAX maxima, publish the block partials, wait for all
// blocks of the team, reduce the partials (same order in every block).  Returns false
// on timeout.
template <int NSUM, int NMAX>
__device__ __forceinline__ bool allreduce(double (&v)[NSUM + NMAX], double* partials, int& parity,
                                          unsigned* bar, long long spin, int* abort_flag, RedShared& sh,
                                          Team team) {
    constexpr int NS = NSUM + NMAX;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int G = team.size;
#pragma unroll
    for (int s = 0; s < NS; s++) {
        v[s] = s < NSUM ? warp_reduce<false>(v[s]) : warp_reduce<true>(v[s]);
        if (lane == 0) sh.warp[warp][s] = v[s];
    }
    __syncthreads();
    double* mine = partials + (size_t)parity * G * kSlots;
    if (warp == 0) {
#pragma unroll
        for (int s = 0; s < NS; s++) {
            double a = lane < nw ? sh.warp[lane][s] : 0.0;
            a = s < NSUM ? warp_reduce<false>(a) : warp_reduce<true>(a);
            if (lane == 0) mine[team.rank * kSlots + s] = a;
        }
    }
    if (!team_barrier(bar, team, spin, abort_flag)) return false;
    if (warp == 0) {
        // all loads first: one L2 round trip for teams of up to 256 blocks
        double x[NS][8];
#pragma unroll
        for (int s = 0; s < NS; s++)
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const int b = lane + 32 * i;
                x[s][i] = b < G ? __ldcg(mine + b * kSlots + s) : 0.0;
            }
#pragma unroll
        for (int s = 0; s < NS; s++) {
            double a = x[s][0];
#pragma unroll
            for (int i = 1; i < 8; i++) a = s < NSUM ? a + x[s][i] : nanmax(a, x[s][i]);
            for (int b = lane + 256; b < G; b += 32) {
                const double z = __ldcg(mine + b * kSlots + s);
                a = s < NSUM ? a + z : nanmax(a, z);
            }
            a = s < NSUM ? warp_reduce<false>(a) : warp_reduce<true>(a);
            if (lane == 0) sh.tot[s] = a;
        }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < NS; s++) v[s] = sh.tot[s];
    parity ^= 1;
    return true;
}

}  // namespace
}  // namespace gq

#include "gq_mg.cuh"
#include "gq_amg.cuh"

namespace gq {
namespace {

// Solve of one problem by one team of co-resident blocks, W cells per thread and pass;
// PC selects the preconditioner: 0 Jacobi (plain CG on A^), 1 aggregation multigrid,
// 2 algebraic multigrid.
// Returns false when a wait of the team timed out (the caller must leave the kernel).
template <bool MIXED, int W, int PC>
__device__ __forceinline__ bool pcg_solve_w(const SolveParams& P, const Workspace& w, Team team, RedShared& sh,
                                            MGShared& msh) {
    using R = std::conditional_t<MIXED, float, double>;
    constexpr bool MG = PC != 0;
    const int N = P.N, nx = P.nx;
    const int nchunk = N / W;          // N is a multiple of W because nx is
    const int tid = team.rank * blockDim.x + threadIdx.x;
    const int stride = team.size * blockDim.x;
    SolveCtl* ctl = w.ctl;
    int* abort_flag = &ctl->abort;
    int parity = 0;

    const double* __restrict__ cW64 = w.wW;
    const double* __restrict__ cS64 = w.wS;
    const double* __restrict__ bh = w.rhs;
    const double* __restrict__ s = w.dloc;
    double* y = w.y;
    double* r64 = w.r64;
    const R* cW;
    const R* cS;
    R* r;
    R* pb[2];
    R* q;
    R* d;
    if constexpr (MIXED) {
        cW = w.cW32; cS = w.cS32; r = w.r32; pb[0] = w.p32[0]; pb[1] = w.p32[1]; q = w.q32; d = w.d32;
    } else {
        cW = w.wW; cS = w.wS; r = w.r64; pb[0] = w.p64[0]; pb[1] = w.p64[1]; q = w.q64; d = w.y;
    }

    const int flags = __ldcg(&ctl->input_flags);
    if (flags) {
        if (tid == 0) ctl->status = (flags & 2) ? kErrNonfinite : kErrInvalid;
        return true;
    }
    if (tid == 0) ctl->t_start = global_ns();
    // multigrid: the rest of the hierarchy, the FP32 level-0 right-hand side and the two
    // preconditioned-residual buffers
    float* r0 = MIXED ? w.r32 : w.mg.r32;
    // mixed aggregation-multigrid path with a vectorised level 0 on the team: the Krylov
    // update is fused with the next cycle's first level-0 sweep, the residual alternating
    // between two buffers
    float* rbuf[2] = {w.r32, w.r32b};
    int rsel = 0;
    const bool fuse = MIXED && PC != 0 && W == 4 &&
                      (PC == 1 ? (w.mg.nlev > 1 && w.mg.L[0].N > P.block_cells) : N > P.block_cells);
    bool pre0_done = false;
    float* zc = w.mg.z;
    float* zo = w.mg.zold;
    if constexpr (PC == 2) {
        if (!amg_build(w, nx, N / nx, P.block_cells, team, tid, stride, P.spin_limit, abort_flag, sh, msh, parity)) {
            if (threadIdx.x == 0) atomicExch(&ctl->status, kErrTimeout);
            return false;
        }
    } else if constexpr (MG) {
        cyc_reset(msh.amg);
        if (!mg_build(w, team, tid, stride, P.spin_limit, abort_flag, msh)) {
            if (threadIdx.x == 0) atomicExch(&ctl->status, kErrTimeout);
            return false;
        }
    }
    if (tid == 0) {
        ctl->t_built = global_ns();
        if constexpr (PC == 2) ctl->levels = msh.amg.nlev;
        else if constexpr (PC == 1) ctl->levels = w.mg.nlev;
        else ctl->levels = 1;
    }

    // ---- FP64 residual r64 = b^ - A^ y and its norms ----------------------------------
    // sums: |r|^2, |r/s|^2 (unscaled residual), |b/s|^2 ; maxima: |r_k / y_k|, |r_k|
    double tr[5];
    auto true_residual = [&](bool first) -> bool {
#pragma unroll
        for (int t = 0; t < 5; t++) tr[t] = 0.0;
        for (int c = tid; c < nchunk; c += stride) {
            const int k = c * W;
            const bool hs = k >= nx, hn = k + nx < N, hw = k > 0, he = k + W < N;
            double yc[W], ys[W], yn[W], cw[W], cs[W], csn[W], bk[W], sk[W];
            double yw = 0.0, ye = 0.0, cwe = 0.0;
            ld64<W>(y + k, yc);
            ld64<W>(cW64 + k, cw);
            ld64<W>(cS64 + k, cs);
            ld64<W>(bh + k, bk);
            ld64<W>(s + k, sk);
            if (hw) yw = __ldcg(y + k - 1);
            if (he) {
                ye = __ldcg(y + k + W);
                cwe = cW64[k + W];
            }
            if (hs) ld64<W>(y + k - nx, ys);
            if (hn) {
                ld64<W>(y + k + nx, yn);
                ld64<W>(cS64 + k + nx, csn);
            }
            double rk[W];
#pragma unroll
            for (int i = 0; i < W; i++) {
                const double left = i == 0 ? yw : yc[i - 1];
                const double right = i == W - 1 ? ye : yc[i + 1];
                const double cright = i == W - 1 ? cwe : cw[i + 1];
                double ax = yc[i] - cw[i] * left - cright * right;
                if (hs) ax -= cs[i] * ys[i];
                if (hn) ax -= csn[i] * yn[i];
                rk[i] = bk[i] - ax;
                const double ru = abs_ratio_approx(rk[i], sk[i]);
                tr[0] += rk[i] * rk[i];
                tr[1] += ru * ru;
                if (first) {
                    const double bu = abs_ratio_approx(bk[i], sk[i]);
                    tr[2] += bu * bu;
                }
                tr[3] = nanmax(tr[3], abs_ratio_approx(rk[i], yc[i]));
                tr[4] = nanmax(tr[4], fabs(rk[i]));
            }
            st64<W>(r64 + k, rk);
        }
        return allreduce<3, 2>(tr, w.partials, parity, w.bar, P.spin_limit, abort_flag, sh, team);
    };

    int it = 0, nref = 0, status = kErrNotConverged;
    double crit = 0.0, l2 = 0.0, bb = 1.0;
    bool timed_out = false;

    if (!true_residual(true)) { timed_out = true; goto done; }
    bb = tr[2];
    crit = tr[3];
    l2 = sqrt(tr[1] / bb);
    if (!isfinite(tr[0]) || !isfinite(bb) || !(crit == crit)) { status = kErrNonfinite; goto done; }
    if (crit <= P.rtol) { status = kOk; goto done; }

    {
        // power-of-two scale that keeps FP32 residual entries O(1): the Krylov residual of
        // the mixed path and the V-cycle input of both paths carry it (the FP64 Krylov
        // vectors of the FP64 path do not)
        const double zs = exp2(-(double)ilogb(tr[4] > 0.0 ? tr[4] : 1.0));
        const double scale = MIXED ? zs : 1.0;
        double rr = tr[0] * scale * scale;
        double rr_ref = rr;
        double beta = 0.0;
        bool use_p = false;
        bool from64 = MIXED;      // next S pass takes r from the FP64 residual
        int cur = 0;
        // FP64 path: target of the recursive criterion, halved whenever the true residual
        // disagrees; both paths: stop once the true residual stalls (FP64 rounding floor)
        double rec_target = P.rtol;
        double best = crit;
        int it_best = 0;
        int stall = 0;
        // multigrid: FP32 copy of the (scaled) FP64 residual for the V-cycle
        bool first = true;
        double rz_prev = 1.0;
        const R rzf = static_cast<R>(MIXED ? 1.0 : 1.0 / zs);
        auto refresh = [&](bool initial) -> bool {
            for (int c = tid; c < nchunk; c += stride) {
                const int k = c * W;
                double t[W];
                float f[W], zero[W];
                ld64<W>(r64 + k, t);
#pragma unroll
                for (int i = 0; i < W; i++) {
                    f[i] = static_cast<float>(t[i] * zs);
                    zero[i] = 0.f;
                }
                stf<W>(r0 + k, f);
                if constexpr (MIXED) stf<W>(reinterpret_cast<float*>(d) + k, zero);
                if (initial) stf<W>(zo + k, zero);
            }
            return team_barrier(w.bar, team, P.spin_limit, abort_flag);
        };
        if constexpr (MG) {
            from64 = false;
            if (!refresh(true)) { timed_out = true; goto done; }
        }

        // FP64 residual (refinement): fold the FP32 correction into y (mixed), recompute
        // b^ - A^ y, apply the stop tests; false ends the solve (status or timed_out set)
        auto refine = [&]() -> bool {
            if constexpr (MIXED) {
                const double inv = 1.0 / scale;
                for (int c = tid; c < nchunk; c += stride) {
                    const int k = c * W;
                    double yk[W];
                    R dk[W], zero[W];
                    ld64<W>(y + k, yk);
                    ldv<R, W>(d + k, dk);
#pragma unroll
                    for (int i = 0; i < W; i++) {
                        yk[i] += static_cast<double>(dk[i]) * inv;
                        zero[i] = R(0);
                    }
                    st64<W>(y + k, yk);
                    stv<R, W>(d + k, zero);
                }
                if (!team_barrier(w.bar, team, P.spin_limit, abort_flag)) {
                    timed_out = true;
                    return false;
                }
            }
            if (!true_residual(false)) {
                timed_out = true;
                return false;
            }
            nref++;
            crit = tr[3];
            l2 = sqrt(tr[1] / bb);
            if (!isfinite(tr[0]) || !(crit == crit)) { status = kErrNonfinite; return false; }
            if (crit <= P.rtol) { status = kOk; return false; }
            if (crit < kStallGain * best) {
                best = crit;
                it_best = it;
                stall = 0;
            } else {
                stall++;
            }
            if (it >= P.max_iter || nref >= P.max_refine || (stall >= kStallChecks && it - it_best >= kStallIters)) {
                status = kErrNotConverged;
                return false;
            }
            rec_target *= 0.5;
            const double rr_true = tr[0] * scale * scale;
            if (MIXED && P.restart) {
                use_p = false;
                beta = 0.0;
                first = true;
            } else {
                use_p = true;
                beta = rr > 0.0 ? rr_true / rr : 0.0;
            }
            rr = rr_true;
            rr_ref = rr_true;
            from64 = MIXED && !MG;
            if constexpr (MG) {
                if (!refresh(false)) {
                    timed_out = true;
                    return false;
                }
            }
            return true;
        };

        while (true) {
            double rho_mg = 0.0;
            bool degenerate = false;
            if constexpr (MG) {
                // ---- z = V-cycle(r) ; r.z and r.z_old (Polak-Ribiere) ---------------------
                double vz[2] = {0.0, 0.0};
                bool ok;
                if constexpr (PC == 2)
                    ok = amg_vcycle(w.amg, msh.amg, r0, zc, zo, w.cW32, w.cS32, nx, P.mg_omega, P.block_cells,
                                    pre0_done && msh.amg.nlev > 1, team, tid, stride, w.bar, P.spin_limit, abort_flag,
                                    &vz[0], &vz[1]);
                else
                    ok = vcycle(w.mg, msh.amg, r0, zc, zo, P.mg_omega, P.mg_over, P.block_cells, pre0_done, team, tid,
                                stride, w.bar, P.spin_limit, abort_flag, &vz[0], &vz[1]);
                pre0_done = false;
                if (!ok) {
                    timed_out = true;
                    break;
                }
                if (!allreduce<2, 0>(vz, w.partials, parity, w.bar, P.spin_limit, abort_flag, sh, team)) {
                    timed_out = true;
                    break;
                }
                if (!isfinite(vz[0]) || !isfinite(vz[1])) { status = kErrNonfinite; break; }
                // a vanished recursive residual (FP32) goes straight to the FP64 check
                degenerate = !(vz[0] > 0.0);
                // Polak-Ribiere beta, restarted (beta = 0) when the new preconditioned
                // residual is far from orthogonal to the old one (Powell's test): near
                // convergence z is rounding noise and the formula could cancel it
                const bool restart_dir = first || fabs(vz[1]) >= 0.2 * vz[0];
                beta = restart_dir ? 0.0 : fmax(0.0, (vz[0] - vz[1]) / rz_prev);
                use_p = !restart_dir;
                rz_prev = vz[0];
                rho_mg = vz[0] * static_cast<double>(rzf) * static_cast<double>(rzf);
                first = false;
            }
            if (!degenerate) {
                // ---- S: p = r + beta p_old ; q = A^ p ; p.q ------------------------------
                if constexpr (MG) cyc_mark(msh.amg, team, kAmgMaxLevels - 4);
                const R* __restrict__ pold = pb[cur];
                R* __restrict__ pnew = pb[cur ^ 1];
                const R rb = static_cast<R>(beta);
                const R rsc = static_cast<R>(scale);
                double v1[1] = {0.0};
                R pqr = R(0);     // mixed path: this thread's p.q in FP32 (FP64 per cell is slow on this part)
                for (int c = tid; c < nchunk; c += stride) {
                    const int k = c * W;
                    const bool hs = k >= nx, hn = k + nx < N, hw = k > 0, he = k + W < N;
                    // r on the cells and their west, east, south and north neighbours
                    R rc[W], rs[W], rn[W], rw = R(0), re = R(0);
                    R pc[W], ps[W], pn[W], pw = R(0), pe = R(0);
    #pragma unroll
                    for (int i = 0; i < W; i++) rs[i] = rn[i] = pc[i] = ps[i] = pn[i] = R(0);
                    if constexpr (MG) {
                        float t[W];
                        ldf<W>(zc + k, t);
    #pragma unroll
                        for (int i = 0; i < W; i++) rc[i] = static_cast<R>(t[i]) * rzf;
                        if (hs) {
                            ldf<W>(zc + k - nx, t);
    #pragma unroll
                            for (int i = 0; i < W; i++) rs[i] = static_cast<R>(t[i]) * rzf;
                        }
                        if (hn) {
                            ldf<W>(zc + k + nx, t);
    #pragma unroll
                            for (int i = 0; i < W; i++) rn[i] = static_cast<R>(t[i]) * rzf;
                        }
                        if (hw) rw = static_cast<R>(__ldcg(zc + k - 1)) * rzf;
                        if (he) re = static_cast<R>(__ldcg(zc + k + W)) * rzf;
                    } else if (MIXED && from64) {
                        double t[W];
                        ld64<W>(r64 + k, t);
    #pragma unroll
                        for (int i = 0; i < W; i++) rc[i] = static_cast<R>(t[i]) * rsc;
                        if (hs) {
                            ld64<W>(r64 + k - nx, t);
    #pragma unroll
                            for (int i = 0; i < W; i++) rs[i] = static_cast<R>(t[i]) * rsc;
                        }
                        if (hn) {
                            ld64<W>(r64 + k + nx, t);
    #pragma unroll
                            for (int i = 0; i < W; i++) rn[i] = static_cast<R>(t[i]) * rsc;
                        }
                        if (hw) rw = static_cast<R>(__ldcg(r64 + k - 1)) * rsc;
                        if (he) re = static_cast<R>(__ldcg(r64 + k + W)) * rsc;
                    } else {
                        ldv<R, W>(r + k, rc);
                        if (hs) ldv<R, W>(r + k - nx, rs);
                        if (hn) ldv<R, W>(r + k + nx, rn);
                        if (hw) rw = __ldcg(r + k - 1);
                        if (he) re = __ldcg(r + k + W);
                    }
                    if (use_p) {
                        ldv<R, W>(pold + k, pc);
                        if (hs) ldv<R, W>(pold + k - nx, ps);
                        if (hn) ldv<R, W>(pold + k + nx, pn);
                        if (hw) pw = __ldcg(pold + k - 1);
                        if (he) pe = __ldcg(pold + k + W);
                    }
                    R cw[W], cs[W], csn[W], cwe = R(0);
    #pragma unroll
                    for (int i = 0; i < W; i++) csn[i] = R(0);
                    ldv<R, W>(cW + k, cw);
                    ldv<R, W>(cS + k, cs);
                    if (he) cwe = cW[k + W];
                    if (hn) ldv<R, W>(cS + k + nx, csn);
                    // p = r + beta p_old on the cells and their neighbours (zero off the grid)
                    R p[W], pS[W], pN[W];
                    const R pW = use_p ? rw + rb * pw : rw;
                    const R pE = use_p ? re + rb * pe : re;
    #pragma unroll
                    for (int i = 0; i < W; i++) {
                        p[i] = use_p ? rc[i] + rb * pc[i] : rc[i];
                        pS[i] = use_p ? rs[i] + rb * ps[i] : rs[i];
                        pN[i] = use_p ? rn[i] + rb * pn[i] : rn[i];
                    }
                    R qv[W];
    #pragma unroll
                    for (int i = 0; i < W; i++) {
                        const R left = i == 0 ? pW : p[i - 1];
                        const R right = i == W - 1 ? pE : p[i + 1];
                        const R cright = i == W - 1 ? cwe : cw[i + 1];
                        qv[i] = p[i] - cw[i] * left - cright * right - cs[i] * pS[i] - csn[i] * pN[i];
                        pqr += p[i] * qv[i];
                    }
                    stv<R, W>(pnew + k, p);
                    stv<R, W>(q + k, qv);
                    if (MIXED && from64) {
                        R zero[W];
    #pragma unroll
                        for (int i = 0; i < W; i++) zero[i] = R(0);
                        stv<R, W>(r + k, rc);
                        stv<R, W>(d + k, zero);
                    }
                }
                v1[0] = static_cast<double>(pqr);
                if (!allreduce<1, 0>(v1, w.partials, parity, w.bar, P.spin_limit, abort_flag, sh, team)) {
                    timed_out = true;
                    break;
                }
                const double pq = v1[0];
                if (!isfinite(pq) || (!MG && !(pq > 0.0))) { status = kErrNonfinite; break; }
                // multigrid: a degenerate direction (rounding noise at convergence) goes to the
                // FP64 check
                degenerate = !(pq > 0.0);
                if (!degenerate) {
                    const double alpha = (MG ? rho_mg : rr) / pq;
                    if constexpr (MG) {
                        float* tz = zc;       // this z becomes z_old of the next cycle
                        zc = zo;
                        zo = tz;
                    }
                    cur ^= 1;
                    from64 = false;

                    // ---- U: x += alpha p ; r -= alpha q ; r.r --------------------------------
                    if constexpr (MG) cyc_mark(msh.amg, team, kAmgMaxLevels - 3);
                    double v2[2] = {0.0, 0.0};
                    const R ra = static_cast<R>(alpha);
                    bool fused = false;
                    if constexpr (MIXED && PC != 0) {
                        if (fuse && (PC == 1 || msh.amg.nlev > 1)) {
                            float* rn = rbuf[rsel ^ 1];
                            // the aggregation cycle pre-smooths into its level-0 scratch, the
                            // algebraic one into the cycle's output z
                            Lv L0 = level_view(w.mg, 0, rn, zc);
                            if constexpr (PC == 2) L0.xa = zc;
                            cyc0_update_presmooth_v(L0, r, rn, q, pnew, d, ra, P.mg_omega, Range{tid, stride},
                                                    &v2[0]);
                            rsel ^= 1;
                            r = rn;
                            r0 = rn;
                            fused = true;
                        }
                    }
                    R rrr = R(0);     // mixed path: this thread's r.r in FP32
                    for (int c = fused ? nchunk : tid; c < nchunk; c += stride) {
                        const int k = c * W;
                        R pk[W], qk[W], rk[W], xk[W];
                        ldv<R, W>(pnew + k, pk);
                        ldv<R, W>(q + k, qk);
                        ldv<R, W>(r + k, rk);
                        ldv<R, W>(d + k, xk);
        #pragma unroll
                        for (int i = 0; i < W; i++) {
                            rk[i] = rk[i] - ra * qk[i];
                            xk[i] = xk[i] + ra * pk[i];
                            rrr += rk[i] * rk[i];
                            // recursive stop estimate in FP32 (FP64 division is slow on this part;
                            // the decisive test uses the exact FP64 residual)
                            if constexpr (!MIXED)
                                v2[1] = nanmax(v2[1], abs_ratio_approx(rk[i], xk[i]));
                        }
                        stv<R, W>(r + k, rk);
                        stv<R, W>(d + k, xk);
                        if constexpr (MG && !MIXED) {
                            float f[W];
        #pragma unroll
                            for (int i = 0; i < W; i++) f[i] = static_cast<float>(rk[i] * zs);
                            stf<W>(r0 + k, f);
                        }
                    }
                    v2[0] += static_cast<double>(rrr);
                    if (!allreduce<1, 1>(v2, w.partials, parity, w.bar, P.spin_limit, abort_flag, sh, team)) {
                        timed_out = true;
                        break;
                    }
                    it++;
                    const double rr_new = v2[0];
                    if (!isfinite(rr_new)) { status = kErrNonfinite; break; }
                    const bool check = MIXED ? (sqrt(rr_new) <= P.drop * sqrt(rr_ref) || it >= P.max_iter)
                                             : (v2[1] <= rec_target || it >= P.max_iter);
                    if (!check) {
                        if constexpr (!MG) {
                            beta = rr_new / rr;
                            use_p = true;
                        }
                        rr = rr_new;
                        pre0_done = fused;
                        continue;
                    }
                }
            }

            if constexpr (MG) cyc_mark(msh.amg, team, kAmgMaxLevels - 2);
            if (!refine()) break;
        }
    }

done:
    if constexpr (PC != 0) {
        if (!timed_out) amg_cycle_report(w.amg, msh.amg, team);
    }
    if (timed_out) {
        if (threadIdx.x == 0) atomicExch(&ctl->status, kErrTimeout);
        return false;
    }
    if (tid == 0) {
        ctl->t_end = global_ns();
        ctl->status = status;
        ctl->iterations = it;
        ctl->refinements = nref;
        ctl->crit = crit;
        ctl->l2 = l2;
    }
    return true;
}

template <bool MIXED>
__device__ __forceinline__ bool pcg_solve(const SolveParams& P, const Workspace& w, Team team, RedShared& sh,
                                          MGShared& msh) {
    constexpr int WV = MIXED ? 4 : 2;
    const bool vec = P.nx % WV == 0;
    if (P.precond == GQ_PRECOND_AMG)
        return vec ? pcg_solve_w<MIXED, WV, 2>(P, w, team, sh, msh) : pcg_solve_w<MIXED, 1, 2>(P, w, team, sh, msh);
    if (P.precond == GQ_PRECOND_MG)
        return vec ? pcg_solve_w<MIXED, WV, 1>(P, w, team, sh, msh) : pcg_solve_w<MIXED, 1, 1>(P, w, team, sh, msh);
    return vec ? pcg_solve_w<MIXED, WV, 0>(P, w, team, sh, msh) : pcg_solve_w<MIXED, 1, 0>(P, w, team, sh, msh);
}

// out-of-line copies for the batched kernel, which holds all the variants: separate
// functions keep each variant's registers to itself
template <bool MIXED, int W, int PC>
__device__ __noinline__ bool pcg_solve_call(const SolveParams& P, const Workspace& w, Team team, RedShared& sh,
                                            MGShared& msh) {
    return pcg_solve_w<MIXED, W, PC>(P, w, team, sh, msh);
}

template <bool MIXED>
__device__ __forceinline__ bool pcg_solve_outlined(const SolveParams& P, const Workspace& w, Team team,
                                                   RedShared& sh, MGShared& msh) {
    constexpr int WV = MIXED ? 4 : 2;
    const bool vec = P.nx % WV == 0;
    if (P.precond == GQ_PRECOND_AMG)
        return vec ? pcg_solve_call<MIXED, WV, 2>(P, w, team, sh, msh)
                   : pcg_solve_call<MIXED, 1, 2>(P, w, team, sh, msh);
    if (P.precond == GQ_PRECOND_MG)
        return vec ? pcg_solve_call<MIXED, WV, 1>(P, w, team, sh, msh)
                   : pcg_solve_call<MIXED, 1, 1>(P, w, team, sh, msh);
    return vec ? pcg_solve_call<MIXED, WV, 0>(P, w, team, sh, msh)
               : pcg_solve_call<MIXED, 1, 0>(P, w, team, sh, msh);
}

template <bool MIXED>
__global__ void __launch_bounds__(kSolveThreads, 1) k_pcg(SolveParams P, Workspace w) {
    __shared__ RedShared sh;
    __shared__ MGShared msh;
    pcg_solve<MIXED>(P, w, Team{static_cast<int>(blockIdx.x), static_cast<int>(gridDim.x)}, sh, msh);
}

}  // namespace

// host-side handles of the single-problem kernels (each defined in its own unit)
const void* solve_kernel_mixed();
const void* solve_kernel_fp64();

}  // namespace gq
