// Persistent Jacobi-preconditioned conjugate-gradient solve of the reduced FLD system
// (the Krylov step of Sec. 3.2.1, stopping rule in the spirit of Eq. linearsystem).
//
// The system is solved in Jacobi-scaled form A^ y = b^ with A^ = S A S (unit diagonal,
// off-diagonals -c_f = -w_f s_k s_m), so Jacobi-PCG on A is plain CG on A^ and the
// matrix-free 5-point product reads two coefficient arrays per cell: c_W (face to the
// west neighbour) and c_S (face to the south neighbour); the east and north
// coefficients of cell k are c_W[k+1] and c_S[k+nx] (zero across the boundary).
//
// One cooperative launch runs the whole solve.  Each iteration is two grid-stride
// passes separated by grid-wide reductions:
//   S: p = r + beta p_old (p double-buffered), q = A^ p, partial p.q
//   U: x += alpha p, r -= alpha q, partial r.r (FP64 path: also max |r_k / y_k|)
// All blocks reduce the per-block partials in the same order, so every block takes
// bitwise-identical control decisions without a broadcast.
//
// FP64 path: x is the FP64 iterate y.  When the recursive cell-wise residual
// max |r_k / y_k| reaches its target (rtol, halved after every disagreeing check), the
// true residual b^ - A^ y is recomputed (in place of r) and the stop test is applied to it.
// Both paths end with GQ_ERR_NOT_CONVERGED (best iterate kept) when the true residual
// has not improved by 10% in 6 consecutive checks: the FP64 rounding floor of the
// cell-wise criterion lies above rtol.
// Mixed path: the Krylov vectors, the coefficients and the correction d are FP32.  When
// |r|_2 has fallen by inner_rtol since the last FP64 residual, y += d (FP64), d = 0, the
// FP64 residual is recomputed and, unless converged, becomes the new FP32 residual; the
// search direction is kept (reliable update) unless `restart` is set.  The FP32 residual
// is carried with a fixed power-of-two scale so that its entries stay O(1).
#include <type_traits>

#include "gq_device.cuh"
#include "gq_internal.h"

namespace gq {

namespace {

constexpr double kStallGain = 0.9;   // a true residual must improve by 10% ...
constexpr int kStallChecks = 6;      // ... within this many consecutive checks

struct RedShared {
    double warp[kSolveThreads / 32][kSlots];
    double tot[kSlots];
};

// Block-reduce NSUM sums and NMAX maxima, publish the block partials, wait for all
// blocks, reduce the partials (same order in every block).  Returns false on timeout.
template <int NSUM, int NMAX>
__device__ __forceinline__ bool allreduce(double (&v)[NSUM + NMAX], double* partials, int& parity,
                                          unsigned* bar, long long spin, int* abort_flag, RedShared& sh) {
    constexpr int NS = NSUM + NMAX;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int G = gridDim.x;
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
            if (lane == 0) mine[blockIdx.x * kSlots + s] = a;
        }
    }
    if (!grid_barrier(bar, G, spin, abort_flag)) return false;
    if (warp == 0) {
#pragma unroll
        for (int s = 0; s < NS; s++) {
            double a = 0.0;
            for (int b = lane; b < G; b += 32) {
                const double x = __ldcg(mine + b * kSlots + s);
                a = s < NSUM ? a + x : nanmax(a, x);
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

template <bool MIXED>
__global__ void __launch_bounds__(kSolveThreads, 2) k_pcg(SolveParams P, Workspace w) {
    using R = std::conditional_t<MIXED, float, double>;
    __shared__ RedShared sh;
    const int N = P.N, nx = P.nx;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
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
        return;
    }

    // ---- FP64 residual r64 = b^ - A^ y and its norms ----------------------------------
    // sums: |r|^2, |r/s|^2 (unscaled residual), |b/s|^2 ; maxima: |r_k / y_k|, |r_k|
    double tr[5];
    auto true_residual = [&](bool first) -> bool {
#pragma unroll
        for (int t = 0; t < 5; t++) tr[t] = 0.0;
        for (int k = tid; k < N; k += stride) {
            const double yk = __ldcg(y + k);
            double ax = yk;
            if (k > 0) ax -= cW64[k] * __ldcg(y + k - 1);
            if (k + 1 < N) ax -= cW64[k + 1] * __ldcg(y + k + 1);
            if (k >= nx) ax -= cS64[k] * __ldcg(y + k - nx);
            if (k + nx < N) ax -= cS64[k + nx] * __ldcg(y + k + nx);
            const double bk = bh[k];
            const double rk = bk - ax;
            r64[k] = rk;
            const double sk = s[k];
            const double ru = rk / sk;
            tr[0] += rk * rk;
            tr[1] += ru * ru;
            if (first) {
                const double bu = bk / sk;
                tr[2] += bu * bu;
            }
            tr[3] = nanmax(tr[3], fabs(rk / yk));
            tr[4] = nanmax(tr[4], fabs(rk));
        }
        return allreduce<3, 2>(tr, w.partials, parity, w.bar, P.spin_limit, abort_flag, sh);
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
        // power-of-two scale for the FP32 residual (1 for the FP64 path)
        const double scale = MIXED ? exp2(-(double)ilogb(tr[4] > 0.0 ? tr[4] : 1.0)) : 1.0;
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
        int stall = 0;

        while (true) {
            // ---- S: p = r + beta p_old ; q = A^ p ; p.q ------------------------------
            const R* pold = pb[cur];
            R* pnew = pb[cur ^ 1];
            const R rb = static_cast<R>(beta);
            const R rsc = static_cast<R>(scale);
            double v1[1] = {0.0};
            for (int k = tid; k < N; k += stride) {
                auto pv = [&](int m) -> R {
                    R rm;
                    if (MIXED && from64) rm = static_cast<R>(__ldcg(r64 + m)) * rsc;
                    else rm = __ldcg(r + m);
                    return use_p ? rm + rb * __ldcg(pold + m) : rm;
                };
                const R pk = pv(k);
                R acc = pk;
                if (k > 0) acc -= cW[k] * pv(k - 1);
                if (k + 1 < N) acc -= cW[k + 1] * pv(k + 1);
                if (k >= nx) acc -= cS[k] * pv(k - nx);
                if (k + nx < N) acc -= cS[k + nx] * pv(k + nx);
                pnew[k] = pk;
                q[k] = acc;
                if (MIXED && from64) {
                    r[k] = static_cast<R>(__ldcg(r64 + k)) * rsc;
                    d[k] = R(0);
                }
                v1[0] += static_cast<double>(pk) * static_cast<double>(acc);
            }
            if (!allreduce<1, 0>(v1, w.partials, parity, w.bar, P.spin_limit, abort_flag, sh)) {
                timed_out = true;
                break;
            }
            const double pq = v1[0];
            if (!(pq > 0.0) || !isfinite(pq)) { status = kErrNonfinite; break; }
            const double alpha = rr / pq;
            cur ^= 1;
            from64 = false;

            // ---- U: x += alpha p ; r -= alpha q ; r.r --------------------------------
            double v2[2] = {0.0, 0.0};
            const R ra = static_cast<R>(alpha);
            for (int k = tid; k < N; k += stride) {
                const R pk = __ldcg(pnew + k);
                const R qk = __ldcg(q + k);
                const R rk = __ldcg(r + k) - ra * qk;
                r[k] = rk;
                if constexpr (MIXED) {
                    d[k] = __ldcg(d + k) + ra * pk;
                    v2[0] += static_cast<double>(rk) * static_cast<double>(rk);
                } else {
                    const double yk = __ldcg(y + k) + alpha * pk;
                    y[k] = yk;
                    v2[0] += rk * rk;
                    v2[1] = nanmax(v2[1], fabs(rk / yk));
                }
            }
            if (!allreduce<1, 1>(v2, w.partials, parity, w.bar, P.spin_limit, abort_flag, sh)) {
                timed_out = true;
                break;
            }
            it++;
            const double rr_new = v2[0];
            if (!isfinite(rr_new)) { status = kErrNonfinite; break; }
            const bool check = MIXED ? (sqrt(rr_new) <= P.drop * sqrt(rr_ref) || it >= P.max_iter)
                                     : (v2[1] <= rec_target || it >= P.max_iter);
            if (!check) {
                beta = rr_new / rr;
                rr = rr_new;
                use_p = true;
                continue;
            }

            // ---- FP64 residual (refinement) -----------------------------------------
            if constexpr (MIXED) {
                const double inv = 1.0 / scale;
                for (int k = tid; k < N; k += stride) {
                    y[k] = __ldcg(y + k) + static_cast<double>(__ldcg(d + k)) * inv;
                    d[k] = R(0);
                }
                if (!grid_barrier(w.bar, gridDim.x, P.spin_limit, abort_flag)) { timed_out = true; break; }
            }
            if (!true_residual(false)) { timed_out = true; break; }
            nref++;
            crit = tr[3];
            l2 = sqrt(tr[1] / bb);
            if (!isfinite(tr[0]) || !(crit == crit)) { status = kErrNonfinite; break; }
            if (crit <= P.rtol) { status = kOk; break; }
            if (crit < kStallGain * best) {
                best = crit;
                stall = 0;
            } else {
                stall++;
            }
            if (it >= P.max_iter || nref >= P.max_refine || stall >= kStallChecks) {
                status = kErrNotConverged;
                break;
            }
            rec_target *= 0.5;
            const double rr_true = tr[0] * scale * scale;
            if (MIXED && P.restart) {
                use_p = false;
                beta = 0.0;
            } else {
                use_p = true;
                beta = rr_true / rr;
            }
            rr = rr_true;
            rr_ref = rr_true;
            from64 = MIXED;
        }
    }

done:
    if (timed_out) {
        if (threadIdx.x == 0) atomicExch(&ctl->status, kErrTimeout);
        return;
    }
    if (tid == 0) {
        ctl->status = status;
        ctl->iterations = it;
        ctl->refinements = nref;
        ctl->crit = crit;
        ctl->l2 = l2;
    }
}

}  // namespace

int solve_max_blocks_per_sm() {
    int a = 0, b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pcg<true>, kSolveThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pcg<false>, kSolveThreads, 0);
    return a < b ? a : b;
}

cudaError_t launch_solve(const SolveParams& p, const Workspace& w, int grid, cudaStream_t st) {
    SolveParams pc = p;
    Workspace wc = w;
    void* args[] = {&pc, &wc};
    const void* fn = p.mixed ? reinterpret_cast<const void*>(k_pcg<true>)
                             : reinterpret_cast<const void*>(k_pcg<false>);
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kSolveThreads), args, 0, st);
}

}  // namespace gq
