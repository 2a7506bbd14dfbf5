// Aggregation-multigrid preconditioned conjugate gradients (included by gq_pcg.cuh).
//
// Preconditioner: one V-cycle on a hierarchy of 2 x 2 aggregates.  Level 0 is the
// Jacobi-scaled system A^ = S A S; level l+1 is the Galerkin product P^T A_l P of
// piecewise-constant aggregation in the unscaled variables (mass summed over the
// aggregate, face weights summed over the aggregate's faces), stored Jacobi-scaled as
// well.  Between scaled levels the transfer is r_{l+1}[I] = sum_k t_k r_l[k] with
// t_k = s_{l+1}[I] / s_l[k] and its transpose.  On each level: two weighted-Jacobi sweeps
// from zero, residual and restriction, the coarser level, prolongation with the factor
// `over`, two weighted-Jacobi sweeps.  The coarsest level (<= 32 cells) is solved with
// its dense inverse.  The cycle is symmetric and positive definite for omega <= 1 and
// over < 2, so it is a valid CG preconditioner; it runs in FP32 for both precisions,
// and the Krylov directions use the Polak-Ribiere beta, which tolerates its rounding.
//
// Levels with more than block_cells cells are processed by the whole team with team
// barriers between sweeps; smaller levels by the team's first block with block
// barriers, while the other blocks wait at one team barrier.
#pragma once

namespace gq {
namespace {

// level table of the algebraic hierarchy, kept per block (every block derives the same
// sizes from the team-wide scans), and scan scratch
struct AMGShared {
    int nlev, stop;
    int n[kAmgMaxLevels], nnz[kAmgMaxLevels], rnz[kAmgMaxLevels];
    int row_off[kAmgMaxLevels], nnz_off[kAmgMaxLevels], rnz_off[kAmgMaxLevels];
    long long red[32];
    int wsc[32];
    long long tns[kAmgMaxLevels + 2];
    long long bph[8];                   // build time per phase (block 0's clock)
    long long tlast;
    long long cyc[kAmgMaxLevels];       // cycle time per level; the last slot: outside the cycle
    long long tcyc;
    int ccur;
};

struct GJShared {
    double a[kCoarseMax][2 * kCoarseMax];   // Gauss-Jordan tableau of the coarsest level
    double col[kCoarseMax];                 // pivot column, read before it is eliminated
};

// per-warp column table of one coarse row of the algebraic Galerkin product
struct RapShared {
    double tval[kSolveThreads / 32][kAmgRowMax];
    double sv[kSolveThreads / 32][32];
    int tcol[kSolveThreads / 32][kAmgRowMax];
};

// cycle timing: the time since the last mark goes to the slot then current (block 0's
// first thread only; the last slot collects the time outside the cycle)
__device__ __forceinline__ void cyc_mark(AMGShared& as, Team team, int slot) {
    if (team.rank == 0 && threadIdx.x == 0) {
        const long long t = global_ns();
        as.cyc[as.ccur] += t - as.tcyc;
        as.tcyc = t;
        as.ccur = slot;
    }
}

// starts the cycle timing of a solve
__device__ __forceinline__ void cyc_reset(AMGShared& as) {
    if (threadIdx.x == 0) {
        for (int k = 0; k < kAmgMaxLevels; k++) as.cyc[k] = 0;
        as.tcyc = global_ns();
        as.ccur = kAmgMaxLevels - 1;
    }
}

struct MGShared {
    union {                                 // never in use at the same time
        GJShared gj;
        RapShared rap;
    };
    AMGShared amg;
};

// iteration range of a level: the whole team, or one block
struct Range {
    int start, step;
};

__device__ __forceinline__ int parent_of(int k, int nx, int cnx) {
    const int j = k / nx, i = k - j * nx;
    return (j >> 1) * cnx + (i >> 1);
}

// ---- hierarchy build (FP64), levels >= 1 -----------------------------------------------

// coarsen level l (>= 1) into level l + 1
__device__ void mg_coarsen(const MGLevel& F, const MGLevel& C, Range rg) {
    for (int c = rg.start; c < C.N; c += rg.step) {
        const int jc = c / C.nx, ic = c - jc * C.nx;
        const int i0 = 2 * ic, j0 = 2 * jc;
        const int i1 = min(i0 + 1, F.nx - 1), j1 = min(j0 + 1, F.ny - 1);
        double m = 0.0, ww = 0.0, ws = 0.0;
        for (int j = j0; j <= j1; j++) {
            for (int i = i0; i <= i1; i++) m += __ldcg(F.m + j * F.nx + i);
            ww += __ldcg(F.wW + j * F.nx + i0);
        }
        for (int i = i0; i <= i1; i++) ws += __ldcg(F.wS + j0 * F.nx + i);
        C.m[c] = m;
        C.wW[c] = ww;
        C.wS[c] = ws;
    }
}

__device__ void mg_scale_diag(const MGLevel& L, Range rg) {
    for (int k = rg.start; k < L.N; k += rg.step) {
        const int j = k / L.nx, i = k - j * L.nx;
        double d = __ldcg(L.m + k) + __ldcg(L.wW + k) + __ldcg(L.wS + k);
        if (i < L.nx - 1) d += __ldcg(L.wW + k + 1);
        if (j < L.ny - 1) d += __ldcg(L.wS + k + L.nx);
        L.s[k] = 1.0 / sqrt(d);
    }
}

__device__ void mg_scale_couplings(const MGLevel& L, Range rg) {
    for (int k = rg.start; k < L.N; k += rg.step) {
        const int j = k / L.nx, i = k - j * L.nx;
        const double sk = __ldcg(L.s + k);
        L.cW[k] = i > 0 ? static_cast<float>(__ldcg(L.wW + k) * sk * __ldcg(L.s + k - 1)) : 0.f;
        L.cS[k] = j > 0 ? static_cast<float>(__ldcg(L.wS + k) * sk * __ldcg(L.s + k - L.nx)) : 0.f;
    }
}

// transfer weights of level l to level l + 1 (s_l of level 0 is the workspace's dloc)
__device__ void mg_transfer(const MGLevel& F, const double* sF, const MGLevel& C, Range rg) {
    for (int k = rg.start; k < F.N; k += rg.step)
        F.t[k] = static_cast<float>(__ldcg(C.s + parent_of(k, F.nx, C.nx)) / __ldcg(sF + k));
}

// dense inverse of the coarsest scaled operator (one block, FP64 Gauss-Jordan; SPD so
// no pivoting); couplings from FP64 data: level 0 uses the workspace's scaled c_W, c_S,
// coarser levels their unscaled weights and s
__device__ void mg_dense_inverse(const MGHierarchy& mg, const Workspace& w, MGShared& sm) {
    const MGLevel& L = mg.L[mg.nlev - 1];
    const int n = L.N, nx = L.nx;
    const bool lvl0 = mg.nlev == 1;
    if (n > kCoarseMax) return;      // the plan layout coarsens below kCoarseMax cells
    for (int e = threadIdx.x; e < n * 2 * n; e += blockDim.x) {
        const int r = e / (2 * n), c = e - r * 2 * n;
        double v = 0.0;
        if (c >= n) {
            v = (c - n == r) ? 1.0 : 0.0;
        } else if (c == r) {
            v = 1.0;
        } else {
            // coupling between r and c if they are neighbours
            const int lo = min(r, c), hi = max(r, c);
            double cw = 0.0;
            if (hi == lo + 1 && (hi % nx) != 0)
                cw = lvl0 ? __ldcg(w.wW + hi) : __ldcg(L.wW + hi) * __ldcg(L.s + hi) * __ldcg(L.s + lo);
            else if (hi == lo + nx)
                cw = lvl0 ? __ldcg(w.wS + hi) : __ldcg(L.wS + hi) * __ldcg(L.s + hi) * __ldcg(L.s + lo);
            v = -cw;
        }
        sm.gj.a[r][c] = v;
    }
    __syncthreads();
    for (int p = 0; p < n; p++) {
        const double piv = sm.gj.a[p][p];
        __syncthreads();
        for (int c = threadIdx.x; c < 2 * n; c += blockDim.x) sm.gj.a[p][c] /= piv;
        for (int r = threadIdx.x; r < n; r += blockDim.x) sm.gj.col[r] = sm.gj.a[r][p];
        __syncthreads();
        // every multiplier comes from the snapshot, so no thread reads an entry another
        // thread of this step writes
        for (int e = threadIdx.x; e < n * 2 * n; e += blockDim.x) {
            const int r = e / (2 * n), c = e - r * 2 * n;
            if (r != p) sm.gj.a[r][c] -= sm.gj.col[r] * sm.gj.a[p][c];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int r = e / n, c = e - r * n;
        mg.inv[e] = static_cast<float>(sm.gj.a[r][n + c]);
    }
    __syncthreads();
}

// whole hierarchy below level 1 (level 1 itself was coarsened in the set-up pass)
__device__ bool mg_build(const Workspace& w, Team team, int tid, int stride, long long spin, int* abort_flag,
                         MGShared& sm) {
    const MGHierarchy& mg = w.mg;
    const Range rg{tid, stride};
    for (int l = 1; l + 1 < mg.nlev; l++) {
        mg_coarsen(mg.L[l], mg.L[l + 1], rg);
        if (!team_barrier(w.bar, team, spin, abort_flag)) return false;
    }
    for (int l = 1; l < mg.nlev; l++) mg_scale_diag(mg.L[l], rg);
    if (!team_barrier(w.bar, team, spin, abort_flag)) return false;
    for (int l = 1; l < mg.nlev; l++) mg_scale_couplings(mg.L[l], rg);
    for (int l = 0; l + 1 < mg.nlev; l++) mg_transfer(mg.L[l], l == 0 ? w.dloc : mg.L[l].s, mg.L[l + 1], rg);
    if (team.rank == 0) mg_dense_inverse(mg, w, sm);
    return team_barrier(w.bar, team, spin, abort_flag);
}

// ---- V-cycle (FP32) ---------------------------------------------------------------------

struct Lv {                  // a level as the cycle sees it
    int nx, ny, N;
    const float* cW;
    const float* cS;
    const float* t;
    const float* r;          // right-hand side
    float* xa;
    float* xb;
    float* out;              // result of the level (xa for l >= 1, z for level 0)
};

// Loads of vectors that other SMs write during the kernel bypass L1 (CG = true): team
// levels.  The block-only levels are written and read by one block, so they go through
// L1 (CG = false), except the right-hand side of the first block level, which the team
// restricts into it (rcg).
template <bool CG>
__device__ __forceinline__ float ldm(const float* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// (A^ v)_k with unit diagonal; v values at k and its 4 neighbours (0 off the grid)
__device__ __forceinline__ float stencil(float vc, float vw, float ve, float vs, float vn, float cw, float ce,
                                         float cs, float cn) {
    return vc - cw * vw - ce * ve - cs * vs - cn * vn;
}

// D1: two Jacobi sweeps from zero: xa = omega (2 r - omega A r)
template <bool CG>
__device__ void cyc_presmooth(const Lv& L, float om, Range rg, bool rcg) {
    const float* __restrict__ r = L.r;
    const float* __restrict__ cW = L.cW;
    const float* __restrict__ cS = L.cS;
    float* __restrict__ xa = L.xa;
    const int nx = L.nx, N = L.N;
#pragma unroll 4
    for (int k = rg.start; k < N; k += rg.step) {
        const bool he = k + 1 < N, hn = k + nx < N;
        auto R = [&](int m) { return (CG || rcg) ? __ldcg(r + m) : r[m]; };
        const float rc = R(k);
        const float rw = k > 0 ? R(k - 1) : 0.f, re = he ? R(k + 1) : 0.f;
        const float rs = k >= nx ? R(k - nx) : 0.f, rn = hn ? R(k + nx) : 0.f;
        const float ce = he ? cW[k + 1] : 0.f, cn = hn ? cS[k + nx] : 0.f;
        const float ar = stencil(rc, rw, re, rs, rn, cW[k], ce, cS[k], cn);
        xa[k] = om * (2.f * rc - om * ar);
    }
}

// D2: residual of xa, restricted to the coarse right-hand side
template <bool CG>
__device__ void cyc_restrict(const Lv& F, const Lv& C, Range rg) {
    const float* __restrict__ xa = F.xa;
    const float* __restrict__ r = F.r;
    const float* __restrict__ cW = F.cW;
    const float* __restrict__ cS = F.cS;
    const float* __restrict__ t = F.t;
    float* __restrict__ rc = const_cast<float*>(C.r);
    const int nx = F.nx, ny = F.ny;
#pragma unroll 2
    for (int c = rg.start; c < C.N; c += rg.step) {
        const int jc = c / C.nx, ic = c - jc * C.nx;
        const int i0 = 2 * ic, j0 = 2 * jc;
        const int i1 = min(i0 + 1, nx - 1), j1 = min(j0 + 1, ny - 1);
        float acc = 0.f;
        for (int j = j0; j <= j1; j++)
            for (int i = i0; i <= i1; i++) {
                const int k = j * nx + i;
                const bool he = i + 1 < nx, hn = j + 1 < ny;
                const float xw = i > 0 ? ldm<CG>(xa + k - 1) : 0.f, xe = he ? ldm<CG>(xa + k + 1) : 0.f;
                const float xs = j > 0 ? ldm<CG>(xa + k - nx) : 0.f, xn = hn ? ldm<CG>(xa + k + nx) : 0.f;
                const float ce = he ? cW[k + 1] : 0.f, cn = hn ? cS[k + nx] : 0.f;
                const float ax = stencil(ldm<CG>(xa + k), xw, xe, xs, xn, cW[k], ce, cS[k], cn);
                acc += t[k] * (ldm<CG>(r + k) - ax);
            }
        rc[c] = acc;
    }
}

// U1: prolongation of the coarse result into xa, then one Jacobi sweep -> xb
template <bool CG>
__device__ void cyc_prolong_smooth(const Lv& F, const Lv& C, float om, float over, Range rg) {
    const float* __restrict__ xa = F.xa;
    const float* __restrict__ r = F.r;
    const float* __restrict__ cW = F.cW;
    const float* __restrict__ cS = F.cS;
    const float* __restrict__ t = F.t;
    const float* __restrict__ xc = C.out;
    float* __restrict__ xb = F.xb;
    const int nx = F.nx, N = F.N, cnx = C.nx;
#pragma unroll 2
    for (int k = rg.start; k < N; k += rg.step) {
        const int j = k / nx, i = k - j * nx;
        const bool hw = i > 0, he = i + 1 < nx, hs = k >= nx, hn = k + nx < N;
        auto xt = [&](int m, int mi, int mj) -> float {
            return ldm<CG>(xa + m) + over * t[m] * ldm<CG>(xc + (mj >> 1) * cnx + (mi >> 1));
        };
        const float x0 = xt(k, i, j);
        const float xw = hw ? xt(k - 1, i - 1, j) : 0.f, xe = he ? xt(k + 1, i + 1, j) : 0.f;
        const float xs = hs ? xt(k - nx, i, j - 1) : 0.f, xn = hn ? xt(k + nx, i, j + 1) : 0.f;
        const float ce = he ? cW[k + 1] : 0.f, cn = hn ? cS[k + nx] : 0.f;
        const float ax = stencil(x0, xw, xe, xs, xn, cW[k], ce, cS[k], cn);
        xb[k] = x0 + om * (ldm<CG>(r + k) - ax);
    }
}

// U2: one Jacobi sweep xb -> out; on level 0 also the partial sums r.z and r.z_old
template <bool CG>
__device__ void cyc_postsmooth(const Lv& L, float om, Range rg, const float* zold, double* rz, double* rzo) {
    const float* __restrict__ xb = L.xb;
    const float* __restrict__ r = L.r;
    const float* __restrict__ cW = L.cW;
    const float* __restrict__ cS = L.cS;
    float* __restrict__ out = L.out;
    const int nx = L.nx, N = L.N;
    float rzf = 0.f, rzof = 0.f;   // this thread's partial sums in FP32 (FP64 per cell is slow on this part)
#pragma unroll 4
    for (int k = rg.start; k < N; k += rg.step) {
        const bool he = k + 1 < N, hn = k + nx < N;
        const float xc = ldm<CG>(xb + k);
        const float xw = k > 0 ? ldm<CG>(xb + k - 1) : 0.f, xe = he ? ldm<CG>(xb + k + 1) : 0.f;
        const float xs = k >= nx ? ldm<CG>(xb + k - nx) : 0.f, xn = hn ? ldm<CG>(xb + k + nx) : 0.f;
        const float ce = he ? cW[k + 1] : 0.f, cn = hn ? cS[k + nx] : 0.f;
        const float ax = stencil(xc, xw, xe, xs, xn, cW[k], ce, cS[k], cn);
        const float rk = ldm<CG>(r + k);
        const float z = xc + om * (rk - ax);
        out[k] = z;
        if (rz) {
            rzf += rk * z;
            rzof += rk * __ldcg(zold + k);
        }
    }
    if (rz) {
        *rz += static_cast<double>(rzf);
        *rzo += static_cast<double>(rzof);
    }
}

// coarsest level: out = inv r (one block)
__device__ void cyc_coarse(const Lv& L, const float* inv, Range rg, bool rcg, const float* zold, double* rz,
                           double* rzo) {
    for (int i = rg.start; i < L.N; i += rg.step) {
        float acc = 0.f;
        for (int j = 0; j < L.N; j++) acc += inv[i * L.N + j] * (rcg ? __ldcg(L.r + j) : L.r[j]);
        L.out[i] = acc;
        if (rz) {
            const double rk = rcg ? __ldcg(L.r + i) : L.r[i];
            *rz += rk * acc;
            *rzo += rk * __ldcg(zold + i);
        }
    }
}

// ---- fine level, four cells per thread (nx a multiple of 4) -----------------------------

struct F4 {
    float v[4];
};

__device__ __forceinline__ F4 ld4(const float* p) {
    const float4 q = __ldcg(reinterpret_cast<const float4*>(p));
    return F4{{q.x, q.y, q.z, q.w}};
}

__device__ __forceinline__ void st4(float* p, const F4& a) {
    *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}

// A^ v on the 4 cells k..k+3 (one row) from v's chunk, its south and north chunks and
// the west and east scalars; coefficients loaded here
__device__ __forceinline__ F4 apply4(const F4& c, const F4& s, const F4& n, float w, float e, const float* cW,
                                     const float* cS, int k, int nx, int N) {
    const bool he = k + 4 < N, hn = k + nx < N;
    const F4 cw = ld4(cW + k), cs = ld4(cS + k);
    const float cwe = he ? __ldcg(cW + k + 4) : 0.f;
    const F4 csn = hn ? ld4(cS + k + nx) : F4{{0.f, 0.f, 0.f, 0.f}};
    F4 a;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const float left = i == 0 ? w : c.v[i - 1];
        const float right = i == 3 ? e : c.v[i + 1];
        const float cright = i == 3 ? cwe : cw.v[i + 1];
        a.v[i] = stencil(c.v[i], left, right, s.v[i], n.v[i], cw.v[i], cright, cs.v[i], csn.v[i]);
    }
    return a;
}

// a vector's chunk with its neighbours (zeros off the grid)
__device__ __forceinline__ void nb4(const float* v, int k, int nx, int N, F4& c, F4& s, F4& n, float& w,
                                    float& e) {
    const F4 zero{{0.f, 0.f, 0.f, 0.f}};
    c = ld4(v + k);
    s = k >= nx ? ld4(v + k - nx) : zero;
    n = k + nx < N ? ld4(v + k + nx) : zero;
    w = k > 0 ? __ldcg(v + k - 1) : 0.f;
    e = k + 4 < N ? __ldcg(v + k + 4) : 0.f;
}

__device__ void cyc0_presmooth_v(const Lv& L, float om, Range rg) {
    const int nx = L.nx, N = L.N, nchunk = N / 4;
    for (int q = rg.start; q < nchunk; q += rg.step) {
        const int k = 4 * q;
        F4 c, s, n;
        float w, e;
        nb4(L.r, k, nx, N, c, s, n, w, e);
        const F4 a = apply4(c, s, n, w, e, L.cW, L.cS, k, nx, N);
        F4 x;
#pragma unroll
        for (int i = 0; i < 4; i++) x.v[i] = om * (2.f * c.v[i] - om * a.v[i]);
        st4(L.xa + k, x);
    }
}

// The Krylov update r' = r - alpha q, d += alpha p fused with the next cycle's level-0
// pre-smoothing (two Jacobi sweeps from zero on r'): r' is formed on the chunk and its
// neighbours from r and q, so no barrier separates the two.  r' goes to rnew (r stays
// intact for the neighbours of other threads); rr receives this thread's sum of r'^2.
__device__ void cyc0_update_presmooth_v(const Lv& L, const float* rold, float* rnew, const float* q, const float* p,
                                        float* d, float alpha, float om, Range rg, double* rr) {
    const int nx = L.nx, N = L.N, nchunk = N / 4;
    float rrf = 0.f;               // this thread's partial sum in FP32
    for (int ch = rg.start; ch < nchunk; ch += rg.step) {
        const int k = 4 * ch;
        F4 c, s, n, qc, qs, qn;
        float w, e, qw, qe;
        nb4(rold, k, nx, N, c, s, n, w, e);
        nb4(q, k, nx, N, qc, qs, qn, qw, qe);
#pragma unroll
        for (int i = 0; i < 4; i++) {
            c.v[i] = c.v[i] - alpha * qc.v[i];
            s.v[i] = s.v[i] - alpha * qs.v[i];
            n.v[i] = n.v[i] - alpha * qn.v[i];
        }
        w = w - alpha * qw;
        e = e - alpha * qe;
        const F4 a = apply4(c, s, n, w, e, L.cW, L.cS, k, nx, N);
        F4 x;
        F4 dk = ld4(d + k);
        const F4 pk = ld4(p + k);
#pragma unroll
        for (int i = 0; i < 4; i++) {
            x.v[i] = om * (2.f * c.v[i] - om * a.v[i]);
            dk.v[i] = dk.v[i] + alpha * pk.v[i];
            rrf += c.v[i] * c.v[i];
        }
        st4(L.xa + k, x);
        st4(rnew + k, c);
        st4(d + k, dk);
    }
    *rr += static_cast<double>(rrf);
}

__device__ void cyc0_postsmooth_v(const Lv& L, float om, Range rg, const float* zold, double* rz, double* rzo) {
    const int nx = L.nx, N = L.N, nchunk = N / 4;
    float rzf = 0.f, rzof = 0.f;   // this thread's partial sums in FP32
    for (int q = rg.start; q < nchunk; q += rg.step) {
        const int k = 4 * q;
        F4 c, s, n;
        float w, e;
        nb4(L.xb, k, nx, N, c, s, n, w, e);
        const F4 a = apply4(c, s, n, w, e, L.cW, L.cS, k, nx, N);
        const F4 rr = ld4(L.r + k);
        const F4 zo = ld4(zold + k);
        F4 z;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            z.v[i] = c.v[i] + om * (rr.v[i] - a.v[i]);
            rzf += rr.v[i] * z.v[i];
            rzof += rr.v[i] * zo.v[i];
        }
        st4(L.out + k, z);
    }
    *rz += static_cast<double>(rzf);
    *rzo += static_cast<double>(rzof);
}

// prolongation + one sweep on 4 fine cells of one row; parents of the chunk are the coarse
// cells i0/2 and i0/2 + 1 of row j/2
__device__ void cyc0_prolong_smooth_v(const Lv& F, const Lv& C, float om, float over, Range rg) {
    const int nx = F.nx, N = F.N, nchunk = N / 4, cnx = C.nx;
    const F4 zero{{0.f, 0.f, 0.f, 0.f}};
    for (int q = rg.start; q < nchunk; q += rg.step) {
        const int k = 4 * q;
        const int j = k / nx, i0 = k - j * nx;
        const bool hs = j > 0, hn = k + nx < N, hw = i0 > 0, he = i0 + 4 < nx;
        // x~ = xa + over t xc(parent) on the chunk, the south and north chunks, west and east
        auto row = [&](int jj, int kk) -> F4 {
            const F4 x = ld4(F.xa + kk), tt = ld4(F.t + kk);
            const float* pc = C.out + (jj >> 1) * cnx + (i0 >> 1);
            const float p0 = __ldcg(pc), p1 = __ldcg(pc + 1);
            F4 o;
            o.v[0] = x.v[0] + over * tt.v[0] * p0;
            o.v[1] = x.v[1] + over * tt.v[1] * p0;
            o.v[2] = x.v[2] + over * tt.v[2] * p1;
            o.v[3] = x.v[3] + over * tt.v[3] * p1;
            return o;
        };
        auto one = [&](int jj, int ii) -> float {
            const int kk = jj * nx + ii;
            return __ldcg(F.xa + kk) + over * __ldcg(F.t + kk) * __ldcg(C.out + (jj >> 1) * cnx + (ii >> 1));
        };
        const F4 c = row(j, k);
        const F4 s = hs ? row(j - 1, k - nx) : zero;
        const F4 n = hn ? row(j + 1, k + nx) : zero;
        const float w = hw ? one(j, i0 - 1) : 0.f;
        const float e = he ? one(j, i0 + 4) : 0.f;
        const F4 a = apply4(c, s, n, w, e, F.cW, F.cS, k, nx, N);
        const F4 rr = ld4(F.r + k);
        F4 x;
#pragma unroll
        for (int i = 0; i < 4; i++) x.v[i] = c.v[i] + om * (rr.v[i] - a.v[i]);
        st4(F.xb + k, x);
    }
}

// residual and restriction for two coarse cells per thread: fine rows j0, j0 + 1 and
// columns i0..i0+3 (i0 a multiple of 4)
__device__ void cyc0_restrict_v(const Lv& F, const Lv& C, Range rg) {
    const int nx = F.nx, ny = F.ny, N = F.N;
    const int npair = (C.nx / 2) * C.ny;       // C.nx = nx / 2 is even
    for (int q = rg.start; q < npair; q += rg.step) {
        const int jc = q / (C.nx / 2), ic2 = q - jc * (C.nx / 2);
        const int i0 = 4 * ic2, j0 = 2 * jc;
        float acc0 = 0.f, acc1 = 0.f;
        for (int jj = 0; jj < 2; jj++) {
            const int j = j0 + jj;
            if (j >= ny) break;
            const int k = j * nx + i0;
            F4 c, s, n;
            float w, e;
            nb4(F.xa, k, nx, N, c, s, n, w, e);
            const F4 a = apply4(c, s, n, w, e, F.cW, F.cS, k, nx, N);
            const F4 rr = ld4(F.r + k), tt = ld4(F.t + k);
            acc0 += tt.v[0] * (rr.v[0] - a.v[0]) + tt.v[1] * (rr.v[1] - a.v[1]);
            acc1 += tt.v[2] * (rr.v[2] - a.v[2]) + tt.v[3] * (rr.v[3] - a.v[3]);
        }
        float* rc = const_cast<float*>(C.r) + jc * C.nx + 2 * ic2;
        rc[0] = acc0;
        rc[1] = acc1;
    }
}

__device__ __forceinline__ Lv level_view(const MGHierarchy& mg, int l, const float* r0, float* z) {
    const MGLevel& M = mg.L[l];
    Lv v;
    v.nx = M.nx;
    v.ny = M.ny;
    v.N = M.N;
    v.cW = M.cW;
    v.cS = M.cS;
    v.t = M.t;
    v.r = l == 0 ? r0 : M.r;
    v.xa = M.xa;
    v.xb = M.xb;
    v.out = l == 0 ? z : M.xa;
    return v;
}

// z = B r0 on the team; rz, rzo receive this thread's partial sums of r0.z and r0.zold.
// Returns false on a timed-out wait.
__device__ bool vcycle(const MGHierarchy& mg, AMGShared& as, const float* r0, float* z, const float* zold, float om,
                       float over, int block_cells, bool pre0_done, Team team, int tid, int stride, unsigned* bar,
                       long long spin, int* abort_flag, double* rz, double* rzo) {
    const int nl = mg.nlev;
    int lg = 0;                          // levels [0, lg) run on the whole team
    while (lg < nl - 1 && mg.L[lg].N > block_cells) lg++;
    const Range tr{tid, stride};
    const Range br{static_cast<int>(threadIdx.x), static_cast<int>(blockDim.x)};
    // the fine level uses 4-cell vectors when its rows allow (and its coarse level has an
    // even width)
    const bool v0 = lg > 0 && (mg.L[0].nx % 4) == 0 && nl > 1;
    for (int l = 0; l < lg; l++) {
        const Lv F = level_view(mg, l, r0, z), C = level_view(mg, l + 1, r0, z);
        cyc_mark(as, team, l);
        // level 0's pre-smoothing may already be done by the fused Krylov update (whose
        // reduction was the barrier)
        if (!(l == 0 && v0 && pre0_done)) {
            if (l == 0 && v0) cyc0_presmooth_v(F, om, Range{tid, stride});
            else cyc_presmooth<true>(F, om, tr, true);
            if (!team_barrier(bar, team, spin, abort_flag)) return false;
        }
        if (l == 0 && v0) cyc0_restrict_v(F, C, tr);
        else cyc_restrict<true>(F, C, tr);
        if (!team_barrier(bar, team, spin, abort_flag)) return false;
    }
    if (team.rank == 0) {
        cyc_mark(as, team, lg);      // all block levels together
        for (int l = lg; l + 1 < nl; l++) {
            const Lv F = level_view(mg, l, r0, z), C = level_view(mg, l + 1, r0, z);
            // the first block level's right-hand side comes from the team (or is r0)
            cyc_presmooth<false>(F, om, br, l == lg);
            __syncthreads();
            if (l == lg) cyc_restrict<true>(F, C, br);
            else cyc_restrict<false>(F, C, br);
            __syncthreads();
        }
        const Lv Z = level_view(mg, nl - 1, r0, z);
        cyc_coarse(Z, mg.inv, br, lg == nl - 1, zold, nl == 1 ? rz : nullptr, rzo);
        __syncthreads();
        for (int l = nl - 2; l >= lg; l--) {
            const Lv F = level_view(mg, l, r0, z), C = level_view(mg, l + 1, r0, z);
            if (l == lg) {
                cyc_prolong_smooth<true>(F, C, om, over, br);
                __syncthreads();
                cyc_postsmooth<true>(F, om, br, zold, l == 0 ? rz : nullptr, rzo);
            } else {
                cyc_prolong_smooth<false>(F, C, om, over, br);
                __syncthreads();
                cyc_postsmooth<false>(F, om, br, zold, l == 0 ? rz : nullptr, rzo);
            }
            __syncthreads();
        }
    }
    if (!team_barrier(bar, team, spin, abort_flag)) return false;
    for (int l = lg - 1; l >= 0; l--) {
        const Lv F = level_view(mg, l, r0, z), C = level_view(mg, l + 1, r0, z);
        cyc_mark(as, team, l);
        if (l == 0 && v0) cyc0_prolong_smooth_v(F, C, om, over, tr);
        else cyc_prolong_smooth<true>(F, C, om, over, tr);
        if (!team_barrier(bar, team, spin, abort_flag)) return false;
        if (l == 0 && v0) cyc0_postsmooth_v(F, om, tr, zold, rz, rzo);
        else cyc_postsmooth<true>(F, om, tr, zold, l == 0 ? rz : nullptr, rzo);
        if (l > 0 && !team_barrier(bar, team, spin, abort_flag)) return false;
    }
    cyc_mark(as, team, kAmgMaxLevels - 1);
    return true;
}

}  // namespace
}  // namespace gq
