// Classical algebraic multigrid preconditioner (included by gq_pcg.cuh).
//
// Why: with cell-by-cell random densities and temperatures the flux-limited face weights
// w_f jump by many orders of magnitude between neighbouring faces, and where the time
// step makes diffusion dominate the mass term the slow modes of A are the near-constant
// vectors on clusters of strongly coupled cells.  A fixed 2 x 2 aggregation cuts those
// clusters and cannot represent them; a coarse grid chosen from the couplings can.
//
// Set-up (every step, on the device, FP64, unscaled operator A_l):
//   strength   j is a strong neighbour of i when -a_ij >= theta max_k(-a_ik), measured on
//              the unscaled entries (the face weights themselves on level 0)
//   splitting  PMIS: weight = number of points that depend on i + a hash in [0, 1); an
//              undecided point whose weight beats every undecided strong neighbour (both
//              directions) becomes C, undecided points depending on a new C point become F,
//              repeated until nothing is undecided; then every F point that depends on
//              some point but on no C point becomes C
//   P          direct interpolation: p_ij = -alpha_i a_ij / (a_ii + sum of positive a_ik)
//              with alpha_i = (sum of negative a_ik) / (sum over strong C neighbours), the
//              kAmgPmax largest kept and rescaled to the same row sum; C points inject
//   A_{l+1}    P^T A_l P, one coarse row per thread: the fine rows that interpolate from
//              coarse point c are c's own point and F neighbours of it, so the product
//              is gathered without atomics; rows are computed once, staged at the pool
//              tails and moved to the places a scan gives them (one warp per row when a
//              row is too long for a thread's table)
// Coarsening stops at <= kCoarseMax rows (dense inverse), when a level does not shrink,
// or when a pool would overflow (the coarsest level is then smoothed instead).
// The V-cycle works on the Jacobi-scaled levels A^_l = S_l A_l S_l (unit diagonal, FP32)
// with P^_l = S_l^{-1} P_l S_{l+1}: two weighted-Jacobi sweeps, residual, restriction
// (P^T), the coarser level, prolongation, two weighted-Jacobi sweeps.  It is symmetric
// and positive definite for omega <= 1 (unit-diagonal levels with spectrum in (0, 2)).
#pragma once

namespace gq {
namespace {

constexpr double kAmgTheta = 0.25;
constexpr int kAmgRounds = 40;
constexpr signed char kStU = 0, kStC = 1, kStF = 2;

// why coarsening stopped (AMGInfo::stop)
enum { kAmgStopSmall = 1, kAmgStopLevels = 2, kAmgStopNoC = 3, kAmgStopRows = 4, kAmgStopNnz = 5,
       kAmgStopRowMax = 6 };

__device__ __forceinline__ double amg_hash(unsigned i, unsigned l) {
    unsigned x = i * 0x9E3779B1u ^ (l + 1u) * 0x85EBCA77u;
    x ^= x >> 15;
    x *= 0x2C1B3C6Du;
    x ^= x >> 12;
    x *= 0x297A2D39u;
    x ^= x >> 15;
    return (double)(x >> 8) * (1.0 / 16777216.0);
}

// loads of hierarchy data during the build: L1-bypassing while the team builds (other SMs
// write it), plain while block 0 builds alone (only it writes, so its L1 stays current)
template <bool CG, class T>
__device__ __forceinline__ T ldp(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// exclusive scan of one value per thread over the block; chunk_total = block sum
__device__ __forceinline__ int block_excl_scan(int v, int& chunk_total, int* wsc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsc[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = lane < nw ? wsc[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) wsc[lane] = t;
    }
    __syncthreads();
    const int pre = warp > 0 ? wsc[warp - 1] : 0;
    chunk_total = wsc[nw - 1];
    __syncthreads();
    return pre + x - v;
}

// Team-wide exclusive scan out[i] = sum_{k < i} cnt[k], i < n; block b scans the b-th
// contiguous segment.  total receives the sum in every thread.  out[] of other blocks is
// readable after the next team barrier.  Returns false on a timed-out wait.
__device__ bool team_scan(const int* cnt, int* out, int n, int& total, double* partials, int& parity,
                          unsigned* bar, long long spin, int* abort_flag, Team team, AMGShared& as) {
    const int G = team.size;
    const int seg = (n + G - 1) / G;
    const int lo = min(n, team.rank * seg), hi = min(n, lo + seg);
    long long s = 0;
    for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) s += __ldcg(cnt + i);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) as.red[warp] = s;
    __syncthreads();
    double* mine = partials + (size_t)parity * G * kSlots;
    if (threadIdx.x == 0) {
        long long b = 0;
        for (int k = 0; k < nw; k++) b += as.red[k];
        mine[team.rank * kSlots] = (double)b;
    }
    if (!team_barrier(bar, team, spin, abort_flag)) return false;
    if (warp == 0) {
        long long pre = 0, tot = 0;
        for (int b = lane; b < G; b += 32) {
            const long long v = (long long)__ldcg(mine + b * kSlots);
            tot += v;
            if (b < team.rank) pre += v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            pre += __shfl_down_sync(0xffffffffu, pre, o);
            tot += __shfl_down_sync(0xffffffffu, tot, o);
        }
        if (lane == 0) {
            as.red[0] = pre;
            as.red[1] = tot;
        }
    }
    __syncthreads();
    int carry = (int)as.red[0];
    total = (int)as.red[1];
    __syncthreads();
    for (int base = lo; base < hi; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < hi ? __ldcg(cnt + i) : 0;
        int chunk = 0;
        const int e = block_excl_scan(v, chunk, as.wsc);
        if (i < hi) out[i] = carry + e;
        carry += chunk;
    }
    parity ^= 1;
    return true;
}

// sum over the warp, identical in every lane (each butterfly step adds the same pair)
__device__ __forceinline__ double warp_sum_all(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One coarse row c of P^T A P, computed by one warp: the fine rows that interpolate from
// c (c's own point, then the F neighbours of it in entry order) are taken one at a time;
// their entries (diagonal first) are spread over the lanes, and each lane's terms are
// merged into a per-warp column table in shared memory.  Terms that hit the same column
// in one round are summed by the lowest lane in lane order, so the sums are bitwise
// reproducible.  FILL = false only counts (distinct off-diagonal columns, restriction
// entries); FILL = true also writes the row, its diagonal and its restriction entries.
// Returns false when the row has more than kAmgRowMax columns.
template <bool FILL, bool CG>
__device__ bool amg_coarse_row_warp(int c, const AMGData& A, int ro, const int* rp, const int* cl, const double* av,
                               const double* dg, RapShared& rs, int wid, int lane, int* col_out, double* a_out,
                               double* diag_out, int* rent_out, int& ncol, int& nr) {
    int* tcol = rs.tcol[wid];
    double* tval = rs.tval[wid];
    double* sv = rs.sv[wid];
    int m = 0;
    bool ovf = false;
    double dgc = 0.0;
    const int f = ldp<CG>(A.cf + c);
    const int fb = ldp<CG>(rp + f), nf = ldp<CG>(rp + f + 1) - fb;
    auto contrib = [&](int i, double wi) {
        const int ib = ldp<CG>(rp + i), ne = ldp<CG>(rp + i + 1) - ib + 1;
        for (int base = 0; base < ne; base += 32) {
            const int e = base + lane;
            int k = -1;
            double aik = 0.0;
            if (e < ne) {
                k = e == 0 ? i : ldp<CG>(cl + ib + e - 1);
                aik = e == 0 ? ldp<CG>(dg + i) : ldp<CG>(av + ib + e - 1);
            }
            int pcq[kAmgPmax];
            double pvq[kAmgPmax];
#pragma unroll
            for (int q = 0; q < kAmgPmax; q++) {
                pcq[q] = (k >= 0 && aik != 0.0) ? ldp<CG>(A.pc + (size_t)kAmgPmax * (ro + k) + q) : -1;
                pvq[q] = pcq[q] >= 0 ? ldp<CG>(A.pv64 + (size_t)kAmgPmax * k + q) : 0.0;
            }
#pragma unroll
            for (int q = 0; q < kAmgPmax; q++) {
                const int cc = pcq[q];
                const double v = cc >= 0 ? wi * aik * pvq[q] : 0.0;
                dgc += warp_sum_all(cc == c ? v : 0.0);
                const bool off = cc >= 0 && cc != c;
                int pos = -1;
                if (off)
                    for (int u = 0; u < m; u++)
                        if (tcol[u] == cc) {
                            pos = u;
                            break;
                        }
                const unsigned grp = __match_any_sync(0xffffffffu, off ? cc : -1 - lane);
                sv[lane] = v;
                __syncwarp();
                const bool leader = off && lane == __ffs(grp) - 1;
                double sum = 0.0;
                if (leader) {
                    unsigned g = grp;
                    while (g) {
                        sum += sv[__ffs(g) - 1];
                        g &= g - 1;
                    }
                }
                const unsigned newm = __ballot_sync(0xffffffffu, leader && pos < 0);
                if (leader) {
                    if (pos >= 0) {
                        tval[pos] += sum;
                    } else {
                        const int slot = m + __popc(newm & ((1u << lane) - 1u));
                        if (slot < kAmgRowMax) {
                            tcol[slot] = cc;
                            tval[slot] = sum;
                        }
                    }
                }
                m += __popc(newm);
                if (m > kAmgRowMax) {
                    ovf = true;
                    m = kAmgRowMax;
                }
                __syncwarp();
            }
        }
    };
    contrib(f, 1.0);
    if constexpr (FILL) {
        if (lane == 0) rent_out[0] = kAmgPmax * (ro + f);
    }
    nr = 1;
    for (int base = 0; base < nf; base += 32) {
        const int h = base + lane;
        int j = -1, slot = -1;
        double wj = 0.0;
        if (h < nf) {
            j = ldp<CG>(cl + fb + h);
            if (ldp<CG>(A.stB + j) == kStF) {
#pragma unroll
                for (int q = 0; q < kAmgPmax; q++)
                    if (ldp<CG>(A.pc + (size_t)kAmgPmax * (ro + j) + q) == c) slot = q;
                if (slot >= 0) wj = ldp<CG>(A.pv64 + (size_t)kAmgPmax * j + slot);
            }
        }
        unsigned mask = __ballot_sync(0xffffffffu, slot >= 0);
        while (mask) {
            const int b = __ffs(mask) - 1;
            mask &= mask - 1;
            const int i = __shfl_sync(0xffffffffu, j, b);
            const int sl = __shfl_sync(0xffffffffu, slot, b);
            const double wi = __shfl_sync(0xffffffffu, wj, b);
            if constexpr (FILL) {
                if (lane == 0) rent_out[nr] = kAmgPmax * (ro + i) + sl;
            }
            nr++;
            contrib(i, wi);
        }
    }
    ncol = m;
    if constexpr (FILL) {
        for (int u = lane; u < m; u += 32) {
            col_out[u] = tcol[u];
            a_out[u] = tval[u];
        }
        if (lane == 0) *diag_out = dgc;
    }
    __syncwarp();
    return !ovf;
}

// The same coarse row computed by one thread with a small column table (levels built by
// the whole team, where rows are many and threads hide each other's latency).  Returns
// false when the row has more than kAmgRowThread columns.
constexpr int kAmgRowThread = 24;

// The coarse row's column table (cols, vals), its diagonal and its restriction count.
template <bool CG>
__device__ __forceinline__ bool amg_row_table(int c, const AMGData& A, int ro, const int* rp, const int* cl,
                                              const double* av, const double* dg, int (&cols)[kAmgRowThread],
                                              double (&vals)[kAmgRowThread], double& dgc, int& m, int& nr) {
    m = 0;
    dgc = 0.0;
    nr = 0;
    const int f = ldp<CG>(A.cf + c);
    const int fb = ldp<CG>(rp + f), fe = ldp<CG>(rp + f + 1);
    // contributors: f itself (slot 0, weight 1) and the F neighbours of f that interpolate from c
    for (int h = -1; h < fe - fb; h++) {
        int i;
        double wi;
        if (h < 0) {
            i = f;
            wi = 1.0;
        } else {
            i = ldp<CG>(cl + fb + h);
            if (ldp<CG>(A.stB + i) != kStF) continue;
            int slot = -1;
            for (int q = 0; q < kAmgPmax; q++)
                if (ldp<CG>(A.pc + (size_t)kAmgPmax * (ro + i) + q) == c) slot = q;
            if (slot < 0) continue;
            wi = ldp<CG>(A.pv64 + (size_t)kAmgPmax * i + slot);
        }
        nr++;
        const int ib = ldp<CG>(rp + i), ie = ldp<CG>(rp + i + 1);
        for (int e = ib - 1; e < ie; e++) {
            const int k = e < ib ? i : ldp<CG>(cl + e);
            const double aik = e < ib ? ldp<CG>(dg + i) : ldp<CG>(av + e);
            if (aik == 0.0) continue;
            const double wa = wi * aik;
            // the 4 interpolation slots of row k: one 16-byte and two 16-byte loads
            const int4 pc4 = ldp<CG>(reinterpret_cast<const int4*>(A.pc) + (ro + k));
            const double2 pv01 = ldp<CG>(reinterpret_cast<const double2*>(A.pv64) + 2 * (size_t)k);
            const double2 pv23 = ldp<CG>(reinterpret_cast<const double2*>(A.pv64) + 2 * (size_t)k + 1);
            const int pcs[kAmgPmax] = {pc4.x, pc4.y, pc4.z, pc4.w};
            const double pvs[kAmgPmax] = {pv01.x, pv01.y, pv23.x, pv23.y};
#pragma unroll
            for (int q = 0; q < kAmgPmax; q++) {
                const int cc = pcs[q];
                if (cc < 0) continue;
                const double v = wa * pvs[q];
                if (cc == c) {
                    dgc += v;
                    continue;
                }
                int u = 0;
                while (u < m && cols[u] != cc) u++;
                if (u == m) {
                    if (m == kAmgRowThread) return false;
                    cols[m] = cc;
                    vals[m] = 0.0;
                    m++;
                }
                vals[u] += v;
            }
        }
    }
    return true;
}

// the restriction entries of coarse row c (indices into the P pool), in contributor order
template <bool CG>
__device__ __forceinline__ void amg_row_rents(int c, const AMGData& A, int ro, const int* rp, const int* cl,
                                              int* rent_out) {
    const int f = ldp<CG>(A.cf + c);
    const int fb = ldp<CG>(rp + f), fe = ldp<CG>(rp + f + 1);
    rent_out[0] = kAmgPmax * (ro + f);
    int nr = 1;
    for (int h = 0; h < fe - fb; h++) {
        const int i = ldp<CG>(cl + fb + h);
        if (ldp<CG>(A.stB + i) != kStF) continue;
        int slot = -1;
        for (int q = 0; q < kAmgPmax; q++)
            if (ldp<CG>(A.pc + (size_t)kAmgPmax * (ro + i) + q) == c) slot = q;
        if (slot >= 0) rent_out[nr++] = kAmgPmax * (ro + i) + slot;
    }
}

enum { kLvlOk = 0, kLvlStop = 1, kLvlTimeout = 2 };

// Coarsens level l into level l + 1 on the team tm (the whole team, or block 0 alone as a
// team of one).  Updates this block's level table; kLvlStop when coarsening must end here.
template <bool CG>
__device__ int amg_level(int l, const Workspace& w, Team tm, int tid, int stride, long long spin, int* abort_flag,
                         RedShared& sh, MGShared& msh, int& parity) {
    const AMGData& A = w.amg;
    AMGShared& as = msh.amg;
    auto sync = [&]() { return team_barrier(w.bar, tm, spin, abort_flag); };
    const int n = as.n[l], ro = as.row_off[l], eo = as.nnz_off[l];
    const int* rp = A.rowptr + ro + l;
    const int* cl = A.col + eo;
    const double* av = A.a64 + eo;
    unsigned char* sf = A.sfl + eo;
    const double* dg = A.diag + ro;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gw = tid >> 5, nwarps = stride >> 5;
    auto mark = [&](int k) {
        if (threadIdx.x == 0) {
            const long long t = global_ns();
            as.bph[k] += t - as.tlast;
            as.tlast = t;
        }
    };
    if (threadIdx.x == 0) as.tlast = global_ns();

    // 1. largest negative coupling of every row
    for (int i = tid; i < n; i += stride) {
        double m = 0.0;
        for (int e = ldp<CG>(rp + i), ee = ldp<CG>(rp + i + 1); e < ee; e++) m = fmax(m, -ldp<CG>(av + e));
        A.rowmax[i] = m;
    }
    if (!sync()) return kLvlTimeout;
    // 2. strength flags, PMIS weights, initial states (isolated points are F)
    for (int i = tid; i < n; i += stride) {
        const double rmi = ldp<CG>(A.rowmax + i);
        int nS = 0, nST = 0;
        for (int e = ldp<CG>(rp + i), ee = ldp<CG>(rp + i + 1); e < ee; e++) {
            const double v = -ldp<CG>(av + e);
            unsigned char fl = 0;
            if (v > 0.0) {
                if (v >= kAmgTheta * rmi) fl |= 1;
                if (v >= kAmgTheta * ldp<CG>(A.rowmax + ldp<CG>(cl + e))) fl |= 2;
            }
            sf[e] = fl;
            nS += fl & 1;
            nST += fl >> 1;
        }
        A.wgt[i] = nST + amg_hash((unsigned)i, (unsigned)l);
        A.stA[i] = (nS == 0 && nST == 0) ? kStF : kStU;
        A.cnt2[i] = nS;
    }
    if (!sync()) return kLvlTimeout;
    mark(0);
    // 3. PMIS rounds (stA -> stB -> stA)
    for (int round = 0; round < kAmgRounds; round++) {
        for (int i = tid; i < n; i += stride) {
            signed char st = ldp<CG>(A.stA + i);
            if (st == kStU) {
                const double wi = ldp<CG>(A.wgt + i);
                bool best = true;
                for (int e = ldp<CG>(rp + i), ee = ldp<CG>(rp + i + 1); e < ee && best; e++) {
                    if (!ldp<CG>(sf + e)) continue;
                    const int j = ldp<CG>(cl + e);
                    if (ldp<CG>(A.stA + j) != kStU) continue;
                    const double wj = ldp<CG>(A.wgt + j);
                    if (wj > wi || (wj == wi && j > i)) best = false;
                }
                if (best) st = kStC;
            }
            A.stB[i] = st;
        }
        if (!sync()) return kLvlTimeout;
        double cu[1] = {0.0};
        for (int i = tid; i < n; i += stride) {
            signed char st = ldp<CG>(A.stB + i);
            if (st == kStU) {
                for (int e = ldp<CG>(rp + i), ee = ldp<CG>(rp + i + 1); e < ee; e++)
                    if ((ldp<CG>(sf + e) & 1) && ldp<CG>(A.stB + ldp<CG>(cl + e)) == kStC) {
                        st = kStF;
                        break;
                    }
                if (st == kStU) cu[0] += 1.0;
            }
            A.stA[i] = st;
        }
        if (!allreduce<1, 0>(cu, w.partials, parity, w.bar, spin, abort_flag, sh, tm)) return kLvlTimeout;
        if (cu[0] == 0.0) break;
    }
    mark(1);
    // 4. undecided points become C; an F point that depends on points but on no C point
    //    becomes C (stA -> stB); C flags for the numbering
    for (int i = tid; i < n; i += stride) {
        signed char st = ldp<CG>(A.stA + i);
        if (st == kStU) {
            st = kStC;
        } else if (st == kStF && ldp<CG>(A.cnt2 + i) > 0) {
            bool has = false;
            for (int e = ldp<CG>(rp + i), ee = ldp<CG>(rp + i + 1); e < ee && !has; e++)
                if (ldp<CG>(sf + e) & 1) {
                    const signed char sj = ldp<CG>(A.stA + ldp<CG>(cl + e));
                    has = sj == kStC || sj == kStU;
                }
            if (!has) st = kStC;
        }
        A.stB[i] = st;
        A.cnt[i] = st == kStC;
    }
    if (!sync()) return kLvlTimeout;
    // 5. coarse numbering
    int nc = 0;
    if (!team_scan(A.cnt, A.cidx, n, nc, w.partials, parity, w.bar, spin, abort_flag, tm, as)) return kLvlTimeout;
    if (!sync()) return kLvlTimeout;
    mark(2);
    if (nc == 0 || nc >= n) {
        if (threadIdx.x == 0) as.stop = kAmgStopNoC;
        return kLvlStop;
    }
    const int ro_c = ro + n;
    if ((long long)ro_c + nc > A.cap_rows) {
        if (threadIdx.x == 0) as.stop = kAmgStopRows;
        return kLvlStop;
    }
    for (int i = tid; i < n; i += stride)
        if (ldp<CG>(A.stB + i) == kStC) A.cf[ldp<CG>(A.cidx + i)] = i;
    // 6. interpolation rows of level l (ELL, kAmgPmax slots)
    for (int i = tid; i < n; i += stride) {
        int* pcr = A.pc + (size_t)kAmgPmax * (ro + i);
        double* pvr = A.pv64 + (size_t)kAmgPmax * i;
        int kc[kAmgPmax];
        double kv[kAmgPmax];
#pragma unroll
        for (int q = 0; q < kAmgPmax; q++) {
            kc[q] = -1;
            kv[q] = 0.0;
        }
        if (ldp<CG>(A.stB + i) == kStC) {
            kc[0] = ldp<CG>(A.cidx + i);
            kv[0] = 1.0;
        } else {
            double negsum = 0.0, possum = 0.0, csum = 0.0;
            const int eb = ldp<CG>(rp + i), ee = ldp<CG>(rp + i + 1);
            for (int e = eb; e < ee; e++) {
                const double a = ldp<CG>(av + e);
                if (a < 0.0) negsum += a;
                else possum += a;
                if ((ldp<CG>(sf + e) & 1) && ldp<CG>(A.stB + ldp<CG>(cl + e)) == kStC) csum += a;
            }
            if (csum < 0.0) {
                const double fac = -(negsum / csum) / (ldp<CG>(dg + i) + possum);
                double tot = 0.0, kept = 0.0;
                for (int e = eb; e < ee; e++) {
                    const int j = ldp<CG>(cl + e);
                    if (!(ldp<CG>(sf + e) & 1) || ldp<CG>(A.stB + j) != kStC) continue;
                    const double p = fac * ldp<CG>(av + e);
                    tot += p;
                    // keep the kAmgPmax largest (insertion into a descending list)
                    if (p > kv[kAmgPmax - 1]) {
                        int q = kAmgPmax - 1;
                        while (q > 0 && kv[q - 1] < p) {
                            kv[q] = kv[q - 1];
                            kc[q] = kc[q - 1];
                            q--;
                        }
                        kv[q] = p;
                        kc[q] = ldp<CG>(A.cidx + j);
                    }
                }
#pragma unroll
                for (int q = 0; q < kAmgPmax; q++) kept += kc[q] >= 0 ? kv[q] : 0.0;
                const double sc = kept > 0.0 ? tot / kept : 0.0;
#pragma unroll
                for (int q = 0; q < kAmgPmax; q++) kv[q] = kc[q] >= 0 ? kv[q] * sc : 0.0;
            }
        }
#pragma unroll
        for (int q = 0; q < kAmgPmax; q++) {
            pcr[q] = kc[q];
            pvr[q] = kv[q];
        }
    }
    if (tid == 0) {
        A.info->ctr = 0;
        A.info->rctr = 0;
    }
    if (!sync()) return kLvlTimeout;
    mark(3);
    // 7. the coarse rows of P^T A P, one thread per row, computed once: each row is staged
    //    at the tail of the entry pool (its restriction entries at the tail of the
    //    restriction pool), with space reserved per warp by one atomic; the final layout
    //    follows from the scans, so the result does not depend on the reservation order.
    //    A row too long for a thread's table sends the level to one warp per row (counted,
    //    then filled); too little tail space to the thread count-and-fill.
    const int eo_c = eo + as.nnz[l];
    const int roff = as.rnz_off[l];
    const long long rcap = (long long)kAmgPmax * A.cap_rows;
    double ovf[2] = {0.0, 0.0};
    for (int base = tid - lane; base < nc; base += stride) {     // whole warps together
        const int c = base + lane;
        int m = 0, nr = 0;
        double dgc = 0.0;
        int cols[kAmgRowThread];
        double vals[kAmgRowThread];
        bool ok = true;
        if (c < nc) ok = amg_row_table<CG>(c, A, ro, rp, cl, av, dg, cols, vals, dgc, m, nr);
        if (!ok) {
            ovf[0] = 1.0;
            m = 0;
            nr = 0;
        }
        int pm = m, pr = nr;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ym = __shfl_up_sync(0xffffffffu, pm, o), yr = __shfl_up_sync(0xffffffffu, pr, o);
            if (lane >= o) {
                pm += ym;
                pr += yr;
            }
        }
        int bm = 0, br = 0;
        if (lane == 31) {
            bm = atomicAdd(&A.info->ctr, pm);
            br = atomicAdd(&A.info->rctr, pr);
        }
        bm = __shfl_sync(0xffffffffu, bm, 31);
        br = __shfl_sync(0xffffffffu, br, 31);
        const long long pos = (long long)A.cap_nnz - (bm + pm), rpos = rcap - (br + pr);
        if (c < nc && ok) {
            if (pos < eo_c || rpos < roff) {
                ovf[1] = 1.0;
            } else {
                for (int u = 0; u < m; u++) {
                    A.col[pos + u] = cols[u];
                    A.a64[pos + u] = vals[u];
                }
                amg_row_rents<CG>(c, A, ro, rp, cl, A.rent + rpos);
            }
            A.diag[ro_c + c] = dgc;
            A.toff[c] = (int)pos;
            A.troff[c] = (int)rpos;
        }
        if (c < nc) {
            A.cnt[c] = m;
            A.cnt2[c] = nr;
        }
    }
    if (!allreduce<0, 2>(ovf, w.partials, parity, w.bar, spin, abort_flag, sh, tm)) return kLvlTimeout;
    const bool warp_rap = ovf[0] != 0.0;
    bool staged = ovf[1] == 0.0 && !warp_rap;
    if (warp_rap) {
        double ov[1] = {0.0};
        for (int c = gw; c < nc; c += nwarps) {
            int m = 0, nr = 0;
            const bool ok = amg_coarse_row_warp<false, CG>(c, A, ro, rp, cl, av, dg, msh.rap, wid, lane, nullptr,
                                                           nullptr, nullptr, nullptr, m, nr);
            if (lane == 0) {
                A.cnt[c] = m;
                A.cnt2[c] = nr;
                if (!ok) ov[0] = 1.0;
            }
        }
        if (!allreduce<0, 1>(ov, w.partials, parity, w.bar, spin, abort_flag, sh, tm)) return kLvlTimeout;
        if (ov[0] != 0.0) {
            if (threadIdx.x == 0) as.stop = kAmgStopRowMax;
            return kLvlStop;
        }
    }
    mark(4);
    // 8. row pointers of level l+1 and of the restriction
    int nnz_c = 0, rtot = 0;
    int* rp_c = A.rowptr + ro_c + (l + 1);
    int* rr_c = A.rrow + ro_c + (l + 1);
    if (!team_scan(A.cnt, rp_c, nc, nnz_c, w.partials, parity, w.bar, spin, abort_flag, tm, as)) return kLvlTimeout;
    if (!team_scan(A.cnt2, rr_c, nc, rtot, w.partials, parity, w.bar, spin, abort_flag, tm, as)) return kLvlTimeout;
    if ((long long)eo_c + nnz_c > A.cap_nnz || (long long)roff + rtot > rcap) {
        if (threadIdx.x == 0) as.stop = kAmgStopNnz;
        return kLvlStop;
    }
    // the staged rows occupy [cap - nnz_c, cap): usable only if the final places lie below
    staged = staged && (long long)eo_c + 2ll * nnz_c <= A.cap_nnz && (long long)roff + 2ll * rtot <= rcap;
    if (tid == 0) {
        rp_c[nc] = nnz_c;
        rr_c[nc] = rtot;
    }
    if (!sync()) return kLvlTimeout;
    mark(5);
    // 9. level l+1 and the restriction of level l in their final places
    if (staged) {
        for (int c = tid; c < nc; c += stride) {
            const int e0 = ldp<CG>(rp_c + c), m = ldp<CG>(A.cnt + c);
            const int src = ldp<CG>(A.toff + c);
            for (int u = 0; u < m; u++) {
                A.col[eo_c + e0 + u] = ldp<CG>(A.col + src + u);
                A.a64[eo_c + e0 + u] = ldp<CG>(A.a64 + src + u);
            }
            const int r0 = ldp<CG>(rr_c + c), nr = ldp<CG>(A.cnt2 + c), rsrc = ldp<CG>(A.troff + c);
            for (int u = 0; u < nr; u++) A.rent[roff + r0 + u] = ldp<CG>(A.rent + rsrc + u);
        }
    } else if (warp_rap) {
        for (int c = gw; c < nc; c += nwarps) {
            int m = 0, nr = 0;
            const int e0 = ldp<CG>(rp_c + c), r0 = ldp<CG>(rr_c + c);
            amg_coarse_row_warp<true, CG>(c, A, ro, rp, cl, av, dg, msh.rap, wid, lane, A.col + eo_c + e0,
                                          A.a64 + eo_c + e0, A.diag + ro_c + c, A.rent + roff + r0, m, nr);
        }
    } else {
        for (int c = tid; c < nc; c += stride) {
            int m = 0, nr = 0;
            double dgc = 0.0;
            int cols[kAmgRowThread];
            double vals[kAmgRowThread];
            amg_row_table<CG>(c, A, ro, rp, cl, av, dg, cols, vals, dgc, m, nr);
            const int e0 = ldp<CG>(rp_c + c), r0 = ldp<CG>(rr_c + c);
            for (int u = 0; u < m; u++) {
                A.col[eo_c + e0 + u] = cols[u];
                A.a64[eo_c + e0 + u] = vals[u];
            }
            A.diag[ro_c + c] = dgc;
            amg_row_rents<CG>(c, A, ro, rp, cl, A.rent + roff + r0);
        }
    }
    if (!sync()) return kLvlTimeout;
    mark(6);
    // 10. scaling of level l+1
    for (int c = tid; c < nc; c += stride) A.s[ro_c + c] = 1.0 / sqrt(ldp<CG>(A.diag + ro_c + c));
    if (threadIdx.x == 0) {
        as.n[l + 1] = nc;
        as.nnz[l + 1] = nnz_c;
        as.row_off[l + 1] = ro_c;
        as.nnz_off[l + 1] = eo_c;
        as.rnz[l] = rtot;
        as.rnz_off[l + 1] = roff + rtot;
        as.nlev = l + 2;
    }
    if (!sync()) return kLvlTimeout;
    // 11. scaled entries of level l+1, scaled interpolation weights of level l
    for (int c = tid; c < nc; c += stride) {
        const double sc = ldp<CG>(A.s + ro_c + c);
        for (int e = ldp<CG>(rp_c + c), ee = ldp<CG>(rp_c + c + 1); e < ee; e++)
            A.a32[eo_c + e] =
                (float)(ldp<CG>(A.a64 + eo_c + e) * sc * ldp<CG>(A.s + ro_c + ldp<CG>(A.col + eo_c + e)));
    }
    for (int i = tid; i < n; i += stride) {
        const double si = l == 0 ? ldp<CG>(w.dloc + i) : ldp<CG>(A.s + ro + i);
#pragma unroll
        for (int q = 0; q < kAmgPmax; q++) {
            const size_t k = (size_t)kAmgPmax * (ro + i) + q;
            const int cc = ldp<CG>(A.pc + k);
            A.pv32[k] =
                cc >= 0 ? (float)(ldp<CG>(A.pv64 + (size_t)kAmgPmax * i + q) * ldp<CG>(A.s + ro_c + cc) / si) : 0.f;
        }
    }
    if (!sync()) return kLvlTimeout;
    mark(7);
    if (threadIdx.x == 0) as.tns[2 + l] = global_ns();
    return kLvlOk;
}

// Builds the hierarchy from the Jacobi-scaled fine system of the workspace (level 0: the
// unscaled operator recovered as a_ij = -c_ij / (s_i s_j), a_ii = 1 / s_i^2).  Levels with
// more than block_cells rows are coarsened by the whole team, the smaller ones by the
// team's first block alone while the others wait at one barrier.  All blocks call it and
// leave with the same level table; returns false on a timed-out wait.
__device__ bool amg_build(const Workspace& w, int nx, int ny, int block_cells, Team team, int tid, int stride,
                          long long spin, int* abort_flag, RedShared& sh, MGShared& msh, int& parity) {
    const AMGData& A = w.amg;
    AMGShared& as = msh.amg;
    const int n0 = A.n0;
    auto sync = [&]() { return team_barrier(w.bar, team, spin, abort_flag); };
    if (threadIdx.x == 0) {
        as.tns[0] = global_ns();
        for (int k = 0; k < 8; k++) as.bph[k] = 0;
    }

    // ---- level 0 ------------------------------------------------------------------------
    for (int i = tid; i < n0; i += stride) {
        const int y = i / nx, x = i - y * nx;
        A.cnt[i] = (x > 0) + (x < nx - 1) + (y > 0) + (y < ny - 1);
    }
    if (!sync()) return false;
    int nnz0 = 0;
    if (!team_scan(A.cnt, A.rowptr, n0, nnz0, w.partials, parity, w.bar, spin, abort_flag, team, as)) return false;
    if (tid == 0) A.rowptr[n0] = nnz0;
    if (!sync()) return false;
    for (int i = tid; i < n0; i += stride) {
        const int y = i / nx, x = i - y * nx;
        const double si = __ldcg(w.dloc + i);
        int e = __ldcg(A.rowptr + i);
        auto put = [&](int j, double c) {
            A.col[e] = j;
            A.a64[e] = -c / (si * __ldcg(w.dloc + j));
            e++;
        };
        if (x > 0) put(i - 1, __ldcg(w.wW + i));
        if (x < nx - 1) put(i + 1, __ldcg(w.wW + i + 1));
        if (y > 0) put(i - nx, __ldcg(w.wS + i));
        if (y < ny - 1) put(i + nx, __ldcg(w.wS + i + nx));
        A.diag[i] = 1.0 / (si * si);
    }
    if (threadIdx.x == 0) {
        as.nlev = 1;
        as.stop = 0;
        as.n[0] = n0;
        as.nnz[0] = nnz0;
        as.row_off[0] = 0;
        as.nnz_off[0] = 0;
        as.rnz_off[0] = 0;
    }
    if (!sync()) return false;
    if (threadIdx.x == 0) as.tns[1] = global_ns();

    // ---- coarsening ---------------------------------------------------------------------
    // 0: continue, 1: done, 2: the rest goes to block 0
    auto next = [&](int l, bool on_team) -> int {
        const int n = as.n[l];
        if (n <= kCoarseMax) {
            if (threadIdx.x == 0) as.stop = kAmgStopSmall;
            return 1;
        }
        if (l + 1 >= kAmgMaxLevels) {
            if (threadIdx.x == 0) as.stop = kAmgStopLevels;
            return 1;
        }
        return (on_team && team.size > 1 && n <= block_cells) ? 2 : 0;
    };
    int l = 0, how = 0;
    while ((how = next(l, true)) == 0) {
        const int r = amg_level<true>(l, w, team, tid, stride, spin, abort_flag, sh, msh, parity);
        if (r == kLvlTimeout) return false;
        if (r == kLvlStop) {
            how = 1;
            break;
        }
        l++;
    }
    if (how == 2 && team.rank == 0) {
        // the small levels on block 0 alone (a team of one: block barriers only); its
        // reduction parity is restored afterwards so that the team stays in step
        const int saved = parity;
        const Team solo{0, 1};
        while (next(l, false) == 0) {
            const int r = amg_level<false>(l, w, solo, threadIdx.x, blockDim.x, spin, abort_flag, sh, msh, parity);
            if (r != kLvlOk) break;
            l++;
        }
        parity = saved;
    }

    // ---- coarsest level: dense inverse of its scaled operator; the level table ----------
    if (team.rank == 0) {
        const int L = as.nlev - 1;
        const int nL = as.n[L];
        if (nL <= kCoarseMax) {
            const int ro = as.row_off[L], eo = as.nnz_off[L];
            const int* rp = A.rowptr + ro + L;
            auto sL = [&](int i) { return L == 0 ? __ldcg(w.dloc + i) : __ldcg(A.s + ro + i); };
            for (int e = threadIdx.x; e < nL * 2 * nL; e += blockDim.x) {
                const int r = e / (2 * nL), c = e - r * 2 * nL;
                msh.gj.a[r][c] = (c == r || c - nL == r) ? 1.0 : 0.0;
            }
            __syncthreads();
            for (int r = threadIdx.x; r < nL; r += blockDim.x) {
                const double sr = sL(r);
                for (int e = __ldcg(rp + r), ee = __ldcg(rp + r + 1); e < ee; e++) {
                    const int c = __ldcg(A.col + eo + e);
                    msh.gj.a[r][c] += __ldcg(A.a64 + eo + e) * sr * sL(c);
                }
            }
            __syncthreads();
            for (int p = 0; p < nL; p++) {
                const double piv = msh.gj.a[p][p];
                __syncthreads();
                for (int c = threadIdx.x; c < 2 * nL; c += blockDim.x) msh.gj.a[p][c] /= piv;
                for (int r = threadIdx.x; r < nL; r += blockDim.x) msh.gj.col[r] = msh.gj.a[r][p];
                __syncthreads();
                for (int e = threadIdx.x; e < nL * 2 * nL; e += blockDim.x) {
                    const int r = e / (2 * nL), c = e - r * 2 * nL;
                    if (r != p) msh.gj.a[r][c] -= msh.gj.col[r] * msh.gj.a[p][c];
                }
                __syncthreads();
            }
            for (int e = threadIdx.x; e < nL * nL; e += blockDim.x) {
                const int r = e / nL, c = e - r * nL;
                A.inv[e] = static_cast<float>(msh.gj.a[r][nL + c]);
            }
        }
        if (threadIdx.x == 0) {
            AMGInfo* I = A.info;
            as.tns[as.nlev + 1] = global_ns();
            for (int k = 0; k <= as.nlev + 1; k++) I->tns[k] = as.tns[k];
            for (int k = 0; k < 8; k++) I->bph[k] = as.bph[k];
            I->nlev = as.nlev;
            I->stop = as.stop;
            for (int k = 0; k < as.nlev; k++) {
                I->n[k] = as.n[k];
                I->nnz[k] = as.nnz[k];
                I->rnz[k] = k + 1 < as.nlev ? as.rnz[k] : 0;
                I->row_off[k] = as.row_off[k];
                I->nnz_off[k] = as.nnz_off[k];
                I->rnz_off[k] = as.rnz_off[k];
            }
        }
    }
    if (!sync()) return false;
    // every block takes the level table that block 0 completed
    if (threadIdx.x == 0) {
        const AMGInfo* I = A.info;
        as.nlev = __ldcg(&I->nlev);
        for (int k = 0; k < as.nlev; k++) {
            as.n[k] = __ldcg(&I->n[k]);
            as.nnz[k] = __ldcg(&I->nnz[k]);
            as.rnz[k] = __ldcg(&I->rnz[k]);
            as.row_off[k] = __ldcg(&I->row_off[k]);
            as.nnz_off[k] = __ldcg(&I->nnz_off[k]);
            as.rnz_off[k] = __ldcg(&I->rnz_off[k]);
        }
    }
    cyc_reset(as);
    __syncthreads();
    return true;
}


// writes the cycle timing of the solve to the device info block
__device__ void amg_cycle_report(const AMGData& A, AMGShared& as, Team team) {
    cyc_mark(as, team, kAmgMaxLevels - 1);
    if (team.rank == 0 && threadIdx.x == 0)
        for (int k = 0; k < kAmgMaxLevels; k++) A.info->cyc[k] = as.cyc[k];
}

// ---- V-cycle (FP32) -------------------------------------------------------------------

// a level as the cycle sees it
struct AV {
    int n, nx;             // nx > 0: level 0 (structured 5-point, cW/cS)
    const int* rp;         // level >= 1: CSR (entries relative to a, col)
    const int* col;
    const float* a;
    const float* cW;
    const float* cS;
    const int* pc;         // P of this level -> next (ELL), absolute pool index base 0
    const float* pv;
    const int* rr;         // restriction rows of the NEXT level are stored with it
    const int* rent;
    const float* b;        // right-hand side
    float* x;              // result
    float* t;              // scratch
};

__device__ __forceinline__ AV amg_view(const AMGData& A, const AMGShared& as, int l, const float* r0, float* z,
                                       const float* cW0, const float* cS0, int nx0) {
    AV v;
    const int ro = as.row_off[l], eo = as.nnz_off[l];
    v.n = as.n[l];
    v.nx = l == 0 ? nx0 : 0;
    v.rp = A.rowptr + ro + l;
    v.col = A.col + eo;
    v.a = A.a32 + eo;
    v.cW = cW0;
    v.cS = cS0;
    v.pc = A.pc + (size_t)kAmgPmax * ro;
    v.pv = A.pv32 + (size_t)kAmgPmax * ro;
    v.rr = A.rrow + ro + l;
    v.rent = A.rent + as.rnz_off[l > 0 ? l - 1 : 0];
    v.b = l == 0 ? r0 : A.b + ro;
    v.x = l == 0 ? z : A.x + ro;
    v.t = A.t + ro;
    return v;
}

// Loads in the cycle.  The hierarchy's arrays are written once by the build (through L2,
// with L1-bypassing loads) and only read afterwards, so plain L1-cached loads see the
// current values.  Vectors that other SMs write during the cycle are loaded with __ldcg
// (CG = true: team levels; BCG: the right-hand side of the first block level, which the
// team restricts into).
template <bool CG>
__device__ __forceinline__ float ldvec(const float* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// (A^ v)_i with unit diagonal
template <bool CG>
__device__ __forceinline__ float amg_apply(const AV& L, const float* v, int i, float vi) {
    float ax = vi;
    if (L.nx > 0) {
        const int nx = L.nx, N = L.n;
        if (i > 0) ax -= L.cW[i] * ldvec<CG>(v + i - 1);
        if (i + 1 < N) ax -= L.cW[i + 1] * ldvec<CG>(v + i + 1);
        if (i >= nx) ax -= L.cS[i] * ldvec<CG>(v + i - nx);
        if (i + nx < N) ax -= L.cS[i + nx] * ldvec<CG>(v + i + nx);
    } else {
        // four gathers in flight per thread
        int e = L.rp[i];
        const int ee = L.rp[i + 1];
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        for (; e + 4 <= ee; e += 4) {
            const int c0 = L.col[e], c1 = L.col[e + 1], c2 = L.col[e + 2], c3 = L.col[e + 3];
            const float w0 = L.a[e], w1 = L.a[e + 1], w2 = L.a[e + 2], w3 = L.a[e + 3];
            a0 += w0 * ldvec<CG>(v + c0);
            a1 += w1 * ldvec<CG>(v + c1);
            a2 += w2 * ldvec<CG>(v + c2);
            a3 += w3 * ldvec<CG>(v + c3);
        }
        for (; e < ee; e++) a0 += L.a[e] * ldvec<CG>(v + L.col[e]);
        ax += (a0 + a1) + (a2 + a3);
    }
    return ax;
}

// two Jacobi sweeps from zero: x = omega (2 b - omega A^ b)
template <bool CG, bool BCG>
__device__ void amg_pre(const AV& L, float om, Range rg) {
    for (int i = rg.start; i < L.n; i += rg.step) {
        const float bi = ldvec<BCG>(L.b + i);
        L.x[i] = om * (2.f * bi - om * amg_apply<BCG>(L, L.b, i, bi));
    }
}

// t = b - A^ x
template <bool CG, bool BCG>
__device__ void amg_resid(const AV& L, Range rg) {
    for (int i = rg.start; i < L.n; i += rg.step) {
        const float xi = ldvec<CG>(L.x + i);
        L.t[i] = ldvec<BCG>(L.b + i) - amg_apply<CG>(L, L.x, i, xi);
    }
}

// b_C = P^T t_F (restriction rows of the coarse level C, entries index F's P pool)
template <bool CG>
__device__ void amg_restrict(const AV& F, const AV& C, const int* pc_base, Range rg) {
    float* bc = const_cast<float*>(C.b);
    const int base = (int)(F.pc - pc_base);
    for (int c = rg.start; c < C.n; c += rg.step) {
        float acc = 0.f;
        for (int e = C.rr[c], ee = C.rr[c + 1]; e < ee; e++) {
            const int k = C.rent[e] - base;                 // index into F's P rows
            acc += F.pv[k] * ldvec<CG>(F.t + k / kAmgPmax);
        }
        bc[c] = acc;
    }
}

// x_F += P x_C (a row's 4 interpolation slots are one 16-byte load each)
template <bool CG>
__device__ void amg_prolong(const AV& F, const AV& C, Range rg) {
    static_assert(kAmgPmax == 4, "one int4 / float4 per interpolation row");
    for (int i = rg.start; i < F.n; i += rg.step) {
        const int4 pc = reinterpret_cast<const int4*>(F.pc)[i];
        const float4 pv = reinterpret_cast<const float4*>(F.pv)[i];
        float acc = ldvec<CG>(F.x + i);
        if (pc.x >= 0) acc += pv.x * ldvec<CG>(C.x + pc.x);
        if (pc.y >= 0) acc += pv.y * ldvec<CG>(C.x + pc.y);
        if (pc.z >= 0) acc += pv.z * ldvec<CG>(C.x + pc.z);
        if (pc.w >= 0) acc += pv.w * ldvec<CG>(C.x + pc.w);
        F.x[i] = acc;
    }
}

// Level 0 with 4 cells per thread (nx a multiple of 4, team levels): 16-byte loads of the
// vector, its south and north rows and the coefficients.  MODE 0: out = omega (2 b - omega
// A^ b) (in = b); 1: out = b - A^ in; 2: out = in + omega (b - A^ in), with the partial sums
// b.out and b.z_old when rz is given.  c_W of a row's first cell is zero, so the west and
// east neighbours may cross rows.
template <int MODE>
__device__ void amg0_v(const AV& L, const float* in, float* out, float om, Range rg, const float* zold, double* rz,
                       double* rzo) {
    const int nx = L.nx, N = L.n, nch = N >> 2;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float rzf = 0.f, rzof = 0.f;   // this thread's partial sums in FP32 (FP64 per cell is slow on this part)
    for (int ch = rg.start; ch < nch; ch += rg.step) {
        const int k = ch << 2;
        const float4 v = __ldcg(reinterpret_cast<const float4*>(in + k));
        const float vw = k > 0 ? __ldcg(in + k - 1) : 0.f;
        const float ve = k + 4 < N ? __ldcg(in + k + 4) : 0.f;
        const float4 vs = k >= nx ? __ldcg(reinterpret_cast<const float4*>(in + k - nx)) : z4;
        const float4 vn = k + nx < N ? __ldcg(reinterpret_cast<const float4*>(in + k + nx)) : z4;
        const float4 cw = *reinterpret_cast<const float4*>(L.cW + k);
        const float4 cs = *reinterpret_cast<const float4*>(L.cS + k);
        const float4 csn = k + nx < N ? *reinterpret_cast<const float4*>(L.cS + k + nx) : z4;
        const float cwe = k + 4 < N ? L.cW[k + 4] : 0.f;
        float a[4];
        a[0] = v.x - cw.x * vw - cw.y * v.y - cs.x * vs.x - csn.x * vn.x;
        a[1] = v.y - cw.y * v.x - cw.z * v.z - cs.y * vs.y - csn.y * vn.y;
        a[2] = v.z - cw.z * v.y - cw.w * v.w - cs.z * vs.z - csn.z * vn.z;
        a[3] = v.w - cw.w * v.z - cwe * ve - cs.w * vs.w - csn.w * vn.w;
        const float4 b = MODE == 0 ? v : __ldcg(reinterpret_cast<const float4*>(L.b + k));
        const float bb[4] = {b.x, b.y, b.z, b.w}, vv[4] = {v.x, v.y, v.z, v.w};
        float o[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if constexpr (MODE == 0) o[j] = om * (2.f * bb[j] - om * a[j]);
            else if constexpr (MODE == 1) o[j] = bb[j] - a[j];
            else o[j] = vv[j] + om * (bb[j] - a[j]);
        }
        *reinterpret_cast<float4*>(out + k) = make_float4(o[0], o[1], o[2], o[3]);
        if (MODE == 2 && rz) {
            const float4 zo = __ldcg(reinterpret_cast<const float4*>(zold + k));
            const float zz[4] = {zo.x, zo.y, zo.z, zo.w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                rzf += bb[j] * o[j];
                rzof += bb[j] * zz[j];
            }
        }
    }
    if (MODE == 2 && rz) {
        *rz += static_cast<double>(rzf);
        *rzo += static_cast<double>(rzof);
    }
}

// one Jacobi sweep out = in + omega (b - A^ in); level 0's second sweep also sums r.z, r.z_old
template <bool CG, bool BCG>
__device__ void amg_sweep(const AV& L, const float* in, float* out, float om, Range rg, const float* zold,
                          double* rz, double* rzo) {
    float rzf = 0.f, rzof = 0.f;   // this thread's partial sums in FP32
    for (int i = rg.start; i < L.n; i += rg.step) {
        const float vi = ldvec<CG>(in + i), bi = ldvec<BCG>(L.b + i);
        const float v = vi + om * (bi - amg_apply<CG>(L, in, i, vi));
        out[i] = v;
        if (rz) {
            rzf += bi * v;
            rzof += bi * __ldcg(zold + i);
        }
    }
    if (rz) {
        *rz += static_cast<double>(rzf);
        *rzo += static_cast<double>(rzof);
    }
}

// coarsest level on block 0: dense inverse or, if coarsening stopped early, Jacobi sweeps
__device__ void amg_coarse(const AV& L, const float* inv, bool dense, float om, Range rg, const float* zold,
                           double* rz, double* rzo) {
    if (dense) {
        const int n = L.n;
        for (int r = rg.start; r < n; r += rg.step) {
            float acc = 0.f;
            for (int c = 0; c < n; c++) acc += inv[r * n + c] * __ldcg(L.b + c);
            L.x[r] = acc;
            if (rz) {
                *rz += (double)__ldcg(L.b + r) * (double)acc;
                *rzo += (double)__ldcg(L.b + r) * (double)__ldcg(zold + r);
            }
        }
        return;
    }
    for (int i = rg.start; i < L.n; i += rg.step) L.x[i] = om * __ldcg(L.b + i);
    __syncthreads();
    for (int s = 0; s < 3; s++) {
        amg_sweep<false, true>(L, L.x, L.t, om, rg, nullptr, nullptr, nullptr);
        __syncthreads();
        for (int i = rg.start; i < L.n; i += rg.step) L.x[i] = L.t[i];
        __syncthreads();
    }
    if (rz) {
        for (int i = rg.start; i < L.n; i += rg.step) {
            *rz += (double)__ldcg(L.b + i) * (double)L.x[i];
            *rzo += (double)__ldcg(L.b + i) * (double)__ldcg(zold + i);
        }
    }
}

// z = B r0 on the team; rz, rzo receive this thread's partial sums of r0.z and r0.z_old.
// Returns false on a timed-out wait.
__device__ bool amg_vcycle(const AMGData& A, AMGShared& as, const float* r0, float* z, const float* zold,
                           const float* cW0, const float* cS0, int nx0, float om, int block_cells, bool pre0_done,
                           Team team, int tid, int stride,
                           unsigned* bar, long long spin, int* abort_flag, double* rz, double* rzo) {
    const int nl = as.nlev;
    const int Lc = nl - 1;
    const bool dense = as.n[Lc] <= kCoarseMax;
    int lg = 0;                                  // levels [0, lg) run on the whole team
    while (lg < nl - 1 && as.n[lg] > block_cells) lg++;
    // a large coarsest level (coarsening stopped early) is smoothed by the team
    const bool team_coarse = !dense && as.n[Lc] > block_cells;
    if (team_coarse) lg = nl - 1;
    const Range tr{tid, stride};
    const Range br{static_cast<int>(threadIdx.x), static_cast<int>(blockDim.x)};
    auto view = [&](int l) { return amg_view(A, as, l, r0, z, cW0, cS0, nx0); };
    auto sync = [&]() { return team_barrier(bar, team, spin, abort_flag); };

    const bool v0 = (nx0 % 4) == 0;
    for (int l = 0; l < lg; l++) {
        const AV F = view(l), C = view(l + 1);
        cyc_mark(as, team, l);
        // level 0's pre-smoothing may already be done by the fused Krylov update (whose
        // reduction was the barrier)
        if (!(l == 0 && v0 && pre0_done)) {
            if (l == 0 && v0) amg0_v<0>(F, F.b, F.x, om, tr, nullptr, nullptr, nullptr);
            else amg_pre<true, true>(F, om, tr);
            if (!sync()) return false;
        }
        if (l == 0 && v0) amg0_v<1>(F, F.x, F.t, om, tr, nullptr, nullptr, nullptr);
        else amg_resid<true, true>(F, tr);
        if (!sync()) return false;
        amg_restrict<true>(F, C, A.pc, tr);
        if (!sync()) return false;
    }
    if (team_coarse) {
        // x = omega b, then three sweeps, all on the team
        const AV Z = view(Lc);
        for (int i = tid; i < Z.n; i += stride) Z.x[i] = om * __ldcg(Z.b + i);
        if (!sync()) return false;
        for (int s = 0; s < 3; s++) {
            amg_sweep<true, true>(Z, Z.x, Z.t, om, tr, nullptr, nullptr, nullptr);
            if (!sync()) return false;
            for (int i = tid; i < Z.n; i += stride) Z.x[i] = __ldcg(Z.t + i);
            if (!sync()) return false;
        }
        if (Lc == 0) {
            for (int i = tid; i < Z.n; i += stride) {
                *rz += (double)__ldcg(Z.b + i) * (double)__ldcg(Z.x + i);
                *rzo += (double)__ldcg(Z.b + i) * (double)__ldcg(zold + i);
            }
        }
    } else if (team.rank == 0) {
        for (int l = lg; l < Lc; l++) {
            const AV F = view(l), C = view(l + 1);
            cyc_mark(as, team, l);
            if (l == lg) amg_pre<false, true>(F, om, br);
            else amg_pre<false, false>(F, om, br);
            __syncthreads();
            if (l == lg) amg_resid<false, true>(F, br);
            else amg_resid<false, false>(F, br);
            __syncthreads();
            amg_restrict<false>(F, C, A.pc, br);
            __syncthreads();
        }
        const AV Z = view(Lc);
        cyc_mark(as, team, Lc);
        amg_coarse(Z, A.inv, dense, om, br, zold, Lc == 0 ? rz : nullptr, rzo);
        __syncthreads();
        for (int l = Lc - 1; l >= lg; l--) {
            const AV F = view(l), C = view(l + 1);
            cyc_mark(as, team, l);
            amg_prolong<false>(F, C, br);
            __syncthreads();
            if (l == lg) {
                amg_sweep<false, true>(F, F.x, F.t, om, br, nullptr, nullptr, nullptr);
                __syncthreads();
                amg_sweep<false, true>(F, F.t, F.x, om, br, zold, l == 0 ? rz : nullptr, rzo);
            } else {
                amg_sweep<false, false>(F, F.x, F.t, om, br, nullptr, nullptr, nullptr);
                __syncthreads();
                amg_sweep<false, false>(F, F.t, F.x, om, br, zold, l == 0 ? rz : nullptr, rzo);
            }
            __syncthreads();
        }
    }
    if (!sync()) return false;
    for (int l = lg - 1; l >= 0; l--) {
        const AV F = view(l), C = view(l + 1);
        cyc_mark(as, team, l);
        amg_prolong<true>(F, C, tr);
        if (!sync()) return false;
        if (l == 0 && v0) amg0_v<2>(F, F.x, F.t, om, tr, nullptr, nullptr, nullptr);
        else amg_sweep<true, true>(F, F.x, F.t, om, tr, nullptr, nullptr, nullptr);
        if (!sync()) return false;
        if (l == 0 && v0) amg0_v<2>(F, F.t, F.x, om, tr, zold, rz, rzo);
        else amg_sweep<true, true>(F, F.t, F.x, om, tr, zold, l == 0 ? rz : nullptr, rzo);
        if (l > 0 && !sync()) return false;
    }
    cyc_mark(as, team, kAmgMaxLevels - 1);
    return true;
}

}  // namespace
}  // namespace gq
