// Tiled single-problem solve: mixed-precision conjugate gradients preconditioned by the
// aggregation-multigrid V-cycle (the Krylov step of Sec. 3.2.1 with the preconditioner of
// gq_mg.cuh), restructured so that every multigrid level the whole grid of blocks works
// on costs two passes and two grid barriers per cycle instead of four.
//
// A pass walks the level in tiles of kTX x kTY cells.  Each block stages a tile's inputs
// with a halo (kHX = 4 cells in x, one 16-byte chunk; kHY = 2 rows in y) into shared
// memory by TMA tensor copies (cp.async.bulk.tensor, one per array, completing on an
// mbarrier; boxes outside the grid read zeros; double-buffered so that the next tile's
// loads overlap this tile's arithmetic), and computes what needs neighbours from
// the staged copy, redundantly on the halo:
//   down pass (level l):  x_a = omega (2 r - omega A r) on the tile and a one-cell ring,
//                         then the residual r - A x_a on the tile, restricted to level
//                         l + 1 (2 x 2 aggregates, transfer weights t);
//   up pass (level l):    x~ = x_a + over t x_{l+1}(parent) on the tile and two rings,
//                         x_b = x~ + omega (r - A x~) on the tile and one ring,
//                         out = x_b + omega (r - A x_b) on the tile;
//   level 0 down pass:    fused with the Krylov update r' = r - alpha q, d += alpha p
//                         (r' formed on the staged region from r and q), with r'.r';
//   level 0 up pass:      out = z, with the partial sums r.z and r.z_old.
// These are the same operations, in the same order, as the cycle of gq_mg.cuh (two
// weighted-Jacobi sweeps from zero fused into one, residual and restriction,
// prolongation with the factor `over` and one sweep, a final sweep); only the pass
// boundaries move.  The levels of at most block_cells cells run in the team's first
// block as before, and the direction pass (p = z + beta p_old, q = A p, p.q), the FP64
// refinement and the stop tests are those of k_pcg.
//
// Used for the mixed path with the aggregation preconditioner when every level the
// whole grid works on has a width divisible by 8 and an even height (16-byte staging
// chunks on the level and on its parent); other problems use k_pcg.
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "gq_pcg.cuh"

namespace gq {
namespace {

constexpr int kTiledThreads = 512;     // threads of a block (1024 measured slower: 64 registers, spills, costlier barriers)
constexpr int kTX = 64, kTY = 32;      // tile of a level (cells); levels below kTallCells use kTY / 2
constexpr int kHX = 4, kHY = 2;        // staged halo: x one 16-byte chunk, y two rows
constexpr int kRW = kTX + 2 * kHX;     // staged region width (72)
constexpr int kRH = kTY + 2 * kHY;     // staged region height (36)
constexpr int kNR = kRW * kRH;
constexpr int kCW = kTX / 2 + 8;       // staged coarse region (40 x 20)
constexpr int kCH = kTY / 2 + 4;
constexpr int kNC = kCW * kCH;
constexpr int kNT = kTX * kTY;         // cells of a tile
constexpr int kRG = kRW / 4;           // groups of 4 cells in a staged region row (18)
constexpr int kTG = kTX / 4;           // groups of 4 cells in a tile row (16)
constexpr int kStaged = 5;             // staged arrays with a halo
constexpr int kOwn = 2;                // staged arrays of the tile alone
constexpr int kNst = 2;                // staging buffers: the tile computed and kNst - 1 tiles ahead
constexpr int kTallCells = 1 << 18;    // levels of at least this many cells use kTY-high tiles

// height of a level's tiles (host and device agree on it): tall tiles halve the halo and
// the per-tile overhead on the large levels, short ones give the small levels more blocks
__host__ __device__ __forceinline__ int tile_h(int cells) { return cells >= kTallCells ? kTY : kTY / 2; }

// tile geometry of tile height TY (the shared-memory buffers are sized for kTY)
template <int TY>
struct Geo {
    static constexpr int RH = TY + 2 * kHY;
    static constexpr int NR = kRW * RH;
    static constexpr int NT = kTX * TY;
    static constexpr int CH = TY / 2 + 4;
    static constexpr int NC = kCW * CH;
    static constexpr unsigned HaloBytes = NR * 4, CoarseBytes = NC * 4, OwnBytes = NT * 4;
};

constexpr int kBlkCap = 1536;          // cells of the block levels kept in shared memory

// The levels one block runs (at most block_cells cells each, coarsened to the dense
// coarsest one): their couplings, transfer weights and coarsest inverse stay in shared
// memory for the whole solve, so that each of their passes costs a block barrier and no
// global-memory round trip.
struct BlockLevels {
    float cw[kBlkCap], cs[kBlkCap], t[kBlkCap];
    float inv[kCoarseMax * kCoarseMax];
};

struct TileSmem {
    float in[kNst][kStaged][kNR];      // staged inputs with a halo (block levels: their vectors)
    float co[kNst][kNC];               // staged coarse values (up passes)
    float own[kNst][kOwn][kNT];        // staged inputs of the tile alone
    float c1[kNR];                     // computed: x_a (down) or x~ (up)
    float c2[kNR];                     // computed: x_b (up)
    BlockLevels blk;
};
static_assert(3 * kBlkCap <= kNst * kStaged * kNR, "block-level vectors must fit the staging buffers");

// ---- TMA staging ---------------------------------------------------------------------
// Every staged array of a level has a tensor map (2-D, FP32, the level's nx x ny with a
// row stride of 4 nx bytes) whose box is the region a tile needs: kRW x kRH with a halo,
// kCW x kCH over the parent level, or kTX x kTY for the tile alone.  Box origins are
// multiples of 4 cells in x (16 bytes), as the tensor copy requires; rows and columns
// outside the grid are filled with zeros.  One thread issues a tile's copies after
// announcing their bytes on the stage's mbarrier; every thread waits on the barrier's
// phase, with a bounded number of polls.
constexpr int kMaxTiledLevels = 12;
constexpr int kMapsPerLevel = 8;
enum { kMapR0 = 0, kMapR1, kMapCW, kMapCS, kMapT, kMapXA, kMapXC, kMapQ };
constexpr int kOwnBase = kMaxTiledLevels * kMapsPerLevel;
enum { kOwnP0 = 0, kOwnP1, kOwnD, kOwnZ, kOwnZold, kOwnCount };
constexpr int kNumMaps = kOwnBase + kOwnCount;

struct TiledMaps {
    CUtensorMap m[kNumMaps];
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma2d(void* dst, const CUtensorMap* map, int x, int y, unsigned long long* b) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(b))
        : "memory");
}
// Proxy fences of the issuing thread.  The full one orders the generic stores of earlier passes
// (other blocks' stores acquired at the grid barrier before this pass, this block's generic
// use of the staging buffers) before this pass's tensor copies: once per pass, because no
// pass reads by tensor copy what the same pass stores.  The shared-memory one orders the
// block's generic reads of a staging buffer before the copies that refill it: once per tile.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// The mbarriers of the staging buffers and the phase each is in (identical in every thread).
struct TilePipe {
    unsigned long long* bar;   // [kNst] in shared memory
    unsigned phase;            // bit k: parity of the phase buffer k completes next
    long long spin;            // poll limit of a wait
};

// The tile passes work on groups of 4 cells of a region row (region index a multiple of
// 4, so every staged and computed array is read and written as float4): a group's
// stencil takes 6 vector and 3 scalar shared-memory loads instead of 36 scalar ones.
__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void sts4(float* p, const float4& v) { *reinterpret_cast<float4*>(p) = v; }

// (A v) on the 4 cells at region index i (i % 4 == 0, a row with rows above and below in
// the region): unit diagonal and couplings staged like v, per cell k
//   v_k - cW_k v_{k-1} - cW_{k+1} v_{k+1} - cS_k v_{k-kRW} - cS_{k+kRW} v_{k+kRW}
__device__ __forceinline__ float4 st5x4(const float* v, const float* cw, const float* cs, int i) {
    const float4 c = lds4(v + i), s = lds4(v + i - kRW), n = lds4(v + i + kRW);
    const float w = v[i - 1], e = v[i + 4];
    const float4 a = lds4(cw + i), b = lds4(cs + i), bn = lds4(cs + i + kRW);
    const float ae = cw[i + 4];
    float4 r;
    r.x = c.x - a.x * w - a.y * c.y - b.x * s.x - bn.x * n.x;
    r.y = c.y - a.y * c.x - a.z * c.z - b.y * s.y - bn.y * n.y;
    r.z = c.z - a.z * c.y - a.w * c.w - b.z * s.z - bn.z * n.z;
    r.w = c.w - a.w * c.z - ae * e - b.w * s.w - bn.w * n.w;
    return r;
}

__device__ __forceinline__ float4 axpy4(const float4& x, float a, const float4& y) {   // x + a y
    return make_float4(x.x + a * y.x, x.y + a * y.y, x.z + a * y.z, x.w + a * y.w);
}
__device__ __forceinline__ float4 sub4(const float4& x, const float4& y) {
    return make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
}
__device__ __forceinline__ float dot4(const float4& x, const float4& y) {
    return x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w;
}

struct TLevel {
    int nx, ny;                // cells (nx % 8 == 0, ny even)
    int mr, mcw, mcs, mt, mxa, mxc;   // tensor maps of r, cW, cS, t, x_a and the parent's result
    const float* cW;
    const float* cS;
    const float* t;            // transfer weight to the parent
    const float* r;            // right-hand side (level 0: the Krylov residual)
    float* xa;                 // pre-smoothed values (kept for the up pass)
    float* out;                // result of the level (level 0: z)
    float* rc;                 // the parent's right-hand side (restriction target)
    const float* xc;           // the parent's result (prolongation source)
    int cnx, cny;              // parent dimensions
};

template <int TY>
__device__ __forceinline__ int ntiles(const TLevel& L) { return ((L.nx + kTX - 1) / kTX) * ((L.ny + TY - 1) / TY); }

template <int TY>
__device__ __forceinline__ void tile_origin(const TLevel& L, int t, int& x0, int& y0) {
    const int tx = (L.nx + kTX - 1) / kTX;
    const int ty = t / tx;
    x0 = (t - ty * tx) * kTX;
    y0 = ty * TY;
}

// The tiles b, b + G, b + 2G, ... of a pass, each staged kNst - 1 tiles ahead of its
// arithmetic: issue(t, buf) (thread 0) starts tile t's copies into buffer buf,
// compute(t, buf) works on it.  Returns false when a wait ran out of polls (the pass's
// copies still in flight are then waited for, again with a bound).
template <class Issue, class Compute>
__device__ __forceinline__ bool tile_loop(int nt, int b, int G, TilePipe& pp, Issue issue, Compute compute) {
    if (threadIdx.x == 0) {
        fence_proxy_async();
#pragma unroll
        for (int k = 0; k < kNst - 1; k++) {
            const int t = b + k * G;
            if (t < nt) issue(t, k);
        }
    }
    int i = 0;
    for (int t = b; t < nt; t += G, i++) {
        const int buf = i % kNst;
        const int tn = t + (kNst - 1) * G;
        if (threadIdx.x == 0 && tn < nt) issue(tn, (i + kNst - 1) % kNst);
        const unsigned par = (pp.phase >> buf) & 1u;
        bool done = mbar_try(&pp.bar[buf], par);
        for (long long n = 0; !done && n < pp.spin; n++) done = mbar_try(&pp.bar[buf], par);
        pp.phase ^= 1u << buf;
        if (__syncthreads_or(!done)) {
            // drain: the tiles issued after this one (bounded waits)
            for (int j = 1; j < kNst; j++) {
                if (t + j * G >= nt) break;
                const int bj = (i + j) % kNst;
                const unsigned pj = (pp.phase >> bj) & 1u;
                bool dj = mbar_try(&pp.bar[bj], pj);
                for (long long n = 0; !dj && n < pp.spin; n++) dj = mbar_try(&pp.bar[bj], pj);
                pp.phase ^= 1u << bj;
            }
            return false;
        }
        compute(t, buf);
        __syncthreads();
    }
    return true;
}

// Kernel-wide arguments of the fused level-0 down pass: the Krylov update.
struct UpdateArgs {
    bool on;                   // false: plain down pass on r
    float alpha;
    int mq, mp, md;            // tensor maps of q, p and d
    const float* q;            // q = A p
    const float* p;            // the direction
    float* d;                  // correction (updated in place)
    float* rnew;               // r' (written for the tile)
};

// Down pass of one level over all of its tiles this block owns (tiles b, b + G, ...).
// Staged with a halo: 0 r (or r_old), 1 q (update only), 2 cW, 3 cS, 4 t; the tile
// alone: 0 p, 1 d (update only).
template <int TY>
__device__ bool down_pass(const TLevel& L, float om, const UpdateArgs& U, TileSmem& S, const TiledMaps& M, TilePipe& pp,
                          int b, int G, double* rr) {
    // this thread's r'.r' over its cells of the pass, in FP32 (a few dozen terms; FP64
    // arithmetic per cell would cost more than the pass's memory traffic on this part)
    float rrf = 0.f;
    using Gm = Geo<TY>;
    const unsigned bytes = 4 * Gm::HaloBytes + (U.on ? Gm::HaloBytes + 2 * Gm::OwnBytes : 0u);
    auto issue = [&](int t, int buf) {
        int x0, y0;
        tile_origin<TY>(L, t, x0, y0);
        const int X0 = x0 - kHX, Y0 = y0 - kHY;
        unsigned long long* bar = &pp.bar[buf];
        fence_proxy_async_smem();
        mbar_expect(bar, bytes);
        tma2d(S.in[buf][0], &M.m[L.mr], X0, Y0, bar);
        tma2d(S.in[buf][2], &M.m[L.mcw], X0, Y0, bar);
        tma2d(S.in[buf][3], &M.m[L.mcs], X0, Y0, bar);
        tma2d(S.in[buf][4], &M.m[L.mt], X0, Y0, bar);
        if (U.on) {
            tma2d(S.in[buf][1], &M.m[U.mq], X0, Y0, bar);
            tma2d(S.own[buf][0], &M.m[U.mp], x0, y0, bar);
            tma2d(S.own[buf][1], &M.m[U.md], x0, y0, bar);
        }
    };
    auto compute = [&](int t, int buf) {
        int x0, y0;
        tile_origin<TY>(L, t, x0, y0);
        float* R = S.in[buf][0];
        const float* Q = S.in[buf][1];
        const float* CW = S.in[buf][2];
        const float* CS = S.in[buf][3];
        const float* T = S.in[buf][4];
        float* XA = S.c1;
        if (U.on) {
            // r' = r - alpha q on the whole staged region (zeros stay zeros)
#pragma unroll
            for (int e = threadIdx.x; e < Gm::NR / 4; e += kTiledThreads)
                sts4(R + 4 * e, axpy4(lds4(R + 4 * e), -U.alpha, lds4(Q + 4 * e)));
            __syncthreads();
        }
        // x_a on the tile and a one-cell ring (whole region rows: the groups at the row ends
        // are formed too and never read)
#pragma unroll
        for (int e = threadIdx.x; e < (TY + 2) * kRG; e += kTiledThreads) {
            const int ly = e / kRG, g = e - ly * kRG;
            const int ix = (kHY - 1 + ly) * kRW + 4 * g;
            const float4 r = lds4(R + ix), a = st5x4(R, CW, CS, ix);
            sts4(XA + ix, make_float4(om * (2.f * r.x - om * a.x), om * (2.f * r.y - om * a.y),
                                      om * (2.f * r.z - om * a.z), om * (2.f * r.w - om * a.w)));
        }
        __syncthreads();
        // the tile, a group a thread: the residual restricted to the parent (the two rows of
        // an aggregate are lanes l and l + 16 of one warp), x_a and, fused with the update,
        // r', d and r'.r'
        if (threadIdx.x < TY * kTG) {
            const int ly = threadIdx.x / kTG, g = threadIdx.x - ly * kTG;
            const int ix = (kHY + ly) * kRW + kHX + 4 * g;
            const float4 r = lds4(R + ix), tw = lds4(T + ix), res = sub4(r, st5x4(XA, CW, CS, ix));
            float c0 = tw.x * res.x + tw.y * res.y, c1 = tw.z * res.z + tw.w * res.w;
            c0 += __shfl_down_sync(0xffffffffu, c0, kTG);
            c1 += __shfl_down_sync(0xffffffffu, c1, kTG);
            const int gx = x0 + 4 * g, gy = y0 + ly;
            if ((ly & 1) == 0) {
                const int gi = gx / 2, gj = gy / 2;
                if (gi < L.cnx && gj < L.cny)
                    *reinterpret_cast<float2*>(L.rc + (size_t)gj * L.cnx + gi) = make_float2(c0, c1);
            }
            if (gx < L.nx && gy < L.ny) {
                const size_t gg = (size_t)gy * L.nx + gx;
                sts4(L.xa + gg, lds4(XA + ix));
                if (U.on) {
                    const int o = ly * kTX + 4 * g;
                    sts4(U.rnew + gg, r);
                    sts4(U.d + gg, axpy4(lds4(S.own[buf][1] + o), U.alpha, lds4(S.own[buf][0] + o)));
                    rrf += dot4(r, r);
                }
            }
        }
    };
    const bool ok = tile_loop(ntiles<TY>(L), b, G, pp, issue, compute);
    *rr += static_cast<double>(rrf);
    return ok;
}

// Up pass of one level.  Staged with a halo: 0 x_a, 1 t, 2 cW, 3 cS, 4 r; coarse: the
// parent's result; the tile alone: 0 z_old (level 0).  Level 0 (zold != null): out is z,
// with the partial sums r.z and r.z_old.
template <int TY>
__device__ bool up_pass(const TLevel& L, float om, float over, TileSmem& S, const TiledMaps& M, TilePipe& pp, int b,
                        int G, int mzold, double* rz, double* rzo) {
    float rzf = 0.f, rzof = 0.f;       // this thread's partial sums (FP32, see down_pass)
    const bool lvl0 = mzold >= 0;
    using Gm = Geo<TY>;
    const unsigned bytes = 5 * Gm::HaloBytes + Gm::CoarseBytes + (lvl0 ? Gm::OwnBytes : 0u);
    auto issue = [&](int t, int buf) {
        int x0, y0;
        tile_origin<TY>(L, t, x0, y0);
        const int X0 = x0 - kHX, Y0 = y0 - kHY;
        unsigned long long* bar = &pp.bar[buf];
        fence_proxy_async_smem();
        mbar_expect(bar, bytes);
        tma2d(S.in[buf][0], &M.m[L.mxa], X0, Y0, bar);
        tma2d(S.in[buf][1], &M.m[L.mt], X0, Y0, bar);
        tma2d(S.in[buf][2], &M.m[L.mcw], X0, Y0, bar);
        tma2d(S.in[buf][3], &M.m[L.mcs], X0, Y0, bar);
        tma2d(S.in[buf][4], &M.m[L.mr], X0, Y0, bar);
        tma2d(S.co[buf], &M.m[L.mxc], x0 / 2 - 4, y0 / 2 - 2, bar);
        if (lvl0) tma2d(S.own[buf][0], &M.m[mzold], x0, y0, bar);
    };
    auto compute = [&](int t, int buf) {
        int x0, y0;
        tile_origin<TY>(L, t, x0, y0);
        const float* XA = S.in[buf][0];
        const float* T = S.in[buf][1];
        const float* CW = S.in[buf][2];
        const float* CS = S.in[buf][3];
        const float* R = S.in[buf][4];
        const float* C = S.co[buf];
        float* XT = S.c1;
        float* XB = S.c2;
        // x~ on the whole region (the tile and two rings are read); the parent of region
        // cell (lx, ly) is coarse region cell ((lx - kHX) / 2 + 4, (ly - kHY) / 2 + 2), floor
        // division: cells 4g, 4g + 1 of a row have parent column 2g + 2, cells 4g + 2, 4g + 3
        // parent column 2g + 3
#pragma unroll
        for (int e = threadIdx.x; e < Gm::RH * kRG; e += kTiledThreads) {
            const int ly = e / kRG, g = e - ly * kRG;
            const int ix = ly * kRW + 4 * g;
            const float2 c = *reinterpret_cast<const float2*>(C + (((ly - kHY) >> 1) + 2) * kCW + 2 * g + 2);
            const float4 xa = lds4(XA + ix), tw = lds4(T + ix);
            sts4(XT + ix, make_float4(xa.x + over * tw.x * c.x, xa.y + over * tw.y * c.x, xa.z + over * tw.z * c.y,
                                      xa.w + over * tw.w * c.y));
        }
        __syncthreads();
        // x_b on the tile and one ring (whole region rows)
#pragma unroll
        for (int e = threadIdx.x; e < (TY + 2) * kRG; e += kTiledThreads) {
            const int ly = e / kRG, g = e - ly * kRG;
            const int ix = (kHY - 1 + ly) * kRW + 4 * g;
            const float4 r = lds4(R + ix), x = lds4(XT + ix), a = st5x4(XT, CW, CS, ix);
            sts4(XB + ix, make_float4(x.x + om * (r.x - a.x), x.y + om * (r.y - a.y), x.z + om * (r.z - a.z),
                                      x.w + om * (r.w - a.w)));
        }
        __syncthreads();
        // the level's result on the tile, a group a thread
        if (threadIdx.x < TY * kTG) {
            const int ly = threadIdx.x / kTG, g = threadIdx.x - ly * kTG;
            const int ix = (kHY + ly) * kRW + kHX + 4 * g;
            const float4 r = lds4(R + ix), x = lds4(XB + ix), a = st5x4(XB, CW, CS, ix);
            const float4 o = make_float4(x.x + om * (r.x - a.x), x.y + om * (r.y - a.y), x.z + om * (r.z - a.z),
                                         x.w + om * (r.w - a.w));
            const int gx = x0 + 4 * g, gy = y0 + ly;
            if (gx < L.nx && gy < L.ny) {
                sts4(L.out + (size_t)gy * L.nx + gx, o);
                if (lvl0) {
                    rzf += dot4(r, o);
                    rzof += dot4(r, lds4(S.own[buf][0] + ly * kTX + 4 * g));
                }
            }
        }
    };
    const bool ok = tile_loop(ntiles<TY>(L), b, G, pp, issue, compute);
    if (lvl0) {
        *rz += static_cast<double>(rzf);
        *rzo += static_cast<double>(rzof);
    }
    return ok;
}

// the tile height a level uses (see tile_h)
__device__ __forceinline__ bool down_any(const TLevel& L, float om, const UpdateArgs& U, TileSmem& S,
                                         const TiledMaps& M, TilePipe& pp, int b, int G, double* rr) {
    return tile_h(L.nx * L.ny) == kTY ? down_pass<kTY>(L, om, U, S, M, pp, b, G, rr)
                                      : down_pass<kTY / 2>(L, om, U, S, M, pp, b, G, rr);
}
__device__ __forceinline__ bool up_any(const TLevel& L, float om, float over, TileSmem& S, const TiledMaps& M,
                                       TilePipe& pp, int b, int G, int mzold, double* rz, double* rzo) {
    return tile_h(L.nx * L.ny) == kTY ? up_pass<kTY>(L, om, over, S, M, pp, b, G, mzold, rz, rzo)
                                      : up_pass<kTY / 2>(L, om, over, S, M, pp, b, G, mzold, rz, rzo);
}

}  // namespace
}  // namespace gq

namespace gq {
namespace {

// The solve of k_pcg<true> with the aggregation V-cycle (gq_pcg.cuh, pcg_solve_w), its
// team levels run by the tiled passes above.  Returns false when a wait timed out.
__device__ bool tiled_solve(const SolveParams& P, const Workspace& w, RedShared& sh, MGShared& msh, TileSmem& S,
                            const TiledMaps& TM, TilePipe& pp) {
    const Team team{static_cast<int>(blockIdx.x), static_cast<int>(gridDim.x)};
    const int N = P.N, nx = P.nx;
    const int nchunk = N / 4;
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
    const float* cW = w.cW32;
    const float* cS = w.cS32;
    float* pb[2] = {w.p32[0], w.p32[1]};
    float* q = w.q32;
    float* d = w.d32;
    float* rbuf[2] = {w.r32, w.r32b};
    int rsel = 0;
    float* zc = w.mg.z;
    int zsel = 0;                        // 0: zc is mg.z and zo mg.zold; 1: swapped
    float* zo = w.mg.zold;
    const MGHierarchy& mg = w.mg;

    const int flags = __ldcg(&ctl->input_flags);
    if (flags) {
        if (tid == 0) ctl->status = (flags & 2) ? kErrNonfinite : kErrInvalid;
        return true;
    }
    if (tid == 0) ctl->t_start = global_ns();
    cyc_reset(msh.amg);
    if (!mg_build(w, team, tid, stride, P.spin_limit, abort_flag, msh)) {
        if (threadIdx.x == 0) atomicExch(&ctl->status, kErrTimeout);
        return false;
    }
    if (tid == 0) {
        ctl->t_built = global_ns();
        ctl->levels = mg.nlev;
    }
    const int nl = mg.nlev;
    int lg = 0;                          // levels [0, lg) run on the whole team (lg >= 1 here)
    while (lg < nl - 1 && mg.L[lg].N > P.block_cells) lg++;
    const float om = P.mg_omega, over = P.mg_over;
    auto tlevel = [&](int l) {
        const MGLevel& M = mg.L[l];
        const MGLevel& C = mg.L[l + 1];
        TLevel t;
        t.nx = M.nx;
        t.ny = M.ny;
        const int base = l * kMapsPerLevel;
        t.mr = base + (l == 0 ? kMapR0 + rsel : kMapR0);
        t.mcw = base + kMapCW;
        t.mcs = base + kMapCS;
        t.mt = base + kMapT;
        t.mxa = base + kMapXA;
        t.mxc = base + kMapXC;
        t.cW = M.cW;
        t.cS = M.cS;
        t.t = M.t;
        t.r = l == 0 ? rbuf[rsel] : M.r;
        t.xa = M.xa;
        t.out = l == 0 ? zc : M.xb;
        t.rc = C.r;
        t.xc = l + 1 == lg ? C.xa : C.xb;
        t.cnx = C.nx;
        t.cny = C.ny;
        return t;
    };
    auto bar = [&]() { return team_barrier(w.bar, team, P.spin_limit, abort_flag); };
    // block levels held in shared memory when they fit (first cell of each level there)
    int blk_off[kAmgMaxLevels];
    int blk_total = 0;
    for (int l = lg; l < nl && l - lg < kAmgMaxLevels; l++) {
        blk_off[l - lg] = blk_total;
        blk_total += mg.L[l].N;
    }
    const bool blk_smem = blk_total <= kBlkCap && mg.L[nl - 1].N <= kCoarseMax;
    if (blk_smem && team.rank == 0) {
        for (int l = lg; l < nl; l++) {
            const MGLevel& M = mg.L[l];
            const int o = blk_off[l - lg];
            for (int k = threadIdx.x; k < M.N; k += blockDim.x) {
                S.blk.cw[o + k] = __ldcg(M.cW + k);
                S.blk.cs[o + k] = __ldcg(M.cS + k);
                S.blk.t[o + k] = l + 1 < nl ? __ldcg(M.t + k) : 0.f;
            }
        }
        const int nc = mg.L[nl - 1].N;
        for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) S.blk.inv[e] = __ldcg(mg.inv + e);
        __syncthreads();
    }
    const UpdateArgs no_update{false, 0.f, 0, 0, 0, nullptr, nullptr, nullptr, nullptr};

    // V-cycle z = B r: down passes (level 0's may be done, fused with the update), the
    // block levels, up passes; rz, rzo receive this thread's r.z and r.z_old
    auto vcycle = [&](bool pre0_done, double* rz, double* rzo) -> bool {
        for (int l = pre0_done ? 1 : 0; l < lg; l++) {
            cyc_mark(msh.amg, team, l);
            double unused = 0.0;
            if (!down_any(tlevel(l), om, no_update, S, TM, pp, team.rank, team.size, &unused)) return false;
            if (!bar()) return false;
        }
        if (team.rank == 0 && blk_smem) {
            // the block levels in shared memory: right-hand side of level lg from the team,
            // the cycle below it, the result of level lg back to global memory
            cyc_mark(msh.amg, team, lg);
            const Range br{static_cast<int>(threadIdx.x), static_cast<int>(blockDim.x)};
            float* vr = &S.in[0][0][0];
            float* vxa = vr + kBlkCap;
            float* vxb = vxa + kBlkCap;
            for (int k = threadIdx.x; k < mg.L[lg].N; k += blockDim.x) vr[k] = __ldcg(mg.L[lg].r + k);
            __syncthreads();
            auto view = [&](int l) {
                const int o = blk_off[l - lg];
                Lv v;
                v.nx = mg.L[l].nx;
                v.ny = mg.L[l].ny;
                v.N = mg.L[l].N;
                v.cW = S.blk.cw + o;
                v.cS = S.blk.cs + o;
                v.t = S.blk.t + o;
                v.r = vr + o;
                v.xa = vxa + o;
                v.xb = vxb + o;
                v.out = vxa + o;
                return v;
            };
            for (int l = lg; l + 1 < nl; l++) {
                const Lv F = view(l), C = view(l + 1);
                cyc_presmooth<false>(F, om, br, false);
                __syncthreads();
                cyc_restrict<false>(F, C, br);
                __syncthreads();
            }
            cyc_coarse(view(nl - 1), S.blk.inv, br, false, nullptr, nullptr, nullptr);
            __syncthreads();
            for (int l = nl - 2; l >= lg; l--) {
                const Lv F = view(l), C = view(l + 1);
                cyc_prolong_smooth<false>(F, C, om, over, br);
                __syncthreads();
                cyc_postsmooth<false>(F, om, br, nullptr, nullptr, nullptr);
                __syncthreads();
            }
            for (int k = threadIdx.x; k < mg.L[lg].N; k += blockDim.x) mg.L[lg].xa[k] = vxa[k];
        } else if (team.rank == 0) {
            cyc_mark(msh.amg, team, lg);
            const Range br{static_cast<int>(threadIdx.x), static_cast<int>(blockDim.x)};
            const float* r0 = rbuf[rsel];
            for (int l = lg; l + 1 < nl; l++) {
                const Lv F = level_view(mg, l, r0, zc), C = level_view(mg, l + 1, r0, zc);
                cyc_presmooth<false>(F, om, br, l == lg);
                __syncthreads();
                if (l == lg) cyc_restrict<true>(F, C, br);
                else cyc_restrict<false>(F, C, br);
                __syncthreads();
            }
            const Lv Z = level_view(mg, nl - 1, r0, zc);
            cyc_coarse(Z, mg.inv, br, lg == nl - 1, zo, nullptr, nullptr);
            __syncthreads();
            for (int l = nl - 2; l >= lg; l--) {
                const Lv F = level_view(mg, l, r0, zc), C = level_view(mg, l + 1, r0, zc);
                if (l == lg) {
                    cyc_prolong_smooth<true>(F, C, om, over, br);
                    __syncthreads();
                    cyc_postsmooth<true>(F, om, br, zo, nullptr, nullptr);
                } else {
                    cyc_prolong_smooth<false>(F, C, om, over, br);
                    __syncthreads();
                    cyc_postsmooth<false>(F, om, br, zo, nullptr, nullptr);
                }
                __syncthreads();
            }
        }
        if (!bar()) return false;
        for (int l = lg - 1; l >= 1; l--) {
            cyc_mark(msh.amg, team, l);
            if (!up_any(tlevel(l), om, over, S, TM, pp, team.rank, team.size, -1, nullptr, nullptr)) return false;
            if (!bar()) return false;
        }
        cyc_mark(msh.amg, team, 0);
        if (!up_any(tlevel(0), om, over, S, TM, pp, team.rank, team.size, kOwnBase + (zsel ? kOwnZ : kOwnZold), rz,
                     rzo))
            return false;
        cyc_mark(msh.amg, team, kAmgMaxLevels - 1);
        return true;
    };

    // FP64 residual r64 = b^ - A^ y and its norms: |r|^2, |r/s|^2, |b/s|^2, max |r_k/y_k|, max |r_k|
    double tr[5];
    auto true_residual = [&](bool first) -> bool {
#pragma unroll
        for (int t = 0; t < 5; t++) tr[t] = 0.0;
        for (int c = tid; c < N / 2; c += stride) {
            const int k = c * 2;
            const bool hs = k >= nx, hn = k + nx < N, hw = k > 0, he = k + 2 < N;
            double yc[2], ys[2] = {0.0, 0.0}, yn[2] = {0.0, 0.0}, cw[2], cs[2], csn[2] = {0.0, 0.0}, bk[2], sk[2];
            double yw = 0.0, ye = 0.0, cwe = 0.0;
            ld64<2>(y + k, yc);
            ld64<2>(cW64 + k, cw);
            ld64<2>(cS64 + k, cs);
            ld64<2>(bh + k, bk);
            ld64<2>(s + k, sk);
            if (hw) yw = __ldcg(y + k - 1);
            if (he) {
                ye = __ldcg(y + k + 2);
                cwe = cW64[k + 2];
            }
            if (hs) ld64<2>(y + k - nx, ys);
            if (hn) {
                ld64<2>(y + k + nx, yn);
                ld64<2>(cS64 + k + nx, csn);
            }
            double rk[2];
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const double left = i == 0 ? yw : yc[0];
                const double right = i == 1 ? ye : yc[1];
                const double cright = i == 1 ? cwe : cw[1];
                const double ax = yc[i] - cw[i] * left - cright * right - cs[i] * ys[i] - csn[i] * yn[i];
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
            st64<2>(r64 + k, rk);
        }
        return allreduce<3, 2>(tr, w.partials, parity, w.bar, P.spin_limit, abort_flag, sh, team);
    };

    int it = 0, nref = 0, status = kErrNotConverged;
    double crit = 0.0, l2 = 0.0, bb = 1.0;
    bool timed_out = false;
    if (!true_residual(true)) {
        timed_out = true;
        goto done;
    }
    bb = tr[2];
    crit = tr[3];
    l2 = sqrt(tr[1] / bb);
    if (!isfinite(tr[0]) || !isfinite(bb) || !(crit == crit)) {
        status = kErrNonfinite;
        goto done;
    }
    if (crit <= P.rtol) {
        status = kOk;
        goto done;
    }
    {
        const double zs = exp2(-(double)ilogb(tr[4] > 0.0 ? tr[4] : 1.0));
        const double scale = zs;
        double rr = tr[0] * scale * scale;
        double rr_ref = rr;
        double beta = 0.0;
        bool use_p = false;
        int cur = 0;
        double best = crit;
        int it_best = 0, stall = 0;
        bool first = true, pre0_done = false;
        double rz_prev = 1.0;
        // FP32 residual from the FP64 one (scaled), correction d = 0
        auto refresh = [&](bool initial) -> bool {
            float* r0 = rbuf[rsel];
            for (int c = tid; c < nchunk; c += stride) {
                const int k = c * 4;
                double t[4];
                float f[4], zero[4];
                ld64<4>(r64 + k, t);
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    f[i] = static_cast<float>(t[i] * zs);
                    zero[i] = 0.f;
                }
                stf<4>(r0 + k, f);
                stf<4>(d + k, zero);
                if (initial) stf<4>(zo + k, zero);
            }
            return bar();
        };
        if (!refresh(true)) {
            timed_out = true;
            goto done;
        }
        auto refine = [&]() -> bool {
            const double inv = 1.0 / scale;
            for (int c = tid; c < nchunk; c += stride) {
                const int k = c * 4;
                double yk[4];
                float dk[4], zero[4];
                ld64<4>(y + k, yk);
                ldf<4>(d + k, dk);
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    yk[i] += static_cast<double>(dk[i]) * inv;
                    zero[i] = 0.f;
                }
                st64<4>(y + k, yk);
                stf<4>(d + k, zero);
            }
            if (!bar()) {
                timed_out = true;
                return false;
            }
            // the FP64 residual b^ - A^ y, written straight to the FP32 Krylov residual
            // (times the fixed scale zs), with its FP32 square sum and the cell-wise
            // criterion: the only FP64 arithmetic per cell is the stencil and two
            // scalings (this part's FP64 rate is a sixtieth of FP32).  The criterion's
            // quotient |r_k / y_k| is taken in FP32 from the scaled r_k zs and y_k zs
            // where both lie well inside the FP32 range (to about two FP32 ulps, as
            // abs_ratio_approx), otherwise (tiny or huge y_k, zero, inf, NaN) from the
            // FP64 values by abs_ratio_approx.
            {
                float rrf = 0.f, crf = 0.f;
                double cr[2] = {0.0, 0.0};
                float* r0 = rbuf[rsel];
                for (int c = tid; c < N / 2; c += stride) {
                    const int k = c * 2;
                    const bool hs = k >= nx, hn = k + nx < N, hw = k > 0, he = k + 2 < N;
                    double yc[2], ys[2] = {0.0, 0.0}, yn[2] = {0.0, 0.0}, cw[2], cs[2], csn[2] = {0.0, 0.0}, bk[2];
                    double yw = 0.0, ye = 0.0, cwe = 0.0;
                    ld64<2>(y + k, yc);
                    ld64<2>(cW64 + k, cw);
                    ld64<2>(cS64 + k, cs);
                    ld64<2>(bh + k, bk);
                    if (hw) yw = __ldcg(y + k - 1);
                    if (he) {
                        ye = __ldcg(y + k + 2);
                        cwe = cW64[k + 2];
                    }
                    if (hs) ld64<2>(y + k - nx, ys);
                    if (hn) {
                        ld64<2>(y + k + nx, yn);
                        ld64<2>(cS64 + k + nx, csn);
                    }
                    float f[2];
#pragma unroll
                    for (int i = 0; i < 2; i++) {
                        const double left = i == 0 ? yw : yc[0];
                        const double right = i == 1 ? ye : yc[1];
                        const double cright = i == 1 ? cwe : cw[1];
                        const double rk = bk[i] - (yc[i] - cw[i] * left - cright * right - cs[i] * ys[i] - csn[i] * yn[i]);
                        f[i] = static_cast<float>(rk * zs);
                        rrf += f[i] * f[i];
                        const float fr = fabsf(f[i]), fy = fabsf(static_cast<float>(yc[i] * zs));
                        const float qk = (fy >= 1e-8f && fy <= 1e30f && fr <= 1e30f)
                                             ? __fdividef(fr, fy)
                                             : static_cast<float>(abs_ratio_approx(rk, yc[i]));
                        crf = (crf != crf || qk != qk) ? qk + crf : fmaxf(crf, qk);
                    }
                    stf<2>(r0 + k, f);
                }
                cr[0] = static_cast<double>(rrf);
                cr[1] = static_cast<double>(crf);
                if (!allreduce<1, 1>(cr, w.partials, parity, w.bar, P.spin_limit, abort_flag, sh, team)) {
                    timed_out = true;
                    return false;
                }
                tr[0] = cr[0] / (scale * scale);
                tr[3] = cr[1];
            }
            nref++;
            crit = tr[3];
            if (!isfinite(tr[0]) || !(crit == crit)) {
                status = kErrNonfinite;
                return false;
            }
            if (crit <= P.rtol) {
                status = kOk;
                return false;
            }
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
            const double rr_true = tr[0] * scale * scale;
            if (P.restart) {
                use_p = false;
                beta = 0.0;
                first = true;
            } else {
                use_p = true;
                beta = rr > 0.0 ? rr_true / rr : 0.0;
            }
            rr = rr_true;
            rr_ref = rr_true;
            return true;
        };

        while (true) {
            double rho_mg = 0.0;
            bool degenerate = false;
            {
                double vz[2] = {0.0, 0.0};
                if (!vcycle(pre0_done, &vz[0], &vz[1])) {
                    timed_out = true;
                    break;
                }
                pre0_done = false;
                if (!allreduce<2, 0>(vz, w.partials, parity, w.bar, P.spin_limit, abort_flag, sh, team)) {
                    timed_out = true;
                    break;
                }
                if (!isfinite(vz[0]) || !isfinite(vz[1])) {
                    status = kErrNonfinite;
                    break;
                }
                degenerate = !(vz[0] > 0.0);
                const bool restart_dir = first || fabs(vz[1]) >= 0.2 * vz[0];
                beta = restart_dir ? 0.0 : fmax(0.0, (vz[0] - vz[1]) / rz_prev);
                use_p = !restart_dir;
                rz_prev = vz[0];
                rho_mg = vz[0];
                first = false;
            }
            if (!degenerate) {
                // ---- S: p = z + beta p_old ; q = A^ p ; p.q --------------------------------
                cyc_mark(msh.amg, team, kAmgMaxLevels - 4);
                const float* __restrict__ pold = pb[cur];
                float* __restrict__ pnew = pb[cur ^ 1];
                const float rb = static_cast<float>(beta);
                double v1[1] = {0.0};
                float pqf = 0.f;      // this thread's p.q in FP32 (see down_pass)
                for (int c = tid; c < nchunk; c += stride) {
                    const int k = c * 4;
                    const bool hs = k >= nx, hn = k + nx < N, hw = k > 0, he = k + 4 < N;
                    float rc[4], rs[4] = {0.f, 0.f, 0.f, 0.f}, rn[4] = {0.f, 0.f, 0.f, 0.f}, rw = 0.f, re = 0.f;
                    float pc[4] = {0.f, 0.f, 0.f, 0.f}, ps[4] = {0.f, 0.f, 0.f, 0.f}, pn[4] = {0.f, 0.f, 0.f, 0.f};
                    float pw = 0.f, pe = 0.f;
                    ldf<4>(zc + k, rc);
                    if (hs) ldf<4>(zc + k - nx, rs);
                    if (hn) ldf<4>(zc + k + nx, rn);
                    if (hw) rw = __ldcg(zc + k - 1);
                    if (he) re = __ldcg(zc + k + 4);
                    if (use_p) {
                        ldf<4>(pold + k, pc);
                        if (hs) ldf<4>(pold + k - nx, ps);
                        if (hn) ldf<4>(pold + k + nx, pn);
                        if (hw) pw = __ldcg(pold + k - 1);
                        if (he) pe = __ldcg(pold + k + 4);
                    }
                    float cw[4], cs[4], csn[4] = {0.f, 0.f, 0.f, 0.f}, cwe = 0.f;
                    ldf<4>(cW + k, cw);
                    ldf<4>(cS + k, cs);
                    if (he) cwe = __ldcg(cW + k + 4);
                    if (hn) ldf<4>(cS + k + nx, csn);
                    float p[4], pS[4], pN[4];
                    const float pW = use_p ? rw + rb * pw : rw;
                    const float pE = use_p ? re + rb * pe : re;
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        p[i] = use_p ? rc[i] + rb * pc[i] : rc[i];
                        pS[i] = use_p ? rs[i] + rb * ps[i] : rs[i];
                        pN[i] = use_p ? rn[i] + rb * pn[i] : rn[i];
                    }
                    float qv[4];
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        const float left = i == 0 ? pW : p[i - 1];
                        const float right = i == 3 ? pE : p[i + 1];
                        const float cright = i == 3 ? cwe : cw[i + 1];
                        qv[i] = p[i] - cw[i] * left - cright * right - cs[i] * pS[i] - csn[i] * pN[i];
                        pqf += p[i] * qv[i];
                    }
                    stf<4>(pnew + k, p);
                    stf<4>(q + k, qv);
                }
                v1[0] = static_cast<double>(pqf);
                if (!allreduce<1, 0>(v1, w.partials, parity, w.bar, P.spin_limit, abort_flag, sh, team)) {
                    timed_out = true;
                    break;
                }
                const double pq = v1[0];
                if (!isfinite(pq)) {
                    status = kErrNonfinite;
                    break;
                }
                degenerate = !(pq > 0.0);
                if (!degenerate) {
                    const double alpha = rho_mg / pq;
                    float* tz = zc;          // this z becomes z_old of the next cycle
                    zc = zo;
                    zsel ^= 1;
                    zo = tz;
                    cur ^= 1;
                    // ---- U fused with the next cycle's level-0 down pass ---------------------
                    cyc_mark(msh.amg, team, kAmgMaxLevels - 3);
                    double v2[2] = {0.0, 0.0};
                    // pnew is pb[cur] now (cur was flipped above)
                    const UpdateArgs upd{true, static_cast<float>(alpha), kMapQ, kOwnBase + kOwnP0 + cur,
                                         kOwnBase + kOwnD, q, pnew, d, rbuf[rsel ^ 1]};
                    const bool okp = down_any(tlevel(0), om, upd, S, TM, pp, team.rank, team.size, &v2[0]);
                    rsel ^= 1;
                    if (!okp) {
                        timed_out = true;
                        break;
                    }
                    if (!allreduce<1, 1>(v2, w.partials, parity, w.bar, P.spin_limit, abort_flag, sh, team)) {
                        timed_out = true;
                        break;
                    }
                    it++;
                    const double rr_new = v2[0];
                    if (!isfinite(rr_new)) {
                        status = kErrNonfinite;
                        break;
                    }
                    const bool check = sqrt(rr_new) <= P.drop * sqrt(rr_ref) || it >= P.max_iter;
                    if (!check) {
                        rr = rr_new;
                        pre0_done = true;
                        continue;
                    }
                    rr = rr_new;
                }
            }
            cyc_mark(msh.amg, team, kAmgMaxLevels - 2);
            if (!refine()) break;
        }
        // the paper's 2-norm |b - A x|_2 / |b|_2 of the final iterate (reported), once
        if (!timed_out && nref > 0 && (status == kOk || status == kErrNotConverged)) {
            double v[1] = {0.0};
            for (int c = tid; c < N / 2; c += stride) {
                const int k = c * 2;
                const bool hs = k >= nx, hn = k + nx < N, hw = k > 0, he = k + 2 < N;
                double yc[2], ys[2] = {0.0, 0.0}, yn[2] = {0.0, 0.0}, cw[2], cs[2], csn[2] = {0.0, 0.0}, bk[2], sk[2];
                double yw = 0.0, ye = 0.0, cwe = 0.0;
                ld64<2>(y + k, yc);
                ld64<2>(cW64 + k, cw);
                ld64<2>(cS64 + k, cs);
                ld64<2>(bh + k, bk);
                ld64<2>(s + k, sk);
                if (hw) yw = __ldcg(y + k - 1);
                if (he) {
                    ye = __ldcg(y + k + 2);
                    cwe = cW64[k + 2];
                }
                if (hs) ld64<2>(y + k - nx, ys);
                if (hn) {
                    ld64<2>(y + k + nx, yn);
                    ld64<2>(cS64 + k + nx, csn);
                }
#pragma unroll
                for (int i = 0; i < 2; i++) {
                    const double left = i == 0 ? yw : yc[0];
                    const double right = i == 1 ? ye : yc[1];
                    const double cright = i == 1 ? cwe : cw[1];
                    const double rk = bk[i] - (yc[i] - cw[i] * left - cright * right - cs[i] * ys[i] - csn[i] * yn[i]);
                    const double ru = abs_ratio_approx(rk, sk[i]);
                    v[0] += ru * ru;
                }
            }
            if (!allreduce<1, 0>(v, w.partials, parity, w.bar, P.spin_limit, abort_flag, sh, team)) timed_out = true;
            else l2 = sqrt(v[0] / bb);
        }
    }

done:
    if (!timed_out) amg_cycle_report(w.amg, msh.amg, team);
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

__global__ void __launch_bounds__(kTiledThreads, 1) k_pcg_tiled(SolveParams P, Workspace w,
                                                                const __grid_constant__ TiledMaps TM) {
    __shared__ RedShared sh;
    __shared__ MGShared msh;
    __shared__ unsigned long long tile_bar[kNst];
    extern __shared__ __align__(128) unsigned char tile_raw[];
    // tensor copies land on 128-byte aligned buffers
    const unsigned pad = (128u - (smem_u32(tile_raw) & 127u)) & 127u;
    TileSmem& S = *reinterpret_cast<TileSmem*>(tile_raw + pad);
    if (threadIdx.x == 0) {
        for (int k = 0; k < kNst; k++) mbar_init(&tile_bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        fence_proxy_async();
    }
    __syncthreads();
    TilePipe pp{tile_bar, 0u, P.spin_limit};
    tiled_solve(P, w, sh, msh, S, TM, pp);
}

}  // namespace

size_t tiled_smem_bytes() { return sizeof(TileSmem) + 128; }

int tiled_threads() { return kTiledThreads; }

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 2-D FP32 tensor map of an nx x ny row-major array (nx % 4 == 0) with box bw x bh
bool encode(CUtensorMap* m, const float* base, int nx, int ny, int bw, int bh) {
    EncodeTiled fn = encode_fn();
    if (!fn || !base || nx % 4 != 0 || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(nx), static_cast<cuuint64_t>(ny)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(nx) * sizeof(float)};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(bw), static_cast<cuuint32_t>(bh)};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// the tensor maps of every array the tiled solve stages, laid out as the kernel indexes them
bool build_tiled_maps(const SolveParams& p, const Workspace& w, TiledMaps* M) {
    const MGHierarchy& mg = w.mg;
    int lg = 0;
    while (lg < mg.nlev - 1 && mg.L[lg].N > p.block_cells) lg++;
    if (lg < 1 || lg > kMaxTiledLevels) return false;
    std::memset(M, 0, sizeof(*M));
    bool ok = true;
    for (int l = 0; l < lg && ok; l++) {
        const MGLevel& L = mg.L[l];
        const MGLevel& C = mg.L[l + 1];
        CUtensorMap* m = M->m + l * kMapsPerLevel;
        const int ty = tile_h(L.N), kRH = ty + 2 * kHY, kCH = ty / 2 + 4;
        const float* r0 = l == 0 ? w.r32 : L.r;
        ok = ok && encode(&m[kMapR0], r0, L.nx, L.ny, kRW, kRH);
        if (l == 0) ok = ok && encode(&m[kMapR1], w.r32b, L.nx, L.ny, kRW, kRH);
        ok = ok && encode(&m[kMapCW], L.cW, L.nx, L.ny, kRW, kRH);
        ok = ok && encode(&m[kMapCS], L.cS, L.nx, L.ny, kRW, kRH);
        ok = ok && encode(&m[kMapT], L.t, L.nx, L.ny, kRW, kRH);
        ok = ok && encode(&m[kMapXA], L.xa, L.nx, L.ny, kRW, kRH);
        ok = ok && encode(&m[kMapXC], l + 1 == lg ? C.xa : C.xb, C.nx, C.ny, kCW, kCH);
        if (l == 0) ok = ok && encode(&m[kMapQ], w.q32, L.nx, L.ny, kRW, kRH);
    }
    const MGLevel& L0 = mg.L[0];
    CUtensorMap* o = M->m + kOwnBase;
    const int kTY = tile_h(L0.N);
    ok = ok && encode(&o[kOwnP0], w.p32[0], L0.nx, L0.ny, kTX, kTY);
    ok = ok && encode(&o[kOwnP1], w.p32[1], L0.nx, L0.ny, kTX, kTY);
    ok = ok && encode(&o[kOwnD], w.d32, L0.nx, L0.ny, kTX, kTY);
    ok = ok && encode(&o[kOwnZ], mg.z, L0.nx, L0.ny, kTX, kTY);
    ok = ok && encode(&o[kOwnZold], mg.zold, L0.nx, L0.ny, kTX, kTY);
    return ok;
}

cudaError_t launch_tiled(const SolveParams& p, const Workspace& w, int grid, cudaStream_t st) {
    static TiledMaps maps;     // host staging of the kernel's parameter (copied at launch)
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (!build_tiled_maps(p, w, &maps)) return cudaErrorInvalidValue;
    SolveParams pc = p;
    Workspace wc = w;
    void* args[] = {&pc, &wc, &maps};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_pcg_tiled), dim3(grid), dim3(kTiledThreads),
                                       args, tiled_smem_bytes(), st);
}

const void* solve_kernel_tiled() { return reinterpret_cast<const void*>(k_pcg_tiled); }

// the tiled kernel takes a problem whose team levels (those above block_cells cells, at
// least level 0) all have widths divisible by 8 and even heights
bool tiled_eligible(const SolveParams& p, const Workspace& w) {
    if (!p.mixed || p.precond != GQ_PRECOND_MG || w.mg.nlev < 2) return false;
    if (p.N <= p.block_cells) return false;
    int l = 0;
    for (; l < w.mg.nlev - 1 && w.mg.L[l].N > p.block_cells; l++) {
        const MGLevel& L = w.mg.L[l];
        if (L.nx % 8 != 0 || L.ny % 2 != 0) return false;
    }
    return l <= kMaxTiledLevels && encode_fn() != nullptr;
}

}  // namespace gq
