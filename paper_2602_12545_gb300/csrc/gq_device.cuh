// Device-side building blocks of the GB300 FLD step: physical constants, the flux
// limiters, warp/block reductions and a bounded inter-block barrier.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gq {

// ---------------------------------------------------------------------------
// physical constants (CGS)
// ---------------------------------------------------------------------------
constexpr double kC = 2.99792458e10;               // speed of light, cm/s
constexpr double kKB = 1.380649e-16;               // Boltzmann constant, erg/K
constexpr double kSigmaSB = 5.670374419e-5;        // Stefan-Boltzmann, erg/(cm^2 s K^4)
constexpr double kAmu = 1.66053906660e-24;         // atomic mass unit, g
constexpr double kMH = 1.00782503207 * kAmu;       // hydrogen atom mass, g
constexpr double kARad = 4.0 * kSigmaSB / kC;      // radiation constant a_R

// status codes (mirror gq_status)
enum : int {
    kOk = 0, kErrInvalid = 1, kErrCuda = 2, kErrOom = 3, kErrNotConverged = 4,
    kErrNonfinite = 5, kErrTimeout = 6, kErrBudget = 7
};

// ---------------------------------------------------------------------------
// flux limiter lambda(R) (Sec. 2): 0 Levermore-Pomraning rational form,
// 1 Minerbo (Eq. limiter, two branches meeting at R = 3/2), 2 lambda = 1/3
// ---------------------------------------------------------------------------
__device__ __forceinline__ double limiter(int kind, double R) {
    if (kind == 2) return 1.0 / 3.0;
    if (kind == 1) {
        return R <= 1.5 ? 2.0 / (3.0 + sqrt(9.0 + 12.0 * R * R))
                        : 1.0 / (1.0 + R + sqrt(1.0 + 2.0 * R));
    }
    return (2.0 + R) / (6.0 + 3.0 * R + R * R);
}

// max that propagates NaN (a NaN anywhere must reach the host as GQ_ERR_NONFINITE)
__device__ __forceinline__ double nanmax(double a, double b) {
    return (a != a || b != b) ? __longlong_as_double(0x7ff8000000000000ULL) : fmax(a, b);
}

template <bool IsMax>
__device__ __forceinline__ double combine(double a, double b) {
    if constexpr (IsMax) return nanmax(a, b);
    else return a + b;
}

template <bool IsMax>
__device__ __forceinline__ double warp_reduce(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = combine<IsMax>(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---------------------------------------------------------------------------
// Bounded barrier of a team of co-resident blocks (rank in [0, size)).  One 32-bit
// word per team: every block adds 1, except rank 0 which adds 2^31 - (size - 1), so
// the word's top bit flips exactly when the last block arrives and its low bits return
// to where they were (no reset between barriers).  The arrival is an acquire-release
// atomic and the poll an acquire load, so writes before the barrier are visible after
// it.  The abort flag is read every 64th poll.  A block that polls more than spin_limit
// times (or sees *abort_flag set) gives up,
// sets *abort_flag and returns false; every caller must then leave the kernel.  No wait
// in this library is unbounded.
// ---------------------------------------------------------------------------
struct Team {
    int rank;
    int size;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// |a / b| to about two FP32 ulps, for any FP64 a and b: the two significands (in [1, 2))
// are divided in FP32 and the exponent difference is applied in FP64 as two exact
// power-of-two factors, so quotients far outside the FP32 range are still right.  Zero,
// subnormal, infinite and NaN operands take the FP64 division.  Used for the cell-wise
// stop criterion and the reported 2-norm, where the FP64 division (slow on this part)
// buys nothing.
__device__ __forceinline__ double abs_ratio_approx(double a, double b) {
    const long long ab = __double_as_longlong(a), bb = __double_as_longlong(b);
    const int ea = (int)((ab >> 52) & 0x7ff), eb = (int)((bb >> 52) & 0x7ff);
    if (ea == 0 || eb == 0 || ea == 0x7ff || eb == 0x7ff) return fabs(a / b);
    const double ma = __longlong_as_double((ab & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    const double mb = __longlong_as_double((bb & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    const double q = (double)__fdividef((float)ma, (float)mb);
    const int d = ea - eb, d1 = d / 2, d2 = d - d1;       // each within [-1023, 1023]
    return q * __longlong_as_double((long long)(d1 + 1023) << 52) *
           __longlong_as_double((long long)(d2 + 1023) << 52);
}

// device clock in nanoseconds (for the timings reported in gq_step_info)
__device__ __forceinline__ long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

__device__ __forceinline__ int ld_volatile_int(const int* p) {
    return *reinterpret_cast<const volatile int*>(p);
}

__device__ __forceinline__ bool team_barrier(unsigned* bar, Team team, long long spin_limit, int* abort_flag) {
    __shared__ int s_ok;
    __syncthreads();
    if (team.size == 1) return true;     // a one-block team needs only the block barrier
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned inc = team.rank == 0 ? 0x80000000u - (unsigned)(team.size - 1) : 1u;
        const unsigned old = atom_add_acq_rel_gpu(bar, inc);
        long long n = 0;
        while (((ld_acquire_gpu(bar) ^ old) & 0x80000000u) == 0u) {
            ++n;
            if (n > spin_limit || ((n & 63) == 0 && ld_volatile_int(abort_flag))) {
                atomicExch(abort_flag, 1);
                ok = 0;
                break;
            }
            __nanosleep(20);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace gq
