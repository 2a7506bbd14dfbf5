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
// bounded inter-block barrier for co-resident (cooperatively launched) grids.
// bar[0] counts arrivals, bar[1] is the generation.  A block that polls longer than
// spin_limit iterations (or sees *abort set) gives up, sets *abort and returns false;
// every caller must then leave the kernel.  No wait in this library is unbounded.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_int(const int* p) {
    return *reinterpret_cast<const volatile int*>(p);
}

__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, long long spin_limit,
                                             int* abort_flag) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned gen = ld_acquire_gpu(bar + 1);
        __threadfence();
        unsigned prev = atomicAdd(bar, 1u);
        if (prev == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            st_release_gpu(bar + 1, gen + 1u);
        } else {
            long long n = 0;
            while (ld_acquire_gpu(bar + 1) == gen) {
                if (++n > spin_limit || ld_volatile_int(abort_flag)) {
                    atomicExch(abort_flag, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace gq
