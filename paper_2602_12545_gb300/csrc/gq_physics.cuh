// Per-cell and per-face physics of the FLD step shared by the single-level set-up and the
// multilevel (composite-grid) step: the power-law mean opacities (Sec. 2), the face
// weight dt A D / d with the flux-limited D of Eq. diffcoeff, and the Milne boundary face
// (Eq. milne).
#pragma once

#include "gq_device.cuh"

namespace gq {
namespace {

// x^e for the exponents power laws use: integers and half-integers up to 8 by repeated
// multiplication (and one square root), anything else through pow.  FP64 pow costs tens
// of FP64 operations, and FP64 arithmetic is the scarce resource of this part.
__device__ __forceinline__ double power(double x, double e) {
    if (e == 1.0) return x;
    if (e == 0.0) return 1.0;
    const double ae = fabs(e);
    const double twice = 2.0 * ae;
    if (ae <= 8.0 && twice == rint(twice)) {
        const int n = static_cast<int>(ae);
        double r = 1.0;
        for (int i = 0; i < n; i++) r *= x;
        if (twice != 2.0 * n) r *= sqrt(x);
        return e < 0.0 ? 1.0 / r : r;
    }
    return pow(x, e);
}

__device__ __forceinline__ double opacity(const double* k, double rho, double T) {
    return k[1] != 0.0 ? k[0] + k[1] * power(rho, k[2]) * power(T, k[3]) : k[0];
}

// weight of an interior face between cells a (lower coordinate) and b
__device__ __forceinline__ double face_weight(double sa, double sb, double Ea, double Eb, double th,
                                              double d, double geo, int lim, double dt) {
    const double sf = sa + th * (sb - sa);
    const double Ef = Ea + th * (Eb - Ea);
    const double R = fabs(Eb - Ea) / (d * sf * Ef);
    const double D = kC * limiter(lim, R) / sf;
    return dt * geo * D;
}

// Milne face (Eq. milne): E_b = k/(1+k) E_cell, k = 2 / (3 sigma h), R_b = 3/2,
// D_b = c lambda(3/2) / sigma; flux D_b (E - E_b)/h = D_b E / (h (1+k)).
// geo = A / h.
__device__ __forceinline__ double milne_weight(double s, double h, double geo, int lim, double dt) {
    const double kk = 2.0 / (3.0 * s * h);
    const double D = kC * limiter(lim, 1.5) / s;
    return dt * geo * D / (1.0 + kk);
}

}  // namespace
}  // namespace gq
