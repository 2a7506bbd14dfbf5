// Per-cell and per-face physics of the FLD step shared by the single-level set-up and the
// multilevel (composite-grid) step: the power-law mean opacities (Sec. 2), the face
// weight dt A D / d with the flux-limited D of Eq. diffcoeff, and the Milne boundary face
// (Eq. milne).
#pragma once

#include "gq_device.cuh"

namespace gq {
namespace {

// x^e for the exponents power laws use: integers and half-integers up to 8 by repeated
// multiplication (and one square root, or for negative half-integers one reciprocal
// square root raised to the odd power 2|e|), anything else through pow.  FP64 pow, sqrt
// and division each cost tens of FP64 operations, and FP64 arithmetic is the scarce
// resource of this part.
__device__ __forceinline__ double power(double x, double e) {
    if (e == 1.0) return x;
    if (e == 0.0) return 1.0;
    const double ae = fabs(e);
    const double twice = 2.0 * ae;
    if (ae <= 8.0 && twice == rint(twice)) {
        const int n = static_cast<int>(ae);
        if (e < 0.0 && twice != 2.0 * n) {
            // x^-(n + 1/2) = (x^-1/2)^(2n + 1), by squaring
            const double q = rsqrt(x);
            double r = q, b = q * q;
            for (int m = n; m > 0; m >>= 1) {
                if (m & 1) r *= b;
                b *= b;
            }
            return r;
        }
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
    if (lim == 0) {
        // Levermore-Pomraning with R = a / u (a = |E_b - E_a|, u = d sigma_f E_f):
        // c lambda / sigma_f = c u (2u + a) / (sigma_f (6u^2 + 3ua + a^2)), one division
        // (u and a kept away from overflow and underflow of their squares)
        const double a = fabs(Eb - Ea), u = d * sf * Ef;
        if (u > 1e-100 && u < 1e100 && a < 1e100)
            return dt * geo * kC * (u * (2.0 * u + a)) / (sf * (u * (6.0 * u + 3.0 * a) + a * a));
    }
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
