// Cell and face geometry of the FLD grid (Sec. 3.2.1 and Eq. fldg), shared by the plan's
// host set-up and the allocation-free step's device kernels so that both evaluate the same
// formulas.  Cartesian (x, y) per unit depth, or axisymmetric spherical-polar (r, theta)
// with the common factor 2 pi dropped:
//   V = (r+^3 - r-^3) / 3 (cos th- - cos th+),  A_r = r^2 (cos th- - cos th+),
//   A_th = sin th (r+^2 - r-^2) / 2;
// volume centres r_c = int r dV / int dV and th_c = int th dV / int dV.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define GQ_HD __host__ __device__ __forceinline__
#else
#define GQ_HD inline
#endif

namespace gq {
namespace geom {

constexpr double kPi = 3.14159265358979323846;

// int_v^{v+h} (t - v) sin t dt and int_v^{v+h} sin t dt, evaluated without cancellation for
// small h (series in h for the two h-only factors)
GQ_HD void theta_moments(double v, double h, double* first, double* zeroth) {
    double A, B;   // A = cos h + h sin h - 1, B = sin h - h cos h
    if (h < 0.05) {
        const double h2 = h * h;
        A = h2 * (0.5 + h2 * (-1.0 / 8.0 + h2 * (1.0 / 144.0 + h2 * (-1.0 / 5760.0))));
        B = h2 * h * (1.0 / 3.0 + h2 * (-1.0 / 30.0 + h2 * (1.0 / 840.0 + h2 * (-1.0 / 45360.0))));
    } else {
        A = cos(h) + h * sin(h) - 1.0;
        B = sin(h) - h * cos(h);
    }
    const double sv = sin(v), cv = cos(v);
    const double half = sin(0.5 * h);
    *first = sv * A + cv * B;
    *zeroth = sv * sin(h) + cv * 2.0 * half * half;
}

// volume centre of [a, b] in x (Cartesian midpoint, or int r^3 dr / int r^2 dr)
GQ_HD double x_centre(double a, double b, bool sph) {
    return sph ? 0.75 * (a + b) * (a * a + b * b) / (a * a + a * b + b * b) : 0.5 * (a + b);
}

// volume centre of [a, b] in y; *dcos receives the cell's cos th- - cos th+ (1 for Cartesian)
GQ_HD double y_centre(double a, double b, bool sph, double* dcos) {
    if (!sph) {
        *dcos = 1.0;
        return 0.5 * (a + b);
    }
    double m1, m0;
    theta_moments(a, b - a, &m1, &m0);
    *dcos = m0;
    return a + m1 / m0;
}

// volume of the cell [xa, xb] x [ya, yb] (dcos from y_centre)
GQ_HD double cell_volume(double xa, double xb, double ya, double yb, bool sph, double dcos) {
    return sph ? (xb - xa) * (xa * xa + xa * xb + xb * xb) / 3.0 * dcos : (xb - xa) * (yb - ya);
}

// area of the x-face at x = r of the row [ya, yb] (dcos from y_centre of that row)
GQ_HD double x_face_area(double r, double ya, double yb, bool sph, double dcos) {
    return sph ? r * r * dcos : yb - ya;
}

// area of the y-face at y = th of the column [xa, xb]; the poles have no area
GQ_HD double y_face_area(double th, double xa, double xb, bool sph) {
    if (!sph) return xb - xa;
    const double sf = (th <= 0.0 || th >= kPi) ? 0.0 : sin(th);
    return sf * (xb - xa) * (xb + xa) * 0.5;
}

}  // namespace geom
}  // namespace gq
