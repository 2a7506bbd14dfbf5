"""Pins for the three discretisation conventions the paper leaves open, each against what
the mathematics fixes rather than against the oracle itself.

* Face values (Eq. diffcoeff says sigma and E at a face are interpolated from the cell
  centres): a linear interpolation in the normal coordinate between the two volume
  centres reproduces every linear field exactly at the face.  On a strongly stretched
  grid, fields linear in x and y (or in r and theta) must therefore give, at every
  interior face, R and D worked out from the fields' closed forms at the face position.
  Interpolation weights taken the wrong way round give the field at the mirrored point.
* Distances on a spherical-polar grid (Sec. 3.2.1 only says the x of Eq. alpha is the
  volume centre): the face flux w (E_m - E_k) / dt must be a second-order approximation
  of the exact flux through that face, D E'(theta_f) sin(theta_f) (r+ - r-) for a
  theta-face and D E'(r_f) r_f^2 (cos theta- - cos theta+) for an r-face, both the
  integral of D grad E . n over the face (axisymmetric, 2 pi dropped).  A metric
  without r misses by an O(1) factor, one at the inner face radius converges at first
  order only.
* The Milne boundary (Eq. milne, E = -(2 / (3 rho kappa_R)) dE/dn at the surface): on a
  slab with a reflecting wall at x = 0 and the Milne condition at x = L, cos(k x) with
  cot(k L) = 2 k / (3 sigma) is an eigenfunction of D d^2/dx^2, so one backward-Euler
  step divides it by 1 + D k^2 dt.  The discrete step must converge to that (second
  order: the ghost at h (1 + k) gives the surface flux D E_cell / (h + 2 / (3 sigma)),
  which matches D E(L) 3 sigma / 2 up to O(h^2)).  A wrong factor in k or a full-cell
  distance does not converge.

CPU only.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from paper_2602_12545_gb300 import workloads as W

C_LIGHT = 2.99792458e10          # typed here, not read from the oracle


def _lp(R):
    """Levermore-Pomraning rational limiter (the benchmark's limiter)."""
    return (2.0 + R) / (6.0 + 3.0 * R + R * R)


def _problem(coord, xf, yf, rho, E, k0=0.4, dt=1e3, bc=(0, 0, 0, 0), limiter=W.LIMITER_LP):
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    e_g = rho * 1e4 * W.EG_PER_RHO_T
    return W.FLDProblem("convention_pin", coord, np.asarray(xf, float), np.asarray(yf, float), rho.copy(), e_g,
                        E.copy(), dt, bc=tuple(bc), opacity_R=(k0, 0.0, 0.0, 0.0), opacity_P=(0.0, 0.0, 0.0, 0.0),
                        limiter=limiter)


def _sph_centres(rf, tf):
    """Volume centroids of spherical-polar cells: r_c = int r dV / int dV with dV ~ r^2 dr,
    th_c = int th sin(th) dth / int sin(th) dth (closed forms of the integrals)."""
    r0, r1 = rf[:-1], rf[1:]
    rc = 0.75 * (r1 ** 4 - r0 ** 4) / (r1 ** 3 - r0 ** 3)
    t0, t1 = tf[:-1], tf[1:]
    F = lambda t: np.sin(t) - t * np.cos(t)              # antiderivative of t sin t
    tc = (F(t1) - F(t0)) / (np.cos(t0) - np.cos(t1))
    return rc, tc


def _check_faces(orc, P, xc, yc, xf, yf, sig_fn, E_fn, dEx, dEy, ymetric):
    """R and D at every interior face against the closed forms at the face position."""
    F = orc.faces(P)
    nx, ny = xc.size, yc.size
    worst = 0.0
    for j in range(ny):
        for i in range(1, nx):
            s, e = sig_fn(xf[i], yc[j]), E_fn(xf[i], yc[j])
            R = abs(dEx(xf[i], yc[j])) / (s * e)
            D = C_LIGHT * _lp(R) / s
            worst = max(worst, abs(F["Rx"][j, i] / R - 1.0), abs(F["Dx"][j, i] / D - 1.0))
    for j in range(1, ny):
        for i in range(nx):
            s, e = sig_fn(xc[i], yf[j]), E_fn(xc[i], yf[j])
            R = abs(dEy(xc[i], yf[j])) / (ymetric(xc[i]) * s * e)
            D = C_LIGHT * _lp(R) / s
            worst = max(worst, abs(F["Ry"][j, i] / R - 1.0), abs(F["Dy"][j, i] / D - 1.0))
    return worst


def test_face_values_interpolate_linear_fields_exactly_cartesian(orc):
    """Stretched Cartesian grid (widths growing 1.6x in x, 1.4x in y): sigma = k0 rho and E
    both linear in (x, y); every interior face gets R and D of the fields at the face."""
    xf = W.geometric_faces(6, 1e11, 1.6)
    yf = W.geometric_faces(5, 2e11, 1.4, x0=3e11)
    xc, yc = 0.5 * (xf[:-1] + xf[1:]), 0.5 * (yf[:-1] + yf[1:])
    k0, r0, ax, ay = 0.4, 1e-9, 2e-12, -0.7e-12
    E0, bx, by = 1e3, 1.5e-12, 0.9e-12
    rho_fn = lambda x, y: r0 * (1.0 + ax * x + ay * y)
    E_fn = lambda x, y: E0 * (1.0 + bx * x + by * y)
    X, Y = np.meshgrid(xc, yc)
    P = _problem(W.CARTESIAN, xf, yf, rho_fn(X, Y), E_fn(X, Y), k0=k0)
    worst = _check_faces(orc, P, xc, yc, xf, yf, lambda x, y: k0 * rho_fn(x, y), E_fn,
                         lambda x, y: E0 * bx, lambda x, y: E0 * by, lambda r: 1.0)
    assert worst < 1e-12, worst


def test_face_values_interpolate_linear_fields_exactly_spherical(orc):
    """Log-spaced r (a factor 3 per cell) and uneven theta cells: sigma and E linear in
    (r, theta) between volume centroids; the theta gradient is dE/dtheta / r_c."""
    rf = np.array([1.0, 3.0, 9.0, 27.0, 81.0]) * 1e11
    tf = np.array([0.2, 0.5, 1.1, 1.4, 2.3, 2.9])
    rc, tc = _sph_centres(rf, tf)
    k0, r0, ar, at = 0.4, 1e-9, 1e-13, 0.3
    E0, br, bt = 1e3, 2e-13, -0.2
    rho_fn = lambda r, t: r0 * (1.0 + ar * r + at * t)
    E_fn = lambda r, t: E0 * (1.0 + br * r + bt * t)
    Rr, Tt = np.meshgrid(rc, tc)
    P = _problem(W.SPHERICAL, rf, tf, rho_fn(Rr, Tt), E_fn(Rr, Tt), k0=k0)
    worst = _check_faces(orc, P, rc, tc, rf, tf, lambda r, t: k0 * rho_fn(r, t), E_fn,
                         lambda r, t: E0 * br, lambda r, t: E0 * bt, lambda r: r)
    assert worst < 1e-12, worst


def _flux_errors(orc, n):
    """Relative error of the discrete face fluxes against the exact face integrals on an
    n x n shell r in [1, 2] cm, theta in [0.3, 2.6], for E = E0 exp(r + theta); constant
    sigma and lambda = 1/3, so D = c / (3 sigma) on every face."""
    rf = np.linspace(1.0, 2.0, n + 1)
    tf = np.linspace(0.3, 2.6, n + 1)
    rc, tc = _sph_centres(rf, tf)
    sigma, dt, E0 = 2.0, 1e-11, 1.0
    Rr, Tt = np.meshgrid(rc, tc)
    E = E0 * np.exp(Rr + Tt)
    P = _problem(W.SPHERICAL, rf, tf, np.full((n, n), sigma / 0.4), E, k0=0.4, dt=dt, limiter=W.LIMITER_NONE)
    F = orc.faces(P)
    D = C_LIGHT / (3.0 * sigma)
    err_t = 0.0
    for j in range(1, n):
        for i in range(n):
            disc = F["wy"][j, i] * (E[j, i] - E[j - 1, i]) / dt
            exact = D * E0 * math.exp(rc[i] + tf[j]) * math.sin(tf[j]) * (rf[i + 1] - rf[i])
            err_t = max(err_t, abs(disc / exact - 1.0))
    err_r = 0.0
    for j in range(n):
        for i in range(1, n):
            disc = F["wx"][j, i] * (E[j, i] - E[j, i - 1]) / dt
            exact = D * E0 * math.exp(rf[i] + tc[j]) * rf[i] ** 2 * (math.cos(tf[j]) - math.cos(tf[j + 1]))
            err_r = max(err_r, abs(disc / exact - 1.0))
    return err_t, err_r


def test_spherical_face_fluxes_converge_at_second_order(orc):
    """The theta distance r_c (th_c,m - th_c,k) and the r distance r_c,m - r_c,k make the
    face flux a second-order approximation of the exact flux through the face."""
    errs = [_flux_errors(orc, n) for n in (32, 64, 128)]
    for axis in (0, 1):
        e = [x[axis] for x in errs]
        orders = [math.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]
        assert min(orders) > 1.8, (axis, e, orders)
        assert e[-1] < 5e-4, (axis, e)


def _milne_error(orc, n, L=1.0, sigma=1.0):
    """Max over cells of |E^{n+1} (1 + D k^2 dt) / E^n - 1| for the Milne eigenmode."""
    ell = 2.0 / (3.0 * sigma)
    z = brentq(lambda z: math.cos(z) - (ell / L) * z * math.sin(z), 1e-6, 0.5 * math.pi - 1e-9)
    k = z / L
    D = C_LIGHT / (3.0 * sigma)
    dt = 1.0 / (D * k * k)                   # D k^2 dt = 1: the mode halves in one step
    xf = np.linspace(0.0, L, n + 1)
    xc = 0.5 * (xf[:-1] + xf[1:])
    E = (1e3 * np.cos(k * xc)).reshape(1, n)
    P = _problem(W.CARTESIAN, xf, np.array([0.0, 1.0]), np.full((1, n), sigma / 0.4), E, k0=0.4, dt=dt,
                 bc=(W.BC_REFLECT, W.BC_MILNE, W.BC_REFLECT, W.BC_REFLECT), limiter=W.LIMITER_NONE)
    out = orc.step(P, "lu")
    return float(np.max(np.abs(out["E_r"] * (1.0 + D * k * k * dt) / E - 1.0)))


def test_milne_eigenmode_decays_as_the_continuum_one(orc):
    """One backward-Euler step of the slab's slowest Milne mode converges at second order
    to the continuum factor 1 / (1 + D k^2 dt)."""
    e = [_milne_error(orc, n) for n in (16, 32, 64, 128)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]
    assert min(orders) > 1.8, (e, orders)
    assert e[-1] < 1e-4, e
