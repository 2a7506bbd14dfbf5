"""Seeded synthetic inputs for the implicit FLD radiation step.

This module only draws numbers: grids (face coordinates), gas density,
gas internal energy and radiation energy density, and the scalar settings of
each workload.  It contains none of the step's arithmetic (no opacities, no
limiter, no matrix, no solver), so that the CUDA path and the FP64 CPU
oracle can both be fed from it without sharing any of the method.

Workloads follow the paper's test set-ups in shape (Chen & Bai, Guangqi):
i.i.d. lognormal density, log-uniform gas temperature and a radiation
temperature perturbed around it on Cartesian grids; power-law profiles on a
spherical-polar grid that spans optically thick to thin (the disk tests of
Sec. 5.3 use a stretched spherical-polar grid).  The paper uses no public
dataset; every array here is synthetic.

Initial-condition recipe: the drawn gas temperature T_g is turned into the
internal energy per unit volume e_g = rho * T_g * EG_PER_RHO_T, the ideal
gamma = 5/3, mu = 0.6 relation (the paper's perfect-gas coupling test, Sec. 5.1.1),
and E_r = A_RAD_RECIPE * T_rad^4.  These two literals are part of the recipe
only: the step itself derives T_g from e_g with its own equation of state.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# --- initial-condition recipe literals (CGS) -------------------------------
# k_B / ((gamma - 1) mu m_H) with gamma = 5/3, mu = 0.6, m_H = 1.00782503207 u.
_KB = 1.380649e-16
_MH = 1.00782503207 * 1.66053906660e-24
EG_PER_RHO_T = _KB / ((5.0 / 3.0 - 1.0) * 0.6 * _MH)
# radiation constant a_R = 4 sigma_SB / c
A_RAD_RECIPE = 4.0 * 5.670374419e-5 / 2.99792458e10

# boundary side order used everywhere: -x, +x, -y, +y
BC_REFLECT = 0
BC_MILNE = 1
CARTESIAN = 0
SPHERICAL = 1
LIMITER_LP = 0
LIMITER_MINERBO = 1
LIMITER_NONE = 2
PREC_FP64 = 0
PREC_MIXED = 1

# opacity law kappa = k0 + k1 * rho^a * T^b (cm^2/g), same for Rosseland and Planck
KRAMERS_LIKE = (0.34, 4.0e25, 1.0, -3.5)


@dataclasses.dataclass
class FLDProblem:
    """One implicit FLD step's inputs (host, float64, row-major [ny][nx])."""
    name: str
    coord: int
    x_faces: np.ndarray          # nx+1 (x, or r for spherical-polar)
    y_faces: np.ndarray          # ny+1 (y, or theta for spherical-polar)
    rho: np.ndarray              # [ny][nx] g/cm^3
    e_g: np.ndarray              # [ny][nx] erg/cm^3
    E_r: np.ndarray              # [ny][nx] erg/cm^3
    dt: float
    bc: tuple = (BC_REFLECT,) * 4
    opacity_R: tuple = KRAMERS_LIKE
    opacity_P: tuple = KRAMERS_LIKE
    gamma: float = 5.0 / 3.0
    mu: float = 0.6
    limiter: int = LIMITER_LP
    precision: int = PREC_FP64
    rtol: float = 1e-10
    S_adv: Optional[np.ndarray] = None   # [ny][nx] explicit radiation source, erg cm^-3 s^-1
    eos_table: Optional[tuple] = None    # (T [K], u [erg/g]) increasing: tabulated u(T); None = ideal gas

    @property
    def nx(self) -> int:
        return self.x_faces.size - 1

    @property
    def ny(self) -> int:
        return self.y_faces.size - 1

    @property
    def ncells(self) -> int:
        return self.nx * self.ny


def _fields_iid(nx: int, ny: int, rng: np.random.Generator):
    """Config-0 field recipe: rho lognormal (median 1e-9, 1.5 dex), log10 T_g ~ U(3,5),
    T_rad = T_g (1 + 0.1 N(0,1)) clamped at 1e-3 T_g."""
    rho = 1e-9 * 10.0 ** (1.5 * rng.standard_normal((ny, nx)))
    T = 10.0 ** rng.uniform(3.0, 5.0, (ny, nx))
    Trad = T * np.maximum(1.0 + 0.1 * rng.standard_normal((ny, nx)), 1e-3)
    return rho, T, Trad


def _pack(name, coord, xf, yf, rho, T, Trad, dt, **kw) -> FLDProblem:
    e_g = rho * T * EG_PER_RHO_T
    E = A_RAD_RECIPE * Trad ** 4
    return FLDProblem(name=name, coord=coord, x_faces=np.ascontiguousarray(xf, dtype=np.float64),
                      y_faces=np.ascontiguousarray(yf, dtype=np.float64),
                      rho=np.ascontiguousarray(rho), e_g=np.ascontiguousarray(e_g),
                      E_r=np.ascontiguousarray(E), dt=float(dt), **kw)


def uniform_faces(n: int, d: float, x0: float = 0.0) -> np.ndarray:
    return x0 + d * np.arange(n + 1, dtype=np.float64)


def geometric_faces(n: int, d0: float, ratio: float, x0: float = 0.0) -> np.ndarray:
    widths = d0 * ratio ** np.arange(n, dtype=np.float64)
    return x0 + np.concatenate([[0.0], np.cumsum(widths)])


def log_faces(n: int, r_in: float, r_out: float) -> np.ndarray:
    f = np.exp(np.linspace(math.log(r_in), math.log(r_out), n + 1))
    f[0], f[-1] = r_in, r_out
    return f


def theta_faces(n: int) -> np.ndarray:
    f = np.linspace(0.0, math.pi, n + 1)
    f[0], f[-1] = 0.0, math.pi
    return f


def config0(seed: int = 1000, n: int = 64) -> FLDProblem:
    """64x64 uniform Cartesian, dx = dy = 1e12 cm, dt = 1e4 s, reflecting, FP64 to 1e-10."""
    rng = np.random.default_rng(seed)
    rho, T, Trad = _fields_iid(n, n, rng)
    f = uniform_faces(n, 1e12)
    return _pack("c0_cart64", CARTESIAN, f, f.copy(), rho, T, Trad, 1e4,
                 bc=(BC_REFLECT,) * 4, precision=PREC_FP64, rtol=1e-10)


def config1(seed: int = 1001, n: int = 1024) -> FLDProblem:
    """1024^2 Cartesian, dx geometric (ratio 1.002, dx0 = 1e12), dy = 1e12, dt = 1e5 s,
    Milne outflow at +x, reflecting elsewhere, FP64 to 1e-10."""
    rng = np.random.default_rng(seed)
    rho, T, Trad = _fields_iid(n, n, rng)
    xf = geometric_faces(n, 1e12, 1.002)
    yf = uniform_faces(n, 1e12)
    return _pack("c1_cart1024_geom", CARTESIAN, xf, yf, rho, T, Trad, 1e5,
                 bc=(BC_REFLECT, BC_MILNE, BC_REFLECT, BC_REFLECT), precision=PREC_FP64, rtol=1e-10)


def spherical_fields(xf: np.ndarray, yf: np.ndarray, rng: np.random.Generator):
    """Config-2 recipe: rho = 1e-8 (r/1e11)^-2 10^(0.5 N), T_g = 1e5 (r/1e11)^-0.5,
    T_rad = T_g (1 + 0.1 N) clamped at 1e-3 T_g; r is the arithmetic cell midpoint."""
    nx, ny = xf.size - 1, yf.size - 1
    r = 0.5 * (xf[1:] + xf[:-1])
    rr = np.broadcast_to(r[None, :], (ny, nx))
    rho = 1e-8 * (rr / 1e11) ** -2 * 10.0 ** (0.5 * rng.standard_normal((ny, nx)))
    T = 1e5 * (rr / 1e11) ** -0.5
    Trad = T * np.maximum(1.0 + 0.1 * rng.standard_normal((ny, nx)), 1e-3)
    return rho, np.ascontiguousarray(T), Trad


def config2(seed: int = 1002, nr: int = 2048, nth: int = 1024) -> FLDProblem:
    """2048 (r, log-spaced 1e11..1e14 cm) x 1024 (theta, 0..pi) spherical-polar, dt = 1e4 s,
    reflecting at inner r and theta ends, Milne at outer r, mixed precision with a
    cell-wise residual of 2e-10: the loosest setting (of 1e-11, 3e-11, 1e-10, 2e-10, 3e-10,
    1e-9 measured) that keeps every cell within 1e-8 of the tightly solved answer with
    room to spare (2.2e-9 measured; 1e-9 gives 3.7e-8)."""
    rng = np.random.default_rng(seed)
    xf = log_faces(nr, 1e11, 1e14)
    yf = theta_faces(nth)
    rho, T, Trad = spherical_fields(xf, yf, rng)
    return _pack("c2_sph2048x1024", SPHERICAL, xf, yf, rho, T, Trad, 1e4,
                 bc=(BC_REFLECT, BC_MILNE, BC_REFLECT, BC_REFLECT), precision=PREC_MIXED, rtol=2e-10)


def batch_sizes(n_problems: int = 256, seed: int = 1003):
    """Side lengths log-uniform in [32, 512], drawn independently for nx and ny."""
    rng = np.random.default_rng(seed)
    lo, hi = math.log(32), math.log(512)
    nxs = np.rint(np.exp(rng.uniform(lo, hi, n_problems))).astype(int)
    nys = np.rint(np.exp(rng.uniform(lo, hi, n_problems))).astype(int)
    dts = 10.0 ** rng.uniform(3.0, 6.0, n_problems)
    return nxs, nys, dts


def config3(n_problems: int = 256, seed: int = 1003, max_side: Optional[int] = None) -> List[FLDProblem]:
    """256 independent problems, nx, ny log-uniform in [32, 512], alternating Cartesian
    (dx = 1e12, reflecting) and spherical-polar (r log-spaced 1e11..1e14, theta 0..pi,
    Milne at outer r), i.i.d. config-0 fields, dt = 10^U(3,6) s, mixed precision with a
    cell-wise residual of 1e-10, which keeps every cell of every problem within 1e-8 of
    the oracle (a residual of 1e-8 leaves errors up to 2e-7 on some spherical draws).
    Problem p draws its fields from seed + 1 + p."""
    nxs, nys, dts = batch_sizes(n_problems, seed)
    out = []
    for p in range(n_problems):
        nx, ny = int(nxs[p]), int(nys[p])
        if max_side is not None:
            nx, ny = min(nx, max_side), min(ny, max_side)
        rng = np.random.default_rng(seed + 1 + p)
        rho, T, Trad = _fields_iid(nx, ny, rng)
        if p % 2 == 0:
            xf, yf = uniform_faces(nx, 1e12), uniform_faces(ny, 1e12)
            pr = _pack(f"c3_p{p}_cart{nx}x{ny}", CARTESIAN, xf, yf, rho, T, Trad, dts[p],
                       bc=(BC_REFLECT,) * 4, precision=PREC_MIXED, rtol=1e-10)
        else:
            xf, yf = log_faces(nx, 1e11, 1e14), theta_faces(ny)
            pr = _pack(f"c3_p{p}_sph{nx}x{ny}", SPHERICAL, xf, yf, rho, T, Trad, dts[p],
                       bc=(BC_REFLECT, BC_MILNE, BC_REFLECT, BC_REFLECT), precision=PREC_MIXED, rtol=1e-10)
        out.append(pr)
    return out


@dataclasses.dataclass
class ServeRequest:
    rid: int
    arrival_s: float
    side: int
    n_steps: int
    seed: int


def config4_trace(n_requests: int = 2000, rate_per_s: float = 2000.0, seed: int = 1004,
                  side_lo: int = 64, side_hi: int = 2048, n_steps: int = 10) -> List[ServeRequest]:
    """Poisson arrivals (mean rate_per_s), square sides log-uniform in [side_lo, side_hi],
    n_steps consecutive implicit steps per request.  The trace is finite."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, n_requests)
    t = np.cumsum(gaps) - gaps[0]
    sides = np.rint(np.exp(rng.uniform(math.log(side_lo), math.log(side_hi), n_requests))).astype(int)
    return [ServeRequest(i, float(t[i]), int(sides[i]), n_steps, seed + 1 + i) for i in range(n_requests)]


def serve_problem(req: ServeRequest) -> FLDProblem:
    """A serving request's initial state: uniform Cartesian square grid, dx = 1e12 cm,
    config-0 fields, dt = 1e4 s, reflecting, mixed precision with a cell-wise residual of
    1e-10 (each step within 1e-8 of the oracle)."""
    n = req.side
    rng = np.random.default_rng(req.seed)
    rho, T, Trad = _fields_iid(n, n, rng)
    f = uniform_faces(n, 1e12)
    return _pack(f"c4_r{req.rid}_cart{n}", CARTESIAN, f, f.copy(), rho, T, Trad, 1e4,
                 bc=(BC_REFLECT,) * 4, precision=PREC_MIXED, rtol=1e-10)


def random_small(nx: int, ny: int, coord: int, bc, seed: int, limiter: int = LIMITER_LP,
                 dt: Optional[float] = None) -> FLDProblem:
    """Small parity cases: config-0 fields on a uniform Cartesian grid (dx = 1e12) or a
    spherical-polar grid (r log-spaced 1e11..1e13, theta 0..pi)."""
    rng = np.random.default_rng(seed)
    rho, T, Trad = _fields_iid(nx, ny, rng)
    if coord == CARTESIAN:
        xf = geometric_faces(nx, 1e12, 1.05)
        yf = uniform_faces(ny, 1e12)
    else:
        xf, yf = log_faces(nx, 1e11, 1e13), theta_faces(ny)
    if dt is None:
        dt = 10.0 ** rng.uniform(3.0, 6.0)
    return _pack(f"small_{'cart' if coord == CARTESIAN else 'sph'}{nx}x{ny}_s{seed}", coord, xf, yf,
                 rho, T, Trad, dt, bc=tuple(bc), limiter=limiter)


def hydrogen_like_table(n: int = 64, T_lo: float = 10.0, T_hi: float = 1e6):
    """A stand-in for a hydrogen EoS table (the paper's Fig. of C_V / rho against T shows
    a dissociation bump near 3e3 K and an ionisation bump near 1e4 K): the specific heat
    c(T) = (k_B / m_H) [1.5 + 20 exp(-(lg T - 3.5)^2 / 0.045) + 60 exp(-(lg T - 4.1)^2 / 0.02)]
    integrated (trapezoid, 50 sub-intervals per table interval) to u(T) at n log-spaced
    temperatures.  Returns (T, u)."""
    T = np.exp(np.linspace(math.log(T_lo), math.log(T_hi), n))
    kB_mH = _KB / _MH

    def c(t):
        lg = np.log10(t)
        return kB_mH * (1.5 + 20.0 * np.exp(-(lg - 3.5) ** 2 / 0.045) + 60.0 * np.exp(-(lg - 4.1) ** 2 / 0.02))

    u = np.empty(n)
    u[0] = kB_mH * 1.5 * T[0]
    for i in range(1, n):
        t = np.linspace(T[i - 1], T[i], 51)
        ct = c(t)
        u[i] = u[i - 1] + float(np.sum(0.5 * (ct[1:] + ct[:-1]) * np.diff(t)))
    return T, u


def advected_packet(nx: int = 1024, v: float = 1.8e5, sigma_R: float = 1e7, E0: float = 2e5, cfl: float = 1.0,
                    limiter: int = LIMITER_LP):
    """The dynamical-diffusion set-up (Sec. 5, radiation advected by a uniform flow and
    diffusing, no coupling): x in [-2, 14] cm, one row of unit height, rho = 1,
    rho kappa_R = sigma_R, kappa_P = 0, T_g = 0.1 K, E_r = 1 with E0 / (2 dx) in the two
    cells whose centres lie within dx of x = 0; reflecting radiation boundaries and the
    mass flux rho v on every x face (the fixed inflow state); dt = cfl dx / v.  Returns
    (problem, fx [1][nx+1], fy [2][nx])."""
    xf = np.linspace(-2.0, 14.0, nx + 1)
    dx = xf[1] - xf[0]
    xc = 0.5 * (xf[:-1] + xf[1:])
    rho = np.ones((1, nx))
    T = np.full((1, nx), 0.1)
    E = np.ones((1, nx))
    E[0, np.abs(xc) < dx] = E0 / (2.0 * dx)
    P = FLDProblem(name=f"packet{nx}", coord=CARTESIAN, x_faces=xf, y_faces=np.array([0.0, 1.0]), rho=rho,
                   e_g=rho * T * EG_PER_RHO_T, E_r=E, dt=float(cfl * dx / v), bc=(BC_REFLECT,) * 4,
                   opacity_R=(float(sigma_R), 0.0, 0.0, 0.0), opacity_P=(0.0, 0.0, 0.0, 0.0), limiter=limiter)
    return P, np.full((1, nx + 1), v * 1.0), np.zeros((2, nx))


def mass_fluxes(P: FLDProblem, seed: int, cfl: float = 0.05):
    """Random face mass fluxes rho v (g cm^-2 s^-1) for problem P: v = cfl N(0,1) (clipped
    to +-1) times the smaller width of the face's cells over dt, rho that of the cell the
    flow comes from (a boundary face: its one cell).  Returns (fx [ny][nx+1], fy [ny+1][nx])."""
    rng = np.random.default_rng(seed)
    nx, ny = P.nx, P.ny
    xf, yf = P.x_faces, P.y_faces
    wx = np.broadcast_to(np.diff(xf)[None, :], (ny, nx))
    if P.coord == CARTESIAN:
        wy = np.broadcast_to(np.diff(yf)[:, None], (ny, nx))
    else:
        wy = np.diff(yf)[:, None] * (0.5 * (xf[:-1] + xf[1:]))[None, :]

    def faces(w, rho, n_f, axis):
        # pad with the edge cell on both sides so that face f sits between cells f-1 and f
        wp = np.concatenate([np.take(w, [0], axis), w, np.take(w, [-1], axis)], axis)
        rp = np.concatenate([np.take(rho, [0], axis), rho, np.take(rho, [-1], axis)], axis)
        lo = [slice(None)] * 2; hi = [slice(None)] * 2
        lo[axis] = slice(0, n_f); hi[axis] = slice(1, n_f + 1)
        dmin = np.minimum(wp[tuple(lo)], wp[tuple(hi)])
        v = cfl * np.clip(rng.standard_normal(dmin.shape), -1.0, 1.0) * dmin / P.dt
        return np.ascontiguousarray(np.where(v > 0, rp[tuple(lo)], rp[tuple(hi)]) * v)

    return faces(wx, P.rho, nx + 1, 1), faces(wy, P.rho, ny + 1, 0)


CONFIGS = {0: config0, 1: config1, 2: config2}
