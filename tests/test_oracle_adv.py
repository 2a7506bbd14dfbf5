"""Pins of the oracle's explicit radiation advection (Sec. 3.2.1, Eq. adv with g = dS / dV
of Eq. fldg), checked against what the mathematics fixes rather than against the oracle's
own formula:

- on a uniform 1-D grid Eq. adv is the textbook first-order upwind difference;
- interior faces cancel in sum_k V_k S_k, which leaves the boundary fluxes;
- a divergence-free flow through a spherical-polar grid with uniform e_r gives S = 0;
- S_adv enters phi_11 as S_adv dt, so with E-independent coefficients a step with the
  source equals a step from E^n + S_adv dt without it; the coupled and reduced systems
  agree with the source on;
- the dynamical-diffusion set-up of Sec. 5 (uniform flow, no coupling): upwind advection
  followed by an implicit diffusion step keeps the packet's energy, moves its centroid by
  v dt per step and adds exactly c(1 - c) dx^2 + 2 D dt to its variance (c = v dt / dx),
  and at the end it matches the paper's analytic Gaussian.
"""
import dataclasses

import numpy as np
import pytest

from paper_2602_12545_gb300 import workloads as W

C_LIGHT = 2.99792458e10


def _uniform_1d(nx, dx, seed):
    rng = np.random.default_rng(seed)
    xf = W.uniform_faces(nx, dx)
    rho = 10.0 ** rng.uniform(-10, -8, (1, nx))
    T = 10.0 ** rng.uniform(3, 5, (1, nx))
    return W._pack("adv1d", W.CARTESIAN, xf, np.array([0.0, 3.0]), rho, T, T * 1.1, 1e3)


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_upwind_closed_form_1d(orc, sign):
    nx, dx, f = 12, 2.0, 0.7 * sign
    P = _uniform_1d(nx, dx, 5)
    e = (P.E_r / P.rho)[0]
    S = orc.adv_source(P, np.full((1, nx + 1), f), np.zeros((2, nx)))[0]
    want = np.zeros(nx)
    for i in range(nx):
        if f > 0:   # flow along +x: each cell receives its left neighbour's e_r
            want[i] = f * ((e[i - 1] if i > 0 else e[0]) - e[i]) / dx
        else:       # flow along -x: each cell receives its right neighbour's e_r
            want[i] = -f * ((e[i + 1] if i < nx - 1 else e[-1]) - e[i]) / dx
    assert np.allclose(S, want, rtol=1e-13, atol=1e-13 * np.abs(want).max())


@pytest.mark.parametrize("coord", [W.CARTESIAN, W.SPHERICAL])
def test_interior_faces_cancel(orc, coord):
    P = W.random_small(17, 11, coord, (0,) * 4, 77)
    fx, fy = W.mass_fluxes(P, 78)
    S = orc.adv_source(P, fx, fy)
    g = orc.geometry(P)
    e = P.E_r / P.rho
    boundary = ((g["Ax"][:, 0] * fx[:, 0] * e[:, 0]).sum() - (g["Ax"][:, -1] * fx[:, -1] * e[:, -1]).sum()
                + (g["Ay"][0] * fy[0] * e[0]).sum() - (g["Ay"][-1] * fy[-1] * e[-1]).sum())
    total = (g["V"] * S).sum()
    scale = (g["V"] * np.abs(S)).sum()
    assert abs(total - boundary) <= 1e-12 * scale


def test_divergence_free_spherical_flow(orc):
    """f_r = C / r^2 and f_theta = C' / sin(theta) carry A f constant along each direction,
    so with uniform e_r every cell's in- and outflow balance."""
    nx, ny = 14, 9
    xf = W.log_faces(nx, 1.0, 10.0)
    yf = np.linspace(0.3, 2.8, ny + 1)
    rng = np.random.default_rng(3)
    rho = 10.0 ** rng.uniform(-10, -8, (ny, nx))
    P = W._pack("divfree", W.SPHERICAL, xf, yf, rho, np.full((ny, nx), 1e4), np.full((ny, nx), 1e4), 1.0)
    P = dataclasses.replace(P, E_r=rho * 3.7e5)
    fx = np.broadcast_to(2.0 / xf[None, :] ** 2, (ny, nx + 1)).copy()
    fy = np.broadcast_to(0.5 / np.sin(yf)[:, None], (ny + 1, nx)).copy()
    S = orc.adv_source(P, fx, fy)
    g = orc.geometry(P)
    e = 3.7e5
    inflow = (g["Ax"][:, :-1] * fx[:, :-1] + g["Ax"][:, 1:] * fx[:, 1:]
              + g["Ay"][:-1] * fy[:-1] + g["Ay"][1:] * fy[1:]) * e / g["V"]
    assert np.all(np.abs(S) <= 1e-13 * inflow)


def test_source_enters_phi11_times_dt(orc):
    """Limiter 'none': D does not depend on E, and nothing else in the step reads E^n, so
    the source is the same as starting from E^n + S_adv dt."""
    P = W.random_small(13, 9, W.SPHERICAL, (0, 1, 1, 0), 91, limiter=W.LIMITER_NONE)
    fx, fy = W.mass_fluxes(P, 92)
    S = orc.adv_source(P, fx, fy)
    assert np.abs(S * P.dt).max() > 1e-3 * P.E_r.min()
    a = orc.step(dataclasses.replace(P, S_adv=S), "lu")
    b = orc.step(dataclasses.replace(P, E_r=P.E_r + S * P.dt), "lu")
    for f in ("E_r", "T_g", "e_g"):
        assert np.allclose(a[f], b[f], rtol=1e-13, atol=0), f


def test_coupled_and_reduced_agree_with_source(orc):
    """Moderate coupling (beta_P ~ 0.3), where the paper-literal coupled system keeps its
    digits: both assemblies include the source."""
    P = W.random_small(11, 7, W.CARTESIAN, (1, 0, 0, 1), 93)
    P = dataclasses.replace(P, opacity_P=(1e-3, 0.0, 0.0, 0.0), opacity_R=(1e-3, 0.0, 0.0, 0.0), dt=1e4)
    fx, fy = W.mass_fluxes(P, 94)
    P = dataclasses.replace(P, S_adv=orc.adv_source(P, fx, fy))
    a = orc.step(P, "lu")
    b = orc.step(P, "coupled")
    for f in ("E_r", "T_g"):
        assert np.allclose(a[f], b[f], rtol=1e-9, atol=0), f
    c = orc.step(dataclasses.replace(P, S_adv=None), "lu")
    assert not np.allclose(a["E_r"], c["E_r"], rtol=1e-6)


def test_subcycled_source_adds_S_dt_in_total(orc):
    """No coupling, reflecting sides: sub-step i adds S_adv dt_i, so the series adds
    S_adv dt in total and sum V E grows by dt sum V S_adv whatever the diffusion does."""
    P, fx, fy = W.advected_packet(nx=64, cfl=0.5)
    P = dataclasses.replace(P, S_adv=orc.adv_source(P, fx, fy))
    g = orc.geometry(P)
    out = orc.step_subcycled(P, 5, 1.4, freeze_D=False)
    before = (g["V"] * P.E_r).sum()
    after = (g["V"] * out["E_r"]).sum()
    assert after == pytest.approx(before + P.dt * (g["V"] * P.S_adv).sum(), rel=1e-13)


def _advance(orc, P, fx, fy, n):
    for _ in range(n):
        S = orc.adv_source(P, fx, fy)
        out = orc.step(dataclasses.replace(P, S_adv=S), "lu")
        P = dataclasses.replace(P, E_r=out["E_r"], e_g=out["e_g"])
    return P


def _moments(x, u):
    M = u.sum()
    mu = (x * u).sum() / M
    return M, mu, ((x - mu) ** 2 * u).sum() / M


@pytest.mark.parametrize("cfl,steps", [(1.0, 714), (0.4, 300)])
def test_advected_packet_moments(orc, cfl, steps):
    """Sec. 5 dynamical diffusion (v = 1.8 km/s, rho kappa_R = 1e7 / cm, kappa_P = 0), with
    limiter 'none' so that D = c / (3 rho kappa_R) exactly.  714 steps at CFL 1 reach the
    paper's t = 6.2e-5 s."""
    v, sig = 1.8e5, 1e7
    P, fx, fy = W.advected_packet(cfl=cfl, limiter=W.LIMITER_NONE)
    x = 0.5 * (P.x_faces[:-1] + P.x_faces[1:])
    dx = P.x_faces[1] - P.x_faces[0]
    D = C_LIGHT / (3.0 * sig)
    M0, mu0, var0 = _moments(x, P.E_r[0] - 1.0)
    Q = _advance(orc, P, fx, fy, steps)
    M, mu, var = _moments(x, Q.E_r[0] - 1.0)
    c = v * P.dt / dx
    assert M == pytest.approx(M0, rel=1e-11)
    assert mu == pytest.approx(mu0 + steps * v * P.dt, abs=1e-11)
    assert var == pytest.approx(var0 + steps * (c * (1 - c) * dx * dx + 2 * D * P.dt), rel=1e-11)
    if cfl == 1.0:
        # the paper's analytic solution, within two diffusion lengths of the packet centre
        t = steps * P.dt
        Ea = 1.0 + 2e5 / np.sqrt(4 * np.pi * D * t) * np.exp(-(x - v * t) ** 2 / (4 * D * t))
        near = np.abs(x - v * t) < 2 * np.sqrt(4 * D * t)
        err = np.abs(Q.E_r[0] - Ea) / Ea
        assert err[near].max() < 1e-2
