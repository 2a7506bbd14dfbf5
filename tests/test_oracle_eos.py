"""Pins of the oracle's non-linear C_V (Sec. 3.2.1 evaluates C_V per cell before the
coefficients; the paper's hydrogen EoS is not available, so a tabulated u(T) with a
dissociation and an ionisation bump stands in):

- a table sampled from the ideal gas reproduces the ideal-gas step;
- without coupling (kappa_P = 0) T^n is the inverse of the table, as numpy's interp
  evaluates it, and e_g is kept;
- the tangent C_V: over a step that keeps T inside one table segment, the returned
  T^{n+1} and e^{n+1} lie on that segment of u(T), so T^{n+1} is numpy's interp of
  e^{n+1} / rho (a secant or wrong-segment C_V breaks this);
- one cell exchanging energy with radiation, sub-cycled, converges at first order to the
  exchange ODE  rho du/dt = c kappa_P rho (E - a T(u)^4) = -dE/dt  integrated by scipy.
  This pins the table inversion and the exchange.  It does not pin C_V: C_V only
  linearises within a sub-step, and T is re-derived from e at the next one.
"""
import dataclasses

import numpy as np
import pytest

from paper_2602_12545_gb300 import workloads as W

KB = 1.380649e-16
MH = 1.00782503207 * 1.66053906660e-24
C_LIGHT = 2.99792458e10
A_RAD = 4.0 * 5.670374419e-5 / C_LIGHT


def test_ideal_gas_table_is_the_ideal_gas(orc):
    P = W.random_small(17, 11, W.SPHERICAL, (0, 1, 0, 1), 21)
    cv = KB / ((P.gamma - 1.0) * P.mu * MH)
    T = np.exp(np.linspace(np.log(10.0), np.log(1e7), 40))
    a = orc.step(dataclasses.replace(P, eos_table=(T, cv * T)))
    b = orc.step(P)
    for f in ("E_r", "T_g", "e_g"):
        assert np.allclose(a[f], b[f], rtol=1e-11, atol=0), f


def test_uncoupled_temperature_inverts_the_table(orc):
    T_tab, u_tab = W.hydrogen_like_table()
    P = W.random_small(13, 9, W.CARTESIAN, (0,) * 4, 22)
    rng = np.random.default_rng(23)
    T0 = 10.0 ** rng.uniform(2.0, 5.5, P.E_r.shape)
    e_g = P.rho * np.interp(T0, T_tab, u_tab)
    P = dataclasses.replace(P, e_g=e_g, eos_table=(T_tab, u_tab), opacity_P=(0.0, 0.0, 0.0, 0.0))
    out = orc.step(P)
    assert np.allclose(out["T_g"], np.interp(e_g / P.rho, u_tab, T_tab), rtol=1e-12, atol=0)
    assert np.allclose(out["e_g"], e_g, rtol=1e-15, atol=0)


def test_tangent_cv_keeps_the_state_on_the_table(orc):
    T_tab, u_tab = W.hydrogen_like_table()
    P = W.random_small(13, 9, W.CARTESIAN, (0, 1, 0, 0), 24)
    rng = np.random.default_rng(25)
    T0 = 10.0 ** rng.uniform(2.5, 5.0, P.E_r.shape)
    e_g = P.rho * np.interp(T0, T_tab, u_tab)
    E = A_RAD * T0 ** 4 * (1.0 + 0.05 * rng.standard_normal(T0.shape))   # near equilibrium: small steps
    P = dataclasses.replace(P, e_g=e_g, E_r=E, eos_table=(T_tab, u_tab), dt=10.0)
    out = orc.step(P)
    seg0 = np.searchsorted(T_tab, T0)
    seg1 = np.searchsorted(T_tab, out["T_g"])
    same = seg0 == seg1
    assert same.mean() > 0.5
    moved = np.abs(out["T_g"] / T0 - 1.0)
    assert moved[same].max() > 1e-6             # the step does change T
    back = np.interp(out["e_g"] / P.rho, u_tab, T_tab)
    assert np.allclose(out["T_g"][same], back[same], rtol=1e-10, atol=0)


def _one_cell(T_g, T_rad, rho, kP, dt, table):
    f = np.array([0.0, 1e10])
    u0 = np.interp(T_g, table[0], table[1])
    return W.FLDProblem(name="cell", coord=W.CARTESIAN, x_faces=f, y_faces=f.copy(), rho=np.full((1, 1), rho),
                        e_g=np.full((1, 1), rho * u0), E_r=np.full((1, 1), A_RAD * T_rad ** 4), dt=dt,
                        opacity_R=(1.0, 0.0, 0.0, 0.0), opacity_P=(kP, 0.0, 0.0, 0.0), eos_table=table)


def test_subcycled_cell_converges_to_the_exchange_ode(orc):
    solve_ivp = pytest.importorskip("scipy.integrate").solve_ivp
    table = W.hydrogen_like_table()
    rho, kP, dt = 1e-9, 1e-2, 20.0       # c kappa_P rho dt = 6: several exchange times
    P = _one_cell(2.0e3, 1.5e4, rho, kP, dt, table)
    E0, e0 = P.E_r[0, 0], P.e_g[0, 0]
    rate = C_LIGHT * kP * rho

    def rhs(t, y):
        u, E = y
        T = np.interp(u, table[1], table[0])
        q = rate * (E - A_RAD * T ** 4)
        return [q / rho, -q]

    sol = solve_ivp(rhs, (0.0, dt), [e0 / rho, E0], method="Radau", rtol=1e-12, atol=[1e-6 * e0 / rho, 1e-12 * E0])
    u_ex, E_ex = sol.y[0, -1], sol.y[1, -1]
    assert u_ex > 1.5 * e0 / rho          # the gas crossed into the dissociation bump
    # errors against the total energy (E falls 300-fold as the gas absorbs it)
    total = E0 + e0
    err = []
    for n in (100, 400):
        out = orc.step_subcycled(P, n, 1.0, freeze_D=False)
        err.append(max(abs(out["e_g"][0, 0] - rho * u_ex), abs(out["E_r"][0, 0] - E_ex)) / total)
    assert err[1] < err[0] / 3.0          # first order: a quarter, within rounding of the ratio
    assert err[1] < 1e-4
