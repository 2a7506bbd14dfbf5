"""Pins of the oracle's sub-cycled step in the order of the paper's radiation algorithm
(Sec. 3.2.1): after each sub-step alpha = dt_i / d is updated and the algorithm re-enters
at the C_V step, so D, with kappa_R rho and the limiter, keeps its value from the start of
the hydro step (freeze_D=True), and the accumulated flux is D^n sum_i alpha_i (E_m - E_k)_i
over dt.

- one sub-step is the plain step;
- where D does not depend on the state (limiter 'none', constant kappa_R) the frozen and
  the re-formed orders coincide;
- where it does (Kramers kappa_R, Levermore-Pomraning) they differ;
- with reflecting sides the frozen order conserves E + e_g, and with Milne sides the
  energy lost equals dt times the flux through them;
- the accumulated flux is the paper's sum, evaluated here from the sub-steps' E and the
  start-of-step D and centre distances.
"""
import dataclasses

import numpy as np
import pytest

from paper_2602_12545_gb300 import workloads as W


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def test_one_substep_is_the_plain_step(orc):
    P = W.random_small(23, 17, W.SPHERICAL, (0, 1, 0, 1), 7)
    a = orc.step_subcycled(P, 1, 1.4, freeze_D=True)
    b = orc.step(P)
    for f in ("E_r", "T_g", "e_g"):
        assert _rel(a[f], b[f]) < 1e-11, f
    assert np.abs(a["Fx"] - b["Fx"]).max() <= 1e-11 * np.abs(b["Fx"]).max()


def test_state_independent_D_orders_coincide(orc):
    P = W.random_small(19, 13, W.CARTESIAN, (1, 0, 0, 1), 11, limiter=W.LIMITER_NONE)
    P = dataclasses.replace(P, opacity_R=(0.4, 0.0, 0.0, 0.0))
    a = orc.step_subcycled(P, 5, 1.3, freeze_D=True)
    b = orc.step_subcycled(P, 5, 1.3, freeze_D=False)
    for f in ("E_r", "T_g", "e_g"):
        assert _rel(a[f], b[f]) < 1e-11, f


def test_state_dependent_D_orders_differ(orc):
    P = W.random_small(19, 13, W.SPHERICAL, (0, 1, 0, 1), 12)
    a = orc.step_subcycled(P, 5, 1.3, freeze_D=True)
    b = orc.step_subcycled(P, 5, 1.3, freeze_D=False)
    assert _rel(a["E_r"], b["E_r"]) > 1e-6


def test_frozen_order_conserves_energy(orc):
    P = W.random_small(21, 15, W.SPHERICAL, (0, 0, 0, 0), 13)
    out = orc.step_subcycled(P, 6, 1.4, freeze_D=True)
    assert out["energy_after"] == pytest.approx(out["energy_before"], rel=1e-12)


def test_frozen_flux_carries_the_lost_energy(orc):
    """Cartesian, Milne at both x sides: dt times the area-weighted flux through them is the
    energy the grid lost; reflecting y sides carry nothing."""
    P = W.random_small(30, 4, W.CARTESIAN, (1, 1, 0, 0), 14)
    out = orc.step_subcycled(P, 6, 1.4, freeze_D=True)
    g = orc.geometry(P)
    lost = out["energy_before"] - out["energy_after"]
    through = P.dt * ((g["Ax"][:, -1] * out["Fx"][:, -1]).sum() - (g["Ax"][:, 0] * out["Fx"][:, 0]).sum())
    assert lost > 0
    assert lost == pytest.approx(through, rel=1e-9)
    assert np.all(out["Fy"][0] == 0) and np.all(out["Fy"][-1] == 0)


def test_frozen_flux_is_the_papers_sum(orc):
    """Interior x faces: F = D^n sum_i (dt_i / dt) (E_{i-1} - E_i)^{(i)} / (x_i - x_{i-1}), with
    D^n the face D of the start state and the sub-steps' E after each sub-step."""
    P = W.random_small(26, 9, W.SPHERICAL, (0, 1, 0, 0), 15)
    n, q = 4, 1.25
    out = orc.step_subcycled(P, n, q, freeze_D=True)
    Dn = orc.faces(P)["Dx"]
    xc = orc.geometry(P)["xc"]
    d = xc[1:] - xc[:-1]
    Q = P
    want = np.zeros((P.ny, P.nx - 1))
    w = orc.faces(P)
    G = (w["wx"] / P.dt, w["wy"] / P.dt)
    for dt in orc.subcycle_dts(P.dt, n, q):
        o = orc.step(dataclasses.replace(Q, dt=dt), G=G)
        E = o["E_r"]
        want += (dt / P.dt) * Dn[:, 1:-1] * (E[:, :-1] - E[:, 1:]) / d[None, :]
        Q = dataclasses.replace(Q, E_r=E, e_g=o["e_g"])
    got = out["Fx"][:, 1:-1]
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
