"""Pins for the oracle's mean opacities: kappa = k0 + k1 rho^a T^b evaluated per cell at
the gas temperature of time n (Sec. 2 defines kappa_R and kappa_P; Sec. 3.2.1 freezes
them over the step).  Every other pin runs the constant law (k1 = 0), so these are the
only ones that fix which exponent goes with rho and which with T, that the constant k0
is kept, that the Rosseland law feeds the diffusion coefficient and the Planck law the
exchange, and that the temperature is T_g^n and not the radiation temperature.

The laws and states are chosen so that each opacity is a short decimal worked out by
hand below (written as literals, not evaluated by the formula):
  Rosseland (k0, k1, a, b) = (0.2, 5e10, 0.5, -2):
    rho = 1e-8, T = 1e4:  0.2 + 5e10 * 1e-4 * 1e-8 = 0.25
    rho = 1e-6, T = 1e2:  0.2 + 5e10 * 1e-3 * 1e-4 = 5000.2
  Planck (k0, k1, a, b) = (0.1, 2e-3, -0.25, 0.5):
    rho = 1e-8, T = 1e4:  0.1 + 2e-3 * 1e2 * 1e2 = 20.1
  The benchmark law (0.34, 4e25, 1, -3.5):
    rho = 1e-12, T = 1e4: 0.34 + 4e25 * 1e-12 * 1e-14 = 0.74
A swapped pair of exponents gives 5e10 * 1e8 * 1e2 = 5e20 in place of 0.05, and a dropped
k0 gives 0.05 in place of 0.25: both fail by orders of magnitude.

CPU only.
"""
import numpy as np
import pytest

from paper_2602_12545_gb300 import workloads as W

# independent literals (CODATA values typed here, not read from the oracle)
C_LIGHT = 2.99792458e10
A_RAD = 7.5657332e-15
K_B = 1.380649e-16
M_H = 1.6735328e-24

ROSS = (0.2, 5e10, 0.5, -2.0)
PLANCK = (0.1, 2e-3, -0.25, 0.5)


def _problem(rho, T, E, kR, kP, nx=2, dt=1e3, limiter=W.LIMITER_NONE):
    """Uniform Cartesian row of nx cells (dx = 1e12 cm), reflecting walls; per-cell rho
    and T (e_g from the ideal-gas recipe), radiation energy E."""
    f = W.uniform_faces(nx, 1e12)
    g = W.uniform_faces(1, 1e12)
    rho = np.asarray(rho, float).reshape(1, nx)
    T = np.asarray(T, float).reshape(1, nx)
    E = np.asarray(E, float).reshape(1, nx)
    return W.FLDProblem("opacity_pin", W.CARTESIAN, f, g, rho.copy(), rho * T * W.EG_PER_RHO_T, E.copy(), dt,
                        bc=(0, 0, 0, 0), opacity_R=tuple(kR), opacity_P=tuple(kP), limiter=limiter)


def _sigma_face(orc, P):
    """sigma at the single interior face, read back from D = c lambda / sigma_f with the
    constant limiter lambda = 1/3."""
    D = orc.faces(P)["Dx"][0, 1]
    return C_LIGHT / (3.0 * D)


def test_rosseland_law_in_the_face_coefficient(orc):
    """Two cells at one state: the face sigma is kappa_R rho = 0.25 * 1e-8 (the radiation
    energy is far from a T^4, so a law taken at the radiation temperature misses)."""
    P = _problem([1e-8, 1e-8], [1e4, 1e4], [1.0e3, 1.3e3], ROSS, PLANCK)
    assert _sigma_face(orc, P) == pytest.approx(0.25 * 1e-8, rel=1e-13)


def test_rosseland_law_per_cell_states(orc):
    """Two cells at different (rho, T): on a uniform grid the face sigma is the mean of
    the cells' kappa_R rho, with kappa_R = 0.25 and 5000.2 worked out by hand."""
    P = _problem([1e-8, 1e-6], [1e4, 1e2], [1.0e3, 1.3e3], ROSS, PLANCK)
    want = 0.5 * (0.25 * 1e-8 + 5000.2 * 1e-6)
    assert _sigma_face(orc, P) == pytest.approx(want, rel=1e-13)


def test_benchmark_law_value(orc):
    """The benchmark workloads' law 0.34 + 4e25 rho T^-3.5 at rho = 1e-12, T = 1e4 is 0.74."""
    P = _problem([1e-12, 1e-12], [1e4, 1e4], [1.0e3, 1.3e3], W.KRAMERS_LIKE, W.KRAMERS_LIKE)
    assert _sigma_face(orc, P) == pytest.approx(0.74 * 1e-12, rel=1e-13)


def test_power_law_equals_its_constant_value(orc):
    """The whole step with the power laws equals the step with constant opacities at the
    hand-evaluated values (kappa_R = 0.25, kappa_P = 20.1): the laws enter only through
    their values at (rho, T_g^n)."""
    rho, T, E = [1e-8, 1e-8], [1e4, 1e4], [1.0e3, 1.3e3]
    a = orc.step(_problem(rho, T, E, ROSS, PLANCK, limiter=W.LIMITER_LP), "lu")
    b = orc.step(_problem(rho, T, E, (0.25, 0.0, 1.0, 0.0), (20.1, 0.0, 1.0, 0.0), limiter=W.LIMITER_LP), "lu")
    for f in ("E_r", "T_g", "e_g"):
        np.testing.assert_allclose(a[f], b[f], rtol=1e-13, atol=0)


def test_planck_law_in_the_exchange_closed_form(orc):
    """One cell with reflecting walls has no diffusion, and the linearised exchange has a
    closed form: with beta = kappa_P rho c dt, q = 4 beta a T^3 and
    beta~ = beta C_V / (C_V + q), E^{n+1} = (E^n + beta~ a T^4) / (1 + beta~), and
    C_V T^{n+1} + E^{n+1} = C_V T^n + E^n.  kappa_P = 20.1 is the hand value."""
    rho, T, E, dt = 1e-8, 1e4, 1.0e3, 1e-3
    P = _problem([rho], [T], [E], ROSS, PLANCK, nx=1, dt=dt)
    out = orc.step(P, "lu")
    cv = rho * K_B / ((5.0 / 3.0 - 1.0) * 0.6 * M_H)
    beta = 20.1 * rho * C_LIGHT * dt
    q = 4.0 * beta * A_RAD * T ** 3
    bt = beta * cv / (cv + q)
    E1 = (E + bt * A_RAD * T ** 4) / (1.0 + bt)
    assert out["E_r"][0, 0] == pytest.approx(E1, rel=1e-7)        # A_RAD, M_H typed to 8 digits
    T1 = T + (E - out["E_r"][0, 0]) / cv
    assert out["T_g"][0, 0] == pytest.approx(T1, rel=1e-7)
    # the step moves E most of the way to a T^4, and beta~ is of order one, so that a
    # kappa_P off by even a few per cent moves E^{n+1} by far more than the tolerance
    assert abs(E1 - E) > 0.5 * E
    assert 0.5 < bt < 50.0
