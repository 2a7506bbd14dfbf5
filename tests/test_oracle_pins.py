"""Pins for the FP64 CPU oracle: each test checks the oracle against something other
than itself -- a number the paper prints, a closed form, an exact discrete identity,
numerical quadrature, an independent ODE integration or a library solver -- so that a
dropped term, a wrong sign or index, or a transposed operand fails one of them.

CPU only (no GPU marker).
"""
import math
import os

import numpy as np
import pytest
import scipy.integrate as si
import scipy.linalg as sla

from paper_2602_12545_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# independent literals for the tests (CODATA / IAU values typed here, not read from the oracle)
C_LIGHT = 2.99792458e10
A_RAD = 7.5657332e-15          # radiation constant, erg cm^-3 K^-4
K_B = 1.380649e-16
M_H = 1.6735328e-24            # 1H atom mass (1.007825 u), g


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            out[parts[0]] = parts[1:]
    return out


def _uniform_problem(nx, ny, dx, rho, T, E, dt, kR=(0.0, 0.0, 1.0, 0.0), kP=(0.0, 0.0, 1.0, 0.0),
                     bc=(0, 0, 0, 0), limiter=W.LIMITER_LP, coord=W.CARTESIAN, xf=None, yf=None):
    xf = W.uniform_faces(nx, dx) if xf is None else xf
    yf = W.uniform_faces(ny, dx) if yf is None else yf
    shape = (ny, nx)
    rho = np.broadcast_to(np.asarray(rho, float), shape).copy()
    T = np.broadcast_to(np.asarray(T, float), shape).copy()
    E = np.broadcast_to(np.asarray(E, float), shape).copy()
    e_g = rho * T * W.EG_PER_RHO_T
    return W.FLDProblem("pin", coord, xf, yf, rho, e_g, E, dt, bc=tuple(bc), opacity_R=tuple(kR),
                        opacity_P=tuple(kP), limiter=limiter)


# ---------------------------------------------------------------------------
# flux limiter (Sec. 2)
# ---------------------------------------------------------------------------

def test_minerbo_golden(orc):
    for R, lam in ((1.5, 2.0 / 9.0), (0.0, 1.0 / 3.0)):
        assert orc.limiter(W.LIMITER_MINERBO, R)[0] == pytest.approx(lam, rel=1e-15)
    g = _golden("minerbo_limiter.txt")
    assert float(g["1.5"][0]) == pytest.approx(2.0 / 9.0, rel=1e-15)
    # continuity across the branch point
    eps = 1e-9
    lo = orc.limiter(W.LIMITER_MINERBO, 1.5 - eps)[0]
    hi = orc.limiter(W.LIMITER_MINERBO, 1.5 + eps)[0]
    assert abs(hi - lo) < 1e-9


@pytest.mark.parametrize("kind", [W.LIMITER_LP, W.LIMITER_MINERBO])
def test_limiter_asymptotics(orc, kind):
    R = np.logspace(-6, 8, 4001)
    lam = orc.limiter(kind, R)
    # optically thick: lambda -> 1/3 ; optically thin: lambda R -> 1 (Eq. asymptotic)
    assert lam[0] == pytest.approx(1.0 / 3.0, rel=1e-10)
    assert lam[-1] * R[-1] == pytest.approx(1.0, abs=2e-4)
    # causality |F| = c lambda R E <= c E, and lambda decreasing
    assert np.all(lam * R <= 1.0 + 1e-15)
    assert np.all(np.diff(lam) <= 0.0)


def test_lp_rational_close_to_exact_lp(orc):
    """The rational Levermore-Pomraning form stays within 8% of the exact LP limiter
    (coth R - 1/R)/R for all R (its known maximum deviation is about 7%)."""
    R = np.logspace(-3, 5, 2001)
    exact = (1.0 / np.tanh(R) - 1.0 / R) / R
    lam = orc.limiter(W.LIMITER_LP, R)
    assert np.max(np.abs(lam - exact) / exact) < 0.08


# ---------------------------------------------------------------------------
# geometry: volumes, areas, centres (Eq. fldg, Eq. alpha)
# ---------------------------------------------------------------------------

def test_cartesian_geometry(orc):
    P = W.random_small(7, 5, W.CARTESIAN, (0, 0, 0, 0), 1)
    g = orc.geometry(P)
    Lx = P.x_faces[-1] - P.x_faces[0]
    Ly = P.y_faces[-1] - P.y_faces[0]
    assert g["V"].sum() == pytest.approx(Lx * Ly, rel=1e-14)
    np.testing.assert_allclose(g["xc"], 0.5 * (P.x_faces[1:] + P.x_faces[:-1]), rtol=1e-15)
    np.testing.assert_allclose(g["Ax"][0], np.full(8, P.y_faces[1] - P.y_faces[0]), rtol=1e-15)


def test_spherical_volume_and_divergence_theorem(orc):
    """Volumes against quadrature of r^2 sin(th); r-face areas from the divergence theorem
    for F = r r_hat (div F = 3); theta-face areas from F = cos(th) th_hat
    (div F = cos(2 th) / (r sin th))."""
    P = W.random_small(9, 7, W.SPHERICAL, (0, 0, 0, 0), 2)
    g = orc.geometry(P)
    rf, tf = P.x_faces, P.y_faces
    assert g["V"].sum() == pytest.approx((rf[-1] ** 3 - rf[0] ** 3) / 3.0 * 2.0, rel=1e-13)
    for (i, j) in [(0, 0), (4, 3), (8, 6), (2, 5)]:
        vol = si.dblquad(lambda r, t: r * r * math.sin(t), tf[j], tf[j + 1], rf[i], rf[i + 1],
                         epsabs=0, epsrel=1e-13)[0]
        assert g["V"][j, i] == pytest.approx(vol, rel=1e-11)
        # F = r r_hat: outward flux through the r faces equals 3 V
        flux_r = rf[i + 1] * g["Ax"][j, i + 1] - rf[i] * g["Ax"][j, i]
        assert flux_r == pytest.approx(3.0 * vol, rel=1e-11)
        # F = cos(th) th_hat: div F integrated over the cell equals the theta-face fluxes
        div_int = si.dblquad(lambda r, t: math.cos(2 * t) / (r * math.sin(t)) * r * r * math.sin(t),
                             tf[j], tf[j + 1], rf[i], rf[i + 1], epsabs=0, epsrel=1e-13)[0]
        flux_t = math.cos(tf[j + 1]) * g["Ay"][j + 1, i] - math.cos(tf[j]) * g["Ay"][j, i]
        assert flux_t == pytest.approx(div_int, rel=1e-9, abs=1e-12 * abs(vol) / rf[i + 1])
        # volume centres (Eq. alpha uses the volume centre)
        rc = si.dblquad(lambda r, t: r ** 3 * math.sin(t), tf[j], tf[j + 1], rf[i], rf[i + 1],
                        epsabs=0, epsrel=1e-13)[0] / vol
        tc = si.dblquad(lambda r, t: t * r * r * math.sin(t), tf[j], tf[j + 1], rf[i], rf[i + 1],
                        epsabs=0, epsrel=1e-13)[0] / vol
        assert g["xc"][i] == pytest.approx(rc, rel=1e-12)
        assert g["yc"][j] == pytest.approx(tc, rel=1e-11)


def test_spherical_theta_centre_fine_grid(orc):
    """Volume centres stay accurate on the fine theta grid of the large spherical case."""
    P = W.random_small(3, 1024, W.SPHERICAL, (0, 0, 0, 0), 3)
    g = orc.geometry(P)
    tf = P.y_faces
    for j in (0, 1, 511, 1022, 1023):
        num = si.quad(lambda t: t * math.sin(t), tf[j], tf[j + 1], epsabs=0, epsrel=1e-13)[0]
        den = si.quad(lambda t: math.sin(t), tf[j], tf[j + 1], epsabs=0, epsrel=1e-13)[0]
        assert g["yc"][j] == pytest.approx(num / den, rel=1e-12)


# ---------------------------------------------------------------------------
# linear algebra: the direct and iterative solvers, symmetry, definiteness
# ---------------------------------------------------------------------------

def test_band_solver_against_lapack(orc):
    import scipy.sparse as sp
    rng = np.random.default_rng(7)
    n, kl, ku = 60, 5, 3
    A = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - kl), min(n, i + ku + 1)):
            A[i, j] = rng.standard_normal()
    A += np.diag(rng.uniform(0.1, 0.5, n))      # not diagonally dominant: pivoting is exercised
    b = rng.standard_normal(n)
    x = orc.band_solve(sp.csr_matrix(A), b)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("coord", [W.CARTESIAN, W.SPHERICAL])
def test_reduced_matrix_symmetric_and_spd(orc, coord):
    P = W.random_small(13, 11, coord, (0, 1, 0, 1) if coord == W.CARTESIAN else (0, 1, 0, 0), 11)
    A, b = orc.assemble_reduced(P)
    A = A.tocsr()
    # exactly symmetric: off-diagonals are the shared face weights
    assert (A != A.T).nnz == 0
    d = A.diagonal()
    off = np.abs(A).sum(axis=1).A1 - np.abs(d)
    assert np.all(d > off)                       # strictly diagonally dominant
    sla.cholesky(A.toarray())                   # positive definite
    assert np.all(b > 0)


def test_coupled_literal_system_matches_reduced(orc):
    """The paper-literal coupled system (Eqs. linearsys1-2, banded LU) and the exactly
    reduced system agree where the coupling leaves FP64 digits to spare (beta_P <~ 1e3)."""
    rng = np.random.default_rng(5)
    nx, ny = 12, 10
    rho = 10.0 ** rng.uniform(-13, -11, (ny, nx))
    T = 10.0 ** rng.uniform(4, 5, (ny, nx))
    E = A_RAD * (T * (1 + 0.2 * rng.standard_normal((ny, nx)))) ** 4
    for bc in ((0, 0, 0, 0), (0, 1, 0, 1)):
        P = _uniform_problem(nx, ny, 1e12, rho, T, E, 1e3, kR=W.KRAMERS_LIKE, kP=W.KRAMERS_LIKE, bc=bc)
        a = orc.step(P, "coupled")
        b = orc.step(P, "lu")
        np.testing.assert_allclose(a["E_r"], b["E_r"], rtol=1e-11)
        np.testing.assert_allclose(a["T_g"], b["T_g"], rtol=1e-11)


def test_cg_matches_direct_config0(orc):
    P = W.config0()
    a = orc.step(P, "lu")
    b = orc.step(P, "cg", tol=1e-15)
    assert b["cell_residual"] < 1e-13
    np.testing.assert_allclose(b["E_r"], a["E_r"], rtol=1e-12)
    np.testing.assert_allclose(b["T_g"], a["T_g"], rtol=1e-12)


# ---------------------------------------------------------------------------
# energy conservation, equation of state, spherical symmetry
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["c0", "sph"])
def test_total_energy_conserved_reflecting(orc, which):
    if which == "c0":
        P = W.config0()
    else:
        P = W.random_small(24, 20, W.SPHERICAL, (0, 0, 0, 0), 9)
    out = orc.step(P, "lu")
    e0, e1 = out["energy_before"], out["energy_after"]
    assert abs(e1 - e0) <= 1e-12 * e0


def test_gas_temperature_matches_recipe_without_coupling(orc):
    """With kappa_P = 0 there is no exchange: T^{n+1} = T^n = e_g / C_V must reproduce the
    drawn temperature, i.e. the oracle's ideal-gas C_V = rho k_B/((gamma-1) mu m_H)."""
    rng = np.random.default_rng(3)
    T = 10.0 ** rng.uniform(3, 5, (6, 5))
    P = _uniform_problem(5, 6, 1e12, 1e-9, T, 1.0, 1e4, kR=(0.4, 0.0, 1.0, 0.0))
    out = orc.step(P, "lu")
    np.testing.assert_allclose(out["T_g"], T, rtol=1e-13)
    # and the recipe itself is the textbook gamma = 5/3, mu = 0.6 gas
    cv_per_rho = K_B / ((5.0 / 3.0 - 1.0) * 0.6 * M_H)
    assert W.EG_PER_RHO_T == pytest.approx(cv_per_rho, rel=1e-5)


def test_spherical_radial_symmetry(orc):
    """theta-independent data stay theta-independent (the theta factor of A_r and V cancel)."""
    rng = np.random.default_rng(4)
    nr, nt = 16, 12
    xf, yf = W.log_faces(nr, 1e11, 1e13), W.theta_faces(nt)
    rho = np.broadcast_to(1e-9 * 10.0 ** (0.5 * rng.standard_normal(nr)), (nt, nr))
    T = np.broadcast_to(10.0 ** rng.uniform(3.5, 4.5, nr), (nt, nr))
    E = A_RAD * T ** 4 * 1.3
    P = _uniform_problem(nr, nt, 0, rho, T, E, 1e4, kR=W.KRAMERS_LIKE, kP=W.KRAMERS_LIKE,
                         bc=(0, 1, 0, 0), coord=W.SPHERICAL, xf=xf, yf=yf)
    out = orc.step(P, "lu")
    for f in ("E_r", "T_g"):
        v = out[f]
        np.testing.assert_allclose(v, np.broadcast_to(v[nt // 2], v.shape), rtol=1e-12)


# ---------------------------------------------------------------------------
# radiation - gas coupling in a uniform box against an ODE integration (Sec. 5.1.1)
# ---------------------------------------------------------------------------

def _coupling_run(orc, e0, growth, t_end):
    g = _golden("coupling_test.txt")
    rho, kP, E0 = float(g["rho"][0]), float(g["kappa_P"][0]), float(g["E_r"][0])
    dt = float(g["dt0"][0])
    cv = rho * K_B / ((5.0 / 3.0 - 1.0) * float(g["mu"][0]) * M_H)
    T0 = e0 / cv
    # large cells: the (uniform) box has no diffusion, and w/V << 1 keeps the diagonal exact
    P = _uniform_problem(2, 2, 1e10, rho, T0, E0, dt, kR=(kP, 0, 1, 0), kP=(kP, 0, 1, 0))
    P.e_g[:] = e0
    ts, es, Es = [0.0], [e0], [E0]
    t = 0.0
    while t < t_end:
        P.dt = dt
        out = orc.step(P, "lu")
        P.e_g = out["e_g"].copy()
        P.E_r = out["E_r"].copy()
        t += dt
        dt *= growth
        ts.append(t); es.append(P.e_g[0, 0]); Es.append(P.E_r[0, 0])
        assert np.ptp(P.e_g) <= 1e-12 * abs(P.e_g[0, 0])
    return np.array(ts), np.array(es), np.array(Es), cv, rho * kP * C_LIGHT


def _ode(cv, krc, e0, E0, ts):
    def f(t, y):
        E, e = y
        src = krc * (E - A_RAD * (e / cv) ** 4)
        return [-src, src]

    def jac(t, y):
        E, e = y
        d = krc * 4 * A_RAD * (e / cv) ** 3 / cv
        return [[-krc, d], [krc, -d]]

    sol = si.solve_ivp(f, (0, ts[-1]), [E0, e0], method="Radau", jac=jac, t_eval=ts, rtol=1e-12,
                       atol=[1e-3, 1e-12 * e0], first_step=1e-22)
    assert sol.success
    return sol.y[0], sol.y[1]


@pytest.mark.parametrize("e0", [1e2, 1e6, 1e10])
def test_coupling_converges_to_ode(orc, e0):
    """Backward Euler with the linearised T^4 follows the exact ODE at first order in the
    step: halving the growth rate of the step roughly halves the error."""
    t_end = 2e-6
    errs = []
    for growth in (1.02, 1.01):
        ts, es, Es, cv, krc = _coupling_run(orc, e0, growth, t_end)
        E_ode, e_ode = _ode(cv, krc, e0, 1e12, ts)
        errs.append(np.max(np.abs(es - e_ode) / e_ode))
        # E + e_g conserved exactly step by step
        np.testing.assert_allclose(Es + es, Es[0] + es[0], rtol=1e-13)
    assert errs[1] < 0.05
    assert 1.5 < errs[0] / errs[1] < 2.6


def test_coupling_equilibrium_quartic(orc):
    """After many steps the box sits at a T^4 = E with E + e_g unchanged: the root of
    a T^4 + C_V T = E0 + e0."""
    e0 = 1e10
    ts, es, Es, cv, krc = _coupling_run(orc, e0, 1.05, 1e-4)
    roots = np.roots([A_RAD, 0, 0, cv, -(1e12 + e0)])
    Teq = max(r.real for r in roots if abs(r.imag) < 1e-6 * abs(r))
    assert es[-1] / cv == pytest.approx(Teq, rel=1e-6)
    assert Es[-1] == pytest.approx(A_RAD * Teq ** 4, rel=1e-6)


# ---------------------------------------------------------------------------
# diffusion of a Gaussian pulse (Sec. 5.2.2 without advection)
# ---------------------------------------------------------------------------

def _gauss_problem(n, dx, E0, Dc, t0, dt):
    half = n * dx / 2
    f = W.uniform_faces(n, dx, -half)
    xc = 0.5 * (f[1:] + f[:-1])
    X, Y = np.meshgrid(xc, xc)
    E = 1.0 + E0 / (4 * math.pi * Dc * t0) * np.exp(-(X * X + Y * Y) / (4 * Dc * t0))
    P = _uniform_problem(n, n, dx, 1.0, 0.1, E, dt, kR=(1e7, 0, 1, 0), kP=(0.0, 0, 1, 0),
                         limiter=W.LIMITER_NONE, xf=f, yf=f.copy())
    return P, X, Y


def test_diffusion_length_golden(orc):
    """D = c / (3 rho kappa_R) at the faces reproduces l_diff = sqrt(4 D t) ~ 0.498 cm."""
    g = _golden("diffusion_length.txt")
    P, _, _ = _gauss_problem(8, 0.1, 1.0, 1000.0, 1e-5, 1e-6)
    fc = orc.faces(P)
    D = fc["Dx"][0, 1]
    assert D == pytest.approx(C_LIGHT / (3 * float(g["rho_kappa_R"][0])), rel=1e-14)
    l_diff = math.sqrt(4 * D * float(g["t"][0]))
    assert l_diff == pytest.approx(float(g["l_diff"][0]), abs=5e-4)
    assert float(g["v_cm_per_s"][0]) * float(g["t"][0]) == pytest.approx(float(g["l_dyn"][0]), rel=1e-3)


def test_gaussian_pulse_moments_and_shape(orc):
    """The 5-point operator is exact on quadratics, so per step the discrete second moment of
    the pulse grows by exactly 4 D dt times its (new) mass in 2D, and mass is conserved.
    Against the analytic 2D Green's function the error is first order in the step
    (backward Euler): doubling the number of steps halves it."""
    Dc = C_LIGHT / 3e7
    n, dx, E0 = 280, 0.03, 2e5       # walls at +-4.2 cm: the implicit kernel's tails stay below 1e-12
    t0, t1 = 1e-5, 6.2e-5
    errs = []
    for nsteps in (10, 20):
        dt = (t1 - t0) / nsteps
        P, X, Y = _gauss_problem(n, dx, E0, Dc, t0, dt)
        V = dx * dx
        r2 = X * X + Y * Y
        pulse = P.E_r - 1.0
        M0, M2 = (V * pulse).sum(), (V * pulse * r2).sum()
        for _ in range(nsteps):
            out = orc.step(P, "cg", tol=1e-15)
            pulse_new = out["E_r"] - 1.0
            M0n, M2n = (V * pulse_new).sum(), (V * pulse_new * r2).sum()
            assert M0n == pytest.approx(M0, rel=1e-11)
            assert (M2n - M2) == pytest.approx(4 * Dc * dt * M0n, rel=1e-9)
            M0, M2 = M0n, M2n
            P.E_r = out["E_r"].copy()
        analytic = E0 / (4 * math.pi * Dc * t1) * np.exp(-r2 / (4 * Dc * t1))
        mask = analytic > 0.01 * analytic.max()
        errs.append(np.max(np.abs(P.E_r - 1.0 - analytic)[mask]) / analytic.max())
    assert errs[1] < 0.05
    assert 1.6 < errs[0] / errs[1] < 2.4


# ---------------------------------------------------------------------------
# boundaries: Milne outflow (Eq. milne) and free streaming
# ---------------------------------------------------------------------------

def test_milne_vacuum_flux_and_energy_balance(orc):
    """Eq. milne with lambda = 1/3 means the boundary flux is c E_b / 2 (a black absorber).
    The energy the grid loses in one step equals dt times the area-weighted boundary flux."""
    nx, ny, dx = 40, 3, 1e10
    sigma = 1e-9
    rng = np.random.default_rng(2)
    E = 1e4 * (1 + 0.3 * rng.random((ny, nx)))
    rho = 1e-10                     # gas energy << radiation energy: the balance is not lost in rounding
    P = _uniform_problem(nx, ny, dx, rho, 10.0, E, 3e3, kR=(sigma / rho, 0, 1, 0), kP=(0.0, 0, 1, 0),
                         bc=(0, 1, 0, 0), limiter=W.LIMITER_NONE)
    out = orc.step(P, "lu")
    Fb = out["Fx"][:, nx]
    assert np.all(Fb > 0)
    V = dx * dx
    lost = (out["energy_before"] - out["energy_after"])
    assert lost == pytest.approx(P.dt * dx * Fb.sum(), rel=1e-10)
    h = dx / 2
    Db = C_LIGHT / (3 * sigma)
    Eb = out["E_r"][:, -1] - Fb * h / Db          # face value from the flux over the half cell
    np.testing.assert_allclose(Fb, 0.5 * C_LIGHT * Eb, rtol=1e-10)
    assert V > 0


@pytest.mark.parametrize("kind", [W.LIMITER_LP, W.LIMITER_MINERBO])
def test_free_streaming_bound(orc, kind):
    """Optically thin, steep E: the limited flux never exceeds c E (Eq. asymptotic)."""
    rng = np.random.default_rng(8)
    nx, ny, dx = 30, 20, 1e12
    E = 10.0 ** rng.uniform(-2, 6, (ny, nx))
    P = _uniform_problem(nx, ny, dx, 1e-15, 1e4, E, 1e5, kR=(0.34, 0, 1, 0), kP=(0.34, 0, 1, 0),
                         limiter=kind, bc=(1, 1, 1, 1))
    fc = orc.faces(P)
    Fx = fc["Dx"][:, 1:-1] * np.abs(np.diff(E, axis=1)) / np.diff(W.uniform_faces(nx, dx))[0]
    assert np.all(Fx <= C_LIGHT * np.maximum(E[:, 1:], E[:, :-1]) * (1 + 1e-12))
    assert np.max(Fx / (C_LIGHT * np.maximum(E[:, 1:], E[:, :-1]))) > 0.3   # really streaming
    out = orc.step(P, "lu")
    En = out["E_r"]
    Fn = np.abs(out["Fx"][:, 1:-1])
    assert np.all(Fn <= C_LIGHT * np.maximum(En[:, 1:], En[:, :-1]))


# ---------------------------------------------------------------------------
# sub-cycling (Eq. subtimesteps)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,q", [(1, 1.3), (5, 1.4), (50, 1.2), (6, 1.0)])
def test_subcycle_series_fills_the_step(orc, n, q):
    """The sub-steps are a geometric series with ratio q that adds up to the hydro step."""
    dts = orc.subcycle_dts(3.7e4, n, q)
    assert len(dts) == n and min(dts) > 0
    assert math.fsum(dts) == pytest.approx(3.7e4, rel=1e-14)
    for a, b in zip(dts, dts[1:]):
        assert b / a == pytest.approx(q, rel=1e-13)


def test_subcycle_single_substep_is_one_step(orc):
    P = W.random_small(9, 7, W.CARTESIAN, (0, 1, 0, 0), 31)
    a = orc.step(P, "lu")
    b = orc.step_subcycled(P, 1, 1.3, freeze_D=False)
    for f in ("E_r", "T_g", "e_g"):
        assert np.array_equal(a[f], b[f])


def test_subcycle_conserves_energy_with_reflecting_walls(orc):
    P = W.random_small(12, 10, W.CARTESIAN, (0, 0, 0, 0), 32)
    out = orc.step_subcycled(P, 6, 1.3, freeze_D=False)
    assert abs(out["energy_after"] - out["energy_before"]) <= 1e-12 * out["energy_before"]


def test_subcycle_follows_the_ode_closer_than_one_step(orc):
    """Radiation-gas exchange in a uniform box (Sec. 5.1.1): one backward-Euler step of the
    whole interval overshoots the stiff exchange; 50 geometric sub-steps with q = 1.2 (the
    paper's choice for this test) stay close to the exact ODE."""
    g = _golden("coupling_test.txt")
    rho, kP, E0 = float(g["rho"][0]), float(g["kappa_P"][0]), float(g["E_r"][0])
    e0 = 1e10
    cv = rho * K_B / ((5.0 / 3.0 - 1.0) * float(g["mu"][0]) * M_H)
    dt = 2e-7
    P = _uniform_problem(2, 2, 1e10, rho, e0 / cv, E0, dt, kR=(kP, 0, 1, 0), kP=(kP, 0, 1, 0))
    P.e_g[:] = e0
    E_ode, e_ode = _ode(cv, rho * kP * C_LIGHT, e0, E0, np.array([0.0, dt]))
    one = orc.step(P, "lu")["e_g"][0, 0]
    sub = orc.step_subcycled(P, 50, 1.2, freeze_D=False)["e_g"][0, 0]
    err_one, err_sub = abs(one - e_ode[-1]) / e_ode[-1], abs(sub - e_ode[-1]) / e_ode[-1]
    assert err_sub < 0.2 * err_one, (err_one, err_sub)


def test_subcycled_flux_carries_the_lost_energy(orc):
    """The hydro step's flux (sub-step fluxes weighted by dt_i / dt): dt times the
    area-weighted flux through the Milne faces equals the energy the grid lost over all
    sub-steps, and reflecting faces carry none."""
    nx, ny, dx = 40, 3, 1e10
    sigma = 1e-9
    rng = np.random.default_rng(3)
    E = 1e4 * (1 + 0.3 * rng.random((ny, nx)))
    rho = 1e-10
    P = _uniform_problem(nx, ny, dx, rho, 10.0, E, 3e3, kR=(sigma / rho, 0, 1, 0), kP=(0.0, 0, 1, 0),
                         bc=(1, 1, 0, 0), limiter=W.LIMITER_NONE)
    out = orc.step_subcycled(P, 6, 1.4, freeze_D=False)
    lost = out["energy_before"] - out["energy_after"]
    through = P.dt * dx * (out["Fx"][:, nx].sum() - out["Fx"][:, 0].sum())
    assert lost > 0
    assert lost == pytest.approx(through, rel=1e-10)
    assert np.all(out["Fy"][0] == 0) and np.all(out["Fy"][-1] == 0)
