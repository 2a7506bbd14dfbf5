"""Pins of the multilevel (SMR) oracle, Sec. 3.2.2 (Eq. linearsys1_amr), against things
other than itself:

- with no refined patch it is the single-level oracle on the base grid, and with the
  whole domain refined it is the single-level oracle on the fine grid (the C oracle,
  pinned on its own);
- a coarse cell beside the patch has five neighbours, the fine cells across from it one
  coarse neighbour each;
- the matrix is symmetric and, with reflecting sides, the step conserves E + e_g;
- for E linear along x, constant kappa_R, no limiting and no coupling, every cell away
  from the x sides receives zero net flux across a stripe of fine cells (the normal
  differences are exact for a linear field).
"""
import numpy as np
import pytest

from paper_2602_12545_gb300 import workloads as W

KB = 1.380649e-16
MH = 1.00782503207 * 1.66053906660e-24


def _fields(n, seed):
    rng = np.random.default_rng(seed)
    rho = 1e-9 * 10.0 ** (1.5 * rng.standard_normal(n))
    T = 10.0 ** rng.uniform(3.0, 5.0, n)
    E = W.A_RAD_RECIPE * (T * np.maximum(1.0 + 0.1 * rng.standard_normal(n), 1e-3)) ** 4
    return rho, rho * T * W.EG_PER_RHO_T, E


KW = dict(kR=W.KRAMERS_LIKE, kP=W.KRAMERS_LIKE, gamma=5.0 / 3.0, mu=0.6, dt=1e5, lim=W.LIMITER_LP)


def _uniform(nx, ny, h, rho, eg, E, bc):
    xf = W.uniform_faces(nx, h)
    yf = W.uniform_faces(ny, h)
    return W.FLDProblem(name="u", coord=W.CARTESIAN, x_faces=xf, y_faces=yf, rho=rho.reshape(ny, nx),
                        e_g=eg.reshape(ny, nx), E_r=E.reshape(ny, nx), dt=KW["dt"], bc=bc)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 0, 1, 1)])
def test_no_patch_is_the_single_level_step(orc, bc):
    from oracle import smr
    g = smr.Composite(9, 7, 1e12, 1e12, 0, 0, 0, 0)
    rho, eg, E = _fields(63, 1)
    out = smr.step(g, rho, eg, E, bc=bc, **KW)
    ref = orc.step(_uniform(9, 7, 1e12, rho, eg, E, bc))
    for f in ("E_r", "T_g", "e_g"):
        assert np.allclose(out[f], ref[f].ravel(), rtol=1e-12, atol=0), f


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (0, 1, 1, 0)])
def test_whole_domain_refined_is_the_fine_grid_step(orc, bc):
    from oracle import smr
    g = smr.Composite(5, 4, 2e12, 2e12, 0, 5, 0, 4)
    rho, eg, E = _fields(10 * 8, 2)
    out = smr.step(g, rho, eg, E, bc=bc, **KW)
    ref = orc.step(_uniform(10, 8, 1e12, rho, eg, E, bc))
    for f in ("E_r", "T_g", "e_g"):
        assert np.allclose(out[f], ref[f].ravel(), rtol=1e-12, atol=0), f


def test_coarse_cells_beside_the_patch_have_five_neighbours():
    from oracle import smr
    g = smr.Composite(8, 6, 1.0, 1.0, 3, 5, 2, 4)
    c = smr.cells(g)
    n = len(c["x"])
    rho, eg, E = _fields(n, 3)
    A = smr.step(g, rho, eg, E, bc=(0,) * 4, **KW)["A"].tocsr()
    nnz = np.diff(A.indptr)
    beside = [c["coarse"][2, 2], c["coarse"][2, 5], c["coarse"][1, 3], c["coarse"][4, 4]]
    for k in beside:
        assert nnz[k] == 6, (k, nnz[k])       # diagonal + 3 coarse + 2 fine neighbours
    assert nnz[c["coarse"][0, 0]] == 3          # a domain corner
    F = c["fine"]
    assert nnz[F[0, 0]] == 5      # the patch's lower-left fine cell: 2 fine + 2 coarse neighbours
    assert nnz[F[1, 1]] == 5      # a fine cell with four fine neighbours


def test_symmetric_and_conservative():
    from oracle import smr
    g = smr.Composite(10, 8, 1e12, 1e12, 2, 7, 3, 6)
    n = len(smr.cells(g)["x"])
    rho, eg, E = _fields(n, 4)
    out = smr.step(g, rho, eg, E, bc=(0,) * 4, **KW)
    A = out["A"]
    assert abs(A - A.T).max() == 0.0
    assert out["energy_after"] == pytest.approx(out["energy_before"], rel=1e-12)


def test_linear_field_has_no_net_flux_across_a_stripe():
    from oracle import smr
    g = smr.Composite(12, 5, 1e11, 1e11, 4, 8, 0, 5)
    c = smr.cells(g)
    n = len(c["x"])
    rho = np.full(n, 1e-9)
    E = 1e3 * (1.0 + 0.02 * c["x"] / 1e11)
    eg = rho * 1e4 * W.EG_PER_RHO_T
    kw = dict(KW, kR=(0.4, 0.0, 0.0, 0.0), kP=(0.0, 0.0, 0.0, 0.0), lim=W.LIMITER_NONE)
    out = smr.step(g, rho, eg, E, bc=(0,) * 4, **kw)
    A = out["A"].tocsr()
    V = c["hx"] * c["hy"]
    net = A @ E - V * E                     # the face terms only (no coupling: the mass term is V)
    scale = (abs(A) @ E - V * E)            # the sum of |w| |E| over the row
    away = (c["x"] - 0.5 * c["hx"] > 1e-3 * g.dx) & (c["x"] + 0.5 * c["hx"] < g.nx * g.dx * (1 - 1e-12))
    assert away.sum() > 0
    assert np.all(np.abs(net[away]) <= 1e-12 * scale[away])
    assert np.abs(net[~away]).max() > 1e-6 * scale[~away].max()
