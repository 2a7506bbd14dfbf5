"""GPU parity of the multilevel (SMR) step, Sec. 3.2.2 (Eq. linearsys1_amr): one implicit
FLD step over a two-level Cartesian grid (a 2:1 refined rectangle) through the C ABI
(gq_smr_step), against the multilevel oracle (oracle/smr.py, assembled explicitly and
solved directly), element by element in composite order.

Cases: the patch inside the grid, against a Milne side, in a corner with Milne sides all
round, no patch and the whole grid refined; FP64 (rtol 1e-12, gate 1e-10) and mixed
(rtol 1e-10, gate 1e-8) with the conditioned gate of parity_gate; energy conservation
with reflecting sides; bad grids and inputs rejected."""
import numpy as np
import pytest

from paper_2602_12545_gb300 import workloads as W
from parity_gate import check_parity_conditioned

pytestmark = pytest.mark.gpu

KW = dict(kR=W.KRAMERS_LIKE, kP=W.KRAMERS_LIKE, gamma=5.0 / 3.0, mu=0.6)


@pytest.fixture(scope="module")
def fld():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_12545_gb300 import build
    build.build()
    from paper_2602_12545_gb300 import fld as F
    return F


def _fields(n, seed):
    """Config-0 statistics per composite cell."""
    rng = np.random.default_rng(seed)
    rho = 1e-9 * 10.0 ** (1.5 * rng.standard_normal(n))
    T = 10.0 ** rng.uniform(3.0, 5.0, n)
    E = W.A_RAD_RECIPE * (T * np.maximum(1.0 + 0.1 * rng.standard_normal(n), 1e-3)) ** 4
    return rho, rho * T * W.EG_PER_RHO_T, E


def _skeel(A, x):
    import scipy.sparse.linalg as spla
    return spla.spsolve(A.tocsc(), abs(A) @ x) / x


def _run(F, geom, bc, dt, lim, prec, rtol, seed):
    import torch
    from oracle import smr
    nx, ny, h, i0, i1, j0, j1 = geom
    g = smr.Composite(nx, ny, h, h, i0, i1, j0, j1)
    n = len(smr.cells(g)["x"])
    rho, eg, E = _fields(n, seed)
    ref = smr.step(g, rho, eg, E, dt=dt, bc=bc, lim=lim, **KW)
    plan = F.SMRPlan(nx, ny, h, h, i0, i1, j0, j1)
    assert plan.cells == n
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    r_, e_, E_ = d(rho), d(eg), d(E)
    T_ = torch.empty_like(E_)
    opts = F.SolverOptions(prec=prec, limiter=lim, rtol=rtol)
    info = plan.step(r_, e_, E_, T_, opacity_R=KW["kR"], opacity_P=KW["kP"], gamma=KW["gamma"], mu=KW["mu"],
                     dt=dt, bc=bc, opts=opts, check=False)
    torch.cuda.synchronize()
    out = {"E_r": E_.cpu().numpy(), "T_g": T_.cpu().numpy(), "e_g": e_.cpu().numpy(), "info": info}
    plan.close()
    return out, ref


GEOMS = {
    "inside": (24, 18, 1e12, 8, 16, 5, 12),
    "on_milne_side": (20, 16, 1e12, 12, 20, 4, 10),
    "corner": (16, 16, 1e12, 0, 6, 0, 5),
    "none": (17, 11, 1e12, 0, 0, 0, 0),
    "all": (9, 7, 2e12, 0, 9, 0, 7),
    "wide": (96, 64, 5e11, 30, 70, 10, 40),
}
CASES = [("inside", (0, 0, 0, 0)), ("on_milne_side", (0, 1, 0, 0)), ("corner", (1, 1, 1, 1)),
         ("none", (1, 0, 1, 0)), ("all", (0, 1, 1, 0)), ("wide", (0, 1, 0, 1))]


@pytest.mark.parametrize("name,bc", CASES)
@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_MIXED])
def test_smr_step_matches_oracle(fld, name, bc, prec):
    seed = 500 + sum(map(ord, name))
    lim = seed % 3
    dt = 10.0 ** (3.0 + (seed % 7) / 2.0)
    out, ref = _run(fld, GEOMS[name], bc, dt, lim, prec, 1e-12 if prec == W.PREC_FP64 else 1e-10, seed)
    assert out["info"]["status"] in (0, 4), out["info"]
    cond = _skeel(ref["A"], ref["E_r"])
    check_parity_conditioned(out, ref, 1e-10 if prec == W.PREC_FP64 else 1e-8, cond,
                             label=f"smr {name} bc={bc} prec={prec}")
    assert out["info"]["energy_before"] == pytest.approx(ref["energy_before"], rel=1e-13)
    if bc == (0, 0, 0, 0):
        e0, e1 = out["info"]["energy_before"], out["info"]["energy_after"]
        assert abs(e1 - e0) <= 1e-12 * e0


def test_smr_without_patch_is_the_single_level_step(fld):
    """No refined rectangle: the composite step is the single-level step (gq_fld_step) on
    the base grid, cell for cell, in both precisions."""
    import torch
    nx, ny, h = 33, 21, 1e12
    rho, eg, E = _fields(nx * ny, 17)
    P = W.FLDProblem("smr_base", W.CARTESIAN, W.uniform_faces(nx, h), W.uniform_faces(ny, h), rho.reshape(ny, nx),
                     eg.reshape(ny, nx), E.reshape(ny, nx), 3e4, bc=(1, 0, 0, 1))
    for prec, rtol, gate in ((W.PREC_FP64, 1e-12, 1e-10), (W.PREC_MIXED, 1e-10, 1e-8)):
        plan = fld.FLDPlan.for_problem(P)
        f = fld.device_fields(P)
        fld.step_problem(plan, P, *f, prec=prec, rtol=rtol, precond=0)
        plan.close()
        out, ref = _run(fld, (nx, ny, h, 0, 0, 0, 0), P.bc, P.dt, P.limiter, prec, rtol, 17)
        for got, want in ((out["E_r"], f[2].cpu().numpy().ravel()), (out["T_g"], f[3].cpu().numpy().ravel())):
            assert np.max(np.abs(got - want) / np.abs(want)) <= 2 * gate


def test_smr_rejects_bad_inputs(fld):
    import torch
    from paper_2602_12545_gb300 import _native as N
    from oracle import smr
    for bad in ((0, 4, 1e12, 0, 0, 0, 0), (4, 4, -1.0, 0, 0, 0, 0), (4, 4, 1e12, 2, 5, 0, 2),
                (4, 4, 1e12, 3, 1, 0, 2), (4, 4, 1e12, 0, 2, -1, 2)):
        nx, ny, h, i0, i1, j0, j1 = bad
        with pytest.raises(N.GQError) as e:
            fld.SMRPlan(nx, ny, h, h, i0, i1, j0, j1)
        assert e.value.code == N.GQ_ERR_INVALID_ARG
    g = smr.Composite(8, 6, 1e12, 1e12, 2, 5, 1, 4)
    n = len(smr.cells(g)["x"])
    plan = fld.SMRPlan(8, 6, 1e12, 1e12, 2, 5, 1, 4)
    rho, eg, E = (torch.from_numpy(a).cuda() for a in _fields(n, 3))
    rho[5] = -1.0
    E0 = E.clone()
    info = plan.step(rho, eg, E, None, opacity_R=KW["kR"], opacity_P=KW["kP"], gamma=KW["gamma"], mu=KW["mu"],
                     dt=1e4, bc=(0, 0, 0, 0), opts=fld.SolverOptions(), check=False)
    assert info["status"] == N.GQ_ERR_INVALID_ARG
    assert torch.equal(E, E0)
    plan.close()
