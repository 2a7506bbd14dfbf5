"""GPU parity of the explicit radiation advection (Sec. 3.2.1, Eq. adv): the source kernel
against the oracle's S_adv, steps with the source attached (single and sub-cycled, both
precisions, both geometries), the dynamical-diffusion set-up of Sec. 5 stepped on both
sides, and the rejection of a source that would make E^n + S_adv dt non-positive."""
import dataclasses

import numpy as np
import pytest

from paper_2602_12545_gb300 import workloads as W
from test_gpu_parity import (FP64_GATE, MIXED_GATE, check_parity_conditioned, componentwise_condition, relerr,
                             run_gpu)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fld():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_12545_gb300 import build
    build.build()
    from paper_2602_12545_gb300 import fld as F
    return F


def _case(coord):
    P = W.random_small(45, 37, coord, (0, 1, 0, 1), 500 + coord)
    fx, fy = W.mass_fluxes(P, 600 + coord)
    return P, fx, fy


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("coord", [W.CARTESIAN, W.SPHERICAL])
def test_adv_source_parity(fld, orc, coord):
    P, fx, fy = _case(coord)
    plan = fld.FLDPlan.for_problem(P)
    rho, e_g, E, T = fld.device_fields(P)
    S = plan.adv_source(rho, E, _dev(fx), _dev(fy)).cpu().numpy()
    want = orc.adv_source(P, fx, fy)
    assert np.isfinite(S).all()
    # a sum of four face terms of either sign: gated against the largest source
    assert np.abs(S - want).max() <= 1e-12 * np.abs(want).max()
    plan.close()


@pytest.mark.parametrize("coord", [W.CARTESIAN, W.SPHERICAL])
@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_MIXED])
def test_step_with_source(fld, orc, coord, prec):
    P, fx, fy = _case(coord)
    P = dataclasses.replace(P, S_adv=orc.adv_source(P, fx, fy))
    ref = orc.step(P, "lu")
    cond = componentwise_condition(orc, P, ref["E_r"])
    out = run_gpu(fld, P, prec, 1e-12 if prec == W.PREC_FP64 else 1e-10)
    assert out["info"]["status"] == 0, out["info"]
    check_parity_conditioned(out, ref, FP64_GATE if prec == W.PREC_FP64 else MIXED_GATE, cond,
                             label=f"adv step coord={coord} prec={prec}")
    # the same step without the source lands elsewhere
    assert relerr(out["E_r"], orc.step(dataclasses.replace(P, S_adv=None), "lu")["E_r"]) > 1e-6


def test_subcycled_step_with_source(fld, orc):
    """Cartesian draw: each sub-step's E + S_adv dt_i stays above 0.69 E (checked below on
    the oracle's sub-steps).  On the spherical draw the coupling drops E a hundredfold in
    some cells within the first sub-step, so the source held from E^n exceeds E there and
    the library rejects the sub-step (GQ_ERR_INVALID_ARG)."""
    P, fx, fy = _case(W.CARTESIAN)
    P = dataclasses.replace(P, S_adv=orc.adv_source(P, fx, fy))
    Q = P
    for dt in orc.subcycle_dts(P.dt, 4, 1.3):
        assert ((Q.E_r + P.S_adv * dt) / Q.E_r).min() > 0.5
        o = orc.step(dataclasses.replace(Q, dt=dt), "lu")
        Q = dataclasses.replace(Q, E_r=o["E_r"], e_g=o["e_g"])
    ref = orc.step_subcycled(P, 4, 1.3, freeze_D=False)
    cond = componentwise_condition(orc, P, ref["E_r"])
    out = run_gpu(fld, P, W.PREC_FP64, 1e-12, n_sub=4, q_t=1.3, subcycle_freeze_D=0)
    assert out["info"]["status"] == 0, out["info"]
    check_parity_conditioned(out, ref, FP64_GATE, cond, label="adv subcycled")


def test_advected_packet_steps(fld, orc):
    """Sec. 5 dynamical diffusion on 1024 cells at CFL 1 with the Levermore-Pomraning
    limiter: 40 steps, each computing S_adv from the current E on the device, attaching
    it and stepping; the oracle does the same on the CPU.  Gate: the cell-wise stop rule
    |r_k| <= rtol A_kk |x_k| leaves a relative error of at most rtol (A^-1 diag(A) |x|)_k / x_k
    per step (A is an M-matrix, so A^-1 >= 0); the test sums its maximum over the steps
    (about 1.1e-10 here) and allows twice that."""
    import torch
    P, fx, fy = W.advected_packet(cfl=1.0)
    n, rtol = 40, 1e-12
    Q = P
    bound = 0.0
    for _ in range(n):
        Qs = dataclasses.replace(Q, S_adv=orc.adv_source(Q, fx, fy))
        o = orc.step(Qs, "lu")
        A, _ = orc.assemble_reduced(Qs)
        x = o["E_r"].ravel()
        bound += (orc.band_solve(A, A.diagonal() * np.abs(x)) / x).max()
        Q = dataclasses.replace(Q, E_r=o["E_r"], e_g=o["e_g"])
    plan = fld.FLDPlan.for_problem(P)
    rho, e_g, E, T = fld.device_fields(P)
    fxd, fyd = _dev(fx), _dev(fy)
    S = torch.empty_like(E)
    opts = fld.SolverOptions(prec=W.PREC_FP64, limiter=P.limiter, rtol=rtol)
    for _ in range(n):
        plan.adv_source(rho, E, fxd, fyd, out=S)
        plan.set_source(S)
        plan.step(rho, e_g, E, T, opacity_R=P.opacity_R, opacity_P=P.opacity_P, gamma=P.gamma, mu=P.mu,
                  dt=P.dt, bc=P.bc, opts=opts)
    plan.set_source(None)
    torch.cuda.synchronize()
    assert relerr(E.cpu().numpy(), Q.E_r) <= max(FP64_GATE, 2.0 * rtol * bound)
    plan.close()


def test_source_making_E_nonpositive_rejected(fld, orc):
    """E^n + S_adv dt <= 0 in one cell: GQ_ERR_INVALID_ARG before the solve, fields kept."""
    import torch
    P, fx, fy = _case(W.CARTESIAN)
    S = np.zeros_like(P.E_r)
    S[5, 7] = -2.0 * P.E_r[5, 7] / P.dt
    plan = fld.FLDPlan.for_problem(P)
    rho, e_g, E, T = fld.device_fields(P)
    E0 = E.clone()
    info = fld.step_problem(plan, dataclasses.replace(P, S_adv=S), rho, e_g, E, T, check=False)
    assert info["status"] == 1
    torch.cuda.synchronize()
    assert torch.equal(E, E0)
    plan.close()
