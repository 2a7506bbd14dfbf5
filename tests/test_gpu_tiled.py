"""GPU checks of the tiled solve kernel (k_pcg_tiled: the aggregation V-cycle's levels run
as two fused shared-memory passes each, gq_pcg_tiled.cu) on problems it takes: against
the oracle element by element (conditioned gate, mixed precision 1e-8), and against the
untiled kernel (same cycle, different pass boundaries and reduction order), including a
grid whose width and height leave partial tiles, Milne sides and a loose refinement
trigger."""
import numpy as np
import pytest

from paper_2602_12545_gb300 import workloads as W
from parity_gate import check_parity_conditioned, componentwise_condition

pytestmark = pytest.mark.gpu

MIXED_GATE = 1e-8


@pytest.fixture(scope="module")
def fld():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_12545_gb300 import build
    build.build()
    from paper_2602_12545_gb300 import fld as F
    return F


def run(F, P, untiled, rtol=1e-10, **kw):
    import torch
    plan = F.FLDPlan.for_problem(P)
    rho, e_g, E, T = F.device_fields(P)
    info = F.step_problem(plan, P, rho, e_g, E, T, prec=W.PREC_MIXED, rtol=rtol, precond=1, untiled=untiled,
                          check=False, **kw)
    torch.cuda.synchronize()
    out = {"E_r": E.cpu().numpy(), "T_g": T.cpu().numpy(), "e_g": e_g.cpu().numpy(), "info": info}
    plan.close()
    return out


def cases():
    out = []
    # the spherical benchmark field on 256 x 128 (team levels 256, 128, 64 wide)
    out.append(("sph256x128", W.config2(nr=256, nth=128)))
    # partial tiles in both directions (352 = 5.5 tiles, 40 = 2.5 tiles), Milne at +x, -y
    P = W.random_small(352, 40, W.CARTESIAN, (0, 1, 1, 0), 91, dt=1e4)
    out.append(("cart352x40", P))
    # spherical with Milne at outer r and both poles reflecting, 512 x 256
    out.append(("sph512x256", W.config2(seed=1702, nr=512, nth=256)))
    return out


@pytest.mark.parametrize("name,P", cases(), ids=[c[0] for c in cases()])
def test_tiled_matches_oracle_and_untiled(fld, orc, name, P):
    a = run(fld, P, untiled=0)
    b = run(fld, P, untiled=1)
    assert a["info"]["status"] in (0, 4) and b["info"]["status"] in (0, 4), (a["info"], b["info"])
    assert a["info"]["solve_kernel"] == 1 and b["info"]["solve_kernel"] == 0
    ref = orc.step(P, "lu") if P.ncells <= 20000 else orc.step(P, "cg", tol=1e-14)
    cond = componentwise_condition(orc, P, ref["E_r"]) if P.ncells <= 20000 else np.ones_like(ref["E_r"])
    check_parity_conditioned(a, ref, MIXED_GATE, cond, label=f"tiled {name}")
    check_parity_conditioned(b, ref, MIXED_GATE, cond, label=f"untiled {name}")
    # the same preconditioner: comparable iteration counts
    ia, ib = a["info"]["iterations"], b["info"]["iterations"]
    assert abs(ia - ib) <= max(3, 0.25 * ib), (ia, ib)


def test_tiled_loose_refinement_trigger(fld, orc):
    """Frequent FP64 refinements (inner_rtol 0.3): each restarts the fused update from the
    refreshed residual; the solve must still converge to parity."""
    P = W.config2(nr=256, nth=128)
    out = run(fld, P, untiled=0, rtol=1e-11, inner_rtol=0.3)
    assert out["info"]["status"] == 0, out["info"]
    ref = orc.step(P, "cg", tol=1e-14)
    for f in ("E_r", "T_g", "e_g"):
        err = float(np.max(np.abs(out[f] - ref[f]) / np.abs(ref[f])))
        assert err <= MIXED_GATE, (f, err)


def test_tiled_deterministic(fld):
    P = W.config2(nr=256, nth=128)
    a = run(fld, P, untiled=0)
    b = run(fld, P, untiled=0)
    assert np.array_equal(a["E_r"], b["E_r"]) and a["info"]["iterations"] == b["info"]["iterations"]
