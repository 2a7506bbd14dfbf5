"""GPU tests of the algebraic-multigrid preconditioner (GQ_PRECOND_AMG): parity with the
FP64 oracle on the small random grids of test_gpu_parity (both precisions, both
geometries), on config 0, and inside a batch; reproducibility; and the iteration count on
a draw whose i.i.d. fields make the flux-limited face weights jump from cell to cell,
where the geometric 2 x 2 aggregation needs hundreds of iterations."""
import numpy as np
import pytest

from paper_2602_12545_gb300 import workloads as W
from test_gpu_batched import gate_for, within
from test_gpu_parity import (CASES, FP64_GATE, MIXED_GATE, check_parity, check_parity_conditioned,
                             componentwise_condition, run_gpu)

pytestmark = pytest.mark.gpu

AMG = 2


@pytest.fixture(scope="module")
def fld():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_12545_gb300 import build
    build.build()
    from paper_2602_12545_gb300 import fld as F
    return F


def small_case(nx, ny, coord):
    """The draw test_gpu_parity.test_small_grids uses for this shape."""
    seed = 100 + nx * 7 + ny * 13 + coord
    rng = np.random.default_rng(seed)
    bc = tuple(int(b) for b in rng.integers(0, 2, 4))
    limiter = int(rng.integers(0, 3))
    return W.random_small(nx, ny, coord, bc, seed, limiter=limiter)


@pytest.mark.parametrize("nx,ny,coord", CASES)
@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_MIXED])
def test_amg_small_grids(fld, orc, nx, ny, coord, prec):
    P = small_case(nx, ny, coord)
    ref = orc.step(P, "lu")
    cond = componentwise_condition(orc, P, ref["E_r"])
    rtol = 1e-12 if prec == W.PREC_FP64 else 1e-10
    out = run_gpu(fld, P, prec, rtol, precond=AMG)
    assert out["info"]["status"] in (0, 4), out["info"]
    check_parity_conditioned(out, ref, FP64_GATE if prec == W.PREC_FP64 else MIXED_GATE, cond,
                             label=f"amg small_grids {P.name} prec={prec}")


@pytest.mark.parametrize("prec,rtol,gate", [(W.PREC_FP64, 1e-12, FP64_GATE), (W.PREC_MIXED, 1e-10, MIXED_GATE)])
def test_amg_config0(fld, orc, prec, rtol, gate):
    P = W.config0()
    ref = orc.step(P, "lu")
    out = run_gpu(fld, P, prec, rtol, precond=AMG)
    assert out["info"]["status"] == 0
    check_parity(out, ref, gate)


def test_amg_cuts_iterations_on_jumping_coefficients(fld, orc):
    """130 x 33 spherical draw (dt 2.9e5 s): the aggregation V-cycle needs over a thousand
    iterations (its 2 x 2 aggregates cut the clusters of strongly coupled cells), the
    algebraic hierarchy a few dozen."""
    P = small_case(130, 33, W.SPHERICAL)
    ref = orc.step(P, "lu")
    cond = componentwise_condition(orc, P, ref["E_r"])
    a = run_gpu(fld, P, W.PREC_MIXED, 1e-10, precond=1)
    b = run_gpu(fld, P, W.PREC_MIXED, 1e-10, precond=AMG)
    check_parity_conditioned(b, ref, MIXED_GATE, cond, label="amg jumping coefficients 130x33")
    assert b["info"]["iterations"] * 10 < a["info"]["iterations"], (a["info"], b["info"])
    assert b["info"]["iterations"] < 100


def test_amg_deterministic(fld):
    P = small_case(67, 45, W.SPHERICAL)
    a = run_gpu(fld, P, W.PREC_MIXED, 1e-10, precond=AMG)
    b = run_gpu(fld, P, W.PREC_MIXED, 1e-10, precond=AMG)
    assert np.array_equal(a["E_r"], b["E_r"]) and a["info"]["iterations"] == b["info"]["iterations"]


def test_amg_in_batch(fld, orc):
    """Problems of the 256-problem batch (spherical draws among them) solved in one batched
    launch with the algebraic preconditioner; each member against the oracle."""
    F = fld
    probs = [P for P in W.config3(24, max_side=96)]
    plans = [F.FLDPlan.for_problem(P) for P in probs]
    fields = [F.device_fields(P) for P in probs]
    B = F.FLDBatch(plans, cells_per_block=2048, max_team=4)
    opts = [F.SolverOptions(prec=P.precision, limiter=P.limiter, rtol=1e-10, precond=AMG) for P in probs]
    rc, infos = B.step(probs, fields, opts_list=opts, check=False)
    assert rc in (0, 4)
    for P, f, info in zip(probs, fields, infos):
        assert info["status"] in (0, 4), (P.name, info)
        ref = orc.step(P, "lu")
        gate = gate_for(orc, P, ref["E_r"])
        assert within(f[2].cpu().numpy(), ref["E_r"], gate, P, f"amg batch {P.name} E", info["status"]) and \
            within(f[3].cpu().numpy(), ref["T_g"], gate, P, f"amg batch {P.name} T", info["status"]), (P.name, info)
    B.close()
    for p in plans:
        p.close()
