"""GPU tests of the batched path: every member of a batch equals its solo step (and the
oracle) within the parity tolerance; graph replay equals eager launch; the autotuner
keeps results unchanged; per-problem statuses stay independent."""
import numpy as np
import pytest

from paper_2602_12545_gb300 import workloads as W
from parity_gate import componentwise_condition, conditioned_gate, within_conditioned

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


def relerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b))))


def plain_gate(P):
    return 1e-10 if P.precision == W.PREC_FP64 else 1e-8


def gate_for(orc, P, E_ref):
    """max(stated tolerance, 16 eps x componentwise condition number) per cell (the
    conditioned gate of parity_gate)."""
    return conditioned_gate(plain_gate(P), componentwise_condition(orc, P, E_ref))


def within(a, b, gate, P=None, label="", status=None):
    """Element-wise within the per-cell gate; with P given, the widening is reported and
    bounded against P's stated tolerance."""
    if P is not None:
        return within_conditioned(a, b, gate, plain_gate(P), label=label, status=status)
    return bool(np.all(np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b)) <= gate))


OK = (0, 4)    # GQ_OK, or GQ_ERR_NOT_CONVERGED at the FP64 floor of an ill-conditioned draw


def small_batch(n=12, seed=50):
    """Uneven sizes, both geometries, both precisions, mixed boundaries and limiters."""
    rng = np.random.default_rng(seed)
    probs = []
    for p in range(n):
        nx, ny = int(rng.integers(1, 90)), int(rng.integers(1, 70))
        coord = p % 2
        bc = tuple(int(b) for b in rng.integers(0, 2, 4))
        P = W.random_small(nx, ny, coord, bc, seed + p, limiter=int(rng.integers(0, 3)))
        P.precision = W.PREC_MIXED if p % 3 else W.PREC_FP64
        P.rtol = 1e-12 if P.precision == W.PREC_FP64 else 1e-10
        probs.append(P)
    return probs


def solo(F, P):
    plan = F.FLDPlan.for_problem(P)
    f = F.device_fields(P)
    info = F.step_problem(plan, P, *f, check=False)
    assert info["status"] in OK
    out = [t.cpu().numpy() for t in f[1:]]
    plan.close()
    return out, info


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_members_match_solo_and_oracle(fld, orc, use_graph):
    F = fld
    probs = small_batch()
    plans = [F.FLDPlan.for_problem(P) for P in probs]
    fields = [F.device_fields(P) for P in probs]
    B = F.FLDBatch(plans, cells_per_block=2048, max_team=4, use_graph=use_graph)
    rc, infos = B.step(probs, fields, check=False)
    assert rc in OK
    for P, f, info in zip(probs, fields, infos):
        assert info["status"] in OK, (P.name, info)
        ref = orc.step(P, "lu")
        gate = gate_for(orc, P, ref["E_r"])
        eg, E, T = (t.cpu().numpy() for t in f[1:])
        lab = f"batch graph={use_graph} {P.name}"
        assert within(E, ref["E_r"], gate, P, lab + " E", info["status"]) and \
            within(T, ref["T_g"], gate, P, lab + " T", info["status"]), (P.name, info)
        (seg, sE, sT), sinfo = solo(F, P)
        assert within(E, sE, 2 * gate) and within(T, sT, 2 * gate)
    assert B.uses_graph == use_graph
    B.close()
    for p in plans:
        p.close()


def test_graph_replay_equals_eager_and_repeats(fld):
    import torch
    F = fld
    probs = small_batch(8, seed=70)
    plans = [F.FLDPlan.for_problem(P) for P in probs]
    f0 = [F.device_fields(P) for P in probs]
    results = []
    for use_graph in (False, True):
        B = F.FLDBatch(plans, cells_per_block=1024, max_team=8, use_graph=use_graph)
        for rep in range(2):           # replay twice: identical inputs give identical outputs
            fields = [(r, e.clone(), E.clone(), T.clone()) for (r, e, E, T) in f0]
            B.step(probs, fields, check=False)
            results.append([E.cpu().numpy() for (_, _, E, _) in fields])
        B.close()
    for r in results[1:]:
        for a, b in zip(results[0], r):
            assert np.array_equal(a, b)
    for p in plans:
        p.close()


def test_autotune_keeps_results(fld, orc):
    F = fld
    probs = small_batch(10, seed=90)
    plans = [F.FLDPlan.for_problem(P) for P in probs]
    fields = [F.device_fields(P) for P in probs]
    E0 = [f[2].clone() for f in fields]
    B = F.FLDBatch(plans)
    best = B.autotune(probs, fields)
    assert best["cells_per_block"] > 0 and best["max_team"] > 0 and best["ms"] > 0
    for f, e in zip(fields, E0):                 # inputs restored by the autotuner
        assert np.array_equal(f[2].cpu().numpy(), e.cpu().numpy())
    rc, infos = B.step(probs, fields, check=False)
    assert rc in OK
    for P, f in zip(probs, fields):
        (seg, sE, sT), _ = solo(F, P)
        ref = orc.step(P, "lu")
        assert within(f[2].cpu().numpy(), sE, 2 * gate_for(orc, P, ref["E_r"]))
    B.close()
    for p in plans:
        p.close()


def test_per_problem_status_independent(fld):
    """A bad input in one problem reports on that problem only; the others are solved."""
    F = fld
    probs = small_batch(6, seed=30)
    plans = [F.FLDPlan.for_problem(P) for P in probs]
    fields = [F.device_fields(P) for P in probs]
    fields[2][0].view(-1)[0] = -1.0
    B = F.FLDBatch(plans, cells_per_block=2048, max_team=4)
    rc, infos = B.step(probs, fields, check=False)
    assert rc == 1 and infos[2]["status"] == 1
    assert all(i["status"] in OK for k, i in enumerate(infos) if k != 2)
    B.close()
    for p in plans:
        p.close()
