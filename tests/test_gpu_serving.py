"""GPU tests of continuous-batching serving: each result is the same alone and in the mix
(within the parity tolerance), admission respects the memory budget, a failing request
does not disturb the others, and requests that arrive while others are resident join
the running batch."""
import numpy as np
import pytest

from paper_2602_12545_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srvmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_12545_gb300 import build
    build.build()
    from paper_2602_12545_gb300 import serve
    return serve


def reqs(n, seed=5, lo=16, hi=160):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        side = int(rng.integers(lo, hi))
        out.append(W.ServeRequest(i, 0.0, side, int(rng.integers(1, 4)), seed * 100 + i))
    return out


def relerr(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def drain(srv, ids):
    res = {}
    for _ in range(10000):
        if len(res) == len(ids):
            break
        srv.poll()
        for rid in ids:
            if rid not in res:
                got = srv.take(rid)
                if got is not None:
                    res[rid] = got
    assert len(res) == len(ids)
    return res


def test_alone_equals_in_the_mix(srvmod):
    S = srvmod
    rs = reqs(7)
    probs = [W.serve_problem(r) for r in rs]
    mix = S.FLDServer(budget_bytes=8 << 30)
    ids = [mix.submit(P, r.n_steps) for P, r in zip(probs, rs)]
    res_mix = drain(mix, ids)
    mix.close()
    for rid, P, r in zip(ids, probs, rs):
        alone = S.FLDServer(budget_bytes=8 << 30)
        a = alone.submit(P, r.n_steps)
        (E1, eg1, T1), cells, info1 = drain(alone, [a])[a]
        alone.close()
        (E0, eg0, T0), _, info0 = res_mix[rid]
        assert info0["status"] == 0 and info1["status"] == 0
        assert info0["steps_done"] == r.n_steps
        for x, y in ((E0, E1), (T0, T1), (eg0, eg1)):
            assert relerr(x, y) <= 1e-8


def test_budget_admission_and_rejection(srvmod):
    S = srvmod
    rs = reqs(5, seed=9, lo=60, hi=70)
    probs = [W.serve_problem(r) for r in rs]
    one = max(S.FLDServer.request_bytes(P.nx, P.ny) for P in probs)
    srv = S.FLDServer(budget_bytes=int(one * 1.5))      # room for one resident request
    ids = [srv.submit(P, 2) for P in probs]
    seen_max = 0
    res = {}
    for _ in range(1000):
        if len(res) == len(ids):
            break
        srv.poll()
        seen_max = max(seen_max, srv.used_bytes)
        for rid in ids:
            if rid not in res:
                got = srv.take(rid)
                if got is not None:
                    res[rid] = got
    assert len(res) == len(ids)
    assert seen_max <= one * 1.5
    infos = [res[i][2] for i in ids]
    for a, b in zip(infos, infos[1:]):              # served one after another, in order
        assert b["admit_s"] >= a["done_s"] - 1e-6
    big = W.serve_problem(W.ServeRequest(99, 0.0, 400, 1, 7))
    from paper_2602_12545_gb300 import _native as N
    with pytest.raises(N.GQError) as e:
        srv.submit(big, 1)
    assert e.value.code == N.GQ_ERR_BUDGET
    srv.close()


def test_failing_request_is_isolated(srvmod):
    S = srvmod
    rs = reqs(4, seed=3)
    probs = [W.serve_problem(r) for r in rs]
    probs[1].rho[2, 2] = float("nan")
    srv = S.FLDServer(budget_bytes=8 << 30)
    ids = [srv.submit(P, r.n_steps) for P, r in zip(probs, rs)]
    res = drain(srv, ids)
    assert res[ids[1]][2]["status"] == 5
    assert all(res[i][2]["status"] == 0 for k, i in enumerate(ids) if k != 1)
    srv.close()


def test_late_arrivals_join_resident_work(srvmod):
    S = srvmod
    first = W.serve_problem(W.ServeRequest(0, 0.0, 120, 1, 11))
    srv = S.FLDServer(budget_bytes=8 << 30)
    a = srv.submit(first, 6)
    srv.poll()                                        # a is resident and has taken a step
    b = srv.submit(W.serve_problem(W.ServeRequest(1, 0.0, 40, 1, 12)), 2)
    res = drain(srv, [a, b])
    ia, ib = res[a][2], res[b][2]
    assert ib["admit_s"] < ia["done_s"]               # b ran while a was resident
    assert ib["done_s"] < ia["done_s"]                # and finished first (fewer steps)
    srv.close()


def test_trace_replay_reports_latency(srvmod):
    S = srvmod
    trace = W.config4_trace(n_requests=12, rate_per_s=200.0, side_lo=32, side_hi=96, n_steps=2)
    out = S.run_trace(trace, budget_bytes=4 << 30)
    assert out["requests"] == 12 and out["failed"] == 0
    assert 0 < out["latency_p50_s"] <= out["latency_p99_s"]
    assert out["throughput_cell_updates_per_s"] > 0
