"""The allocation-free step (gq_fld_step_noalloc) against the plan-based step.

Callers that cannot allocate device memory (hosts whose device memory is fixed at
start-up, plug-ins inside another application's memory manager, loops that cannot afford
the device synchronisation of cudaMalloc / cudaFree) use this entry point; it keeps all
scratch in one static device array.  This test calls it through the C ABI and
checks its output against gq_fld_step's on the same inputs, within the parity tolerances
used elsewhere (1e-10 FP64, 1e-8 mixed), on two calls in a row (the second reuses the
array the first left behind).  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2602_12545_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_12545_gb300 import build
    build.build()
    from paper_2602_12545_gb300 import _native as N
    from paper_2602_12545_gb300 import fld as F
    return torch, N, F


def noalloc_step(torch, N, F, P, prec, rtol):
    L = N.load()
    xf = torch.from_numpy(P.x_faces).cuda()
    yf = torch.from_numpy(P.y_faces).cuda()
    rho, e_g, E, T = F.device_fields(P)
    op = N.OpacityLaw(*[float(v) for v in tuple(P.opacity_R) + tuple(P.opacity_P)])
    eos = N.Eos(float(P.gamma), float(P.mu))
    bc = N.Bc()
    for s in range(4):
        bc.side[s] = int(P.bc[s])
    o = F.SolverOptions(prec=prec, limiter=P.limiter, rtol=rtol).to_c()
    info = N.StepInfo()
    st = torch.cuda.current_stream().cuda_stream
    rc = L.gq_fld_step_noalloc(P.nx, P.ny, int(P.coord), xf.data_ptr(), yf.data_ptr(), rho.data_ptr(),
                               e_g.data_ptr(), E.data_ptr(), T.data_ptr(), ctypes.byref(op), ctypes.byref(eos),
                               float(P.dt), ctypes.byref(bc), ctypes.byref(o), ctypes.c_void_p(st),
                               ctypes.byref(info))
    return rc, E.cpu().numpy(), T.cpu().numpy(), e_g.cpu().numpy(), info


def plan_step(F, P, prec, rtol):
    plan = F.FLDPlan.for_problem(P)
    rho, e_g, E, T = F.device_fields(P)
    info = F.step_problem(plan, P, rho, e_g, E, T, prec=prec, rtol=rtol)
    out = E.cpu().numpy(), T.cpu().numpy(), e_g.cpu().numpy()
    plan.close()
    return out, info


def relerr(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.mark.parametrize("which,prec,rtol,gate", [
    ("c0", W.PREC_FP64, 1e-12, 1e-10),
    ("sph", W.PREC_MIXED, 1e-10, 1e-8),
])
def test_noalloc_matches_plan_step_twice(env, which, prec, rtol, gate):
    torch, N, F = env
    P = W.config0() if which == "c0" else W.random_small(67, 45, W.SPHERICAL, (0, 1, 0, 0), 21, dt=1e4)
    (E0, T0, eg0), info0 = plan_step(F, P, prec, rtol)
    assert info0["status"] == 0
    for _ in range(2):
        rc, E1, T1, eg1, info1 = noalloc_step(torch, N, F, P, prec, rtol)
        assert rc == 0, N.status_string(rc)
        assert relerr(E1, E0) <= gate and relerr(T1, T0) <= gate and relerr(eg1, eg0) <= gate


def test_noalloc_rejects_oversized_grid(env):
    torch, N, F = env
    P = W.random_small(600, 600, W.CARTESIAN, (0, 0, 0, 0), 1)
    rc, E1, *_ = noalloc_step(torch, N, F, P, W.PREC_FP64, 1e-10)
    assert rc == N.GQ_ERR_INVALID_ARG
    assert np.array_equal(E1, P.E_r)          # nothing ran
    assert N.load().gq_fld_step_noalloc_max_bytes() == 32 << 20
