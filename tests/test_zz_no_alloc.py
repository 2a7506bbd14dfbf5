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


def noalloc_step(torch, N, F, P, prec, rtol, x_faces=None, y_faces=None):
    L = N.load()
    xf = torch.from_numpy(np.ascontiguousarray(P.x_faces if x_faces is None else x_faces)).cuda()
    yf = torch.from_numpy(np.ascontiguousarray(P.y_faces if y_faces is None else y_faces)).cuda()
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


def plan_step(F, P, prec, rtol, check=True):
    plan = F.FLDPlan.for_problem(P)
    rho, e_g, E, T = F.device_fields(P)
    info = F.step_problem(plan, P, rho, e_g, E, T, prec=prec, rtol=rtol, check=check)
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


def test_noalloc_sequence_of_shapes(env):
    """Calls of different shapes in a row: every call lays its arrays out afresh in the
    shared array, so small -> large -> small must each match the plan-based step."""
    torch, N, F = env
    shapes = [(23, 17, W.CARTESIAN), (150, 120, W.SPHERICAL), (31, 9, W.CARTESIAN), (150, 120, W.SPHERICAL)]
    for k, (nx, ny, coord) in enumerate(shapes):
        P = W.random_small(nx, ny, coord, (0, 1, 0, 0), 60 + k, dt=1e4)
        (E0, T0, eg0), info0 = plan_step(F, P, W.PREC_FP64, 1e-11, check=False)
        rc, E1, T1, eg1, info1 = noalloc_step(torch, N, F, P, W.PREC_FP64, 1e-11)
        # the same kernels on the same inputs: the same status (GQ_ERR_NOT_CONVERGED only at
        # the FP64 floor of an ill-conditioned draw)
        assert rc in (0, 4) and rc == info0["status"], (nx, ny, N.status_string(rc), info0)
        assert relerr(E1, E0) <= 1e-10 and relerr(T1, T0) <= 1e-10 and relerr(eg1, eg0) <= 1e-10, (nx, ny)


def _largest_square_side(N):
    """Largest n whose n x n footprint fits the static array (the footprint of the
    allocation-free step is the plan's arena less its 256 bytes of slack)."""
    L = N.load()
    cap = L.gq_fld_step_noalloc_max_bytes()
    fits = lambda n: 0 < L.gq_fld_plan_bytes_for(n, n) - 256 <= cap
    lo, hi = 1, 4096
    assert fits(lo) and not fits(hi)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        lo, hi = (mid, hi) if fits(mid) else (lo, mid)
    return lo


def test_noalloc_at_the_size_limit(env):
    """The largest square grid that fits uses the last bytes of the array and must match
    the plan-based step; one cell row more is rejected before anything runs."""
    torch, N, F = env
    n = _largest_square_side(N)
    assert 40_000 <= n * n <= 60_000            # about 50 000 cells, as documented
    P = W.random_small(n, n, W.CARTESIAN, (0, 1, 0, 0), 77, dt=1e4)
    (E0, T0, eg0), info0 = plan_step(F, P, W.PREC_FP64, 1e-11, check=False)
    rc, E1, T1, eg1, info1 = noalloc_step(torch, N, F, P, W.PREC_FP64, 1e-11)
    assert rc in (0, 4) and rc == info0["status"], (N.status_string(rc), info0)
    assert relerr(E1, E0) <= 1e-10 and relerr(T1, T0) <= 1e-10 and relerr(eg1, eg0) <= 1e-10
    Q = W.random_small(n + 1, n + 1, W.CARTESIAN, (0, 1, 0, 0), 78, dt=1e4)
    rc, E2, *_ = noalloc_step(torch, N, F, Q, W.PREC_FP64, 1e-11)
    assert rc == N.GQ_ERR_INVALID_ARG
    assert np.array_equal(E2, Q.E_r)


def test_noalloc_rejects_bad_faces(env):
    """Faces gq_fld_setup would reject (reversed, repeated, not finite, r <= 0, theta past
    pi) are caught on the device: GQ_ERR_INVALID_ARG and the fields untouched."""
    torch, N, F = env
    P = W.random_small(20, 12, W.CARTESIAN, (0, 0, 0, 0), 5)
    S = W.random_small(20, 12, W.SPHERICAL, (0, 1, 0, 0), 6)
    xr = P.x_faces[::-1].copy()
    rep = P.x_faces.copy()
    rep[7] = rep[6]
    nan = P.y_faces.copy()
    nan[3] = float("nan")
    r0 = S.x_faces.copy()
    r0[0] = 0.0
    th = S.y_faces.copy()
    th[-1] = 3.5
    for Q, xf, yf in ((P, xr, None), (P, rep, None), (P, None, nan), (S, r0, None), (S, None, th)):
        rc, E1, T1, eg1, _ = noalloc_step(torch, N, F, Q, W.PREC_FP64, 1e-10, x_faces=xf, y_faces=yf)
        assert rc == N.GQ_ERR_INVALID_ARG, N.status_string(rc)
        assert np.array_equal(E1, Q.E_r) and np.array_equal(eg1, Q.e_g)
    # and a good call right after works
    (E0, T0, eg0), info0 = plan_step(F, S, W.PREC_FP64, 1e-11, check=False)
    rc, E1, T1, eg1, _ = noalloc_step(torch, N, F, S, W.PREC_FP64, 1e-11)
    assert rc in (0, 4) and rc == info0["status"] and relerr(E1, E0) <= 1e-10
