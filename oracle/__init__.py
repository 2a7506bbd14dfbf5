"""FP64 CPU oracle for the implicit FLD radiation step (Guangqi, Sec. 3.2).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It is a plain, slow C
implementation (``gq_oracle.c``) that shares no code with the CUDA library; this
module marshals numpy arrays into it and strings its single steps into sub-cycled ones.
``smr.py`` assembles the two-level (SMR) matrix of Sec. 3.2.2 with numpy and scipy.
"""
from __future__ import annotations

import ctypes
import threading
from typing import Optional

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("coord", ctypes.c_int),
        ("xf", _dp), ("yf", _dp), ("V_in", _dp), ("Ax_in", _dp), ("Ay_in", _dp),
        ("rho", _dp), ("eg", _dp), ("E", _dp),
        ("kR", ctypes.c_double * 4), ("kP", ctypes.c_double * 4),
        ("gamma", ctypes.c_double), ("mu", ctypes.c_double), ("dt", ctypes.c_double),
        ("bc", ctypes.c_int * 4), ("limiter", ctypes.c_int), ("S_adv", _dp),
        ("Gx_in", _dp), ("Gy_in", _dp),
        ("eos_n", ctypes.c_int), ("eos_T", _dp), ("eos_u", _dp),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER(_Problem)
            L.orc_limiter.restype = ctypes.c_double
            L.orc_limiter.argtypes = [ctypes.c_int, ctypes.c_double]
            for name in ("orc_const_c", "orc_const_aR", "orc_const_kB", "orc_const_mH"):
                getattr(L, name).restype = ctypes.c_double
                getattr(L, name).argtypes = []
            L.orc_geometry.argtypes = [P, _dp, _dp, _dp, _dp, _dp]
            L.orc_faces.argtypes = [P, _dp, _dp, _dp, _dp, _dp, _dp]
            L.orc_assemble_coupled.argtypes = [P, _ip, _ip, _dp, _dp]
            L.orc_assemble_reduced.argtypes = [P, _ip, _ip, _dp, _dp]
            L.orc_band_solve.argtypes = [ctypes.c_int, _ip, _ip, _dp, _dp, _dp]
            L.orc_pcg.argtypes = [ctypes.c_int, _ip, _ip, _dp, _dp, _dp, ctypes.c_double, ctypes.c_int,
                                  _ip, _dp]
            L.orc_step.argtypes = [P, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp, _dp, _dp]
            L.orc_adv_source.argtypes = [P, _dp, _dp, _dp]
            _lib = L
    return _lib


def _d(a: Optional[np.ndarray]):
    if a is None:
        return ctypes.cast(None, _dp)
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _i(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_ip)


class _Bound:
    """Keeps the numpy arrays referenced by a _Problem alive."""

    def __init__(self, prob, V=None, Ax=None, Ay=None, G=None):
        self.arrs = [np.ascontiguousarray(prob.x_faces, dtype=np.float64),
                     np.ascontiguousarray(prob.y_faces, dtype=np.float64),
                     None if V is None else np.ascontiguousarray(V, dtype=np.float64),
                     None if Ax is None else np.ascontiguousarray(Ax, dtype=np.float64),
                     None if Ay is None else np.ascontiguousarray(Ay, dtype=np.float64),
                     np.ascontiguousarray(prob.rho, dtype=np.float64),
                     np.ascontiguousarray(prob.e_g, dtype=np.float64),
                     np.ascontiguousarray(prob.E_r, dtype=np.float64)]
        S_adv = getattr(prob, "S_adv", None)
        self.arrs.append(None if S_adv is None else np.ascontiguousarray(S_adv, dtype=np.float64).ravel())
        self.arrs += [None, None] if G is None else [np.ascontiguousarray(g, dtype=np.float64).ravel() for g in G]
        tab = getattr(prob, "eos_table", None)
        self.arrs += [None, None] if tab is None else [np.ascontiguousarray(t, dtype=np.float64) for t in tab]
        xf, yf, V_, Ax_, Ay_, rho, eg, E, S, Gx, Gy, eT, eu = self.arrs
        s = _Problem()
        s.nx, s.ny, s.coord = prob.nx, prob.ny, int(prob.coord)
        s.xf, s.yf, s.V_in, s.Ax_in, s.Ay_in = _d(xf), _d(yf), _d(V_), _d(Ax_), _d(Ay_)
        s.rho, s.eg, s.E = _d(rho.ravel()), _d(eg.ravel()), _d(E.ravel())
        for t in range(4):
            s.kR[t] = float(prob.opacity_R[t])
            s.kP[t] = float(prob.opacity_P[t])
            s.bc[t] = int(prob.bc[t])
        s.gamma, s.mu, s.dt = float(prob.gamma), float(prob.mu), float(prob.dt)
        s.limiter = int(prob.limiter)
        s.S_adv = _d(S)
        s.Gx_in, s.Gy_in = _d(Gx), _d(Gy)
        s.eos_n = 0 if eT is None else int(eT.size)
        s.eos_T, s.eos_u = _d(eT), _d(eu)
        self.s = s

    def ref(self):
        return ctypes.byref(self.s)


def constants() -> dict:
    L = lib()
    return {"c": L.orc_const_c(), "aR": L.orc_const_aR(), "kB": L.orc_const_kB(), "mH": L.orc_const_mH()}


def limiter(kind: int, R) -> np.ndarray:
    L = lib()
    R = np.atleast_1d(np.asarray(R, dtype=np.float64))
    return np.array([L.orc_limiter(int(kind), float(r)) for r in R.ravel()]).reshape(R.shape)


def geometry(prob, V=None, Ax=None, Ay=None) -> dict:
    nx, ny = prob.nx, prob.ny
    out = {"V": np.zeros((ny, nx)), "Ax": np.zeros((ny, nx + 1)), "Ay": np.zeros((ny + 1, nx)),
           "xc": np.zeros(nx), "yc": np.zeros(ny)}
    b = _Bound(prob, V, Ax, Ay)
    rc = lib().orc_geometry(b.ref(), _d(out["V"]), _d(out["Ax"]), _d(out["Ay"]), _d(out["xc"]), _d(out["yc"]))
    if rc:
        raise RuntimeError(f"orc_geometry failed ({rc})")
    return out


def faces(prob, V=None, Ax=None, Ay=None) -> dict:
    nx, ny = prob.nx, prob.ny
    out = {k: np.zeros((ny, nx + 1)) for k in ("Rx", "Dx", "wx")}
    out.update({k: np.zeros((ny + 1, nx)) for k in ("Ry", "Dy", "wy")})
    b = _Bound(prob, V, Ax, Ay)
    rc = lib().orc_faces(b.ref(), _d(out["Rx"]), _d(out["Ry"]), _d(out["Dx"]), _d(out["Dy"]),
                         _d(out["wx"]), _d(out["wy"]))
    if rc:
        raise RuntimeError(f"orc_faces failed ({rc})")
    return out


def adv_source(prob, fx, fy) -> np.ndarray:
    """Eq. adv: the explicit advection source S_adv [ny][nx] (erg cm^-3 s^-1) from face mass
    fluxes fx [ny][nx+1], fy [ny+1][nx] (g cm^-2 s^-1, positive along +x / +y) and the
    upwind e_r = E / rho of prob's fields."""
    nx, ny = prob.nx, prob.ny
    fx = np.ascontiguousarray(fx, dtype=np.float64).reshape(ny, nx + 1)
    fy = np.ascontiguousarray(fy, dtype=np.float64).reshape(ny + 1, nx)
    S = np.zeros((ny, nx))
    b = _Bound(prob)
    rc = lib().orc_adv_source(b.ref(), _d(fx), _d(fy), _d(S))
    if rc:
        raise RuntimeError(f"orc_adv_source failed ({rc})")
    return S


def _csr(n, rp, cl, vl, nnz):
    import scipy.sparse as sp
    return sp.csr_matrix((vl[:nnz].copy(), cl[:nnz].copy(), rp.copy()), shape=(n, n))


def assemble_coupled(prob):
    """Paper-literal coupled system (2N x 2N, interleaved [E_k, T_k]) as scipy CSR, rhs."""
    N = prob.ncells
    rp = np.zeros(2 * N + 1, np.int32); cl = np.zeros(8 * N, np.int32)
    vl = np.zeros(8 * N); rhs = np.zeros(2 * N)
    b = _Bound(prob)
    nnz = lib().orc_assemble_coupled(b.ref(), _i(rp), _i(cl), _d(vl), _d(rhs))
    if nnz < 0:
        raise RuntimeError(f"orc_assemble_coupled failed ({nnz})")
    return _csr(2 * N, rp, cl, vl, nnz), rhs


def assemble_reduced(prob, V=None, Ax=None, Ay=None):
    """Schur-reduced symmetric system (N x N, rows times V_k) as scipy CSR, rhs."""
    N = prob.ncells
    rp = np.zeros(N + 1, np.int32); cl = np.zeros(5 * N, np.int32)
    vl = np.zeros(5 * N); rhs = np.zeros(N)
    b = _Bound(prob, V, Ax, Ay)
    nnz = lib().orc_assemble_reduced(b.ref(), _i(rp), _i(cl), _d(vl), _d(rhs))
    if nnz < 0:
        raise RuntimeError(f"orc_assemble_reduced failed ({nnz})")
    return _csr(N, rp, cl, vl, nnz), rhs


def band_solve(A, rhs) -> np.ndarray:
    A = A.tocsr()
    n = A.shape[0]
    rp = np.ascontiguousarray(A.indptr, dtype=np.int32); cl = np.ascontiguousarray(A.indices, dtype=np.int32)
    vl = np.ascontiguousarray(A.data, dtype=np.float64)
    x = np.zeros(n)
    rc = lib().orc_band_solve(n, _i(rp), _i(cl), _d(vl), _d(np.ascontiguousarray(rhs, dtype=np.float64)), _d(x))
    if rc:
        raise RuntimeError(f"orc_band_solve failed ({rc})")
    return x


def pcg(A, rhs, x0, tol=1e-15, maxit=1000000):
    A = A.tocsr()
    n = A.shape[0]
    rp = np.ascontiguousarray(A.indptr, dtype=np.int32); cl = np.ascontiguousarray(A.indices, dtype=np.int32)
    vl = np.ascontiguousarray(A.data, dtype=np.float64)
    x = np.array(x0, dtype=np.float64, copy=True)
    it = ctypes.c_int(0); crit = ctypes.c_double(0.0)
    rc = lib().orc_pcg(n, _i(rp), _i(cl), _d(vl), _d(np.ascontiguousarray(rhs, dtype=np.float64)), _d(x),
                       float(tol), int(maxit), ctypes.byref(it), ctypes.byref(crit))
    return x, it.value, crit.value, rc


def step(prob, method: str = "lu", tol: float = 1e-15, V=None, Ax=None, Ay=None, G=None) -> dict:
    """One implicit step.  method 'lu': banded LU on the reduced system; 'cg': Jacobi-PCG on
    the reduced system to the cell-wise relative residual tol; 'coupled': banded LU on the
    paper-literal coupled system (accurate only for moderate coupling).  G = (Gx, Gy): frozen
    face conductances A D / d (face weights dt G instead of those of this state)."""
    nx, ny = prob.nx, prob.ny
    E = np.zeros((ny, nx)); T = np.zeros((ny, nx)); eg = np.zeros((ny, nx))
    info = np.zeros(5)
    Fx = np.zeros((ny, nx + 1)); Fy = np.zeros((ny + 1, nx))
    b = _Bound(prob, V, Ax, Ay, G)
    m = {"lu": 0, "cg": 1, "coupled": 2}[method]
    rc = lib().orc_step(b.ref(), m, float(tol), _d(E), _d(T), _d(eg), _d(info), _d(Fx), _d(Fy))
    if rc < 0:
        raise RuntimeError(f"orc_step failed ({rc})")
    return {"E_r": E, "T_g": T, "e_g": eg, "iterations": int(info[0]), "cell_residual": info[1],
            "l2_residual": info[2], "energy_before": info[3], "energy_after": info[4],
            "Fx": Fx, "Fy": Fy, "status": rc}


def subcycle_dts(dt_total: float, n_sub: int, q_t: float) -> list:
    """Sub-step lengths of Eq. subtimesteps (Sec. 3.2): dt_i = dt_0 q^(i-1), i = 1..n_sub,
    dt_0 = dt_total (1 - q) / (1 - q^n_sub), so that they add up to the hydro step;
    q = 1, the limit of the formula, gives equal sub-steps."""
    if q_t == 1.0:
        return [dt_total / n_sub] * n_sub
    dt0 = dt_total * (1.0 - q_t) / (1.0 - q_t ** n_sub)
    return [dt0 * q_t ** (i - 1) for i in range(1, n_sub + 1)]


def step_subcycled(prob, n_sub: int, q_t: float, method: str = "lu", tol: float = 1e-15,
                   freeze_D: bool = True) -> dict:
    """prob.dt split into n_sub implicit steps (Eq. subtimesteps), each taken from the state
    the previous one left, so opacities, C_V and the linearisation are re-evaluated.  With
    freeze_D (the default), in the order of the paper's radiation algorithm (alpha updated,
    D kept), every sub-step uses the face conductances A D / d of the hydro step's start
    with its own dt; without it, D (with kappa_R rho and the limiter) is re-formed from
    each sub-step's state too.  Fx, Fy: the radiative face flux of the hydro step, the sub-steps'
    post-step fluxes weighted by dt_i / dt (so that dt times it is the energy each face
    carried); with freeze_D this is D^n sum_i (dt_i / dt) (E_m - E_k)_i / d, the
    accumulation of Sec. 3.2.1."""
    import copy
    P = copy.copy(prob)
    P.E_r = np.array(prob.E_r, dtype=np.float64, copy=True)
    P.e_g = np.array(prob.e_g, dtype=np.float64, copy=True)
    first, out, its = None, None, 0
    G = None
    if freeze_D:
        w = faces(prob)
        G = (w["wx"] / prob.dt, w["wy"] / prob.dt)
    Fx = np.zeros((prob.ny, prob.nx + 1))
    Fy = np.zeros((prob.ny + 1, prob.nx))
    for dt in subcycle_dts(prob.dt, n_sub, q_t):
        P.dt = dt
        out = step(P, method, tol, G=G)
        if first is None:
            first = out
        P.E_r = out["E_r"].copy()
        P.e_g = out["e_g"].copy()
        its += out["iterations"]
        Fx += (dt / prob.dt) * out["Fx"]
        Fy += (dt / prob.dt) * out["Fy"]
    return {"E_r": out["E_r"], "T_g": out["T_g"], "e_g": out["e_g"], "iterations": its,
            "energy_before": first["energy_before"], "energy_after": out["energy_after"], "Fx": Fx, "Fy": Fy}
