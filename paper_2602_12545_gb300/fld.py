"""Python binding of the implicit FLD step: argument marshalling over the C ABI.

Every step of the path runs in the CUDA library (libgqfld.so); this module only
checks tensors (float64, contiguous, on the plan's CUDA device) and passes raw
pointers and the current CUDA stream.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional, Sequence

import numpy as np
import torch

from . import _native as N
from .workloads import FLDProblem


def _host_ptr(a: Optional[np.ndarray]):
    if a is None:
        return ctypes.cast(None, ctypes.POINTER(ctypes.c_double)), None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a


@dataclasses.dataclass
class SolverOptions:
    prec: int = 0                 # 0 FP64, 1 mixed (FP32 inner, FP64 refinement)
    limiter: int = 0              # 0 LP, 1 Minerbo, 2 none
    rtol: float = 1e-10           # cell-wise relative residual
    max_iter: int = 200000
    inner_rtol: float = 0.1
    max_refine: int = 200
    spin_limit: int = 0
    restart: int = 0
    timing: int = 0
    precond: int = 2              # 0 Jacobi, 1 aggregation multigrid, 2 algebraic multigrid
    mg_omega: float = 0.0         # 0 = library default
    mg_over: float = 0.0
    mg_block_cells: int = 0       # 0 = library default
    subcycle_freeze_D: int = 1    # sub-cycled steps: 1 = D from the hydro step's start (the paper's order),
                                  # 0 = D re-formed from each sub-step's state
    untiled: int = 0              # 1 = never the tiled solve kernel

    def to_c(self) -> N.SolverOpts:
        o = N.SolverOpts()
        N.load().gq_solver_opts_default(ctypes.byref(o))
        o.prec, o.limiter, o.rtol, o.max_iter = int(self.prec), int(self.limiter), float(self.rtol), int(self.max_iter)
        o.inner_rtol, o.max_refine = float(self.inner_rtol), int(self.max_refine)
        o.spin_limit, o.restart, o.timing = int(self.spin_limit), int(self.restart), int(self.timing)
        o.precond, o.mg_omega, o.mg_over = int(self.precond), float(self.mg_omega), float(self.mg_over)
        o.mg_block_cells = int(self.mg_block_cells)
        o.subcycle_freeze_D = int(self.subcycle_freeze_D)
        o.untiled = int(self.untiled)
        return o


class FLDPlan:
    """gq_fld_setup / gq_fld_step / gq_fld_destroy for one grid on the current CUDA device."""

    def __init__(self, x_faces, y_faces, coord: int = 0, area_x=None, area_y=None, volume=None):
        L = N.load()
        xf = np.ascontiguousarray(x_faces, dtype=np.float64)
        yf = np.ascontiguousarray(y_faces, dtype=np.float64)
        self.nx, self.ny, self.coord = xf.size - 1, yf.size - 1, int(coord)
        g = N.GridDesc()
        g.nx, g.ny, g.coord = self.nx, self.ny, self.coord
        g.x_faces, _a = _host_ptr(xf)
        g.y_faces, _b = _host_ptr(yf)
        g.area_x, _c = _host_ptr(area_x)
        g.area_y, _d = _host_ptr(area_y)
        g.volume, _e = _host_ptr(volume)
        h = ctypes.c_void_p()
        self.device = torch.cuda.current_device()
        rc = L.gq_fld_setup(ctypes.byref(g), ctypes.byref(h))
        if rc != N.GQ_OK:
            raise N.GQError(rc, "gq_fld_setup")
        self._h = h

    @classmethod
    def for_problem(cls, p: FLDProblem) -> "FLDPlan":
        return cls(p.x_faces, p.y_faces, p.coord)

    @property
    def nbytes(self) -> int:
        return int(N.load().gq_fld_plan_bytes(self._h))

    def precond_info(self) -> dict:
        """gq_fld_precond_info: the multigrid hierarchy of the last step (levels, rows,
        entries, device build times)."""
        out = N.PrecondInfo()
        rc = N.load().gq_fld_precond_info(self._h, ctypes.byref(out))
        if rc != N.GQ_OK:
            raise N.GQError(rc, "gq_fld_precond_info")
        return out.as_dict()

    def adv_source(self, rho: torch.Tensor, E_r: torch.Tensor, fx: torch.Tensor, fy: torch.Tensor,
                   out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """gq_fld_adv_source (Eq. adv): S_adv [ny][nx] from the face mass fluxes fx [ny][nx+1],
        fy [ny+1][nx] and the upwind E_r / rho, on the current stream."""
        shapes = ((rho, self.ny * self.nx, "rho"), (E_r, self.ny * self.nx, "E_r"),
                  (fx, self.ny * (self.nx + 1), "fx"), (fy, (self.ny + 1) * self.nx, "fy"))
        for t, n, name in shapes:
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
                raise ValueError(f"{name} must be a contiguous float64 CUDA tensor of {n} elements")
        if out is None:
            out = torch.empty((self.ny, self.nx), dtype=torch.float64, device=rho.device)
        st = torch.cuda.current_stream(rho.device).cuda_stream
        rc = N.load().gq_fld_adv_source(self._h, rho.data_ptr(), E_r.data_ptr(), fx.data_ptr(), fy.data_ptr(),
                                        out.data_ptr(), ctypes.c_void_p(st))
        if rc != N.GQ_OK:
            raise N.GQError(rc, "gq_fld_adv_source")
        return out

    def set_source(self, S_adv: Optional[torch.Tensor]):
        """gq_fld_set_source: attach S_adv [ny][nx] (float64 CUDA) to the plan's later steps,
        or detach with None.  The plan keeps a reference while attached."""
        if S_adv is not None and (S_adv.dtype != torch.float64 or not S_adv.is_cuda or not S_adv.is_contiguous()
                                  or S_adv.numel() != self.nx * self.ny):
            raise ValueError(f"S_adv must be a contiguous float64 CUDA tensor of {self.nx * self.ny} elements")
        rc = N.load().gq_fld_set_source(self._h, S_adv.data_ptr() if S_adv is not None else None)
        if rc != N.GQ_OK:
            raise N.GQError(rc, "gq_fld_set_source")
        self._source = S_adv

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.load().gq_fld_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, t: torch.Tensor, name: str):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch.Tensor")
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
        if t.numel() != self.nx * self.ny:
            raise ValueError(f"{name} has {t.numel()} elements, expected {self.nx * self.ny}")
        if t.device.index != self.device:
            raise ValueError(f"{name} is on cuda:{t.device.index}, plan on cuda:{self.device}")

    def step(self, rho: torch.Tensor, e_g: torch.Tensor, E_r: torch.Tensor, T_out: Optional[torch.Tensor] = None,
             *, opacity_R: Sequence[float], opacity_P: Sequence[float], gamma: float, mu: float, dt: float,
             bc: Sequence[int], opts: SolverOptions, stream: Optional[torch.cuda.Stream] = None,
             check: bool = True, n_sub: int = 0, q_t: float = 1.0, Fx: Optional[torch.Tensor] = None,
             Fy: Optional[torch.Tensor] = None, eos_table=None) -> dict:
        """One implicit step; e_g and E_r are updated in place, T_out receives T_g^{n+1}.
        With n_sub >= 1, dt is split into n_sub geometric sub-steps of ratio q_t
        (gq_fld_step_subcycled); Fx [ny][nx+1] and Fy [ny+1][nx] (float64 CUDA tensors) then
        receive the hydro step's face flux."""
        for t, n in ((rho, "rho"), (e_g, "e_g"), (E_r, "E_r")):
            self._check(t, n)
        if T_out is not None:
            self._check(T_out, "T_out")
        op = N.OpacityLaw(*[float(v) for v in tuple(opacity_R) + tuple(opacity_P)])
        eos = N.Eos(float(gamma), float(mu))
        if eos_table is not None:
            # a tabulated u(T): two float64 CUDA tensors of the same length (kept alive by the caller)
            tT, tu = eos_table
            if (tT.dtype != torch.float64 or tu.dtype != torch.float64 or not tT.is_cuda or not tu.is_cuda
                    or not tT.is_contiguous() or not tu.is_contiguous() or tT.numel() != tu.numel()):
                raise ValueError("eos_table must be two contiguous float64 CUDA tensors of one length")
            eos.table_n, eos.table_T, eos.table_u = int(tT.numel()), tT.data_ptr(), tu.data_ptr()
        b = N.Bc()
        for i in range(4):
            b.side[i] = int(bc[i])
        o = opts.to_c()
        info = N.StepInfo()
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        T_ptr = T_out.data_ptr() if T_out is not None else None
        if n_sub >= 1:
            for t, shape, name in ((Fx, (self.ny, self.nx + 1), "Fx"), (Fy, (self.ny + 1, self.nx), "Fy")):
                if t is not None and (t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous()
                                      or t.numel() != shape[0] * shape[1]):
                    raise ValueError(f"{name} must be a contiguous float64 CUDA tensor of {shape[0]} x {shape[1]}")
            rc = N.load().gq_fld_step_subcycled(self._h, rho.data_ptr(), e_g.data_ptr(), E_r.data_ptr(), T_ptr,
                                                ctypes.byref(op), ctypes.byref(eos), float(dt), int(n_sub),
                                                float(q_t), ctypes.byref(b), ctypes.byref(o),
                                                Fx.data_ptr() if Fx is not None else None,
                                                Fy.data_ptr() if Fy is not None else None, ctypes.c_void_p(st),
                                                ctypes.byref(info))
        else:
            rc = N.load().gq_fld_step(self._h, rho.data_ptr(), e_g.data_ptr(), E_r.data_ptr(), T_ptr,
                                      ctypes.byref(op), ctypes.byref(eos), float(dt), ctypes.byref(b),
                                      ctypes.byref(o), ctypes.c_void_p(st), ctypes.byref(info))
        out = info.as_dict()
        out["status"] = rc
        if check and rc not in (N.GQ_OK,):
            raise N.GQError(rc, "gq_fld_step_subcycled" if n_sub >= 1 else "gq_fld_step")
        return out


class SMRPlan:
    """gq_smr_setup / gq_smr_step / gq_smr_destroy: one implicit step on a two-level
    Cartesian grid (nx x ny base cells of widths dx, dy; base cells [i0, i1) x [j0, j1)
    refined 2 x 2).  Fields are float64 CUDA tensors of `cells` values in composite order
    (base cells outside the rectangle row-major, then the fine cells row-major)."""

    def __init__(self, nx: int, ny: int, dx: float, dy: float, i0: int = 0, i1: int = 0, j0: int = 0, j1: int = 0):
        g = N.SmrGrid(int(nx), int(ny), float(dx), float(dy), int(i0), int(i1), int(j0), int(j1))
        h = ctypes.c_void_p()
        self.device = torch.cuda.current_device()
        rc = N.load().gq_smr_setup(ctypes.byref(g), ctypes.byref(h))
        if rc != N.GQ_OK:
            raise N.GQError(rc, "gq_smr_setup")
        self._h = h
        self.cells = int(N.load().gq_smr_cells(h))

    def step(self, rho: torch.Tensor, e_g: torch.Tensor, E_r: torch.Tensor, T_out: Optional[torch.Tensor] = None,
             *, opacity_R: Sequence[float], opacity_P: Sequence[float], gamma: float, mu: float, dt: float,
             bc: Sequence[int], opts: SolverOptions, stream: Optional[torch.cuda.Stream] = None,
             check: bool = True) -> dict:
        for t, n in ((rho, "rho"), (e_g, "e_g"), (E_r, "E_r"), (T_out, "T_out")):
            if t is None and n == "T_out":
                continue
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != self.cells:
                raise ValueError(f"{n} must be a contiguous float64 CUDA tensor of {self.cells} elements")
        op = N.OpacityLaw(*[float(v) for v in tuple(opacity_R) + tuple(opacity_P)])
        eos = N.Eos(float(gamma), float(mu))
        b = N.Bc()
        for i in range(4):
            b.side[i] = int(bc[i])
        o = opts.to_c()
        info = N.StepInfo()
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        rc = N.load().gq_smr_step(self._h, rho.data_ptr(), e_g.data_ptr(), E_r.data_ptr(),
                                  T_out.data_ptr() if T_out is not None else None, ctypes.byref(op),
                                  ctypes.byref(eos), float(dt), ctypes.byref(b), ctypes.byref(o),
                                  ctypes.c_void_p(st), ctypes.byref(info))
        out = info.as_dict()
        out["status"] = rc
        if check and rc != N.GQ_OK:
            raise N.GQError(rc, "gq_smr_step")
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.load().gq_smr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def device_fields(p: FLDProblem, device="cuda"):
    """Copy a problem's fields to the device (float64): rho, e_g, E_r, T_out."""
    rho = torch.from_numpy(np.ascontiguousarray(p.rho)).to(device)
    e_g = torch.from_numpy(np.ascontiguousarray(p.e_g)).to(device)
    E_r = torch.from_numpy(np.ascontiguousarray(p.E_r)).to(device)
    T = torch.empty_like(rho)
    return rho, e_g, E_r, T


def step_problem(plan: FLDPlan, p: FLDProblem, rho, e_g, E_r, T_out=None, *, prec=None, rtol=None,
                 check=True, n_sub=0, q_t=1.0, Fx=None, Fy=None, **kw) -> dict:
    """One step of problem p with its own settings (limiter, bc, dt, precision, rtol);
    n_sub >= 1 sub-cycles it (Eq. subtimesteps)."""
    opts = SolverOptions(prec=p.precision if prec is None else prec, limiter=p.limiter,
                         rtol=p.rtol if rtol is None else rtol, **kw)
    if p.S_adv is not None:
        # the problem's explicit source, attached for this step only
        plan.set_source(torch.as_tensor(np.ascontiguousarray(p.S_adv, dtype=np.float64)).to(rho.device))
        try:
            return plan.step(rho, e_g, E_r, T_out, opacity_R=p.opacity_R, opacity_P=p.opacity_P, gamma=p.gamma,
                             mu=p.mu, dt=p.dt, bc=p.bc, opts=opts, check=check, n_sub=n_sub, q_t=q_t, Fx=Fx, Fy=Fy)
        finally:
            plan.set_source(None)
    return plan.step(rho, e_g, E_r, T_out, opacity_R=p.opacity_R, opacity_P=p.opacity_P, gamma=p.gamma,
                     mu=p.mu, dt=p.dt, bc=p.bc, opts=opts, check=check, n_sub=n_sub, q_t=q_t, Fx=Fx, Fy=Fy)


class FLDBatch:
    """gq_batch_*: independent problems (each with its own FLDPlan) stepped together in one
    persistent launch, replayed from a CUDA graph."""

    def __init__(self, plans, cells_per_block: int = 0, max_team: int = 0, use_graph: bool = True):
        L = N.load()
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        o = N.BatchOpts()
        L.gq_batch_opts_default(ctypes.byref(o))
        o.cells_per_block, o.max_team, o.use_graph = int(cells_per_block), int(max_team), int(bool(use_graph))
        h = ctypes.c_void_p()
        rc = L.gq_batch_create(ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), len(self.plans), ctypes.byref(o),
                               ctypes.byref(h))
        if rc != N.GQ_OK:
            raise N.GQError(rc, "gq_batch_create")
        self._h = h
        self._keep = None

    def _items(self, problems, fields, opts_list):
        items = (N.BatchItem * len(self.plans))()
        for i, (P, (rho, e_g, E, T), o) in enumerate(zip(problems, fields, opts_list)):
            plan = self.plans[i]
            for t, n in ((rho, "rho"), (e_g, "e_g"), (E, "E_r")):
                plan._check(t, n)
            if T is not None:
                plan._check(T, "T_out")
            it = items[i]
            it.rho, it.e_g, it.E_r = rho.data_ptr(), e_g.data_ptr(), E.data_ptr()
            it.T_g_out = T.data_ptr() if T is not None else None
            it.opacity = N.OpacityLaw(*[float(v) for v in tuple(P.opacity_R) + tuple(P.opacity_P)])
            it.eos = N.Eos(float(P.gamma), float(P.mu))
            it.dt = float(P.dt)
            for s in range(4):
                it.bc.side[s] = int(P.bc[s])
            it.opts = o.to_c()
        return items

    @staticmethod
    def default_opts(problems, **kw):
        return [SolverOptions(prec=P.precision, limiter=P.limiter, rtol=P.rtol, **kw) for P in problems]

    def step(self, problems, fields, opts_list=None, stream=None, check=True):
        """One step of every problem; fields is a list of (rho, e_g, E_r, T_out) tensors."""
        opts_list = opts_list or self.default_opts(problems)
        items = self._items(problems, fields, opts_list)
        infos = (N.StepInfo * len(self.plans))()
        st = (stream or torch.cuda.current_stream()).cuda_stream
        rc = N.load().gq_batch_step(self._h, items, ctypes.c_void_p(st), infos)
        out = [i.as_dict() for i in infos]
        if check and rc != N.GQ_OK:
            raise N.GQError(rc, "gq_batch_step")
        return rc, out

    def autotune(self, problems, fields, opts_list=None, stream=None):
        opts_list = opts_list or self.default_opts(problems)
        items = self._items(problems, fields, opts_list)
        best = N.BatchOpts()
        ms = ctypes.c_double()
        st = (stream or torch.cuda.current_stream()).cuda_stream
        rc = N.load().gq_batch_autotune(self._h, items, ctypes.c_void_p(st), ctypes.byref(best), ctypes.byref(ms))
        if rc != N.GQ_OK:
            raise N.GQError(rc, "gq_batch_autotune")
        return {"cells_per_block": best.cells_per_block, "max_team": best.max_team, "ms": ms.value}

    def reschedule(self, cells_per_block=0, max_team=0, use_graph=True):
        o = N.BatchOpts()
        o.cells_per_block, o.max_team, o.use_graph = int(cells_per_block), int(max_team), int(bool(use_graph))
        rc = N.load().gq_batch_reschedule(self._h, ctypes.byref(o))
        if rc != N.GQ_OK:
            raise N.GQError(rc, "gq_batch_reschedule")

    @property
    def last_ms(self) -> float:
        return float(N.load().gq_batch_last_step_ms(self._h))

    @property
    def uses_graph(self) -> bool:
        return bool(N.load().gq_batch_uses_graph(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.load().gq_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
