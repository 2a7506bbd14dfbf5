"""ctypes declarations of the C ABI in include/gq_fld.h and the library loader.

The CUDA library is required: there is no fallback.  Loading fails with a clear error
when libgqfld.so has not been built (``python -m paper_2602_12545_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgqfld.so")

GQ_OK = 0
GQ_ERR_INVALID_ARG = 1
GQ_ERR_CUDA = 2
GQ_ERR_OOM = 3
GQ_ERR_NOT_CONVERGED = 4
GQ_ERR_NONFINITE = 5
GQ_ERR_TIMEOUT = 6
GQ_ERR_BUDGET = 7
GQ_PRECOND_JACOBI = 0
GQ_PRECOND_MG = 1
GQ_PRECOND_AMG = 2

_dp = ctypes.POINTER(ctypes.c_double)


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("coord", ctypes.c_int),
                ("x_faces", _dp), ("y_faces", _dp), ("area_x", _dp), ("area_y", _dp), ("volume", _dp)]


class OpacityLaw(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("k0_R", "k1_R", "a_R", "b_R", "k0_P", "k1_P", "a_P", "b_P")]


class Eos(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("mu", ctypes.c_double), ("table_n", ctypes.c_int),
                ("table_T", ctypes.c_void_p), ("table_u", ctypes.c_void_p)]


class Bc(ctypes.Structure):
    _fields_ = [("side", ctypes.c_int * 4)]


class SolverOpts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("limiter", ctypes.c_int), ("rtol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("inner_rtol", ctypes.c_double), ("max_refine", ctypes.c_int),
                ("spin_limit", ctypes.c_int64), ("restart", ctypes.c_int), ("timing", ctypes.c_int),
                ("precond", ctypes.c_int), ("mg_block_cells", ctypes.c_int), ("mg_omega", ctypes.c_double),
                ("mg_over", ctypes.c_double), ("subcycle_freeze_D", ctypes.c_int), ("untiled", ctypes.c_int)]


class StepInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("refinements", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("rel_residual_l2", ctypes.c_double), ("energy_before", ctypes.c_double),
                ("energy_after", ctypes.c_double), ("status", ctypes.c_int), ("solve_blocks", ctypes.c_int),
                ("t_setup_ms", ctypes.c_double), ("t_solve_ms", ctypes.c_double), ("t_finish_ms", ctypes.c_double),
                ("t_precond_ms", ctypes.c_float), ("t_iter_us", ctypes.c_float), ("precond_levels", ctypes.c_int),
                ("solve_kernel", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class PrecondInfo(ctypes.Structure):
    _fields_ = [("precond", ctypes.c_int), ("levels", ctypes.c_int), ("stop_reason", ctypes.c_int),
                ("rows", ctypes.c_int * 24), ("entries", ctypes.c_int * 24), ("build_ms", ctypes.c_float * 24),
                ("fine_copy_ms", ctypes.c_float), ("coarsest_ms", ctypes.c_float),
                ("build_phase_ms", ctypes.c_float * 8), ("cycle_ms", ctypes.c_float * 24)]

    def as_dict(self) -> dict:
        n = self.levels
        return {"precond": self.precond, "levels": n, "stop_reason": self.stop_reason,
                "rows": list(self.rows[:n]), "entries": list(self.entries[:n]),
                "build_ms": list(self.build_ms[:max(n - 1, 0)]), "fine_copy_ms": self.fine_copy_ms,
                "coarsest_ms": self.coarsest_ms, "build_phase_ms": list(self.build_phase_ms),
                "cycle_ms": list(self.cycle_ms[:min(n, 20)]), "direction_ms": self.cycle_ms[20],
                "update_ms": self.cycle_ms[21], "refine_ms": self.cycle_ms[22],
                "after_cycle_ms": self.cycle_ms[23],
                "outside_cycle_ms": sum(self.cycle_ms[20:24])}


class SmrGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("i0", ctypes.c_int), ("i1", ctypes.c_int), ("j0", ctypes.c_int), ("j1", ctypes.c_int)]


class BatchItem(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_void_p), ("e_g", ctypes.c_void_p), ("E_r", ctypes.c_void_p),
                ("T_g_out", ctypes.c_void_p), ("opacity", OpacityLaw), ("eos", Eos), ("dt", ctypes.c_double),
                ("bc", Bc), ("opts", SolverOpts)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("cells_per_block", ctypes.c_int), ("max_team", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("reserved", ctypes.c_int * 5)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("max_active", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("solo_cells", ctypes.c_int), ("reserved", ctypes.c_int * 5)]


class Request(ctypes.Structure):
    _fields_ = [("grid", GridDesc), ("rho", _dp), ("e_g", _dp), ("E_r", _dp), ("opacity", OpacityLaw),
                ("eos", Eos), ("dt", ctypes.c_double), ("bc", Bc), ("opts", SolverOpts), ("n_steps", ctypes.c_int),
                ("E_r_out", _dp), ("e_g_out", _dp), ("T_g_out", _dp)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int), ("steps_done", ctypes.c_int),
                ("iterations", ctypes.c_int), ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("energy_before", ctypes.c_double), ("energy_after", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("reserved", ctypes.c_int * 4)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


# every symbol include/gq_fld.h declares, with (restype, argtypes)
SIGNATURES = {
    "gq_fld_setup": (ctypes.c_int, [ctypes.POINTER(GridDesc), ctypes.POINTER(ctypes.c_void_p)]),
    "gq_fld_plan_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "gq_fld_plan_bytes_for": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int]),
    "gq_server_create": (ctypes.c_int, [ctypes.POINTER(ServerOpts), ctypes.POINTER(ctypes.c_void_p)]),
    "gq_server_request_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int]),
    "gq_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_int64)]),
    "gq_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "gq_server_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(RequestInfo)]),
    "gq_server_release": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "gq_server_pending": (ctypes.c_int, [ctypes.c_void_p]),
    "gq_server_used_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "gq_server_destroy": (None, [ctypes.c_void_p]),
    "gq_fld_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.POINTER(OpacityLaw), ctypes.POINTER(Eos),
                                   ctypes.c_double, ctypes.POINTER(Bc), ctypes.POINTER(SolverOpts),
                                   ctypes.c_void_p, ctypes.POINTER(StepInfo)]),
    "gq_fld_destroy": (None, [ctypes.c_void_p]),
    "gq_fld_step_subcycled": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.POINTER(OpacityLaw), ctypes.POINTER(Eos),
                                             ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.POINTER(Bc),
                                             ctypes.POINTER(SolverOpts), ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.POINTER(StepInfo)]),
    "gq_fld_precond_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(PrecondInfo)]),
    "gq_fld_adv_source": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 5 + [ctypes.c_void_p]),
    "gq_fld_set_source": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gq_fld_step_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.POINTER(OpacityLaw), ctypes.POINTER(Eos), ctypes.c_double,
                                           ctypes.POINTER(Bc), ctypes.POINTER(SolverOpts), ctypes.c_void_p,
                                           ctypes.POINTER(StepInfo)]),
    "gq_fld_step_noalloc_max_bytes": (ctypes.c_size_t, []),
    "gq_smr_setup": (ctypes.c_int, [ctypes.POINTER(SmrGrid), ctypes.POINTER(ctypes.c_void_p)]),
    "gq_smr_cells": (ctypes.c_int, [ctypes.c_void_p]),
    "gq_smr_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.POINTER(OpacityLaw), ctypes.POINTER(Eos),
                                   ctypes.c_double, ctypes.POINTER(Bc), ctypes.POINTER(SolverOpts),
                                   ctypes.c_void_p, ctypes.POINTER(StepInfo)]),
    "gq_smr_destroy": (None, [ctypes.c_void_p]),
    "gq_solver_opts_default": (None, [ctypes.POINTER(SolverOpts)]),
    "gq_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gq_version": (ctypes.c_char_p, []),
    "gq_batch_opts_default": (None, [ctypes.POINTER(BatchOpts)]),
    "gq_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(BatchOpts),
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "gq_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(BatchItem), ctypes.c_void_p,
                                     ctypes.POINTER(StepInfo)]),
    "gq_batch_reschedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(BatchOpts)]),
    "gq_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(BatchItem), ctypes.c_void_p,
                                         ctypes.POINTER(BatchOpts), ctypes.POINTER(ctypes.c_double)]),
    "gq_batch_last_step_ms": (ctypes.c_double, [ctypes.c_void_p]),
    "gq_batch_uses_graph": (ctypes.c_int, [ctypes.c_void_p]),
    "gq_batch_destroy": (None, [ctypes.c_void_p]),
    "gq_fld_step_batched": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(BatchItem),
                                           ctypes.c_void_p, ctypes.POINTER(StepInfo)]),
}

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libgqfld.so and declare its signatures (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path} is missing "
                                   "(run `python -m paper_2602_12545_gb300.build`)")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def status_string(code: int) -> str:
    return load().gq_status_string(int(code)).decode()


class GQError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = int(code)
        super().__init__(f"{where}: {status_string(code)} (status {code})")
