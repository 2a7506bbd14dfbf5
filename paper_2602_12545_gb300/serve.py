"""Continuous-batching serving of implicit FLD solves (Python driver over gq_server_*).

FLDServer wraps the C server: submit() queues a request (host numpy inputs, copied),
poll() runs one engine tick (admit by memory budget, step every resident request once in
one batched launch, retire finished ones).  run_trace() replays a seeded Poisson arrival
trace in real time and reports throughput and latency percentiles.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import threading
import time
from collections import deque
from typing import Dict, List, Optional

import numpy as np

from . import _native as N
from .fld import SolverOptions
from .workloads import FLDProblem, ServeRequest, serve_problem


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclasses.dataclass
class Completed:
    rid: int
    status: int
    steps: int
    iterations: int
    cells: int
    arrival_s: float
    submit_s: float
    admit_s: float
    done_s: float
    E_r: Optional[np.ndarray] = None
    T_g: Optional[np.ndarray] = None
    e_g: Optional[np.ndarray] = None
    energy_before: float = 0.0
    energy_after: float = 0.0


class FLDServer:
    def __init__(self, budget_bytes: int, max_active: int = 256, use_graph: bool = False, solo_cells: int = 0):
        L = N.load()
        o = N.ServerOpts()
        o.budget_bytes, o.max_active, o.use_graph = int(budget_bytes), int(max_active), int(bool(use_graph))
        o.solo_cells = int(solo_cells)
        h = ctypes.c_void_p()
        rc = L.gq_server_create(ctypes.byref(o), ctypes.byref(h))
        if rc != N.GQ_OK:
            raise N.GQError(rc, "gq_server_create")
        self._h = h
        self._keep: Dict[int, tuple] = {}

    @staticmethod
    def request_bytes(nx: int, ny: int) -> int:
        return int(N.load().gq_server_request_bytes(nx, ny))

    def submit(self, P: FLDProblem, n_steps: int, opts: Optional[SolverOptions] = None, keep_output=True) -> int:
        opts = opts or SolverOptions(prec=P.precision, limiter=P.limiter, rtol=P.rtol)
        r = N.Request()
        xf = np.ascontiguousarray(P.x_faces, dtype=np.float64)
        yf = np.ascontiguousarray(P.y_faces, dtype=np.float64)
        rho = np.ascontiguousarray(P.rho, dtype=np.float64)
        eg = np.ascontiguousarray(P.e_g, dtype=np.float64)
        E = np.ascontiguousarray(P.E_r, dtype=np.float64)
        r.grid.nx, r.grid.ny, r.grid.coord = P.nx, P.ny, int(P.coord)
        r.grid.x_faces, r.grid.y_faces = _dp(xf), _dp(yf)
        r.rho, r.e_g, r.E_r = _dp(rho), _dp(eg), _dp(E)
        r.opacity = N.OpacityLaw(*[float(v) for v in tuple(P.opacity_R) + tuple(P.opacity_P)])
        r.eos = N.Eos(float(P.gamma), float(P.mu))
        r.dt = float(P.dt)
        for s in range(4):
            r.bc.side[s] = int(P.bc[s])
        r.opts = opts.to_c()
        r.n_steps = int(n_steps)
        outs = None
        if keep_output:
            outs = (np.empty((P.ny, P.nx)), np.empty((P.ny, P.nx)), np.empty((P.ny, P.nx)))
            r.E_r_out, r.e_g_out, r.T_g_out = _dp(outs[0]), _dp(outs[1]), _dp(outs[2])
        rid = ctypes.c_int64()
        rc = N.load().gq_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid))
        if rc != N.GQ_OK:
            raise N.GQError(rc, "gq_server_submit")
        self._keep[rid.value] = (outs, P.ncells)
        return rid.value

    def poll(self) -> int:
        done = ctypes.c_int()
        rc = N.load().gq_server_poll(self._h, ctypes.byref(done))
        if rc != N.GQ_OK:
            raise N.GQError(rc, "gq_server_poll")
        return done.value

    def info(self, rid: int) -> dict:
        i = N.RequestInfo()
        rc = N.load().gq_server_info(self._h, int(rid), ctypes.byref(i))
        if rc != N.GQ_OK:
            raise N.GQError(rc, "gq_server_info")
        return i.as_dict()

    def take(self, rid: int):
        """Outputs (E_r, e_g, T_g) and info of a finished request; releases it."""
        info = self.info(rid)
        if info["state"] != 2:
            return None
        outs, cells = self._keep.pop(rid)
        N.load().gq_server_release(self._h, int(rid))
        return outs, cells, info

    @property
    def pending(self) -> int:
        return int(N.load().gq_server_pending(self._h))

    @property
    def used_bytes(self) -> int:
        return int(N.load().gq_server_used_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.load().gq_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _percentile(xs: List[float], q: float) -> float:
    if not xs:
        return float("nan")
    s = sorted(xs)
    k = min(len(s) - 1, max(0, int(math.ceil(q / 100.0 * len(s))) - 1))
    return s[k]


def run_trace(trace: List[ServeRequest], budget_bytes: int, max_active: int = 256, keep_output=False,
              opts: Optional[SolverOptions] = None, lookahead: int = 64, problem_fn=serve_problem,
              solo_cells: int = 0) -> dict:
    """Replay a trace in real time: request i is submitted when the wall clock reaches its
    arrival time (or as soon as its inputs are ready), the server is polled continuously,
    and latency is arrival -> completion.  Inputs are generated by a producer thread ahead
    of the clock (bounded lookahead)."""
    srv = FLDServer(budget_bytes, max_active, solo_cells=solo_cells)
    ready: deque = deque()
    lock = threading.Condition()
    stop = [False]

    def producer():
        for req in trace:
            P = problem_fn(req)
            with lock:
                while len(ready) >= lookahead and not stop[0]:
                    lock.wait(0.05)
                if stop[0]:
                    return
                ready.append((req, P, time.perf_counter()))
                lock.notify_all()

    th = threading.Thread(target=producer, daemon=True)
    th.start()
    t0 = time.perf_counter()
    inflight: Dict[int, tuple] = {}
    done: List[Completed] = []
    submitted = 0
    ticks = 0
    lag = []
    while len(done) < len(trace):
        now = time.perf_counter() - t0
        with lock:
            while ready and ready[0][0].arrival_s <= now:
                req, P, t_ready = ready.popleft()
                rid = srv.submit(P, req.n_steps, opts, keep_output=keep_output)
                inflight[rid] = (req, time.perf_counter() - t0)
                lag.append(max(0.0, (t_ready - t0) - req.arrival_s))
                submitted += 1
            lock.notify_all()
        if srv.pending:
            n_done = srv.poll()
            ticks += 1
            if n_done:
                for rid in list(inflight):
                    got = srv.take(rid)
                    if got is None:
                        continue
                    outs, cells, info = got
                    req, t_sub = inflight.pop(rid)
                    done.append(Completed(req.rid, info["status"], info["steps_done"], info["iterations"], cells,
                                          req.arrival_s, t_sub, info["admit_s"], time.perf_counter() - t0,
                                          *(outs if outs is not None else (None, None, None)),
                                          energy_before=info["energy_before"], energy_after=info["energy_after"]))
        else:
            time.sleep(0.0005)
    stop[0] = True
    th.join(timeout=5)
    srv.close()
    t_end = max(c.done_s for c in done)
    lat = [c.done_s - c.arrival_s for c in done]
    cell_steps = sum(c.cells * c.steps for c in done)
    span = t_end - min(c.arrival_s for c in done)
    return {"requests": len(done), "ticks": ticks, "cell_steps": cell_steps, "makespan_s": span,
            "throughput_cell_updates_per_s": cell_steps / span,
            "latency_p50_s": _percentile(lat, 50), "latency_p99_s": _percentile(lat, 99),
            "latency_max_s": max(lat), "input_lag_p99_s": _percentile(lag, 99),
            "failed": sum(1 for c in done if c.status not in (0, 4)),
            "offered_cell_updates_per_s": cell_steps / max(1e-9, trace[-1].arrival_s - trace[0].arrival_s)
            if len(trace) > 1 else float("nan"),
            "completed": done}
