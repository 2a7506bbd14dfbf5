#!/usr/bin/env python3
"""Benchmark of the GB300 implicit FLD radiation step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c2|c1|c0] [--rtol R]

A step is one implicit FLD step (coefficients, opacities, limiter, reduced 5-point
system, Krylov solve, back-substitution, energy sums) over the whole grid.  The default
workload is the 2048 (r) x 1024 (theta) spherical-polar grid in mixed precision (FP32
inner PCG, FP64 refinement).  Rank 0 prints one JSON line.

Timing: W untimed warm-up steps, then K steps bracketed by a barrier and a device
synchronisation; each step is timed with CUDA events on the launching stream.  Before
every step the inputs are restored from a pristine copy and L2 is flushed (a 512 MiB
write); both happen outside the per-step events.

--impl reference times the FP64 CPU oracle (plain C, one host core): one full oracle
step to convergence, then bounded samples of the same workload (the full assembly plus a
fixed number of CG iterations) extrapolated to that step's iteration count.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FLD cell-updates/s at 1e-8 rel residual (FP32+refine vs FP64 GPU); p99 latency"
UNIT = "cell-updates/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0

# algorithmic bytes per cell (each array touched once per pass)
BYTES_ITER = {1: 32.0, 0: 64.0}       # 2 coefficients + (x, r, p) read and written
# one multigrid V-cycle per iteration, per fine cell: 4 level-0 sweeps (value, c_W, c_S
# in, value out: 16 B each), transfers (t twice, 8 B), z_old read (4 B), times 4/3 for
# the coarser levels, plus reading z in the direction pass (4 B); the FP64 path also
# writes the FP32 copy of its residual (4 B)
BYTES_VCYCLE = (4 * 16 + 8 + 4) * 4.0 / 3.0 + 4
BYTES_ITER_MG = {1: 32.0 + BYTES_VCYCLE, 0: 64.0 + BYTES_VCYCLE + 4.0}
BYTES_RESID = {1: 60.0, 0: 40.0}      # FP64 residual (c_W, c_S, b, y in; r out) [+ y += d for mixed]
KERNELS_PER_STEP = 7                  # cells, faces, diag, scale, solve, backsub, finalize (+ coarsen0: aggregation MG)
PRECOND_NAMES = {0: "Jacobi", 1: "aggregation multigrid V-cycle (FP32)",
                 2: "algebraic multigrid V-cycle (FP32), hierarchy built on the device every step"}
# default preconditioner per workload: the smooth spherical field converges fastest with
# the 2 x 2 aggregation cycle; i.i.d. fields (config-0 statistics) need the algebraic one
DEFAULT_PRECOND = {"c2": 1, "c1": 2, "c0": 2, "batched": 2, "serving": 2}


def amg_cycle_bytes(pi: dict, n0: int) -> float:
    """Algorithmic bytes of one algebraic V-cycle per fine cell, from the hierarchy the
    device built: level 0 (structured, FP32) 4 sweep/residual passes of 20 B and the
    transfers (P in ELL: 32 B, plus values) 120 B per cell; every coarse level applies its
    CSR operator 4 times (row pointer 4 B, column + value 8 B per entry) and moves its
    vectors (44 B per row); transfers 60 B per row of every level but the coarsest."""
    rows, ents = pi["rows"], pi["entries"]
    b = 120.0 * rows[0]
    for l in range(1, len(rows)):
        b += 60.0 * rows[l] + 32.0 * ents[l]
    for l in range(len(rows) - 1):
        b += 60.0 * rows[l]
    return b / n0
# batched and served problems (config-0 fields): the cell-wise residual that keeps every
# cell within 1e-8 of the oracle
SERVE_RTOL = 1e-10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["c2", "c1", "c0", "batched", "serving"], default="c2")
    ap.add_argument("--problems", type=int, default=256, help="batched: number of problems")
    ap.add_argument("--requests", type=int, default=400, help="serving: requests in the trace")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: mean arrival rate (1/s)")
    ap.add_argument("--budget-gb", type=float, default=60.0, help="serving: device memory budget")
    ap.add_argument("--rtol", type=float, default=None)
    ap.add_argument("--c2-grid", default=None,
                    help="NRxNTH: draw the spherical workload on a smaller grid (profiling captures only)")
    ap.add_argument("--precond", type=int, default=None,
                    help="0 Jacobi, 1 aggregation multigrid, 2 algebraic multigrid (default: per workload)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison path")
    ap.add_argument("--untiled", action="store_true", help="use the untiled solve kernel (comparison)")
    ap.add_argument("--block-cells", type=int, default=0,
                    help="multigrid levels of at most this many cells run in one block (0: library default)")
    ap.add_argument("--inner-rtol", type=float, default=None,
                    help="mixed precision: FP32 residual drop that triggers an FP64 refinement (default: library's)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="single-grid workloads: skip the compact batched and serving measurements")
    args = ap.parse_args()
    if args.precond is None:
        args.precond = DEFAULT_PRECOND[args.workload]
    return args


def workload(name, c2_grid=None):
    """The named workload; c2_grid = (nr, ntheta) draws the spherical one's fields on a
    smaller grid (profiling captures; the benchmark's line uses 2048 x 1024)."""
    from paper_2602_12545_gb300 import workloads as W
    if name == "c2" and c2_grid is not None:
        nr, nth = c2_grid
        P = W.config2(nr=nr, nth=nth)
        P.name = f"c2_sph{nr}x{nth}"
        return P, (f"{nr} (r, log 1e11-1e14 cm) x {nth} (theta 0-pi) spherical-polar, Milne at outer r, "
                   "dt=1e4 s (reduced grid)")
    P = {"c0": W.config0, "c1": W.config1, "c2": W.config2}[name]()
    desc = {"c0": "64x64 uniform Cartesian, reflecting, dt=1e4 s",
            "c1": "1024x1024 Cartesian, dx geometric x1.002, Milne at +x, dt=1e5 s",
            "c2": "2048 (r, log 1e11-1e14 cm) x 1024 (theta 0-pi) spherical-polar, Milne at outer r, dt=1e4 s"}[name]
    return P, desc


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
    return local_rank


def traffic_from_profile(kernel_tag, src_hash):
    """Per-launch DRAM bytes of the solve kernel from a committed ncu summary, if that
    summary was taken on the current kernel source (same hash), else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("source_sha256") != src_hash:
            return None
        return float(d["dram_bytes_per_launch_full_size"])
    except Exception:
        return None


def kernel_source_hash():
    """Hash of the solver kernel's sources with comments and blank space removed, so that
    a committed ncu figure stays attached to the code it was measured on."""
    import re
    h = hashlib.sha256()
    for name in ("gq_pcg.cuh", "gq_pcg_mixed.cu", "gq_pcg_fp64.cu", "gq_pcg_batch.cu", "gq_pcg_tiled.cu", "gq_mg.cuh",
                 "gq_amg.cuh", "gq_device.cuh", "gq_internal.h"):
        with open(os.path.join(ROOT, "paper_2602_12545_gb300", "csrc", name)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("".join(src.split()).encode())
    return h.hexdigest()


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ---------------------------------------------------------------------------

def oracle_sample(P, iters_needed, cg_iters=60):
    import numpy as np
    import oracle
    t0 = time.perf_counter()
    A, b = oracle.assemble_reduced(P)
    t1 = time.perf_counter()
    _, it, _, _ = oracle.pcg(A, b, P.E_r.ravel().copy(), tol=0.0, maxit=cg_iters)
    t2 = time.perf_counter()
    t_iter = (t2 - t1) / max(it, 1)
    t_step = (t1 - t0) + iters_needed * t_iter
    return {"value": P.ncells / t_step, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"oracle assembly of the full {P.nx}x{P.ny} reduced system plus {it} Jacobi-PCG "
                       f"iterations on it, extrapolated to {iters_needed} iterations (the oracle's own "
                       f"Jacobi-PCG count for the full step at the same tolerance); single host thread"),
            "t_assembly_s": t1 - t0, "t_per_iteration_s": t_iter}, t2 - t0


# ---------------------------------------------------------------------------
# ranks: one process per GPU, independent replicas (no data-path collective)
# ---------------------------------------------------------------------------

def dist_init(world, local):
    """Joins the process group of a torchrun launch: NCCL on GPUs, gloo without one."""
    import torch
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        if torch.cuda.is_available():
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")


def job_ms(local_ms, world):
    """The slowest rank's timed total: a barrier, then a max over the ranks."""
    if world <= 1:
        return local_ms
    import torch
    import torch.distributed as dist
    dist.barrier()
    t = torch.tensor([local_ms], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank / (ms / 1e3)


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2602_12545_gb300 import fld as F

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist_init(world, local)

    def barrier():
        if world > 1:
            dist.barrier()

    c2_grid = tuple(int(v) for v in args.c2_grid.lower().split("x")) if args.c2_grid else None
    P, desc = workload(args.workload, c2_grid)
    # the workload's cell-wise residual target (for the spherical grid the loosest setting
    # whose E and T agree with the tightly solved FP64 answer to 1e-8 per cell, reported)
    rtol = args.rtol if args.rtol is not None else P.rtol
    prec = 1 if args.workload == "c2" else P.precision
    plan = F.FLDPlan.for_problem(P)
    rho0, eg0, E0, _ = F.device_fields(P)
    rho = rho0
    e_g, E, T = eg0.clone(), E0.clone(), torch.empty_like(E0)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def one(opts, check=True):
        e_g.copy_(eg0)
        E.copy_(E0)
        flush.fill_(1.0)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        info = plan.step(rho, e_g, E, T, opacity_R=P.opacity_R, opacity_P=P.opacity_P, gamma=P.gamma, mu=P.mu,
                         dt=P.dt, bc=P.bc, opts=opts, check=check)
        s1.record(stream)
        s1.synchronize()
        info["ms"] = s0.elapsed_time(s1)
        return info

    extra = {} if args.inner_rtol is None else {"inner_rtol": args.inner_rtol}
    opts = F.SolverOptions(prec=prec, limiter=P.limiter, rtol=rtol, timing=1, precond=args.precond,
                           untiled=int(args.untiled), mg_block_cells=args.block_cells, **extra)
    # accuracy reference: FP64 path solved tightly (untimed)
    ref_opts = F.SolverOptions(prec=0, limiter=P.limiter, rtol=1e-13, timing=0, max_iter=1000000)
    ref_info = one(ref_opts, check=False)       # may stop at the FP64 floor (status 4)
    if ref_info["status"] not in (0, 4):
        raise RuntimeError(f"reference solve failed: {ref_info}")
    E_ref, T_ref = E.clone(), T.clone()

    for _ in range(args.warmup):
        one(opts)

    clocks = Clocks(gpu_index(local))
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall0 = time.perf_counter()
    infos = [one(opts) for _ in range(args.steps)]
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    barrier()
    ck = clocks.stop()
    err_E = float(((E - E_ref).abs() / E_ref.abs()).max())
    err_T = float(((T - T_ref).abs() / T_ref.abs()).max())

    total_ms = job_ms(sum(i["ms"] for i in infos), world)
    N = P.ncells
    value = job_value(N * args.steps, world, total_ms)
    lat = sorted(i["ms"] for i in infos)
    p50 = statistics.median(lat)
    p99 = lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]
    its = statistics.mean(i["iterations"] for i in infos)
    refs = statistics.mean(i["refinements"] for i in infos)
    t_solve = statistics.mean(i["t_solve_ms"] for i in infos)
    t_setup = statistics.mean(i["t_setup_ms"] for i in infos)
    t_finish = statistics.mean(i["t_finish_ms"] for i in infos)
    t_pre = statistics.mean(i["t_precond_ms"] for i in infos)
    if args.precond == 2:
        b_iter = BYTES_ITER[prec] + 4.0 + amg_cycle_bytes(plan.precond_info(), N)
    elif args.precond == 1:
        b_iter = BYTES_ITER_MG[prec]
    else:
        b_iter = BYTES_ITER[prec]
    alg_bytes = N * (its * b_iter + (refs + 1) * BYTES_RESID[prec])
    # device-clock breakdown of the last timed step's solve, per Krylov iteration
    cycle_us = None
    if args.precond in (1, 2):
        pi = plan.precond_info()
        n_it = max(1, infos[-1]["iterations"])
        cycle_us = {"levels": [round(1e3 * v / n_it, 2) for v in pi["cycle_ms"]],
                    "direction": round(1e3 * pi["direction_ms"] / n_it, 2),
                    "update": round(1e3 * pi["update_ms"] / n_it, 2),
                    "refine": round(1e3 * pi["refine_ms"] / n_it, 2),
                    "after_cycle": round(1e3 * pi["after_cycle_ms"] / n_it, 2)}
    solve_kernel = "k_pcg_tiled" if infos[-1]["solve_kernel"] == 1 else f"k_pcg<{'true' if prec else 'false'}>"
    achieved = alg_bytes / (t_solve / 1e3) / 1e9
    peak, peak_kind = peaks()
    tag = ("pcg_tiled_c2" if solve_kernel == "k_pcg_tiled" else
           f"pcg_{'mixed' if prec else 'fp64'}_{args.workload}")
    # the committed DRAM figure is for the full-size grid: none for a reduced one
    traffic = traffic_from_profile(tag, kernel_source_hash()) if c2_grid is None else None
    if traffic is not None:
        traffic = traffic

    # FP64 GPU path on the same workload and tolerance
    fp64 = None
    if not args.no_fp64 and prec == 1:
        f_opts = F.SolverOptions(prec=0, limiter=P.limiter, rtol=rtol, timing=1, precond=args.precond)
        one(f_opts)
        f_infos = [one(f_opts) for _ in range(max(1, min(args.steps, 3)))]
        f_ms = statistics.mean(i["ms"] for i in f_infos)
        f_err = float(((E - E_ref).abs() / E_ref.abs()).max())
        fp64 = {"value": N / (f_ms / 1e3), "unit": UNIT, "ms_per_step": f_ms,
                "iterations": statistics.mean(i["iterations"] for i in f_infos),
                "max_rel_err_E_vs_fp64_tight": f_err, "steps": len(f_infos)}

    # end to end: pinned host inputs -> device, step, results -> host, every step
    e2e = None
    if not args.no_e2e:
        h_rho = rho0.cpu().pin_memory()
        h_eg = eg0.cpu().pin_memory()
        h_E = E0.cpu().pin_memory()
        o_E, o_eg, o_T = (torch.empty_like(h_E).pin_memory() for _ in range(3))
        d_rho = torch.empty_like(rho0)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n_e2e = max(1, min(args.steps, 3))
        for _ in range(n_e2e):
            d_rho.copy_(h_rho, non_blocking=True)
            e_g.copy_(h_eg, non_blocking=True)
            E.copy_(h_E, non_blocking=True)
            plan.step(d_rho, e_g, E, T, opacity_R=P.opacity_R, opacity_P=P.opacity_P, gamma=P.gamma, mu=P.mu,
                      dt=P.dt, bc=P.bc, opts=opts)
            o_E.copy_(E, non_blocking=True)
            o_eg.copy_(e_g, non_blocking=True)
            o_T.copy_(T, non_blocking=True)
            torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        barrier()
        e2e = {"value": world * N * n_e2e / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 3 * 8 * N,
               "d2h_bytes_per_step": 3 * 8 * N, "steps": n_e2e}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # the oracle's solver is Jacobi-PCG: a bounded sample (assembly + 60 iterations)
        # extrapolated to the iteration count of the oracle's own full step, which
        # oracle/iteration_counts.json records (the reference arm re-measures it)
        cnt = oracle_iterations(args.workload)
        cpu, _ = oracle_sample(P, int(cnt["iterations"]))
        cpu["extrapolated"] = True
        cpu["full_step_seconds_recorded"] = cnt["seconds_one_thread"]

    # compact batched (the 256-problem batch) and serving (a short trace, saturated and
    # below saturation) measurements beside the headline, single-GPU runs only
    batched = serving = None
    if world == 1 and not args.no_extra and args.workload == "c2":
        _, _, batched, _ = batched_measure(256, 3, 1, 2, local, oracle_members=(0, 64, 128, 192))
        sat = serving_measure(48, 2000.0, args.budget_gb, 2, fp64_sample=8)
        sub = serving_measure(16, 4.0, args.budget_gb, 2, fp64_sample=0)
        # below saturation: the offered load against the saturated throughput (the trace's
        # own makespan includes the last requests' service time, so its ratio says nothing)
        sub["overloaded"] = sub["offered_cell_updates_per_s"] > sat["throughput_cell_updates_per_s"]
        sub["offered_over_capacity"] = sub["offered_cell_updates_per_s"] / sat["throughput_cell_updates_per_s"]
        keys = ("requests", "throughput_cell_updates_per_s", "offered_cell_updates_per_s", "overloaded",
                "latency_p50_s", "latency_p99_s", "makespan_s", "failed", "rate_per_s")
        serving = {"saturated": {k: sat[k] for k in keys},
                   "below_saturation": {k: sub[k] for k in keys + ("offered_over_capacity",)},
                   "one_at_a_time_fp64": sat["one_at_a_time_fp64"],
                   "trace": "Poisson arrivals, square sides log-uniform in [64, 2048], 10 steps each, "
                            f"{args.budget_gb:g} GB budget, mixed precision, cell-wise residual {SERVE_RTOL:g}, "
                            "algebraic multigrid"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if prec == 1 else "f64",
        "data": "synthetic",
        "config": {"workload": f"{P.name}_{'mixed' if prec else 'fp64'}", "grid": desc, "nx": P.nx, "ny": P.ny,
                   "cells": N, "precision": "FP32 inner PCG + FP64 refinement" if prec else "FP64 PCG",
                   "rtol": rtol, "residual": "cell-wise max |b-Ax|_k/(A_kk x_k) of the reduced system",
                   "preconditioner": PRECOND_NAMES[args.precond],
                   "l2": "inputs restored and L2 flushed (512 MiB write) before every step, outside the timed events",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "step_latency_ms": {"p50": p50, "p99": p99},
        "solver": {"iterations": its, "refinements": refs, "rel_residual": infos[-1]["rel_residual"],
                   "rel_residual_l2": infos[-1]["rel_residual_l2"], "max_rel_err_E_vs_fp64_tight": err_E,
                   "max_rel_err_T_vs_fp64_tight": err_T, "t_setup_ms": t_setup, "t_solve_ms": t_solve,
                   "t_finish_ms": t_finish, "t_precond_build_ms": t_pre,
                   "t_per_iteration_us": statistics.mean(i["t_iter_us"] for i in infos),
                   "precond_levels": infos[-1]["precond_levels"], "solve_blocks": infos[-1]["solve_blocks"],
                   "solve_kernel": solve_kernel, "cycle_us_per_iteration": cycle_us},
        "roofline": {"kernel": f"{solve_kernel} (persistent cooperative Krylov solve)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": peak_kind, "traffic": traffic,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "bytes_per_cell": {"iteration": b_iter, "fp64_residual": BYTES_RESID[prec]}},
        "fp64_gpu": fp64,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": (KERNELS_PER_STEP + (1 if args.precond == 1 else 0)) * args.steps,
        "clocks": ck,
        "wall_s_timed_loop": t_wall,
        "batched": batched,
        "serving": serving,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def _batch_line(args, world, value, total_ms, infos, extra):
    statuses = {}
    for i in infos:
        statuses[i["status"]] = statuses.get(i["status"], 0) + 1
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", **extra,
        "status_counts": statuses,
    }


def _c3_oracle_member(p):
    """Oracle answer for member p of the 256-problem batch (spawned worker)."""
    import oracle
    from paper_2602_12545_gb300 import workloads as W
    P = W.config3(256)[p]
    return p, oracle.step(P, "cg", tol=1e-14)["E_r"]


def batched_measure(n_problems, steps, warmup, precond, local, oracle_members=()):
    """The batched workload: n_problems independent problems of uneven size (32..512 per
    side, Cartesian and spherical-polar alternating, dt 1e3..1e6 s) in one persistent
    launch replayed from a CUDA graph, schedule chosen by the autotuner (untimed, once).
    Returns the per-step device times, the step infos and a summary; oracle_members are
    compared cell by cell with the oracle (computed in spawned workers meanwhile)."""
    import multiprocessing as mp
    import numpy as np
    import torch
    from paper_2602_12545_gb300 import fld as F
    from paper_2602_12545_gb300 import workloads as W
    pool = res = None
    if oracle_members:
        pool = mp.get_context("spawn").Pool(min(len(oracle_members), max(1, (os.cpu_count() or 2) - 1)))
        res = pool.map_async(_c3_oracle_member, list(oracle_members), chunksize=1)
    probs = W.config3(n_problems)
    plans = [F.FLDPlan.for_problem(P) for P in probs]
    pristine = [F.device_fields(P) for P in probs]
    fields = [(r, e.clone(), E.clone(), T.clone()) for (r, e, E, T) in pristine]
    opts = [F.SolverOptions(prec=1, limiter=P.limiter, rtol=P.rtol, precond=precond) for P in probs]
    B = F.FLDBatch(plans)
    t_tune = time.perf_counter()
    tuned = B.autotune(probs, fields, opts)
    t_tune = time.perf_counter() - t_tune
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def restore():
        for (r, e, E, T), (r0, e0, E0, T0) in zip(fields, pristine):
            e.copy_(e0)
            E.copy_(E0)
        flush.fill_(1.0)
        torch.cuda.synchronize()

    for _ in range(warmup):
        restore()
        B.step(probs, fields, opts, check=False)
    clocks = Clocks(gpu_index(local))
    torch.cuda.synchronize()
    clocks.start()
    ms, infos = [], None
    for _ in range(steps):
        restore()
        rc, infos = B.step(probs, fields, opts, check=False)
        ms.append(B.last_ms)
    ck = clocks.stop()
    cells = sum(P.ncells for P in probs)
    errs = {}
    if res is not None:
        for p, E_ref in res.get(timeout=900):
            E = fields[p][2].cpu().numpy()
            errs[probs[p].name] = float(np.max(np.abs(E - E_ref) / np.abs(E_ref)))
        pool.close()
        pool.join()
    its = [i["iterations"] for i in infos]
    statuses = {}
    for i in infos:
        statuses[i["status"]] = statuses.get(i["status"], 0) + 1
    summary = {"problems": len(probs), "cells": cells, "value": cells * steps / (sum(ms) / 1e3), "unit": UNIT,
               "ms_per_step": statistics.mean(ms), "steps": steps, "autotuned": tuned, "autotune_s": t_tune,
               "graph": B.uses_graph, "iterations_mean": float(np.mean(its)), "iterations_max": int(np.max(its)),
               "status_counts": statuses, "rtol": probs[0].rtol,
               "max_rel_err_E_vs_oracle_sampled": max(errs.values()) if errs else None,
               "oracle_members": sorted(errs)}
    B.close()
    for p in plans:
        p.close()
    return ms, infos, summary, ck


def run_batched(args):
    """256 independent problems of uneven size in one persistent launch (batched_measure)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    torch.cuda.set_device(local)
    dist_init(world, local)
    members = tuple(range(0, args.problems, max(1, args.problems // 4))) if rank == 0 else ()
    ms, infos, summary, ck = batched_measure(args.problems, args.steps, args.warmup, args.precond, local, members)
    total_ms = job_ms(sum(ms), world)
    line = _batch_line(args, world, job_value(summary["cells"] * args.steps, world, total_ms), total_ms, infos, {
        "config": {"workload": f"c3_batch{summary['problems']}_mixed", "problems": summary["problems"],
                   "cells": summary["cells"],
                   "sides": "nx, ny log-uniform in [32, 512], Cartesian and spherical-polar alternating",
                   "rtol": summary["rtol"], "preconditioner": PRECOND_NAMES[args.precond],
                   "l2": "inputs restored and L2 flushed before every step, outside the timed events",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "batch": summary,
        "step_latency_ms": {"p50": statistics.median(ms), "p99": max(ms)},
        "gpu_launches": 9 * args.steps, "clocks": ck})
    if rank == 0:
        print(json.dumps(line), flush=True)


def serving_measure(requests, rate, budget_gb, precond, fp64_sample=40, side_hi=2048):
    """A finite Poisson trace (square grids 64..side_hi, 10 steps each) replayed in real
    time through the continuous-batching server, and the same requests (a sample) served
    one at a time on the plain FP64 path."""
    import torch
    from paper_2602_12545_gb300 import fld as F
    from paper_2602_12545_gb300 import serve as S
    from paper_2602_12545_gb300 import workloads as W
    trace = W.config4_trace(requests, rate_per_s=rate, side_hi=side_hi)
    # cell-wise residual 1e-10: every request's cells within 1e-8 of the oracle
    opts = F.SolverOptions(prec=1, limiter=0, rtol=SERVE_RTOL, precond=precond)
    budget = int(budget_gb * (1 << 30))
    warm = W.config4_trace(4, rate_per_s=rate, side_lo=64, side_hi=128, n_steps=2, seed=99)
    S.run_trace(warm, budget)
    out = S.run_trace(trace, budget, opts=opts)
    done = out.pop("completed")
    sample = trace[: min(len(trace), fp64_sample)]
    # one request at a time on the FP64 path: the steps alone, and (as the server counts a
    # request) with its plan set-up, the upload of its fields and the download of its results
    t_seq, t_all, cells_seq = 0.0, 0.0, 0
    for req in sample:
        P = W.serve_problem(req)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan = F.FLDPlan.for_problem(P)
        rho, e_g, E, T = F.device_fields(P)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(req.n_steps):
            F.step_problem(plan, P, rho, e_g, E, T, prec=0, rtol=SERVE_RTOL, check=False, precond=precond)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        host = (E.cpu(), e_g.cpu(), T.cpu())
        plan.close()
        t_all += time.perf_counter() - t0
        t_seq += t2 - t1
        cells_seq += P.ncells * req.n_steps
        del host
    out["one_at_a_time_fp64"] = ({"value": cells_seq / t_seq, "value_with_setup": cells_seq / t_all, "unit": UNIT,
                                  "requests_sampled": len(sample),
                                  "value_counts": "the steps alone",
                                  "value_with_setup_counts": "plan set-up, field upload, steps and result download"}
                                 if sample else None)
    out["overloaded"] = out["offered_cell_updates_per_s"] > out["throughput_cell_updates_per_s"]
    out["rate_per_s"] = rate
    out["requests_done"] = len(done)
    return out


def run_serving(args):
    """Continuous-batching serving of a finite Poisson trace (serving_measure)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist_init(world, local)
    clocks = Clocks(gpu_index(local))
    clocks.start()
    out = serving_measure(args.requests, args.rate, args.budget_gb, args.precond)
    ck = clocks.stop()
    # every rank serves the same trace on its own GPU: the job's time is the slowest makespan
    mk_ms = job_ms(1e3 * out["makespan_s"], world)
    line = {
        "metric": METRIC, "value": job_value(out["cell_steps"], world, mk_ms), "unit": UNIT, "n_gpus": world,
        "steps": args.requests, "warmup": 4, "ms_per_step": 1e3 * out["makespan_s"] / max(1, out["requests_done"]),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"c4_serving_{args.requests}req_{int(args.rate)}per_s", "requests": args.requests,
                   "rate_per_s": args.rate, "sides": "square, log-uniform in [64, 2048]", "steps_per_request": 10,
                   "budget_gb": args.budget_gb, "rtol": SERVE_RTOL,
                   "preconditioner": PRECOND_NAMES[args.precond]},
        "serving": out,
        "latency_s": {"p50": out["latency_p50_s"], "p99": out["latency_p99_s"]},
        "one_at_a_time_fp64": out["one_at_a_time_fp64"],
        "overloaded": out["overloaded"],
        "clocks": ck,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def oracle_iterations(name):
    """The oracle's own Jacobi-PCG iteration count for one full step of a workload, from
    oracle/iteration_counts.json (written by running the oracle alone to convergence)."""
    with open(os.path.join(ROOT, "oracle", "iteration_counts.json")) as f:
        return json.load(f)[name]


def run_reference(args):
    """The FP64 CPU oracle on the host cores (rank 0 only).  One full oracle step is run
    to convergence first (its time and iteration count are reported); each of the W + K
    steps after it is a bounded sample (the full assembly plus 30 iterations) extrapolated
    to the full step's iteration count, so that the run ends within a few minutes.  On the
    64 x 64 workload every step is a full step."""
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    if args.workload in ("batched", "serving"):
        print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle baseline is defined for the single-grid workloads (c0, c1, c2)"}))
        return
    P, desc = workload(args.workload)
    rtol = args.rtol if args.rtol is not None else P.rtol
    t0 = time.perf_counter()
    full = oracle.step(P, "cg", tol=rtol)
    t_full = time.perf_counter() - t0
    iters = int(full["iterations"])
    samples = []
    if args.workload == "c0":
        for _ in range(args.warmup):
            oracle.step(P, "cg", tol=rtol)
        for _ in range(args.steps):
            t0 = time.perf_counter()
            oracle.step(P, "cg", tol=rtol)
            samples.append(P.ncells / (time.perf_counter() - t0))
        sample_desc = f"{args.steps} full oracle steps (assembly + Jacobi-PCG to {rtol:g}); single host thread"
        extrapolated = False
    else:
        for _ in range(args.warmup):
            oracle_sample(P, iters, cg_iters=10)
        for _ in range(args.steps):
            s, _ = oracle_sample(P, iters, cg_iters=30)
            samples.append(s["value"])
        sample_desc = (f"one full oracle step ({iters} Jacobi-PCG iterations to {rtol:g}, {t_full:.1f} s), then "
                       f"{args.steps} samples of the full assembly plus 30 iterations, each extrapolated to "
                       f"{iters} iterations; single host thread")
        extrapolated = True
    v = statistics.mean(samples)
    ms = P.ncells / v * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{P.name}_{'mixed' if args.workload == 'c2' else 'fp64'}", "grid": desc,
                       "nx": P.nx, "ny": P.ny, "cells": P.ncells, "rtol": rtol},
            "extrapolated": extrapolated,
            "full_oracle_step": {"steps_run": 1, "seconds": t_full, "iterations": iters,
                                 "cell_residual": full["cell_residual"],
                                 "value": P.ncells / t_full, "unit": UNIT},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample_desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
