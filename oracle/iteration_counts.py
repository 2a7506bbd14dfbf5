"""Write oracle/iteration_counts.json: the number of Jacobi-PCG iterations the oracle's
own solver takes for one full step of each benchmark workload, at the cell-wise
tolerance the benchmark uses for it.

    python -m oracle.iteration_counts

Test and benchmark infrastructure only.  The CPU baseline extrapolates a bounded sample
of the oracle (assembly plus a few dozen iterations) to this count; the count comes from
running the oracle alone, to convergence, on the same seeded inputs.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OUT = os.path.join(HERE, "iteration_counts.json")

# workload -> cell-wise tolerance of the benchmark's line for it
TOLERANCES = {"c0": 1e-10, "c1": 1e-10, "c2": 2e-10}


def main():
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2602_12545_gb300 import workloads as W
    make = {"c0": W.config0, "c1": W.config1, "c2": W.config2}
    out = {}
    for name, tol in TOLERANCES.items():
        P = make[name]()
        t0 = time.perf_counter()
        r = oracle.step(P, "cg", tol=tol)
        out[name] = {"iterations": r["iterations"], "tol": tol, "cell_residual": r["cell_residual"],
                     "status": r["status"], "seconds_one_thread": time.perf_counter() - t0,
                     "cells": P.ncells}
        print(name, out[name], flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
