"""The benchmark's reference arm (the FP64 CPU oracle on the host cores) runs without a GPU:
its JSON line carries the contract keys, only rank 0 prints under a multi-rank launch, and
the workloads the oracle baseline does not cover say so in one line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=e,
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return [json.loads(l) for l in p.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_line():
    (line,) = run(["--impl", "reference", "--workload", "c0", "--steps", "1", "--warmup", "0"])
    assert line["impl"] == "reference"
    assert line["unit"] == "cell-updates/s" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 0 and line["n_gpus"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["cells"] == 64 * 64
    # the 64 x 64 workload is timed on full oracle steps, and one full step is reported
    assert line["extrapolated"] is False
    assert line["full_oracle_step"]["steps_run"] == 1 and line["full_oracle_step"]["iterations"] > 0


def test_oracle_iteration_counts_recorded():
    """The CPU baseline's extrapolation count comes from the oracle's own full steps."""
    with open(os.path.join(ROOT, "oracle", "iteration_counts.json")) as f:
        counts = json.load(f)
    for name in ("c0", "c1", "c2"):
        assert counts[name]["iterations"] > 0 and counts[name]["status"] == 0
        assert counts[name]["cell_residual"] <= counts[name]["tol"] * 1.01


def test_reference_arm_only_rank0_prints():
    out = run(["--impl", "reference", "--workload", "c0", "--steps", "1", "--warmup", "0"],
              env={"RANK": "1", "WORLD_SIZE": "2"})
    assert out == []


@pytest.mark.parametrize("workload", ["batched", "serving"])
def test_reference_arm_unavailable_for_multi_problem_workloads(workload):
    (line,) = run(["--impl", "reference", "--workload", workload])
    assert line["impl"] == "reference" and "unavailable" in line
