"""Compile the FP64 CPU oracle (plain C) into oracle/_build/liboracle.so.

Test infrastructure only: the oracle is the reference the CUDA path is checked
against, never part of the product path.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gq_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Build (if stale) and return the shared-library path.  -ffp-contract=off keeps the
    arithmetic identical on x86-64 and aarch64 hosts (no fused multiply-add contraction)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    hdr = os.path.join(HERE, "gq_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
           "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
