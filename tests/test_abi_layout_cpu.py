"""Host-side ABI check: every struct the binding passes through the C ABI has the size and
field offsets that include/gq_fld.h gives it, as gcc lays it out.  A probe program is
compiled against the header and prints sizeof / offsetof of each field; the ctypes
classes must agree.  No GPU, no CUDA."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2602_12545_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = {
    "gq_grid_desc": N.GridDesc, "gq_opacity_law": N.OpacityLaw, "gq_eos": N.Eos, "gq_bc": N.Bc,
    "gq_solver_opts": N.SolverOpts, "gq_step_info": N.StepInfo, "gq_precond_info": N.PrecondInfo,
    "gq_batch_item": N.BatchItem, "gq_batch_opts": N.BatchOpts, "gq_server_opts": N.ServerOpts,
    "gq_request": N.Request, "gq_request_info": N.RequestInfo, "gq_smr_grid": N.SmrGrid,
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gq_fld.h"', 'int main(void) {']
    for cname, cls in PAIRS.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ['return 0;', '}']
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "probe.c", d / "probe"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        cname, key, val = line.split()
        table[(cname, key)] = int(val)
    return table


@pytest.mark.parametrize("cname", list(PAIRS))
def test_struct_layout_matches_the_header(c_layout, cname):
    cls = PAIRS[cname]
    assert ctypes.sizeof(cls) == c_layout[(cname, "size")], cname
    for fname, _ in cls._fields_:
        assert getattr(cls, fname).offset == c_layout[(cname, fname)], (cname, fname)
