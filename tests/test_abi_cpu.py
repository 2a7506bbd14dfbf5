"""CPU checks of the C ABI: the library builds, loads and exports every entry point the
public header declares; host-only helpers answer.  No CUDA compute call is made."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(gq_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_2602_12545_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("gq_fld_setup", "gq_fld_step", "gq_fld_destroy", "gq_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_every_symbol(lib_path):
    from paper_2602_12545_gb300 import _native as N
    assert set(declared_functions()) <= set(N.SIGNATURES), set(declared_functions()) - set(N.SIGNATURES)
    L = N.load()
    for name in declared_functions():
        assert getattr(L, name) is not None


def test_host_helpers(lib_path):
    from paper_2602_12545_gb300 import _native as N
    L = N.load()
    assert L.gq_version().decode().count(".") == 2
    for code in range(8):
        assert len(L.gq_status_string(code)) > 0
    o = N.SolverOpts()
    L.gq_solver_opts_default(ctypes.byref(o))
    assert o.prec == 0 and o.rtol == 1e-10 and o.max_iter > 0 and 0 < o.inner_rtol < 1


def test_setup_rejects_bad_geometry_without_gpu(lib_path):
    """Argument validation happens before any CUDA call."""
    from paper_2602_12545_gb300 import _native as N
    import numpy as np
    L = N.load()
    g = N.GridDesc()
    h = ctypes.c_void_p()
    g.nx, g.ny, g.coord = 0, 4, 0
    assert L.gq_fld_setup(ctypes.byref(g), ctypes.byref(h)) == N.GQ_ERR_INVALID_ARG
    xf = np.array([0.0, 1.0, 0.5])            # not increasing
    yf = np.array([0.0, 1.0])
    g.nx, g.ny = 2, 1
    g.x_faces = xf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    g.y_faces = yf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.gq_fld_setup(ctypes.byref(g), ctypes.byref(h)) == N.GQ_ERR_INVALID_ARG
    assert L.gq_fld_step(None, None, None, None, None, None, None, 1.0, None, None, None, None) == N.GQ_ERR_INVALID_ARG


def test_package_fails_loudly_without_library(tmp_path):
    from paper_2602_12545_gb300 import _native as N
    with pytest.raises(RuntimeError, match="not built"):
        N.load.__wrapped__(str(tmp_path / "missing.so")) if hasattr(N.load, "__wrapped__") else _fresh_load(N, tmp_path)


def _fresh_load(N, tmp_path):
    saved = N._lib
    try:
        N._lib = None
        N.load(str(tmp_path / "missing.so"))
    finally:
        N._lib = saved


def test_smr_setup_rejects_bad_grids_on_the_host(lib_path):
    """gq_smr_setup validates the grid before touching the device: no GPU needed."""
    from paper_2602_12545_gb300 import _native as N
    L = N.load()
    for nx, ny, dx, dy, i0, i1, j0, j1 in ((0, 4, 1.0, 1.0, 0, 0, 0, 0), (4, 4, -1.0, 1.0, 0, 0, 0, 0),
                                           (4, 4, 1.0, float("nan"), 0, 0, 0, 0), (4, 4, 1.0, 1.0, 2, 5, 0, 2),
                                           (4, 4, 1.0, 1.0, 3, 1, 0, 2), (4, 4, 1.0, 1.0, 0, 2, -1, 2)):
        g = N.SmrGrid(nx, ny, dx, dy, i0, i1, j0, j1)
        h = ctypes.c_void_p()
        assert L.gq_smr_setup(ctypes.byref(g), ctypes.byref(h)) == N.GQ_ERR_INVALID_ARG
        assert not h.value
