"""CPU checks of the seeded workload generators (shapes, ranges, determinism)."""
import math

import numpy as np

from paper_2602_12545_gb300 import workloads as W


def test_deterministic_and_shaped():
    a, b = W.config0(), W.config0()
    assert np.array_equal(a.rho, b.rho) and np.array_equal(a.E_r, b.E_r)
    assert a.rho.shape == (64, 64) and a.x_faces.size == 65
    T = a.e_g / (a.rho * W.EG_PER_RHO_T)
    assert T.min() >= 1e3 * (1 - 1e-12) and T.max() <= 1e5 * (1 + 1e-12)
    med = np.median(np.log10(a.rho))
    assert abs(med + 9) < 0.2


def test_config1_and_2_grids():
    P1 = W.config1(n=64)
    dx = np.diff(P1.x_faces)
    np.testing.assert_allclose(dx[1:] / dx[:-1], 1.002, rtol=1e-12)
    assert P1.bc == (0, 1, 0, 0)
    P2 = W.config2(nr=64, nth=32)
    assert P2.x_faces[0] == 1e11 and abs(P2.x_faces[-1] / 1e14 - 1) < 1e-12
    assert P2.y_faces[0] == 0.0 and P2.y_faces[-1] == math.pi
    assert P2.precision == W.PREC_MIXED and P2.coord == W.SPHERICAL


def test_batch_sizes_and_trace():
    nxs, nys, dts = W.batch_sizes(256)
    assert nxs.min() >= 32 and nxs.max() <= 512 and 1e3 <= dts.min() and dts.max() <= 1e6
    expected = (512 ** 2 - 32 ** 2) / (2 * math.log(16))     # E[n^2] for log-uniform n
    assert 0.5 * expected < np.mean(nxs.astype(float) ** 2) < 2 * expected
    tr = W.config4_trace(2000)
    gaps = np.diff([r.arrival_s for r in tr])
    assert abs(np.mean(gaps) - 1 / 2000) < 0.1 / 2000
    sides = np.array([r.side for r in tr])
    assert sides.min() >= 64 and sides.max() <= 2048
