"""FP64 CPU oracle for the multilevel (SMR) matrix of Sec. 3.2.2 (Eq. linearsys1_amr).

TEST INFRASTRUCTURE ONLY.  Only the tests may import this module; it shares nothing with
the CUDA library.

The grid is a uniform Cartesian base grid of nx x ny cells (widths dx, dy) in which one
rectangle of base cells, columns [i0, i1) by rows [j0, j1), is replaced by fine cells
of half the width (refinement ratio 2).  The radiation step is the single-level step
(Sec. 3.2.1: backward Euler, linearised (T^{n+1})^4, FLD face coefficients, T eliminated
from the local psi row), assembled over the composite cell list in one matrix, as
Sec. 3.2.2 does: a coarse cell next to the patch couples directly to each fine cell
across its side, so that side carries two faces, each with the fine face's area and its
own D, and the coarse cell has five neighbours (Eq. linearsys1_amr).  Both cells of a
face use the same weight, so the fluxes leaving the coarse cell are those entering the
fine cells.

Readings where the text leaves the discretisation open (the same as on one level):
- face values of E and kappa_R rho are linear in the normal coordinate between the two
  cell centres, and the gradient in R is their normal difference over the normal
  distance (3/4 of a coarse width across the level jump); the tangential offset of the
  coarse centre from the fine face is not used;
- D = c lambda(R) / sigma_face > 0; Milne faces as on one level; reflecting faces carry
  nothing; ideal-gas C_V, opacities at T^n, kappa_e = kappa_P.

The matrix is assembled explicitly and solved by scipy's sparse direct solver.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import constants, limiter as _limiter


@dataclasses.dataclass
class Composite:
    nx: int
    ny: int
    dx: float
    dy: float
    i0: int
    i1: int
    j0: int
    j1: int

    def refined(self, i: int, j: int) -> bool:
        return self.i0 <= i < self.i1 and self.j0 <= j < self.j1


def cells(g: Composite):
    """Composite cell list: the base cells outside the patch (row-major), then the fine
    cells (row-major over the 2 (i1-i0) x 2 (j1-j0) fine grid).  Returns a dict of arrays
    x, y (centres), hx, hy (widths), level (0 / 1) and the index maps coarse[j, i] and
    fine[J, I] (-1 where absent)."""
    x, y, hx, hy, lev = [], [], [], [], []
    coarse = -np.ones((g.ny, g.nx), dtype=np.int64)
    for j in range(g.ny):
        for i in range(g.nx):
            if not g.refined(i, j):
                coarse[j, i] = len(x)
                x.append((i + 0.5) * g.dx); y.append((j + 0.5) * g.dy)
                hx.append(g.dx); hy.append(g.dy); lev.append(0)
    nfx, nfy = 2 * (g.i1 - g.i0), 2 * (g.j1 - g.j0)
    fine = -np.ones((max(nfy, 0), max(nfx, 0)), dtype=np.int64)
    for J in range(nfy):
        for I in range(nfx):
            fine[J, I] = len(x)
            x.append(g.i0 * g.dx + (I + 0.5) * 0.5 * g.dx); y.append(g.j0 * g.dy + (J + 0.5) * 0.5 * g.dy)
            hx.append(0.5 * g.dx); hy.append(0.5 * g.dy); lev.append(1)
    return {"x": np.array(x), "y": np.array(y), "hx": np.array(hx), "hy": np.array(hy),
            "level": np.array(lev), "coarse": coarse, "fine": fine}


def _owner(g: Composite, c, px, py):
    """The composite cell containing point (px, py) (inside the domain)."""
    i, j = int(px // g.dx), int(py // g.dy)
    if g.refined(i, j):
        I = int((px - g.i0 * g.dx) // (0.5 * g.dx))
        J = int((py - g.j0 * g.dy) // (0.5 * g.dy))
        return int(c["fine"][J, I])
    return int(c["coarse"][j, i])


def faces(g: Composite, c):
    """Interior faces (k, m, axis, area, position of the face along the normal), k on the
    lower side, and boundary faces (k, side, area) with side -x, +x, -y, +y = 0..3.  Each
    face is the smaller of the two cells' sides, so a coarse side next to the patch
    splits into two faces."""
    inner, bnd = [], []
    n = len(c["x"])
    for k in range(n):
        xk, yk, hxk, hyk = c["x"][k], c["y"][k], c["hx"][k], c["hy"][k]
        # the +x side of k, in pieces as small as the finer neighbour's side
        for axis in (0, 1):
            h_norm, h_tan = (hxk, hyk) if axis == 0 else (hyk, hxk)
            face_pos = (xk if axis == 0 else yk) + 0.5 * h_norm
            edge = g.nx * g.dx if axis == 0 else g.ny * g.dy
            lo_tan = (yk if axis == 0 else xk) - 0.5 * h_tan
            if face_pos >= edge * (1 - 1e-14):
                bnd.append((k, 1 if axis == 0 else 3, h_tan))
                continue
            pieces = 2 if c["level"][k] == 0 else 1
            # a coarse cell whose +side neighbour region is refined splits into two
            # pieces; otherwise the side is one face
            probe = [lo_tan + (p + 0.5) * h_tan / pieces for p in range(pieces)]
            owners = [(_owner(g, c, face_pos + 1e-9 * g.dx, t) if axis == 0 else
                       _owner(g, c, t, face_pos + 1e-9 * g.dy)) for t in probe]
            if pieces == 2 and owners[0] == owners[1]:
                inner.append((k, owners[0], axis, h_tan, face_pos))
            else:
                for m in owners:
                    inner.append((k, m, axis, h_tan / pieces, face_pos))
        # -x and -y sides: only the domain boundary here (every interior face is added
        # once, from the cell on its lower side)
        if abs(xk - 0.5 * hxk) < 1e-14 * g.dx:
            bnd.append((k, 0, hyk))
        if abs(yk - 0.5 * hyk) < 1e-14 * g.dy:
            bnd.append((k, 2, hxk))
    return inner, bnd


def _opacity(k, rho, T):
    k0, k1, a, b = k
    return np.full_like(rho, k0) if k1 == 0.0 else k0 + k1 * rho ** a * T ** b


def step(g: Composite, rho, eg, E, *, kR, kP, gamma, mu, dt, bc, lim, S_adv=None) -> dict:
    """One implicit step on the composite grid; rho, eg, E are per composite cell (the
    order of cells()).  Returns E_r, T_g, e_g, the reduced matrix A (scipy CSR, rows times
    V) and its right-hand side, and the energies before and after."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    K = constants()
    c = cells(g)
    n = len(c["x"])
    V = c["hx"] * c["hy"]
    CV = rho * K["kB"] / ((gamma - 1.0) * mu * K["mH"])
    T = eg / CV
    sig = _opacity(kR, rho, T) * rho
    beta = _opacity(kP, rho, T) * rho * K["c"] * dt
    aT3 = K["aR"] * T ** 3
    psi6 = CV + 4.0 * beta * aT3
    inner, bnd = faces(g, c)
    rows, cols, vals = [], [], []
    diag = V * (1.0 + beta * CV / psi6)
    for (k, m, axis, area, fpos) in inner:
        pk = c["x"][k] if axis == 0 else c["y"][k]
        pm = c["x"][m] if axis == 0 else c["y"][m]
        d = pm - pk
        th = (fpos - pk) / d
        sf = sig[k] + th * (sig[m] - sig[k])
        Ef = E[k] + th * (E[m] - E[k])
        R = abs(E[m] - E[k]) / (d * sf * Ef)
        D = K["c"] * float(_limiter(lim, R)[0]) / sf
        w = dt * area * D / d
        diag[k] += w
        diag[m] += w
        rows += [k, m]; cols += [m, k]; vals += [-w, -w]
    for (k, side, area) in bnd:
        if bc[side] != 1:
            continue
        h = 0.5 * (c["hx"][k] if side < 2 else c["hy"][k])
        kk = 2.0 / (3.0 * sig[k] * h)
        Db = K["c"] * float(_limiter(lim, 1.5)[0]) / sig[k]
        diag[k] += dt * area * Db / (h * (1.0 + kk))
    rows += list(range(n)); cols += list(range(n)); vals += list(diag)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    Ea = E + (0.0 if S_adv is None else S_adv * dt)
    rhs = V * (Ea + beta * K["aR"] * T ** 4 * CV / psi6)
    En = spl.spsolve(A.tocsc(), rhs)
    Tn = (CV * T + 3.0 * beta * K["aR"] * T ** 4 + beta * En) / psi6
    en = eg + CV * (Tn - T)
    return {"E_r": En, "T_g": Tn, "e_g": en, "A": A, "rhs": rhs,
            "energy_before": float((V * (E + eg)).sum()), "energy_after": float((V * (En + en)).sum())}
