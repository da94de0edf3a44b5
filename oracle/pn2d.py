"""The 2D reduction of the staggered P_N system (section "2D checkerboard").

TEST INFRASTRUCTURE ONLY (part of the FP64 CPU oracle; see oracle/__init__.py).

When every parameter, source and boundary condition is independent of z, so
is the solution.  In the 3D system, the coefficients that are odd under
z-reflection then vanish: those with l + m odd (parity bit p_z = (l + |m|)
mod 2 = 1).  The z-derivative terms also drop out. What remains is a system on
the square for the coefficients with l + m even:

  row (l, m) at location p = (x, y):
      sum_{d in {x, y}} sum_{k'} A_d[k, k'] (u_{k'}(p + h/2 e_d) - u_{k'}(p - h/2 e_d)) / h
    + (sigma_t(p) - sigma_s(p) g^l) u_k(p)                 = Q_k(p)

with the same angular couplings A_x, A_y as in 3D (they never mix l + m
parities), the parity placement restricted to (p_x, p_y), central differences
between grids half a cell apart, Dirichlet dropping at the boundary of the
closed square, and parameters interpolated as the mean of the adjacent
in-domain cell centres.

This module assembles that system directly in 2D (it does not call the 3D
assembler).  tests/test_oracle_2d.py pins it against the 3D oracle with a
z-periodic wrap and z-independent data.

Vector order: coefficient-major over the 2D coefficient list (l + m even, in
3D order k = l^2 + l + m), each coefficient's grid in C order [y][x].
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .sh import coupling_matrices, lm_list


def lm_list_2d(N: int):
    """[(l, m)] with l + m even, in 3D coefficient order."""
    return [(l, m) for (l, m) in lm_list(N) if (l + m) % 2 == 0]


def class_2d(l: int, m: int):
    """(p_x, p_y) of coefficient (l, m): odd under reflection of x, resp. y."""
    am = abs(m)
    px = (m % 2) if m >= 0 else ((am + 1) % 2)
    py = 1 if m < 0 else 0
    return px, py


class Layout2D:
    """Unknown locations of the 2D P_N system on an R x R grid of the unit square."""

    def __init__(self, N: int, R: int):
        if R < 2:
            raise ValueError("grid must have at least 2 cells per axis")
        self.N, self.R, self.h = N, R, 1.0 / R
        self.lm = lm_list_2d(N)
        self.K = len(self.lm)
        all_lm = lm_list(N)
        self.k3 = [all_lm.index(lm) for lm in self.lm]
        self.classes = [class_2d(l, m) for (l, m) in self.lm]
        self.shapes = [(R + c[1], R + c[0]) for c in self.classes]  # (ny, nx)
        sizes = [ny * nx for ny, nx in self.shapes]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.n = int(self.offsets[-1])

    def split(self, u: np.ndarray):
        return [u[self.offsets[k]:self.offsets[k + 1]].reshape(self.shapes[k]) for k in range(self.K)]

    def join(self, parts) -> np.ndarray:
        return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def interpolate_2d(F: np.ndarray, px: int, py: int) -> np.ndarray:
    """Centre field F[y, x] (R x R) -> mean over the in-domain centres adjacent
    to each location of class (px, py): along an odd axis, location i lies
    between centres i - 1 and i, and a boundary location sees one centre."""
    F = np.asarray(F, dtype=np.float64)
    R = F.shape[0]
    ny, nx = R + py, R + px
    out = np.zeros((ny, nx))
    for iy in range(ny):
        cy = [iy] if not py else [j for j in (iy - 1, iy) if 0 <= j < R]
        for ix in range(nx):
            cx = [ix] if not px else [j for j in (ix - 1, ix) if 0 <= j < R]
            out[iy, ix] = np.mean([F[a, b] for a in cy for b in cx])
    return out


def assemble_2d(N: int, R: int, sigma_t, albedo, g: float, Q, sigma_t_min: float = 0.0):
    """(Layout2D, A CSR, b) of the 2D system.  sigma_t, albedo (scalar or
    field) and Q are cell-centre arrays [y][x]; Q is the Q^{0,0} field (R, R)
    or the moments of the 2D coefficient list (K2, R, R)."""
    lay = Layout2D(N, R)
    A = coupling_matrices(N)
    st = np.maximum(np.asarray(sigma_t, dtype=np.float64), sigma_t_min)
    ss = np.asarray(albedo, dtype=np.float64) * st
    rows, cols, vals = [], [], []
    b = np.zeros(lay.n)
    Qa = np.asarray(Q, dtype=np.float64)
    for k, (l, m) in enumerate(lay.lm):
        px, py = lay.classes[k]
        ny, nx = lay.shapes[k]
        fl = 1.0 if l == 0 else g ** l
        diag = interpolate_2d(st, px, py) - fl * interpolate_2d(ss, px, py)
        base = lay.offsets[k]
        for iy in range(ny):
            for ix in range(nx):
                r = base + iy * nx + ix
                rows.append(r)
                cols.append(r)
                vals.append(diag[iy, ix])
        if Qa.shape == (R, R):
            if k == 0:
                b[base:base + ny * nx] = Qa.ravel()
        else:
            b[base:base + ny * nx] = interpolate_2d(Qa[k], px, py).ravel()
        for d, cd in enumerate((px, py)):
            for kp in range(lay.K):
                a = A[d, lay.k3[k], lay.k3[kp]]
                if a == 0.0:
                    continue
                qx, qy = lay.classes[kp]
                assert (qx != px) == (d == 0) and (qy != py) == (d == 1), "coupled grids must be half a cell apart"
                sny, snx = lay.shapes[kp]
                for iy in range(ny):
                    for ix in range(nx):
                        r = base + iy * nx + ix
                        i = ix if d == 0 else iy
                        n_nb = snx if d == 0 else sny
                        for sign, j in ((1.0, i + 1 - cd), (-1.0, i - cd)):
                            if 0 <= j < n_nb:
                                jx, jy = (j, iy) if d == 0 else (ix, j)
                                rows.append(r)
                                cols.append(lay.offsets[kp] + jy * snx + jx)
                                vals.append(sign * a / lay.h)
    M = sp.csr_matrix((vals, (rows, cols)), shape=(lay.n, lay.n))
    M.sum_duplicates()
    return lay, M, b


def solve_direct_2d(A, b: np.ndarray) -> np.ndarray:
    """Sparse LU (SuperLU) solve in FP64."""
    return spla.splu(sp.csc_matrix(A)).solve(b)
