"""Brute-force, term-by-term evaluation of the printed P_N equations on a grid.

TEST INFRASTRUCTURE ONLY (part of the FP64 CPU oracle; see oracle/__init__.py).

For tiny grids this builds the dense system matrix by walking every unknown,
every printed term of its equation (printed.printed_terms: the appendix "Final
equation" read term by term) and locating each referenced unknown by its
world coordinate, half a cell away along the derivative's axis (central
difference over one cell, section "Precomputation").  It shares with the
assembler in pn.py only the final numbering of unknowns (grid.Layout offsets);
couplings come from the printed closed forms instead of projection integrals,
and neighbours, the domain test and parameter averaging are found from
coordinates instead of index arithmetic.

Coordinates are integers in units of h/2: a cell centre (i + 1/2) h is 2i+1,
a face i h is 2i; the closed domain is [0, 2R] on every axis.
"""
from __future__ import annotations

import itertools

import numpy as np

from .grid import Layout
from .printed import printed_terms, scattering_factor_printed
from .sh import lm_index


def _centre_average(F, X, Y, Z, R):
    """Mean of F over the voxel centres adjacent to half-unit point (X, Y, Z)
    that lie inside the domain."""
    cand = []
    for c in (X, Y, Z):
        if c % 2 == 1:
            cand.append([c])
        else:
            cand.append([v for v in (c - 1, c + 1) if 0 < v < 2 * R])
    vals = [F[(cz - 1) // 2, (cy - 1) // 2, (cx - 1) // 2]
            for cx, cy, cz in itertools.product(cand[0], cand[1], cand[2])]
    return sum(vals) / len(vals)


def dense_matrix(N: int, R: int, sigma_t, albedo, g: float) -> np.ndarray:
    """Dense A (vacuum boundary) in the oracle's unknown order."""
    lay = Layout(N, R)
    st = np.asarray(sigma_t, dtype=np.float64)
    ss = np.asarray(albedo, dtype=np.float64) * st
    h = 1.0 / R
    index = {}
    for k in range(lay.K):
        px, py, pz = lay.classes[k]
        nz, ny, nx = lay.shapes[k]
        for iz in range(nz):
            for iy in range(ny):
                for ix in range(nx):
                    key = (k, 2 * ix + (1 - px), 2 * iy + (1 - py), 2 * iz + (1 - pz))
                    index[key] = lay.offsets[k] + (iz * ny + iy) * nx + ix
    A = np.zeros((lay.n, lay.n))
    for (k, X, Y, Z), row in index.items():
        l, m = lay.lm[k]
        fl = scattering_factor_printed(l, g)
        A[row, row] += _centre_average(st, X, Y, Z, R) - fl * _centre_average(ss, X, Y, Z, R)
        for coef, axis, lp, mp in printed_terms(N, l, m):
            kp = lm_index(lp, mp)
            for sign in (+1, -1):
                P = [X, Y, Z]
                P[axis] += sign
                if not all(0 <= c <= 2 * R for c in P):
                    continue  # outside the closed domain: Dirichlet, dropped
                key = (kp, P[0], P[1], P[2])
                if key not in index:
                    raise AssertionError(f"no unknown {lay.lm[kp]} at {P}: placement inconsistent")
                A[row, index[key]] += sign * coef / h
    return A
