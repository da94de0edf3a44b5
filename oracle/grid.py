"""Staggered grid layout of the P_N unknowns, and parameter interpolation.

TEST INFRASTRUCTURE ONLY (part of the FP64 CPU oracle; see oracle/__init__.py).

The paper distributes the SH coefficients over disjoint staggered grids
(section "Runtime"/"Precomputation", Fig. staggeredgrid, following StaRMAP) so
that every first derivative is a central difference over one cell, and defers
the exact placement to StaRMAP.  Reading used here (parity placement): the
coefficient (l, m) lives on the grid whose offset along axis d is h/2 exactly
when Ytilde^{l,m} is odd under reflection of axis d:

    p_x = m mod 2 (m >= 0),  (|m| + 1) mod 2 (m < 0)
    p_y = 1 if m < 0 else 0
    p_z = (l + |m|) mod 2

Along an axis with p_d = 0 the unknowns sit at cell centres (i + 1/2) h,
i = 0..R-1; with p_d = 1 they sit on cell faces i h, i = 0..R (the closed
domain [0, 1]; boundary faces carry unknowns).  Because w_d is odd in axis d
and even in the other two, int Ytilde_i w_d Ytilde_j vanishes unless the
classes of i and j differ exactly in axis d, so every d/dx_d couples two grids
that are exactly half a cell apart along d.

Boundary (section "Runtime", Dirichlet): a term that would reference a
location outside the domain is dropped (that unknown is zero).

Parameters (sigma_t, sigma_s, Q) are given at voxel centres and are
interpolated to an unknown's location as the arithmetic mean of the adjacent
voxel centres that lie inside the domain (section "Precomputation": parameters
are interpolated to the staggered locations; the rule itself is a reading).

A periodic test mode (R locations per axis for every class, wrap-around;
all axes, or a chosen subset of them) exists only for the exact closed-form
pins and for pinning the 2D reduction (z-periodic, z-independent data).

Oracle vector order: coefficient-major, k = l^2 + l + m, each coefficient's
grid in C order [z][y][x] with its own extents.
"""
from __future__ import annotations

import numpy as np

from .sh import lm_list, n_coeffs


def parity_class(l: int, m: int):
    """(p_x, p_y, p_z) of coefficient (l, m)."""
    am = abs(m)
    px = (m % 2) if m >= 0 else ((am + 1) % 2)
    py = 1 if m < 0 else 0
    pz = (l + am) % 2
    return (px, py, pz)


class Layout:
    """Unknown locations of one P_N system on an R^3 grid of the unit cube."""

    def __init__(self, N: int, R: int, periodic=False):
        """periodic: bool (all axes) or a tuple of three bools (x, y, z)."""
        if R < 2:
            raise ValueError("grid must have at least 2 cells per axis")
        self.N = N
        self.R = R
        self.h = 1.0 / R
        if isinstance(periodic, (tuple, list)):
            self.periodic_axes = tuple(bool(v) for v in periodic)
        else:
            self.periodic_axes = (bool(periodic),) * 3
        self.periodic = any(self.periodic_axes)
        self.K = n_coeffs(N)
        self.lm = lm_list(N)
        self.classes = [parity_class(l, m) for (l, m) in self.lm]
        self.shapes = []  # (nz, ny, nx) per k
        for c in self.classes:
            ext = [R if self.periodic_axes[d] else R + c[d] for d in range(3)]  # x, y, z
            self.shapes.append((ext[2], ext[1], ext[0]))
        sizes = [int(np.prod(s)) for s in self.shapes]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.n = int(self.offsets[-1])

    def split(self, u: np.ndarray):
        """View a flat vector as a list of per-coefficient 3D arrays."""
        return [u[self.offsets[k]:self.offsets[k + 1]].reshape(self.shapes[k]) for k in range(self.K)]

    def join(self, parts) -> np.ndarray:
        return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])

    def positions(self, k: int):
        """World coordinates (z, y, x) of the locations of coefficient k, as 1D axes."""
        c = self.classes[k]
        out = []
        for axis_cls, n in zip((c[2], c[1], c[0]), self.shapes[k]):
            i = np.arange(n, dtype=np.float64)
            out.append(i * self.h if axis_cls == 1 else (i + 0.5) * self.h)
        return out  # [z_axis, y_axis, x_axis]


def _face_average(F: np.ndarray, axis: int, periodic: bool) -> np.ndarray:
    """Average a centre-located field onto the faces along one axis.

    Face i lies between centres i-1 and i; only in-domain centres take part
    (vacuum: faces 0 and R see one centre).  Periodic: R faces, wrap-around.
    """
    F = np.moveaxis(F, axis, 0)
    R = F.shape[0]
    if periodic:
        G = 0.5 * (np.roll(F, 1, axis=0) + F)
    else:
        G = np.empty((R + 1,) + F.shape[1:])
        G[0] = F[0]
        G[R] = F[R - 1]
        G[1:R] = 0.5 * (F[:-1] + F[1:])
    return np.moveaxis(G, 0, axis)


def interpolate_to_class(F: np.ndarray, cls, periodic) -> np.ndarray:
    """Centre field F[z, y, x] (R^3) -> values at the locations of parity class cls.

    The mean over the adjacent in-domain centres is a tensor product of 1D
    means, applied along each odd axis.  periodic: bool or (x, y, z) bools.
    """
    per = tuple(periodic) if isinstance(periodic, (tuple, list)) else (bool(periodic),) * 3
    G = np.asarray(F, dtype=np.float64)
    px, py, pz = cls
    if px:
        G = _face_average(G, 2, per[0])
    if py:
        G = _face_average(G, 1, per[1])
    if pz:
        G = _face_average(G, 0, per[2])
    return G
