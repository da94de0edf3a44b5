"""Single-scatter source of a collimated beam, and unstaggering.

TEST INFRASTRUCTURE ONLY (part of the FP64 CPU oracle; see oracle/__init__.py).

Section "Rendering" of the paper splits the radiance into single- and
multiple-scattered light and folds the single-scattered part into the
emission term:  Q(x, w) = sigma_s(x) int p(w' -> w) L_u(x, w') dw', with L_u
the uncollided light of the source, attenuated by the medium.

For a collimated beam of unit irradiance travelling along the unit direction
w_b, L_u(x, w') = E(x) delta(w' - w_b) inside the beam, with transmittance
E(x) = exp(-int sigma_t ds) from the entry face to x.  Projecting onto the
basis (Funk-Hecke, normalised Henyey-Greenstein p with Legendre weights
(2l+1)/(4 pi) g^l) gives the moments

    Q^{l,m}(x) = sigma_s(x) E(x) g^l Ytilde_{l,m}(w_b).

Readings (the paper gives no formula for the beam): the beam is axis-aligned
along +-x, +-y or +-z, enters through the domain face it points away from,
has a circular cross-section of given radius around a given transverse
centre, and is evaluated at voxel centres; the optical depth to a voxel
centre is the sum of sigma_t h over the whole cells before it plus half its
own cell (midpoint rule on the piecewise-constant medium).  Attenuation uses
the medium's sigma_t as given (the solver's sigma_t_min clamp is a property
of the linear system, not of the uncollided light).

Unstaggering (section "Rendering": coefficients are interpolated to voxel
centres and the extra boundary coefficients dropped): along every axis on
which a coefficient lives on faces, the centre value is the mean of the two
faces of the cell.
"""
from __future__ import annotations

import math

import numpy as np

from .grid import Layout
from .sh import Y_tilde, lm_list, n_coeffs

AXIS_DIRECTIONS = {0: (0.5 * math.pi, 0.0), 1: (0.5 * math.pi, 0.5 * math.pi), 2: (0.0, 0.0)}


def beam_direction_angles(axis: int, sign: int):
    """(theta, phi) of the unit vector sign * e_axis."""
    theta, phi = AXIS_DIRECTIONS[axis]
    if sign < 0:
        theta, phi = math.pi - theta, phi + math.pi
    return theta, phi


def beam_transmittance(sigma_t: np.ndarray, axis: int, sign: int, radius: float, centre=(0.5, 0.5)) -> np.ndarray:
    """E(x) at the R^3 voxel centres ([z][y][x]); zero outside the beam."""
    st = np.asarray(sigma_t, dtype=np.float64)
    R = st.shape[0]
    h = 1.0 / R
    ax = 2 - axis  # array axis
    cells = np.moveaxis(st, ax, 0)
    if sign < 0:
        cells = cells[::-1]
    tau = np.cumsum(cells, axis=0) * h - 0.5 * cells * h
    E = np.exp(-tau)
    if sign < 0:
        E = E[::-1]
    E = np.moveaxis(E, 0, ax)
    c = (np.arange(R) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    coords = [x, y, z]
    t = [coords[a] for a in range(3) if a != axis]
    inside = (t[0] - centre[0]) ** 2 + (t[1] - centre[1]) ** 2 <= radius * radius
    return np.where(inside, E, 0.0)


def single_scatter_beam(sigma_t, albedo, g: float, N: int, axis: int, sign: int, radius: float,
                        centre=(0.5, 0.5)) -> np.ndarray:
    """Centre moments Q^{l,m} (shape (K, R, R, R)) of the single-scattered beam."""
    st = np.asarray(sigma_t, dtype=np.float64)
    ss = np.asarray(albedo, dtype=np.float64) * st
    E = beam_transmittance(st, axis, sign, radius, centre)
    theta, phi = beam_direction_angles(axis, sign)
    out = np.empty((n_coeffs(N),) + st.shape)
    for k, (l, m) in enumerate(lm_list(N)):
        out[k] = ss * E * (g ** l if l > 0 else 1.0) * float(Y_tilde(l, m, theta, phi))
    return out


def unstagger(layout: Layout, parts) -> np.ndarray:
    """Per-coefficient grids -> (K, R, R, R) values at voxel centres."""
    R = layout.R
    out = np.empty((layout.K, R, R, R))
    for k in range(layout.K):
        a = np.asarray(parts[k], dtype=np.float64)
        px, py, pz = layout.classes[k]
        if px:
            a = 0.5 * (a[:, :, :-1] + a[:, :, 1:])
        if py:
            a = 0.5 * (a[:, :-1, :] + a[:, 1:, :])
        if pz:
            a = 0.5 * (a[:-1, :, :] + a[1:, :, :])
        out[k] = a
    return out
