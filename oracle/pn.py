"""The discrete staggered-grid P_N system: explicit sparse assembly, a
matrix-free FP64 apply, a sparse direct solve and the paper's CG on the normal
equations.

TEST INFRASTRUCTURE ONLY (part of the FP64 CPU oracle; see oracle/__init__.py).

System (paper, section "Discretized Radiative Transfer Equation", A u = Q with
A = T + C - S, and the real-valued P_N equations of the appendix):

  row (l, m) at location p:
      sum_d sum_{k'} A_d[k, k'] (u_{k'}(p + h/2 e_d) - u_{k'}(p - h/2 e_d)) / h
    + (sigma_t(p) - sigma_s(p) f_l) u_k(p)                 = Q_k(p)

with A_d the angular coupling matrices (sh.coupling_matrices), f_l =
lambda_l p^{l,0} = g^l for a normalised Henyey-Greenstein phase function
(appendix "Scattering Term"; isotropic is g = 0, f_l = delta_{l,0}), central
differences over one cell between staggered grids (grid.py), Dirichlet
boundary: references to locations outside the domain are dropped (section
"Runtime"), and sigma_t clamped below by a threshold sigma_t_min (sections
"Runtime" and "Nebulae": vacuum makes A singular).

Vectors use the oracle order of grid.Layout (coefficient-major, each
coefficient's own grid in C order [z][y][x]).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .grid import Layout, interpolate_to_class
from .printed import scattering_factor_printed
from .sh import coupling_matrices


@dataclass
class Medium:
    """Voxel-centre parameter fields (arrays indexed [z][y][x], shape (R, R, R)).

    sigma_t: extinction; albedo: scalar or field, sigma_s = albedo * sigma_t;
    g: Henyey-Greenstein mean cosine; Q: either a centre field of Q^{0,0}
    (shape (R, R, R)) or all K centre moments (shape (K, R, R, R)).
    """
    sigma_t: np.ndarray
    albedo: object
    g: float
    Q: np.ndarray
    sigma_t_min: float = 0.0


@dataclass
class System:
    layout: Layout
    A: sp.csr_matrix
    b: np.ndarray
    diag: np.ndarray          # D as a flat vector (oracle order)
    f_l: np.ndarray = field(default=None)


def centre_fields(medium: Medium, R: int):
    st = np.maximum(np.asarray(medium.sigma_t, dtype=np.float64), medium.sigma_t_min)
    if st.shape != (R, R, R):
        raise ValueError("sigma_t must have shape (R, R, R)")
    ss = np.asarray(medium.albedo, dtype=np.float64) * st
    return st, ss


def diagonal(layout: Layout, medium: Medium) -> np.ndarray:
    """Collision minus scattering, sigma_t(p) - sigma_s(p) g^l, per unknown."""
    st, ss = centre_fields(medium, layout.R)
    parts = []
    for k, (l, m) in enumerate(layout.lm):
        c = layout.classes[k]
        fl = scattering_factor_printed(l, medium.g)
        per = layout.periodic_axes
        parts.append(interpolate_to_class(st, c, per) - fl * interpolate_to_class(ss, c, per))
    return layout.join(parts)


def rhs(layout: Layout, medium: Medium) -> np.ndarray:
    """Q_k at every unknown location (centre moments interpolated like sigma)."""
    R = layout.R
    Q = np.asarray(medium.Q, dtype=np.float64)
    parts = []
    if Q.shape == (R, R, R):
        for k in range(layout.K):
            parts.append(Q.copy() if k == 0 else np.zeros(layout.shapes[k]))
    elif Q.shape == (layout.K, R, R, R):
        for k in range(layout.K):
            parts.append(interpolate_to_class(Q[k], layout.classes[k], layout.periodic_axes))
    else:
        raise ValueError("Q must have shape (R,R,R) or (K,R,R,R)")
    return layout.join(parts)


def _neighbour_index(i, cls_d, R, periodic):
    """Indices of the +h/2 and -h/2 neighbours along one axis, and validity."""
    plus = i + 1 - cls_d
    minus = i - cls_d
    if periodic:
        return plus % R, minus % R, np.ones_like(i, bool), np.ones_like(i, bool)
    n_nb = R + 1 - cls_d  # extent of the neighbour grid along this axis
    return plus, minus, (plus >= 0) & (plus < n_nb), (minus >= 0) & (minus < n_nb)


def transport_coo(layout: Layout):
    """(rows, cols, vals) of the transport matrix T (before summing duplicates)."""
    A = coupling_matrices(layout.N)
    h = layout.h
    R = layout.R
    rows, cols, vals = [], [], []
    for k in range(layout.K):
        ck = layout.classes[k]
        nz, ny, nx = layout.shapes[k]
        iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        idx = [ix.ravel(), iy.ravel(), iz.ravel()]
        row = layout.offsets[k] + np.arange(nz * ny * nx, dtype=np.int64)
        for d in range(3):
            for kp in np.nonzero(A[d, k])[0]:
                a = A[d, k, kp]
                cp = layout.classes[kp]
                if any((cp[e] != ck[e]) != (e == d) for e in range(3)):
                    raise AssertionError("coupling between grids not half a cell apart")
                snz, sny, snx = layout.shapes[kp]
                for sign, which in ((+1.0, 0), (-1.0, 1)):
                    nb = list(idx)
                    pl, mi, vp, vm = _neighbour_index(idx[d], ck[d], R, layout.periodic_axes[d])
                    nb[d] = pl if which == 0 else mi
                    valid = vp if which == 0 else vm
                    col = layout.offsets[kp] + (nb[2] * sny + nb[1]) * snx + nb[0]
                    rows.append(row[valid])
                    cols.append(col[valid])
                    vals.append(np.full(int(valid.sum()), sign * a / h))
    if rows:
        return np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0)


def assemble(N: int, R: int, medium: Medium, periodic=False) -> System:
    """Explicit sparse A (CSR, FP64) and right-hand side, row by row as the
    paper's runtime does (section "Runtime": the stencil is executed for every
    unknown to fill A and Q)."""
    layout = Layout(N, R, periodic)
    r, c, v = transport_coo(layout)
    D = diagonal(layout, medium)
    n = layout.n
    r = np.concatenate([r, np.arange(n)])
    c = np.concatenate([c, np.arange(n)])
    v = np.concatenate([v, D])
    A = sp.csr_matrix((v, (r, c)), shape=(n, n))
    A.sum_duplicates()
    return System(layout=layout, A=A, b=rhs(layout, medium), diag=D)


def apply_matrix_free(layout: Layout, medium: Medium, u: np.ndarray, transpose: bool = False) -> np.ndarray:
    """y = A u (or A^T u) without forming A, by the same row definition.

    A^T follows from the structure: the transport part is skew-symmetric (the
    +h/2 entry of row i and the -h/2 entry of row j are the same coupling with
    opposite sign, and the Dirichlet rule removes both together), so
    A^T = D - T.
    """
    A = coupling_matrices(layout.N)
    h = layout.h
    R = layout.R
    D = diagonal(layout, medium)
    parts = layout.split(u)
    ys = [np.zeros(s) for s in layout.shapes]
    tsign = -1.0 if transpose else 1.0
    for k in range(layout.K):
        ck = layout.classes[k]
        for d in range(3):
            ax = 2 - d  # array axis of world axis d
            for kp in np.nonzero(A[d, k])[0]:
                src = parts[kp]
                n_out = layout.shapes[k][ax]
                i = np.arange(n_out)
                pl, mi, vp, vm = _neighbour_index(i, ck[d], R, layout.periodic_axes[d])
                plus = np.zeros(layout.shapes[k])
                minus = np.zeros(layout.shapes[k])
                sl_out = [slice(None)] * 3
                sl_in = [slice(None)] * 3
                sl_out[ax] = np.nonzero(vp)[0]
                sl_in[ax] = pl[vp]
                plus[tuple(sl_out)] = src[tuple(sl_in)]
                sl_out[ax] = np.nonzero(vm)[0]
                sl_in[ax] = mi[vm]
                minus[tuple(sl_out)] = src[tuple(sl_in)]
                ys[k] += tsign * (A[d, k, kp] / h) * (plus - minus)
    return layout.join(ys) + D * u


def relative_residual(A, b: np.ndarray, u: np.ndarray) -> float:
    """||Q - A u||_2 / ||Q||_2 of the original (not the normal) system."""
    return float(np.linalg.norm(b - A @ u) / np.linalg.norm(b))


def solve_direct(system: System) -> np.ndarray:
    """Sparse LU (SuperLU) solve of A u = Q in FP64."""
    lu = spla.splu(system.A.tocsc())
    return lu.solve(system.b)


def cgls(A, b: np.ndarray, tol: float = 1e-10, max_iter: int = 100000, x0=None, history=None):
    """CG on the normal equations A^T A u = A^T Q without forming A^T A.

    The paper's solver (section "Results": a CG modified so that the normal
    form is never computed explicitly; section "Runtime": solving the normal
    form because A is non-symmetric).  Textbook CGLS steps; convergence is
    tested on the residual of the original system, ||Q - A u|| / ||Q||.
    A: a matrix (anything with A @ v and A.T @ v) or a pair of functions
    (v -> A v, v -> A^T v).
    Returns (u, iterations, relative residual).
    """
    if isinstance(A, tuple):
        matvec, rmatvec = A
    else:
        def matvec(v):
            return A @ v

        def rmatvec(v):
            return A.T @ v
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - matvec(x)
    s = rmatvec(r)
    p = s.copy()
    gamma = float(s @ s)
    bnorm = float(np.linalg.norm(b))
    rel = float(np.linalg.norm(r)) / bnorm
    it = 0
    while rel > tol and it < max_iter:
        q = matvec(p)
        qq = float(q @ q)
        if qq == 0.0:
            break
        alpha = gamma / qq
        x += alpha * p
        r -= alpha * q
        s = rmatvec(r)
        gamma_new = float(s @ s)
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        it += 1
        rel = float(np.linalg.norm(r)) / bnorm
        if history is not None:
            history.append(rel)
    return x, it, rel


def apply_rows(layout: Layout, medium: Medium, parts, rows, transpose: bool = False) -> np.ndarray:
    """(A u)[row] (or (A^T u)[row]) for a list of rows (k, iz, iy, ix), one by
    one, straight from the row definition in this module's docstring.

    `parts` are the per-coefficient grids of u (any array-like supporting
    integer indexing, e.g. large numpy arrays).  Used to check full-size
    applies at sampled outputs.  Vacuum boundary only.
    """
    if layout.periodic:
        raise ValueError("apply_rows supports the vacuum boundary only")
    A = coupling_matrices(layout.N)
    R, h = layout.R, layout.h
    st = np.maximum(np.asarray(medium.sigma_t, dtype=np.float64), medium.sigma_t_min)
    al = np.asarray(medium.albedo, dtype=np.float64)
    tsign = -1.0 if transpose else 1.0
    out = []
    for (k, iz, iy, ix) in rows:
        l, m = layout.lm[k]
        c = layout.classes[k]
        idx = (ix, iy, iz)
        # parameter means over adjacent in-domain centres
        cand = []
        for d in range(3):
            i = idx[d]
            cand.append([i] if c[d] == 0 else [j for j in (i - 1, i) if 0 <= j < R])
        sts, sss = [], []
        for cz in cand[2]:
            for cy in cand[1]:
                for cx in cand[0]:
                    t = st[cz, cy, cx]
                    a = al if al.ndim == 0 else al[cz, cy, cx]
                    sts.append(t)
                    sss.append(a * t)
        diag = np.mean(sts) - scattering_factor_printed(l, medium.g) * np.mean(sss)
        acc = diag * float(parts[k][iz, iy, ix])
        for d in range(3):
            for kp in np.nonzero(A[d, k])[0]:
                shp = layout.shapes[kp]
                vals = []
                for off in (1 - c[d], -c[d]):
                    j = list(idx)
                    j[d] += off
                    inside = all(0 <= j[e] < shp[2 - e] for e in range(3))
                    vals.append(float(parts[kp][j[2], j[1], j[0]]) if inside else 0.0)
                acc += tsign * A[d, k, kp] / h * (vals[0] - vals[1])
        out.append(acc)
    return np.array(out)
