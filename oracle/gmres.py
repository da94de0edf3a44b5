"""Restarted GMRES(m) in FP64 for A u = Q.

TEST INFRASTRUCTURE ONLY (part of the FP64 CPU oracle; see oracle/__init__.py).

A plain Krylov solve of the original (non-normal) system: Arnoldi with
modified Gram-Schmidt, Givens rotations on the Hessenberg matrix, restart
after m steps (Saad and Schultz, 1986).  The paper solves the normal equations
instead (section "Runtime"); this solver reaches the same unique solution
(A is nonsingular when sigma_a > 0) and is used where a sparse direct solve is
too slow.  Convergence is measured by ||Q - A u|| / ||Q||.
"""
from __future__ import annotations

import numpy as np


def gmres(matvec, b: np.ndarray, tol: float = 1e-10, m: int = 50, max_iter: int = 20000, x0=None):
    """Returns (u, total inner iterations, final relative residual)."""
    if not callable(matvec):
        A = matvec
        matvec = lambda v: A @ v  # noqa: E731
    x = np.zeros_like(b, dtype=np.float64) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    total = 0
    r = b - matvec(x)
    beta = float(np.linalg.norm(r))
    while beta / bnorm > tol and total < max_iter:
        V = np.zeros((m + 1, b.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            w = matvec(V[j])
            for i in range(j + 1):
                H[i, j] = float(V[i] @ w)
                w -= H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            j_done = j + 1
            if abs(g[j + 1]) / bnorm <= tol or total >= max_iter:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x += V[:j_done].T @ y
        r = b - matvec(x)
        beta = float(np.linalg.norm(r))
    return x, total, beta / bnorm
