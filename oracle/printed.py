"""The real-valued P_N equations exactly as printed in the paper, term by term.

TEST INFRASTRUCTURE ONLY (part of the FP64 CPU oracle; see oracle/__init__.py).

This is the second, independent derivation path of the transport couplings:
`sh.coupling_matrices` integrates Ytilde_i w_d Ytilde_j numerically, while this
module reads them off the closed-form equations of the appendix section "Final
equation" (the m = 0, m < 0 and m > 0 cases) with the coefficient definitions
a..f, beta, delta and lambda_l printed below them.

Readings of the printed text (each pinned by tests/test_oracle_sh.py, which
compares these terms against the projection integrals):

* a^{l,m}: printed with denominator (2l+1)(2l-1).  That gives a^{0,0} =
  sqrt(-1).  The z-recursion needs the coefficient of Y^{l+1,m} in cos(theta)
  Y^{l,m}, whose denominator is (2l+3)(2l+1); that is used.
* m > 0, x-derivative of L^{l-1,m-1}: printed with e^{l-1,m-1}.  The term next
  to it uses f^{l+1,-m+1}, and the m<0 case pairs e^{l-1,m+1} with
  f^{l+1,m+1}; the same pairing for m>0 needs e^{l-1,-m+1}.  That is used (the
  two agree for m = 1).
* m > 0, first term: printed "c^{l-1,-m-1} d_x" with the unknown dropped; the
  unknown is L^{l-1,m+1} (as in the compact main-text form).
* m = 0: two "+" signs are missing between terms in the printed line; read
  as "+".
* beta^m = sqrt(2) for |m| = 1 else 1; delta_{m != v} = 0 if m == v else 1
  (appendix definitions; the main-text beta_x/beta_y are self-contradictory).
* Terms whose unknown L^{l',m'} does not exist (l' < 0, l' > N or |m'| > l')
  are dropped: they are outside the truncated expansion.
"""
from __future__ import annotations

import math

import numpy as np

from .sh import lm_index, lm_list, n_coeffs

SQ2 = math.sqrt(2.0)


def _sqrt_nonneg(v: float) -> float:
    if v < -1e-12:
        raise ValueError(f"negative radicand {v}")
    return math.sqrt(max(v, 0.0))


def coef_a(l, m):
    # corrected denominator (see module docstring)
    return _sqrt_nonneg((l - m + 1) * (l + m + 1) / ((2 * l + 3) * (2 * l + 1)))


def coef_b(l, m):
    if l == 0:
        return 0.0
    return _sqrt_nonneg((l - m) * (l + m) / ((2 * l + 1) * (2 * l - 1)))


def coef_c(l, m):
    return _sqrt_nonneg((l + m + 1) * (l + m + 2) / ((2 * l + 3) * (2 * l + 1)))


def coef_d(l, m):
    if l == 0:
        return 0.0
    return _sqrt_nonneg((l - m) * (l - m - 1) / ((2 * l + 1) * (2 * l - 1)))


def coef_e(l, m):
    return _sqrt_nonneg((l - m + 1) * (l - m + 2) / ((2 * l + 3) * (2 * l + 1)))


def coef_f(l, m):
    if l == 0:
        return 0.0
    return _sqrt_nonneg((l + m) * (l + m - 1) / ((2 * l + 1) * (2 * l - 1)))


def beta(m):
    return SQ2 if abs(m) == 1 else 1.0


def delta_ne(m, v):
    return 0.0 if m == v else 1.0


def _exists(N, l, m):
    return 0 <= l <= N and abs(m) <= l


def printed_terms(N: int, l: int, m: int):
    """Transport terms of equation (l, m): list of (coef, axis, l', m').

    axis 0, 1, 2 = d/dx, d/dy, d/dz.  A coefficient is only evaluated when its
    unknown exists (otherwise the term is dropped before its radicand is
    formed, since some radicands are negative exactly where the unknown is
    outside the expansion).
    """
    T = []

    def add(coef_fn, axis, lp, mp):
        if _exists(N, lp, mp):
            T.append((coef_fn(), axis, lp, mp))

    if m == 0:
        add(lambda: coef_c(l - 1, -1) / SQ2, 0, l - 1, 1)
        add(lambda: -coef_d(l + 1, -1) / SQ2, 0, l + 1, 1)
        add(lambda: coef_c(l - 1, -1) / SQ2, 1, l - 1, -1)
        add(lambda: -coef_d(l + 1, -1) / SQ2, 1, l + 1, -1)
        add(lambda: coef_a(l - 1, 0), 2, l - 1, 0)
        add(lambda: coef_b(l + 1, 0), 2, l + 1, 0)
    elif m < 0:
        add(lambda: -0.5 * coef_c(l - 1, m - 1), 1, l - 1, -m + 1)
        add(lambda: 0.5 * coef_d(l + 1, m - 1), 1, l + 1, -m + 1)
        add(lambda: -0.5 * beta(m) * coef_e(l - 1, m + 1), 1, l - 1, -m - 1)
        add(lambda: 0.5 * beta(m) * coef_f(l + 1, m + 1), 1, l + 1, -m - 1)
        add(lambda: 0.5 * coef_c(l - 1, m - 1), 0, l - 1, m - 1)
        if delta_ne(m, -1):
            add(lambda: -0.5 * coef_e(l - 1, m + 1), 0, l - 1, m + 1)
            add(lambda: 0.5 * coef_f(l + 1, m + 1), 0, l + 1, m + 1)
        add(lambda: -0.5 * coef_d(l + 1, m - 1), 0, l + 1, m - 1)
        add(lambda: coef_a(l - 1, m), 2, l - 1, m)
        add(lambda: coef_b(l + 1, m), 2, l + 1, m)
    else:
        add(lambda: 0.5 * coef_c(l - 1, -m - 1), 0, l - 1, m + 1)
        add(lambda: -0.5 * coef_d(l + 1, -m - 1), 0, l + 1, m + 1)
        add(lambda: -0.5 * beta(m) * coef_e(l - 1, -m + 1), 0, l - 1, m - 1)
        add(lambda: 0.5 * beta(m) * coef_f(l + 1, -m + 1), 0, l + 1, m - 1)
        add(lambda: 0.5 * coef_c(l - 1, -m - 1), 1, l - 1, -m - 1)
        add(lambda: -0.5 * coef_d(l + 1, -m - 1), 1, l + 1, -m - 1)
        if delta_ne(m, 1):
            add(lambda: 0.5 * coef_e(l - 1, -m + 1), 1, l - 1, -m + 1)
            add(lambda: -0.5 * coef_f(l + 1, -m + 1), 1, l + 1, -m + 1)
        add(lambda: coef_a(l - 1, -m), 2, l - 1, m)
        add(lambda: coef_b(l + 1, -m), 2, l + 1, m)
    return T


def printed_coupling_matrices(N: int) -> np.ndarray:
    """A[d, k, k'] summed from the printed terms (same shape as sh.coupling_matrices)."""
    K = n_coeffs(N)
    A = np.zeros((3, K, K))
    for (l, m) in lm_list(N):
        for coef, axis, lp, mp in printed_terms(N, l, m):
            A[axis, lm_index(l, m), lm_index(lp, mp)] += coef
    return A


def scattering_factor_printed(l: int, g: float) -> float:
    """lambda_l p^{l,0} for a normalised Henyey-Greenstein phase function.

    With p normalised over the sphere, p^{l,0} = sqrt((2l+1)/(4 pi)) g^l, so
    lambda_l p^{l,0} = g^l (the isotropic case g = 0 gives delta_{l,0}).
    """
    return 1.0 if l == 0 else g ** l
