"""Spherical harmonics and the angular coupling matrices of the real P_N equations.

TEST INFRASTRUCTURE ONLY: this module belongs to the FP64 CPU oracle.  Only the
test-suite, the smoke check and the CPU-baseline leg of the benchmark may use
it; the CUDA library never imports, links or calls it.

What it computes (Koerner, Portsmouth, Jakob, "P_N-Method for Multiple
Scattering in Participating Media", EGSR 2018):

* Complex SH with the Condon-Shortley phase (appendix, definition of the complex
  basis): Y_C^{l,m} = (-1)^m sqrt((2l+1)/(4pi) (l-m)!/(l+m)!) e^{i m phi}
  P^{l,m}(cos theta) for m >= 0, and Y_C^{l,-m} = (-1)^m conj(Y_C^{l,m}); here
  P^{l,m} does NOT carry the (-1)^m.
* The real basis Y_R of the appendix (section "Derivation of the real-valued
  P_N-equations", Eq. real_sh_basis): i/sqrt2 (Y_C^{l,m} - (-1)^m Y_C^{l,-m})
  for m<0, Y_C^{l,0}, 1/sqrt2 (Y_C^{l,-m} + (-1)^m Y_C^{l,m}) for m>0.
  (The main-text version, Eq. sh_real_basis, has a sign that makes the m>0
  functions imaginary; the appendix form is used.)
* The printed real P_N equations (appendix "Final equation") are the Galerkin
  projection in the sign-adjusted basis Ytilde^{l,m} = (-1)^m Y_R^{l,m}, i.e.
  the real SH *with* the Condon-Shortley phase.  This reading is what makes the
  printed coupling coefficients agree with the projection integrals; it is
  pinned in tests by comparing against those printed equations.
* Transport coupling matrices A_d[i, j] = int_S2 Ytilde_i(w) w_d Ytilde_j(w) dw
  (the projection of (w . grad) L-hat, appendix "Transport Term"), evaluated by
  a product quadrature (Gauss-Legendre in cos(theta) x uniform in phi) that is
  exact for these polynomial integrands.

Coefficient order: k = l*l + l + m, for l = 0..N, m = -l..l.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np


def n_coeffs(N: int) -> int:
    """K = (N+1)^2 real SH coefficients per location."""
    return (N + 1) * (N + 1)


def lm_index(l: int, m: int) -> int:
    return l * l + l + m


def lm_list(N: int):
    """[(l, m)] in coefficient order k = l^2 + l + m."""
    return [(l, m) for l in range(N + 1) for m in range(-l, l + 1)]


def assoc_legendre_nocs(l: int, m: int, x: np.ndarray) -> np.ndarray:
    """P^{l,m}(x) for m >= 0 WITHOUT the Condon-Shortley phase.

    Standard three-term recurrence in l at fixed m, started from
    P^{m,m} = (2m-1)!! (1-x^2)^{m/2} and P^{m+1,m} = x (2m+1) P^{m,m}.
    """
    if m < 0 or m > l:
        raise ValueError("need 0 <= m <= l")
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    pmm = np.ones_like(x)
    for i in range(1, m + 1):
        pmm = pmm * (2 * i - 1) * s
    if l == m:
        return pmm
    pm1 = x * (2 * m + 1) * pmm
    if l == m + 1:
        return pm1
    p_lm2, p_lm1 = pmm, pm1
    for ll in range(m + 2, l + 1):
        p = ((2 * ll - 1) * x * p_lm1 - (ll + m - 1) * p_lm2) / (ll - m)
        p_lm2, p_lm1 = p_lm1, p
    return p_lm1


def sh_norm(l: int, m: int) -> float:
    """sqrt((2l+1)/(4 pi) * (l-|m|)! / (l+|m|)!)."""
    am = abs(m)
    return math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))


def Y_complex(l: int, m: int, theta, phi) -> np.ndarray:
    """Complex SH with Condon-Shortley phase, as defined in the appendix."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    am = abs(m)
    base = ((-1) ** am) * sh_norm(l, am) * np.exp(1j * am * phi) * assoc_legendre_nocs(l, am, np.cos(theta))
    if m >= 0:
        return base
    return ((-1) ** am) * np.conj(base)


def Y_real_appendix(l: int, m: int, theta, phi) -> np.ndarray:
    """Y_R of the appendix definition, built literally from Y_complex.

    Returns the real part after asserting that the imaginary part vanishes.
    """
    if m < 0:
        v = (1j / math.sqrt(2.0)) * (Y_complex(l, m, theta, phi) - ((-1) ** m) * Y_complex(l, -m, theta, phi))
    elif m == 0:
        v = Y_complex(l, 0, theta, phi)
    else:
        v = (1.0 / math.sqrt(2.0)) * (Y_complex(l, -m, theta, phi) + ((-1) ** m) * Y_complex(l, m, theta, phi))
    v = np.asarray(v)
    if np.max(np.abs(np.imag(v)), initial=0.0) > 1e-12:
        raise AssertionError("real SH basis produced an imaginary value")
    return np.real(v)


def Y_tilde(l: int, m: int, theta, phi) -> np.ndarray:
    """The basis of the printed real P_N equations: (-1)^m Y_R^{l,m}."""
    return ((-1) ** abs(m)) * Y_real_appendix(l, m, theta, phi)


@lru_cache(maxsize=None)
def sphere_quadrature(n_mu: int, n_phi: int):
    """Product rule on S^2: Gauss-Legendre in mu = cos(theta), uniform in phi.

    Exact for polynomials in (x, y, z) of degree < 2*n_mu in mu and trig
    polynomials of degree < n_phi in phi.  Returns (theta, phi, w) flat arrays.
    """
    mu, wmu = np.polynomial.legendre.leggauss(n_mu)
    phi = (np.arange(n_phi) + 0.5) * (2.0 * math.pi / n_phi)
    wphi = np.full(n_phi, 2.0 * math.pi / n_phi)
    MU, PHI = np.meshgrid(mu, phi, indexing="ij")
    W = np.outer(wmu, wphi)
    return np.arccos(MU).ravel(), PHI.ravel(), W.ravel()


def direction(theta, phi):
    """Unit vector components (x, y, z) for polar angle theta, azimuth phi."""
    st = np.sin(theta)
    return st * np.cos(phi), st * np.sin(phi), np.cos(theta)


@lru_cache(maxsize=None)
def basis_table(N: int, n_mu: int | None = None, n_phi: int | None = None):
    """Ytilde_k evaluated at the quadrature nodes: array (K, n_nodes), plus nodes."""
    if n_mu is None:
        n_mu = N + 4
    if n_phi is None:
        n_phi = 2 * N + 6
    th, ph, w = sphere_quadrature(n_mu, n_phi)
    Y = np.stack([Y_tilde(l, m, th, ph) for (l, m) in lm_list(N)])
    return Y, th, ph, w


@lru_cache(maxsize=None)
def coupling_matrices(N: int) -> np.ndarray:
    """A[d, i, j] = int Ytilde_i w_d Ytilde_j dw for d = x, y, z (FP64, (3, K, K)).

    Entries below 1e-13 in magnitude are exact zeros of the integral (parity or
    selection rules) and are set to 0.
    """
    Y, th, ph, w = basis_table(N)
    dx, dy, dz = direction(th, ph)
    A = np.empty((3, Y.shape[0], Y.shape[0]))
    for d, wd in enumerate((dx, dy, dz)):
        A[d] = (Y * (w * wd)) @ Y.T
    A[np.abs(A) < 1e-13] = 0.0
    return A


def gram_matrix(N: int) -> np.ndarray:
    """int Ytilde_i Ytilde_j dw (identity for an orthonormal basis)."""
    Y, th, ph, w = basis_table(N)
    return (Y * w) @ Y.T


def phase_factors_hg(N: int, g: float) -> np.ndarray:
    """Per-coefficient scattering factor lambda_l p^{l,0} for a normalised
    Henyey-Greenstein phase function, evaluated from the definitions
    (appendix "Phase Function" and "Scattering Term"): p^{l,0} = int p(w.e3)
    Y^{l,0}(w) dw, lambda_l = sqrt(4 pi / (2l+1)).  Computed by Gauss-Legendre
    quadrature in mu with many nodes (HG is not a polynomial), so it is accurate
    to quadrature error only.  Returns an array of length K (one value per k).
    """
    mu, wmu = np.polynomial.legendre.leggauss(400)
    if abs(g) < 1e-300:
        p = np.full_like(mu, 1.0 / (4.0 * math.pi))
    else:
        p = (1.0 - g * g) / (4.0 * math.pi * (1.0 + g * g - 2.0 * g * mu) ** 1.5)
    out = []
    for (l, m) in lm_list(N):
        # Y^{l,0}(theta) = sh_norm(l,0) P_l(mu), azimuth integral gives 2 pi.
        pl0 = 2.0 * math.pi * np.sum(wmu * p * sh_norm(l, 0) * assoc_legendre_nocs(l, 0, mu))
        lam = math.sqrt(4.0 * math.pi / (2 * l + 1))
        out.append(lam * pl0)
    return np.array(out)
