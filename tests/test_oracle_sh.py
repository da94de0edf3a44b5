"""Pins of the oracle's spherical harmonics and angular coupling matrices.

Each test checks oracle/sh.py or oracle/printed.py against something other
than itself: a library routine (scipy), closed-form low-order harmonics, exact
identities of the projected operator w_d, the hand-read P1 equations, or the
other derivation path (projection integrals vs printed closed forms).
"""
import math
import os

import numpy as np
import pytest
import scipy.special as ss

from oracle import printed, sh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_associated_legendre_matches_scipy():
    x = np.linspace(-0.999, 0.999, 41)
    for l in range(0, 9):
        for m in range(0, l + 1):
            ours = sh.assoc_legendre_nocs(l, m, x)
            # scipy's lpmv includes the Condon-Shortley phase (-1)^m
            ref = ((-1) ** m) * ss.lpmv(m, l, x)
            np.testing.assert_allclose(ours, ref, rtol=1e-12, atol=1e-12)


def test_complex_sh_matches_scipy():
    th = np.linspace(0.05, math.pi - 0.05, 13)[:, None]
    ph = np.linspace(0.0, 2 * math.pi, 17)[None, :]
    for l in range(0, 8):
        for m in range(-l, l + 1):
            ours = sh.Y_complex(l, m, th, ph)
            ref = ss.sph_harm_y(l, m, th, ph)
            np.testing.assert_allclose(ours, ref, rtol=1e-11, atol=1e-12)


def test_real_basis_is_orthonormal():
    for N in (1, 3, 5, 7):
        G = sh.gram_matrix(N)
        np.testing.assert_allclose(G, np.eye(len(G)), atol=1e-13)


def test_low_order_real_harmonics_closed_form():
    th = np.linspace(0.1, 3.0, 11)[:, None]
    ph = np.linspace(0.0, 6.0, 9)[None, :]
    x, y, z = np.broadcast_arrays(*sh.direction(th, ph))
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    np.testing.assert_allclose(sh.Y_tilde(0, 0, th, ph), np.full_like(x, 0.5 / math.sqrt(math.pi)), atol=1e-15)
    # with the Condon-Shortley phase the l=1 real harmonics are (-y, z, -x) * sqrt(3/4pi)
    np.testing.assert_allclose(sh.Y_tilde(1, -1, th, ph), -c1 * y, atol=1e-14)
    np.testing.assert_allclose(sh.Y_tilde(1, 0, th, ph), c1 * z, atol=1e-14)
    np.testing.assert_allclose(sh.Y_tilde(1, 1, th, ph), -c1 * x, atol=1e-14)
    c2 = 0.5 * math.sqrt(15.0 / math.pi)
    np.testing.assert_allclose(sh.Y_tilde(2, -2, th, ph), c2 * x * y, atol=1e-14)
    np.testing.assert_allclose(sh.Y_tilde(2, 2, th, ph), 0.5 * c2 * (x * x - y * y), atol=1e-14)
    np.testing.assert_allclose(sh.Y_tilde(2, 0, th, ph),
                               0.25 * math.sqrt(5.0 / math.pi) * (3 * z * z - 1), atol=1e-14)


@pytest.mark.parametrize("N", range(0, 8))
def test_projection_integrals_equal_printed_equations(N):
    """The two derivation paths agree: integrals of Ytilde_i w_d Ytilde_j and
    the appendix's closed-form equations (with the readings in printed.py)."""
    A = sh.coupling_matrices(N)
    P = printed.printed_coupling_matrices(N)
    np.testing.assert_allclose(A, P, atol=1e-13)


def test_p1_couplings_match_hand_read_equations():
    A = sh.coupling_matrices(1)
    ref = np.zeros_like(A)
    with open(os.path.join(GOLDEN, "p1_couplings.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            d, k, kp, v = line.split()
            ref[int(d), int(k), int(kp)] = float(v)
    np.testing.assert_allclose(A, ref, atol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
def test_coupling_matrices_symmetric(N):
    A = sh.coupling_matrices(N)
    for d in range(3):
        np.testing.assert_allclose(A[d], A[d].T, atol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_z_coupling_m0_block_eigenvalues_are_legendre_roots(N):
    """On the m = 0 harmonics, projected multiplication by cos(theta) is the
    Jacobi matrix of the Legendre polynomials: its eigenvalues are the roots
    of P_{N+1} (the Gauss-Legendre nodes)."""
    A = sh.coupling_matrices(N)
    idx = [sh.lm_index(l, 0) for l in range(N + 1)]
    ev = np.sort(np.linalg.eigvalsh(A[2][np.ix_(idx, idx)]))
    nodes = np.sort(np.polynomial.legendre.leggauss(N + 1)[0])
    np.testing.assert_allclose(ev, nodes, atol=1e-13)


@pytest.mark.parametrize("N", [1, 3, 4, 7])
def test_coupling_spectra_rotation_invariant(N):
    """The degree-<=N harmonics are closed under rotations, so the projected
    operators w_x, w_y, w_z are unitarily similar: equal spectra.  A wrong
    sign or coefficient in an x or y term breaks this."""
    A = sh.coupling_matrices(N)
    evs = [np.sort(np.linalg.eigvalsh(A[d])) for d in range(3)]
    np.testing.assert_allclose(evs[0], evs[2], atol=1e-12)
    np.testing.assert_allclose(evs[1], evs[2], atol=1e-12)
    assert np.max(np.abs(evs[2])) < 1.0


@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_sum_of_squares_is_identity_below_truncation(N):
    """w_x^2 + w_y^2 + w_z^2 = 1.  For rows and columns with l <= N-1 the
    product w_d Y_j stays inside the expansion, so the identity is exact there."""
    A = sh.coupling_matrices(N)
    S = sum(A[d] @ A[d] for d in range(3))
    n = N * N  # coefficients with l <= N-1
    np.testing.assert_allclose(S[:n, :n], np.eye(n), atol=1e-13)
    assert np.max(np.abs(S[n:, n:] - np.eye(len(S) - n))) > 1e-3  # truncation shows at l = N


@pytest.mark.parametrize("g", [0.0, 0.3, 0.6, -0.4])
def test_hg_phase_projection_is_g_power_l(g):
    """lambda_l p^{l,0} of a normalised Henyey-Greenstein phase function,
    from its projection integral, equals g^l (isotropic: delta_{l0})."""
    N = 7
    f = sh.phase_factors_hg(N, g)
    ref = [printed.scattering_factor_printed(l, g) for (l, m) in sh.lm_list(N)]
    np.testing.assert_allclose(f, ref, atol=1e-10)
    if g == 0.0:
        np.testing.assert_allclose(f, [1.0] + [0.0] * (len(f) - 1), atol=1e-12)


# --- planted mistakes: the pins above must catch plausible errors -------------

def test_uncorrected_a_coefficient_is_caught(monkeypatch):
    def a_as_printed(l, m):
        den = (2 * l + 1) * (2 * l - 1)
        return math.sqrt(abs((l - m + 1) * (l + m + 1) / den))
    monkeypatch.setattr(printed, "coef_a", a_as_printed)
    assert np.max(np.abs(printed.printed_coupling_matrices(3) - sh.coupling_matrices(3))) > 1e-2


def test_uncorrected_e_index_is_caught(monkeypatch):
    orig = printed.printed_terms

    def terms_as_printed(N, l, m):
        T = orig(N, l, m)
        if m <= 1:
            return T
        out = []
        for coef, axis, lp, mp in T:
            if axis == 0 and lp == l - 1 and mp == m - 1:
                coef = -0.5 * printed.beta(m) * printed.coef_e(l - 1, m - 1)
            out.append((coef, axis, lp, mp))
        return out
    monkeypatch.setattr(printed, "printed_terms", terms_as_printed)
    assert np.max(np.abs(printed.printed_coupling_matrices(4) - sh.coupling_matrices(4))) > 1e-2


def test_basis_without_cs_sign_is_caught():
    """Y_R itself (without the (-1)^m) does not reproduce the printed signs."""
    N = 3
    Y, th, ph, w = sh.basis_table(N)
    s = np.array([(-1) ** abs(m) for (l, m) in sh.lm_list(N)], dtype=float)
    YR = Y * s[:, None]
    dx, dy, dz = sh.direction(th, ph)
    AR = (YR * (w * dx)) @ YR.T
    assert np.max(np.abs(AR - printed.printed_coupling_matrices(N)[0])) > 0.1
