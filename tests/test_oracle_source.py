"""Pins of the oracle's single-scatter beam source and unstaggering
(oracle/source.py): closed-form transmittance in a homogeneous medium, the
isotropic case, the spherical-harmonic addition theorem (the moments rebuild
the truncated Henyey-Greenstein lobe around the beam direction), energy, and
exact unstaggering of linear fields."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre

from oracle import grid, sh, source


@pytest.mark.parametrize("axis,sign", [(0, 1), (0, -1), (1, 1), (2, -1)])
def test_homogeneous_transmittance_closed_form(axis, sign):
    R, st = 8, 3.0
    E = source.beam_transmittance(np.full((R, R, R), st), axis, sign, radius=2.0)
    c = (np.arange(R) + 0.5) / R
    depth = c if sign > 0 else 1.0 - c
    ref1d = np.exp(-st * depth)
    shape = [1, 1, 1]
    shape[2 - axis] = R
    np.testing.assert_allclose(E, np.broadcast_to(ref1d.reshape(shape), E.shape), rtol=1e-14)


def test_beam_radius_and_heterogeneous_depth():
    R = 10
    rng = np.random.default_rng(0)
    st = rng.uniform(0.0, 5.0, (R, R, R))
    E = source.beam_transmittance(st, 0, 1, radius=0.25, centre=(0.5, 0.5))
    h = 1.0 / R
    for (z, y) in [(5, 5), (4, 6)]:
        tau = 0.0
        for x in range(R):
            ref = math.exp(-(tau + 0.5 * st[z, y, x] * h))
            assert abs(E[z, y, x] - ref) < 1e-14
            tau += st[z, y, x] * h
    assert E[0, 0, :].max() == 0.0  # far outside the beam
    c = (np.arange(R) + 0.5) / R
    inside = ((c[:, None] - 0.5) ** 2 + (c[None, :] - 0.5) ** 2 <= 0.0625)
    assert ((E[:, :, 0] > 0) == inside).all()


def test_isotropic_scattering_gives_only_l0():
    R, N = 6, 3
    Q = source.single_scatter_beam(np.full((R, R, R), 2.0), 0.8, 0.0, N, 2, 1, radius=1.0)
    E = source.beam_transmittance(np.full((R, R, R), 2.0), 2, 1, 1.0)
    np.testing.assert_allclose(Q[0], 0.8 * 2.0 * E / (2.0 * math.sqrt(math.pi)), rtol=1e-14)
    assert np.abs(Q[1:]).max() == 0.0


@pytest.mark.parametrize("axis,sign,g", [(0, 1, 0.6), (1, -1, 0.3), (2, 1, -0.4)])
def test_moments_rebuild_truncated_hg_lobe(axis, sign, g):
    """sum_lm Q^{lm} Ytilde_lm(w) = sigma_s E sum_l g^l (2l+1)/(4 pi) P_l(w_b . w)
    (addition theorem): checks normalisation and every sign of the basis."""
    N, R = 5, 2
    Q = source.single_scatter_beam(np.full((R, R, R), 1.0), 1.0, g, N, axis, sign, radius=5.0)
    E = source.beam_transmittance(np.full((R, R, R), 1.0), axis, sign, 5.0)[0, 0, 0]
    wb = np.zeros(3)
    wb[axis] = sign
    th = np.linspace(0.2, 2.9, 7)[:, None]
    ph = np.linspace(0.1, 6.0, 9)[None, :]
    dx, dy, dz = np.broadcast_arrays(*sh.direction(th, ph))
    mu = wb[0] * dx + wb[1] * dy + wb[2] * dz
    rebuilt = sum(Q[k, 0, 0, 0] * sh.Y_tilde(l, m, th, ph) for k, (l, m) in enumerate(sh.lm_list(N)))
    coeffs = [(g ** l) * (2 * l + 1) / (4 * math.pi) for l in range(N + 1)]
    ref = E * legendre.legval(mu, coeffs)
    np.testing.assert_allclose(rebuilt, ref, atol=1e-12)


def test_scattered_power_equals_sigma_s_times_transmittance():
    R, N = 4, 2
    rng = np.random.default_rng(3)
    st = rng.uniform(0.5, 3.0, (R, R, R))
    al = rng.uniform(0.2, 0.9, (R, R, R))
    Q = source.single_scatter_beam(st, al, 0.5, N, 1, 1, radius=1.0)
    E = source.beam_transmittance(st, 1, 1, 1.0)
    # int Q dw = Q^{00} * int Y00 dw = Q^{00} sqrt(4 pi)
    np.testing.assert_allclose(Q[0] * math.sqrt(4 * math.pi), al * st * E, rtol=1e-13)


def test_unstagger_is_exact_for_linear_fields():
    N, R = 3, 5
    lay = grid.Layout(N, R)
    parts = []
    for k in range(lay.K):
        z, y, x = np.meshgrid(*lay.positions(k), indexing="ij")
        parts.append(1.0 + k + 2.0 * x - 0.5 * y + 3.0 * z)
    out = source.unstagger(lay, parts)
    c = (np.arange(R) + 0.5) / R
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    for k in range(lay.K):
        np.testing.assert_allclose(out[k], 1.0 + k + 2.0 * x - 0.5 * y + 3.0 * z, atol=1e-13)
