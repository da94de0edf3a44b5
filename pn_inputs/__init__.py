"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds input generation only -- no step of the P_N method's
arithmetic: voxel-centre parameter fields (extinction, albedo), the
Henyey-Greenstein g, and a point source given as a Q^{0,0} centre field.

Media stand in for the paper's scenes (section "Results": a homogeneous
point-source medium, a procedural heterogeneous cloud with vacuum regions);
the paper's nebulae dataset is not available, so clouds are seeded value-noise
fBm:

* value noise on an integer lattice of `base` cells per unit length, lattice
  values uniform in [0, 1) from numpy's PCG64 seeded generator, smoothstep
  weights, trilinear interpolation, evaluated at voxel centres (i + 1/2) / R;
* `octaves` octaves, lacunarity 2, gain 1/2;
* min-max normalised to [0, 1], then mapped affinely onto the wanted range.

All arrays are float64, indexed [z][y][x], shape (R, R, R).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Problem:
    """One P_N problem: order N, R^3 cells on the unit cube, centre fields."""
    name: str
    N: int
    R: int
    sigma_t: np.ndarray
    albedo: float
    g: float
    Q00: np.ndarray
    sigma_t_min: float = 0.0
    source_voxel: tuple = None


def _smoothstep(t):
    return t * t * (3.0 - 2.0 * t)


def _interp_matrix(R: int, freq: int) -> np.ndarray:
    """(R, freq+1) weights of lattice nodes at voxel centres along one axis."""
    u = (np.arange(R) + 0.5) / R * freq
    i0 = np.minimum(np.floor(u).astype(np.int64), freq - 1)
    t = _smoothstep(u - i0)
    W = np.zeros((R, freq + 1))
    W[np.arange(R), i0] = 1.0 - t
    W[np.arange(R), i0 + 1] += t
    return W


def value_noise_fbm(R: int, seed: int, octaves: int = 4, base: int = 4) -> np.ndarray:
    """fBm of smoothstep value noise at the R^3 voxel centres, normalised to [0, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros((R, R, R))
    amp = 1.0
    for o in range(octaves):
        f = base * (2 ** o)
        L = rng.random((f + 1, f + 1, f + 1))  # [z][y][x]
        W = _interp_matrix(R, f)
        v = np.einsum("zc,cba->zba", W, L)
        v = np.einsum("yb,zba->zya", W, v)
        v = np.einsum("xa,zya->zyx", W, v)
        out += amp * v
        amp *= 0.5
    lo, hi = out.min(), out.max()
    return (out - lo) / (hi - lo)


def point_source(R: int, voxel, strength: float = 1.0) -> np.ndarray:
    """Q^{0,0} = strength in one voxel (z, y, x), zero elsewhere."""
    Q = np.zeros((R, R, R))
    Q[tuple(voxel)] = strength
    return Q


def seeded_voxel(R: int, seed: int, lo: int, hi: int):
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    return tuple(int(v) for v in rng.integers(lo, hi, size=3))


def homogeneous_point(N: int = 1, R: int = 16, sigma_t: float = 10.0, albedo: float = 0.9,
                      g: float = 0.0) -> Problem:
    """P_N point source in a homogeneous medium: Q^{0,0} = 1 in voxel (R/2, R/2, R/2)."""
    c = R // 2
    return Problem(name=f"P{N} {R}^3 homogeneous point source", N=N, R=R,
                   sigma_t=np.full((R, R, R), float(sigma_t)), albedo=albedo, g=g,
                   Q00=point_source(R, (c, c, c)), source_voxel=(c, c, c))


def fbm_point(N: int, R: int, seed: int, sig_lo: float, sig_hi: float, albedo: float,
              g: float, name: str = None) -> Problem:
    """Heterogeneous fBm medium with a point source at a seeded voxel in the middle half."""
    st = sig_lo + (sig_hi - sig_lo) * value_noise_fbm(R, seed)
    v = seeded_voxel(R, seed, R // 4, (3 * R) // 4)
    return Problem(name=name or f"P{N} {R}^3 fBm[{sig_lo},{sig_hi}] point source seed {seed}",
                   N=N, R=R, sigma_t=st, albedo=albedo, g=g, Q00=point_source(R, v), source_voxel=v)


def cloud_point(N: int, R: int, seed: int, sig_max: float = 100.0, albedo: float = 0.99,
                g: float = 0.6, sigma_t_min: float = 0.1) -> Problem:
    """Cloud-like medium: sigma_t = sig_max * clamp((fBm - 1/2) / (1/2), 0, 1),
    zero (vacuum) where the noise is below its midpoint, clamped below by
    sigma_t_min in the solver; point source at a seeded voxel."""
    n = value_noise_fbm(R, seed)
    st = sig_max * np.clip((n - 0.5) / 0.5, 0.0, 1.0)
    v = seeded_voxel(R, seed, R // 4, (3 * R) // 4)
    return Problem(name=f"P{N} {R}^3 thresholded-fBm cloud seed {seed}", N=N, R=R, sigma_t=st,
                   albedo=albedo, g=g, Q00=point_source(R, v), sigma_t_min=sigma_t_min,
                   source_voxel=v)


# The workloads the benchmark and the parity tests are sized on.

def p1_16_homogeneous() -> Problem:
    """P1, 16^3, sigma_t = 10, albedo 0.9, isotropic, Q = 1 at the centre voxel."""
    return homogeneous_point(1, 16, 10.0, 0.9, 0.0)


def p5_64_fbm(seed: int = 0) -> Problem:
    """P5, 64^3, fBm sigma_t in [0.5, 40], albedo 0.95, g 0.3, seeded point source."""
    return fbm_point(5, 64, seed, 0.5, 40.0, 0.95, 0.3)


def p3_64_fbm(seed: int = 0) -> Problem:
    """P3, 64^3, fBm sigma_t in [0.5, 80], albedo and g drawn from the seed."""
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    albedo = float(rng.uniform(0.8, 0.99))
    g = float(rng.uniform(0.0, 0.6))
    return fbm_point(3, 64, seed, 0.5, 80.0, albedo, g)


def p7_256_cloud(seed: int = 0, R: int = 256) -> Problem:
    """P7, 256^3, thresholded-fBm cloud (sigma_t up to 100, empty regions 0),
    albedo 0.99, g 0.6."""
    return cloud_point(7, R, seed, 100.0, 0.99, 0.6, 0.1)


def p7_256_cloud_beam(seed: int = 0, R: int = 256):
    """The P7 256^3 cloud of p7_256_cloud lit by a collimated beam instead of a
    point source: (problem, beam) with beam = (axis, sign, radius, centre), the
    axis and direction seeded, radius 0.1, the line through a seeded point of
    the middle of the entry face (the source moments are built from it by the
    single-scatter source builder)."""
    p = cloud_point(7, R, seed, 100.0, 0.99, 0.6, 0.1)
    rng = np.random.Generator(np.random.PCG64(seed + 31337))
    axis = int(rng.integers(3))
    sign = int(rng.choice([-1, 1]))
    centre = tuple(float(c) for c in rng.uniform(0.35, 0.65, size=2))
    return p, (axis, sign, 0.1, centre)


def random_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Uniform random values (test vectors)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=shape)


def checkerboard_2d(R: int = 71, blocks: int = 7, sigma_a: float = 10.0, sigma_s: float = 1.0,
                    source: float = 1.0):
    """The 2D checkerboard workload (section "2D checkerboard": a 7 x 7
    domain at 71 x 71 cells, unit blocks alternately purely absorbing,
    sigma_a = 10, and purely scattering, sigma_s = 1) on R x R cells.

    The paper gives neither the pattern's phase nor the source; the reading
    here: cell (iy, ix) belongs to unit block (floor(y), floor(x)) of its
    centre (x, y) in [0, blocks)^2; block (i, j) absorbs when i + j is odd
    and scatters otherwise; an isotropic source of unit strength per unit
    area fills the centre block (which scatters).  The problem is scaled to
    the unit square (cell size h = 1 / R): extinction and source scale by
    `blocks`, which leaves sigma h and Q h, and so the solution, unchanged.

    Returns (sigma_t, albedo, Q00), float64 arrays [y][x] of shape (R, R).
    """
    c = (np.arange(R) + 0.5) * blocks / R
    by, bx = np.meshgrid(np.floor(c).astype(int), np.floor(c).astype(int), indexing="ij")
    absorbing = (by + bx) % 2 == 1
    sigma_t = np.where(absorbing, sigma_a, sigma_s) * float(blocks)
    albedo = np.where(absorbing, 0.0, 1.0)
    mid = blocks // 2
    Q00 = np.where((by == mid) & (bx == mid), source, 0.0) * float(blocks)
    return sigma_t, albedo, Q00


@dataclass
class BatchInstance:
    """One instance of a batched workload: order, grid, centre fields and a
    source given either as a point (Q^{0,0} at `voxel`) or as a collimated
    beam (axis, sign, radius, centre), to be turned into moments by the
    single-scatter source builder."""
    N: int
    R: int
    sigma_t: np.ndarray
    albedo: float
    g: float
    source: tuple


def batch_instances(count: int = 64, base_seed: int = 0, r_lo: int = 24, r_hi: int = 96, orders=(1, 3, 5),
                    sig_lo: float = 0.1, sig_hi: float = 60.0):
    """The many-instance workload: instance i (seed base_seed + i) draws its
    grid R uniformly in [r_lo, r_hi], its order from `orders`, an fBm
    extinction field mapped onto [sig_lo, sig_hi], albedo ~ U[0.7, 0.99],
    g ~ U[0, 0.7], and a point source (a seeded voxel in the middle half) or a
    collimated beam of radius 0.1 along a seeded axis and direction, with
    equal probability."""
    out = []
    for i in range(count):
        seed = base_seed + i
        rng = np.random.Generator(np.random.PCG64(seed + 7919))
        R = int(rng.integers(r_lo, r_hi + 1))
        N = int(orders[int(rng.integers(len(orders)))])
        albedo = float(rng.uniform(0.7, 0.99))
        g = float(rng.uniform(0.0, 0.7))
        st = sig_lo + (sig_hi - sig_lo) * value_noise_fbm(R, seed)
        if rng.uniform() < 0.5:
            v = tuple(int(t) for t in rng.integers(R // 4, R - R // 4, size=3))
            src = ("point", v)
        else:
            src = ("beam", int(rng.integers(3)), int(rng.choice([-1, 1])), 0.1,
                   (float(rng.uniform(0.3, 0.7)), float(rng.uniform(0.3, 0.7))))
        out.append(BatchInstance(N, R, st, albedo, g, src))
    return out
