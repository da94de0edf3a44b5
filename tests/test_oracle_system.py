"""Pins of the oracle's discrete P_N system (oracle/grid.py, pn.py, gmres.py).

Each test checks the oracle against something other than itself: brute-force
term-by-term evaluation of the printed equations, exact structural identities,
closed-form solutions (homogeneous media, the diffusion Green's function),
the textbook 7-point diffusion operator that P1 collapses to, the second-order
truncation error of staggered central differences, and a planted mistake that
the pins must catch.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import pn_inputs
from oracle import bruteforce, gmres, grid, pn, sh


def _rand_medium(R, seed, g=0.4, q_moments=False, N=1):
    rng = np.random.default_rng(seed)
    st = rng.uniform(0.5, 5.0, (R, R, R))
    al = rng.uniform(0.3, 0.95, (R, R, R))
    if q_moments:
        Q = rng.uniform(-1, 1, ((N + 1) ** 2, R, R, R))
    else:
        Q = rng.uniform(0, 1, (R, R, R))
    return pn.Medium(st, al, g, Q)


# --- layout -----------------------------------------------------------------

@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
def test_couplings_join_grids_half_a_cell_apart(N):
    """Every nonzero A_d couples two parity classes that differ exactly in
    axis d (so each derivative is a one-cell central difference)."""
    A = sh.coupling_matrices(N)
    cls = [grid.parity_class(l, m) for (l, m) in sh.lm_list(N)]
    for d in range(3):
        for i, j in zip(*np.nonzero(A[d])):
            diff = [cls[i][e] != cls[j][e] for e in range(3)]
            assert diff == [e == d for e in range(3)]


def test_parity_class_counts():
    """P1 uses 4 staggered grids (MAC placement), P3 and up all 8."""
    assert len({grid.parity_class(l, m) for (l, m) in sh.lm_list(1)}) == 4
    for N in (3, 5, 7):
        assert len({grid.parity_class(l, m) for (l, m) in sh.lm_list(N)}) == 8
    assert grid.parity_class(0, 0) == (0, 0, 0)
    assert grid.parity_class(1, 1) == (1, 0, 0)
    assert grid.parity_class(1, -1) == (0, 1, 0)
    assert grid.parity_class(1, 0) == (0, 0, 1)


def test_interpolation_rule():
    """Mean of adjacent in-domain centres: exact for a linear field on interior
    faces and edges, the single neighbour's value on boundary faces."""
    R = 5
    z, y, x = np.meshgrid(*(((np.arange(R) + 0.5) / R,) * 3), indexing="ij")
    F = 1.0 + 2.0 * x - 3.0 * y + 0.5 * z
    G = grid.interpolate_to_class(F, (1, 1, 0), periodic=False)
    assert G.shape == (R, R + 1, R + 1)
    xf = np.arange(R + 1) / R
    yf = np.arange(R + 1) / R
    zc = (np.arange(R) + 0.5) / R
    exact = 1.0 + 2.0 * xf[None, None, :] - 3.0 * yf[None, :, None] + 0.5 * zc[:, None, None]
    np.testing.assert_allclose(G[:, 1:R, 1:R], exact[:, 1:R, 1:R], atol=1e-14)
    np.testing.assert_allclose(G[:, 3, 0], F[:, 2, 0] * 0.5 + F[:, 3, 0] * 0.5, atol=1e-14)
    np.testing.assert_allclose(G[:, 0, 0], F[:, 0, 0], atol=1e-14)


# --- assembly vs brute force ----------------------------------------------------

@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_assembly_matches_bruteforce_printed_equations(N):
    R = 4
    rng = np.random.default_rng(100 + N)
    st = rng.uniform(0.5, 5.0, (R, R, R))
    al = rng.uniform(0.3, 0.95, (R, R, R))
    g = 0.35
    B = bruteforce.dense_matrix(N, R, st, al, g)
    S = pn.assemble(N, R, pn.Medium(st, al, g, np.zeros((R, R, R))))
    scale = np.abs(B).max()
    np.testing.assert_allclose(S.A.toarray(), B, atol=1e-13 * scale)


def test_planted_neighbour_swap_is_caught(monkeypatch):
    """Swapping the +h/2 and -h/2 neighbour in the assembler must break the
    brute-force agreement."""
    orig = pn._neighbour_index

    def swapped(i, cls_d, R, periodic):
        p, m, vp, vm = orig(i, cls_d, R, periodic)
        return m, p, vm, vp
    monkeypatch.setattr(pn, "_neighbour_index", swapped)
    R, N = 3, 1
    st = np.full((R, R, R), 2.0)
    B = bruteforce.dense_matrix(N, R, st, 0.5, 0.0)
    S = pn.assemble(N, R, pn.Medium(st, 0.5, 0.0, np.zeros((R, R, R))))
    assert np.abs(S.A.toarray() - B).max() > 1.0


# --- structure ------------------------------------------------------------------

@pytest.mark.parametrize("N,periodic", [(1, False), (3, False), (5, False), (3, True)])
def test_transport_is_skew_and_diagonal_is_collision_minus_scattering(N, periodic):
    """A + A^T = 2 D: the transport part is skew under the Dirichlet rule."""
    R = 5
    med = _rand_medium(R, 7, g=0.5)
    S = pn.assemble(N, R, med, periodic=periodic)
    sym = (S.A + S.A.T - 2 * sp.diags(S.diag)).toarray()
    assert np.abs(sym).max() <= 1e-14 * np.abs(S.A).max()
    np.testing.assert_allclose(S.A.diagonal(), S.diag, atol=1e-14)


@pytest.mark.parametrize("N", [1, 3, 5])
def test_matrix_free_apply_equals_csr(N):
    R = 6
    med = _rand_medium(R, 3, g=0.2)
    S = pn.assemble(N, R, med)
    u = np.random.default_rng(1).standard_normal(S.layout.n)
    np.testing.assert_allclose(pn.apply_matrix_free(S.layout, med, u), S.A @ u, atol=1e-12)
    np.testing.assert_allclose(pn.apply_matrix_free(S.layout, med, u, transpose=True), S.A.T @ u, atol=1e-12)


def test_source_moments_interpolated_like_parameters():
    R, N = 4, 3
    med = _rand_medium(R, 5, q_moments=True, N=N)
    lay = grid.Layout(N, R)
    b = lay.split(pn.rhs(lay, med))
    for k in range(lay.K):
        np.testing.assert_allclose(b[k], grid.interpolate_to_class(med.Q[k], lay.classes[k], False))


# --- closed forms ----------------------------------------------------------------

@pytest.mark.parametrize("N,g", [(1, 0.0), (3, 0.5), (5, 0.3)])
def test_homogeneous_periodic_uniform_source_exact(N, g):
    """Homogeneous medium, uniform source, periodic box: transport vanishes, so
    L^{0,0} = Q/sigma_a and every other moment is Q^{lm}/(sigma_t - sigma_s g^l)
    (zero where Q^{lm} = 0)."""
    R = 4
    st, al = 3.0, 0.8
    Q = np.zeros(((N + 1) ** 2, R, R, R))
    Q[0] = 2.0
    Q[2] = 0.5  # (l, m) = (1, 0)
    S = pn.assemble(N, R, pn.Medium(np.full((R, R, R), st), al, g, Q), periodic=True)
    u = S.layout.split(pn.solve_direct(S))
    sa = st * (1 - al)
    np.testing.assert_allclose(u[0], 2.0 / sa, rtol=1e-13)
    np.testing.assert_allclose(u[2], 0.5 / (st - st * al * g), rtol=1e-13)
    for k in range(1, S.layout.K):
        if k != 2:
            assert np.abs(u[k]).max() < 1e-13


def test_homogeneous_vacuum_centre_approaches_infinite_medium():
    """Vacuum box much larger than the diffusion length: the centre value of
    L^{0,0} under a uniform source approaches Q/sigma_a."""
    R = 12
    st, al = 40.0, 0.5
    S = pn.assemble(1, R, pn.Medium(np.full((R, R, R), st), al, 0.0, np.ones((R, R, R))))
    u = S.layout.split(pn.solve_direct(S))[0]
    sa = st * (1 - al)
    c = R // 2
    assert abs(u[c, c, c] * sa - 1.0) < 1e-6
    assert u[0, c, c] * sa < 0.97  # energy leaks at the vacuum boundary


def test_p1_is_classical_diffusion_exactly():
    """Eliminating the face unknowns of the staggered P1 system leaves the
    textbook 7-point finite-volume diffusion operator
    (1/(3 h^2)) sum_faces (u_i - u_j) / sigma_t'(face) + sigma_a u_i = Q_i,
    sigma_t' = sigma_t - g sigma_s, with u_j = 0 across the vacuum boundary.
    The diffusion matrix below is assembled independently of the oracle."""
    R = 7
    rng = np.random.default_rng(42)
    st = rng.uniform(0.5, 8.0, (R, R, R))
    al = rng.uniform(0.2, 0.95, (R, R, R))
    g = 0.3
    Q = rng.uniform(0.0, 1.0, (R, R, R))
    S = pn.assemble(1, R, pn.Medium(st, al, g, Q))
    L00 = S.layout.split(pn.solve_direct(S))[0]
    # independent 7-point FV diffusion
    h = 1.0 / R
    sp_ = st - g * al * st  # sigma_t' at centres
    sa = st * (1 - al)
    n = R ** 3
    idx = lambda z, y, x: (z * R + y) * R + x  # noqa: E731
    rows, cols, vals = [], [], []
    for z in range(R):
        for y in range(R):
            for x in range(R):
                i = idx(z, y, x)
                diag = sa[z, y, x]
                for dz, dy, dx in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    zz, yy, xx = z + dz, y + dy, x + dx
                    inside = 0 <= zz < R and 0 <= yy < R and 0 <= xx < R
                    sf = 0.5 * (sp_[z, y, x] + sp_[zz, yy, xx]) if inside else sp_[z, y, x]
                    w = 1.0 / (3.0 * h * h * sf)
                    diag += w
                    if inside:
                        rows.append(i)
                        cols.append(idx(zz, yy, xx))
                        vals.append(-w)
                rows.append(i)
                cols.append(i)
                vals.append(diag)
    M = sp.csc_matrix((vals, (rows, cols)), shape=(n, n))
    ref = spla.spsolve(M, Q.ravel()).reshape(R, R, R)
    np.testing.assert_allclose(L00, ref, rtol=1e-11, atol=1e-14)


def test_p1_point_source_converges_to_diffusion_greens_function():
    """Infinite-medium point source of total strength 1: L^{0,0}(r) =
    3 sigma_t' exp(-kappa r) / (4 pi r), kappa = sqrt(3 sigma_a sigma_t').
    Away from the source and the (optically distant) boundary the discrete
    P1 solution approaches it at second order in h."""
    errs = {}
    for R in (16, 24, 32):
        st, al = 40.0, 0.9
        kap = math.sqrt(3 * st * (1 - al) * st)
        c = R // 2
        Q = np.zeros((R, R, R))
        Q[c, c, c] = float(R ** 3)  # total strength Q h^3 = 1
        S = pn.assemble(1, R, pn.Medium(np.full((R, R, R), st), al, 0.0, Q))
        u, it, rel = gmres.gmres(S.A, S.b, tol=1e-11, m=60)
        assert rel < 1e-10
        L00 = S.layout.split(u)[0][c, c, :]
        xs = (np.arange(R) + 0.5) / R
        r = np.abs(xs - xs[c])
        sel = (r >= 0.1) & (r <= 0.3)
        ref = 3 * st * np.exp(-kap * r[sel]) / (4 * math.pi * r[sel])
        errs[R] = np.max(np.abs(L00[sel] - ref) / ref)
    assert errs[16] > errs[24] > errs[32]
    assert errs[16] / errs[32] > 3.5  # second order: ~4 per halving of h
    assert errs[32] < 0.2


def test_2d_problem_has_no_odd_moments():
    """z-independent medium and source with z-periodic wrap: all moments with
    l + m odd vanish (the 2D reduction of the paper's checkerboard section)."""
    R, N = 6, 3
    rng = np.random.default_rng(9)
    st2 = rng.uniform(0.5, 5.0, (R, R))
    q2 = rng.uniform(0.0, 1.0, (R, R))
    st = np.broadcast_to(st2, (R, R, R)).copy()
    Q = np.broadcast_to(q2, (R, R, R)).copy()
    S = pn.assemble(N, R, pn.Medium(st, 0.9, 0.2, Q), periodic=True)
    u = S.layout.split(pn.solve_direct(S))
    for k, (l, m) in enumerate(sh.lm_list(N)):
        if (l + m) % 2 == 1:
            assert np.abs(u[k]).max() < 1e-13
        elif k == 0:
            assert np.abs(u[k]).max() > 1e-3


def test_staggered_discretisation_is_second_order():
    """Manufactured smooth periodic solution: the truncation error
    ||A_h u_exact - Q_exact||_inf falls by about 4 per halving of h."""
    N = 3
    K = (N + 1) ** 2
    rng = np.random.default_rng(2)
    wave = rng.integers(-2, 3, size=(K, 3))
    wave[wave.sum(axis=1) == 0, 0] = 1
    phase = rng.uniform(0, 2 * math.pi, K)
    st, al, g = 2.0, 0.7, 0.4
    A3 = sh.coupling_matrices(N)
    errs = []
    for R in (8, 16, 32):
        lay = grid.Layout(N, R, periodic=True)
        med = pn.Medium(np.full((R, R, R), st), al, g, np.zeros((R, R, R)))
        S = pn.assemble(N, R, med, periodic=True)

        def field(k, deriv=None, kk=None):
            z, y, x = np.meshgrid(*lay.positions(kk), indexing="ij")
            arg = 2 * math.pi * (wave[k, 0] * x + wave[k, 1] * y + wave[k, 2] * z) + phase[k]
            if deriv is None:
                return np.sin(arg)
            return 2 * math.pi * wave[k, deriv] * np.cos(arg)
        u = lay.join([field(k, kk=k) for k in range(K)])
        q = []
        for k, (l, m) in enumerate(lay.lm):
            acc = (st - st * al * g ** l) * field(k, kk=k)
            for d in range(3):
                for kp in np.nonzero(A3[d, k])[0]:
                    acc = acc + A3[d, k, kp] * field(kp, deriv=d, kk=k)
            q.append(acc)
        errs.append(np.abs(S.A @ u - lay.join(q)).max())
    assert 3.5 < errs[0] / errs[1] < 4.5
    assert 3.5 < errs[1] / errs[2] < 4.5


def test_vacuum_reading_leaks_energy_through_boundary_faces():
    """Summing the L^{0,0} rows telescopes the transport differences to the
    boundary faces: sum h^3 (Q - sigma_a L00) = h^2 sum_d A_d[0,k'] (outflow
    of the l=1 moments through the faces at 1 minus those at 0).  With the
    closed-domain reading that outflow is positive (energy leaves the box)."""
    R, N = 6, 3
    med = _rand_medium(R, 21, g=0.3)
    S = pn.assemble(N, R, med)
    u = pn.solve_direct(S)
    parts = S.layout.split(u)
    h = 1.0 / R
    st = med.sigma_t
    sa = st * (1 - np.asarray(med.albedo))
    absorbed = np.sum(sa * parts[0]) * h ** 3
    emitted = np.sum(med.Q) * h ** 3
    A3 = sh.coupling_matrices(N)
    flux = 0.0
    for d in range(3):
        ax = 2 - d
        for kp in np.nonzero(A3[d, 0])[0]:
            arr = parts[kp]
            hi = np.take(arr, -1, axis=ax).sum()
            lo = np.take(arr, 0, axis=ax).sum()
            flux += A3[d, 0, kp] * (hi - lo) * h ** 2
    assert abs(emitted - (absorbed + flux)) < 1e-12 * emitted
    assert flux > 0.01 * emitted


@pytest.mark.parametrize("N", [1, 3])
def test_iterative_solvers_reach_the_direct_solution(N):
    R = 5
    med = _rand_medium(R, 11, g=0.25)
    S = pn.assemble(N, R, med)
    x = pn.solve_direct(S)
    assert pn.relative_residual(S.A, S.b, x) < 1e-13
    xc, it, rel = pn.cgls(S.A, S.b, tol=1e-12)
    assert rel <= 1e-12
    np.testing.assert_allclose(xc, x, atol=1e-9 * np.abs(x).max())
    # the operator as a pair of functions takes the same iterates
    xp, itp, relp = pn.cgls((lambda v: S.A @ v, lambda v: S.A.T @ v), S.b, tol=1e-12)
    assert itp == it and relp == rel and np.array_equal(xp, xc)
    xg, it, rel = gmres.gmres(S.A, S.b, tol=1e-12, m=30)
    assert rel <= 1e-12
    np.testing.assert_allclose(xg, x, atol=1e-9 * np.abs(x).max())


def test_vacuum_without_threshold_is_singular_and_threshold_restores_it():
    """sigma_t = 0 in a region with no threshold: the diagonal vanishes there
    and A is singular for odd-sized isolated blocks (the transport part is a
    skew matrix); the threshold sigma_t_min makes D positive again."""
    R, N = 4, 1
    st = np.zeros((R, R, R))
    med = pn.Medium(st, 0.9, 0.0, np.ones((R, R, R)))
    S = pn.assemble(N, R, med)
    assert np.abs(S.diag).max() == 0.0
    smin = np.linalg.svd(S.A.toarray(), compute_uv=False).min()
    assert smin < 1e-10
    med.sigma_t_min = 0.1
    S2 = pn.assemble(N, R, med)
    assert S2.diag.min() > 0.0
    smin2 = np.linalg.svd(S2.A.toarray(), compute_uv=False).min()
    assert smin2 >= S2.diag.min() * (1 - 1e-12)  # x^T A x = x^T D x


def test_input_generators_are_seeded_and_in_range():
    p = pn_inputs.fbm_point(3, 16, 5, 0.5, 40.0, 0.9, 0.3)
    q = pn_inputs.fbm_point(3, 16, 5, 0.5, 40.0, 0.9, 0.3)
    np.testing.assert_array_equal(p.sigma_t, q.sigma_t)
    assert abs(p.sigma_t.min() - 0.5) < 1e-12 and abs(p.sigma_t.max() - 40.0) < 1e-12
    c = pn_inputs.cloud_point(7, 16, 1)
    assert c.sigma_t.min() == 0.0 and c.sigma_t.max() <= 100.0
    assert (c.sigma_t == 0).mean() > 0.2


def test_row_by_row_apply_equals_csr():
    """The sampled-row evaluator used for full-size GPU checks agrees with the
    assembled matrix on every row of a small grid (and for A^T)."""
    R, N = 5, 3
    med = _rand_medium(R, 31, g=0.45)
    S = pn.assemble(N, R, med)
    u = np.random.default_rng(4).standard_normal(S.layout.n)
    parts = S.layout.split(u)
    rows = [(k, iz, iy, ix) for k in range(S.layout.K)
            for iz in range(S.layout.shapes[k][0]) for iy in range(S.layout.shapes[k][1])
            for ix in range(S.layout.shapes[k][2])]
    np.testing.assert_allclose(pn.apply_rows(S.layout, med, parts, rows), S.A @ u, atol=1e-12)
    np.testing.assert_allclose(pn.apply_rows(S.layout, med, parts, rows, transpose=True), S.A.T @ u, atol=1e-12)
