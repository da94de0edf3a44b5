"""GPU parity of the CUDA library against the FP64 CPU oracle.

Every test calls the C ABI (through the ctypes binding) and compares element
by element with the oracle on the same seeded inputs.  Tolerances:

* FP64 apply / transpose / residual: max |y_gpu - y_ref| <= 1e-12 * max(|A| |x|)
  and ||y_gpu - y_ref|| / ||y_ref|| <= 1e-12;
* FP32: the same with 1e-5 (inputs rounded to FP32 first, reference in FP64);
* solves: the oracle's own FP64 residual ||Q - A u|| / ||Q|| of the GPU
  solution, and the L2 error of L^{0,0} against the oracle's direct solution.
"""
import math

import numpy as np
import pytest

import pn_inputs
from oracle import pn as opn

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1807_00410_gb300 import build
    build.build()


def _system(N, R, seed, g=0.35, q_moments=False, albedo_field=True, sigma_t_min=0.0, lo=0.5, hi=20.0):
    from paper_1807_00410_gb300 import System
    st = lo + (hi - lo) * pn_inputs.value_noise_fbm(R, seed, base=2)
    al = pn_inputs.random_field((R, R, R), seed + 1, 0.3, 0.97) if albedo_field else 0.9
    K = (N + 1) ** 2
    Q = pn_inputs.random_field((K, R, R, R) if q_moments else (R, R, R), seed + 2, -1.0, 1.0)
    med = opn.Medium(st, al, g, Q, sigma_t_min)
    gpu = System(N, R, st, al, g, Q, sigma_t_min=sigma_t_min)
    return med, gpu


def _rand_planes(layout_o, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [rng.uniform(-1, 1, s) for s in layout_o.shapes]


def _compare(y_gpu, y_ref, scale, tol):
    err = np.max(np.abs(y_gpu - y_ref))
    assert err <= tol * scale, f"max err {err:.3e} > {tol:.0e} * {scale:.3e}"
    rel = np.linalg.norm(y_gpu - y_ref) / max(np.linalg.norm(y_ref), 1e-300)
    assert rel <= tol, f"relative L2 {rel:.3e}"


# sizes span one and several x-tiles (32 wide), the columns right of the
# tiles (R a multiple of 32), several z-chunks, and ragged y-tiles
CASES = [(0, 5), (1, 2), (1, 9), (3, 5), (3, 17), (5, 9), (7, 3), (7, 6), (3, 32), (1, 33), (2, 40), (5, 20)]


@pytest.mark.parametrize("N,R", CASES)
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_apply_transpose_residual_match_oracle(N, R, dtype):
    med, gpu = _system(N, R, 10 * N + R, q_moments=(N % 2 == 1))
    S = opn.assemble(N, R, med)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    tol = 1e-12 if dtype == "f64" else 1e-5
    planes = _rand_planes(S.layout, 7 * R + N)
    if dtype == "f32":
        planes = [p.astype(np.float32).astype(np.float64) for p in planes]
    u = S.layout.join(planes)
    x = gpu.from_planes(planes, dtype=tdt)
    y = gpu.zeros(tdt)
    absA = abs(S.A)
    scale = np.max(absA @ np.abs(u))
    gpu.apply(x, y)
    _compare(S.layout.join(gpu.to_planes(y)), S.A @ u, scale, tol)
    gpu.apply_t(x, y)
    _compare(S.layout.join(gpu.to_planes(y)), S.A.T @ u, scale, tol)
    rel = gpu.residual(x, y)
    r_ref = S.b - S.A @ u
    _compare(S.layout.join(gpu.to_planes(y)), r_ref, scale + np.max(np.abs(S.b)), tol)
    assert abs(rel - np.linalg.norm(r_ref) / np.linalg.norm(S.b)) <= 10 * tol * rel
    gpu.close()


def test_inactive_slots_ignored_and_zeroed():
    N, R = 3, 6
    med, gpu = _system(N, R, 3)
    S = opn.assemble(N, R, med)
    planes = _rand_planes(S.layout, 1)
    x = gpu.from_planes(planes, dtype=torch.float64)
    y_clean = gpu.zeros(torch.float64)
    gpu.apply(x, y_clean)
    # poison every padding slot of x with NaN
    mask = gpu.from_planes([np.ones(s) for s in S.layout.shapes], dtype=torch.float64) == 0
    x2 = x.clone()
    x2[mask] = float("nan")
    y = torch.full_like(x, 7.0)
    gpu.apply(x2, y)
    assert torch.isfinite(y).all()
    assert torch.equal(y, y_clean)
    assert (y[mask] == 0).all()
    gpu.close()


def test_fp64_apply_and_dot_are_deterministic():
    med, gpu = _system(5, 9, 4)
    S = opn.assemble(5, 9, med)
    x = gpu.from_planes(_rand_planes(S.layout, 2), dtype=torch.float64)
    y1, y2 = gpu.zeros(torch.float64), gpu.zeros(torch.float64)
    gpu.apply(x, y1)
    gpu.apply(x, y2)
    assert torch.equal(y1, y2)
    assert gpu.dot(x, y1) == gpu.dot(x, y1)
    gpu.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_dot_and_axpby(dtype):
    med, gpu = _system(3, 7, 5)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    g = torch.Generator(device="cpu").manual_seed(0)
    a = torch.rand(gpu.layout.n_elems, generator=g, dtype=torch.float64).to(tdt)
    b = torch.rand(gpu.layout.n_elems, generator=g, dtype=torch.float64).to(tdt)
    ref = float(np.dot(a.double().numpy(), b.double().numpy()))
    d = gpu.dot(a.cuda(), b.cuda())
    assert abs(d - ref) <= (1e-13 if dtype == "f64" else 1e-6) * abs(ref)
    y = b.cuda().clone()
    gpu.axpby(2.0, a.cuda(), -0.5, y)
    np.testing.assert_allclose(y.cpu().double().numpy(), 2.0 * a.double().numpy() - 0.5 * b.double().numpy(),
                               rtol=1e-6 if dtype == "f32" else 1e-15, atol=1e-7 if dtype == "f32" else 1e-15)
    gpu.close()


# --- solves ---------------------------------------------------------------------

def _p1_centre_problem():
    p = pn_inputs.p1_16_homogeneous()
    med = opn.Medium(p.sigma_t, p.albedo, p.g, p.Q00)
    return p, med


@pytest.mark.parametrize("solver", ["cgls", "gmres"])
def test_p1_point_source_solves_to_1e10_in_fp64(solver):
    """P1, 16^3, sigma_t = 10, albedo 0.9, isotropic, Q = 1 at the centre voxel,
    FP64 on the GPU to rel. residual 1e-10; matches the oracle's direct solve."""
    from paper_1807_00410_gb300 import System
    p, med = _p1_centre_problem()
    S = opn.assemble(p.N, p.R, med)
    u_ref = opn.solve_direct(S)
    gpu = System(p.N, p.R, p.sigma_t, p.albedo, p.g, p.Q00)
    u = gpu.zeros(torch.float64)
    st = gpu.solve(u, solver=solver, tol=1e-10, max_iter=20000, restart=80)
    assert st["rel_residual"] <= 1e-10
    uo = S.layout.join(gpu.to_planes(u))
    assert opn.relative_residual(S.A, S.b, uo) <= 1.5e-10
    err = np.linalg.norm(uo - u_ref) / np.linalg.norm(u_ref)
    assert err <= 1e-8, err
    gpu.close()


def test_ir_gmres_fp32_inner_reaches_1e6_and_oracle_l00():
    """FP32 GMRES inner solves with FP64 iterative refinement: the oracle's FP64
    residual is <= 1e-6 and L^{0,0} is within 1e-5 (relative L2) of the oracle's
    direct solution."""
    N, R = 3, 10
    p = pn_inputs.fbm_point(N, R, 3, 0.5, 40.0, 0.95, 0.3)
    med = opn.Medium(p.sigma_t, p.albedo, p.g, p.Q00)
    S = opn.assemble(N, R, med)
    u_ref = opn.solve_direct(S)
    from paper_1807_00410_gb300 import System
    gpu = System(N, R, p.sigma_t, p.albedo, p.g, p.Q00)
    u = gpu.zeros(torch.float64)
    st = gpu.solve(u, solver="ir", tol=1e-6, max_iter=20000, restart=40)
    assert st["rel_residual"] <= 1e-6 and st["outer_iterations"] >= 1
    uo = S.layout.join(gpu.to_planes(u))
    assert opn.relative_residual(S.A, S.b, uo) <= 1.0001e-6
    L00, L00_ref = gpu.to_planes(u)[0], S.layout.split(u_ref)[0]
    assert np.linalg.norm(L00 - L00_ref) / np.linalg.norm(L00_ref) <= 1e-5
    gpu.close()


def test_zero_source_solves_immediately():
    from paper_1807_00410_gb300 import System
    R = 4
    gpu = System(1, R, np.full((R, R, R), 2.0), 0.5, 0.0, None)
    u = gpu.zeros(torch.float64)
    st = gpu.solve(u, solver="gmres", tol=1e-8)
    assert st["iterations"] == 0 and float(u.abs().max()) == 0.0
    gpu.close()


def test_cgls_fp32_reaches_moderate_tolerance():
    N, R = 1, 10
    med, gpu = _system(N, R, 8, albedo_field=False)
    u = gpu.zeros(torch.float32)
    st = gpu.solve(u, solver="cgls", tol=1e-4, max_iter=20000)
    S = opn.assemble(N, R, med)
    assert opn.relative_residual(S.A, S.b, S.layout.join(gpu.to_planes(u))) <= 2e-4
    assert st["iterations"] > 0
    gpu.close()


# --- errors ---------------------------------------------------------------------

def test_argument_and_nonfinite_errors():
    from paper_1807_00410_gb300 import PnError, System
    from paper_1807_00410_gb300 import pn as ppn
    R = 4
    st = np.full((R, R, R), 2.0)
    st[1, 1, 1] = np.nan
    with pytest.raises(PnError) as e:
        System(1, R, st, 0.5, 0.0, np.ones((R, R, R)))
    assert e.value.code == ppn.PN_ERR_ARG
    gpu = System(1, R, np.full((R, R, R), 2.0), 0.5, 0.0, np.ones((R, R, R)))
    x = gpu.zeros(torch.float64)
    with pytest.raises(ValueError):
        gpu.apply(x[:-1], x[:-1].clone())
    with pytest.raises(PnError) as e:
        gpu.apply(x, x)
    assert e.value.code == ppn.PN_ERR_ARG
    x[0] = float("nan")
    with pytest.raises(PnError) as e:
        gpu.residual(x, gpu.zeros(torch.float64))
    assert e.value.code == ppn.PN_ERR_NONFINITE
    gpu.close()


# --- full-size sampled parity ----------------------------------------------------

def _sampled_rows(layout_o, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    rows = []
    for _ in range(n):
        k = int(rng.integers(layout_o.K))
        sh = layout_o.shapes[k]
        rows.append((k, *[int(rng.integers(s)) for s in sh]))
    # every boundary face / last centre of some coefficients
    for k in range(0, layout_o.K, max(1, layout_o.K // 8)):
        nz, ny, nx = layout_o.shapes[k]
        rows += [(k, 0, 0, 0), (k, nz - 1, ny - 1, nx - 1), (k, nz // 2, 0, nx - 1), (k, 0, ny - 1, nx // 2)]
    return rows


@pytest.mark.parametrize("which", ["p5_64", "p7_256"])
def test_full_size_fp32_apply_sampled(which):
    """Full-size workloads in FP32, in the launch configuration the benchmark
    times: sampled outputs against the oracle's row-by-row evaluation."""
    from paper_1807_00410_gb300 import System
    p = pn_inputs.p5_64_fbm(0) if which == "p5_64" else pn_inputs.p7_256_cloud(0)
    med = opn.Medium(p.sigma_t, p.albedo, p.g, p.Q00, p.sigma_t_min)
    lay_o = opn.Layout(p.N, p.R)
    gpu = System(p.N, p.R, p.sigma_t, p.albedo, p.g, p.Q00, sigma_t_min=p.sigma_t_min)
    lay = gpu.layout
    rng = np.random.Generator(np.random.PCG64(11))
    host = rng.random(lay.n_elems, dtype=np.float32) - np.float32(0.5)
    x = torch.from_numpy(host).cuda()
    y = torch.empty_like(x)
    gpu.apply(x, y)
    r = torch.empty_like(x)
    gpu.residual(x, r)
    torch.cuda.synchronize()
    yh = y.cpu().numpy()
    rh = r.cpu().numpy()
    R = p.R
    parts_x, parts_y, parts_r = [None] * lay.K, [None] * lay.K, [None] * lay.K
    for q in range(lay.K):
        nz, ny, nx = lay.active_shape(q)
        sl = slice(q * lay.plane_stride, q * lay.plane_stride + lay.pitch_y * (R + 1))
        k = lay.plane_k[q]
        parts_x[k] = host[sl].reshape(R + 1, R + 1, lay.pitch_x)[:nz, :ny, :nx]
        parts_y[k] = yh[sl].reshape(R + 1, R + 1, lay.pitch_x)[:nz, :ny, :nx]
        parts_r[k] = rh[sl].reshape(R + 1, R + 1, lay.pitch_x)[:nz, :ny, :nx]
    rows = _sampled_rows(lay_o, 1500, 5)
    ref = opn.apply_rows(lay_o, med, parts_x, rows)
    got = np.array([parts_y[k][iz, iy, ix] for (k, iz, iy, ix) in rows], dtype=np.float64)
    scale = 10.0 * R + 100.0  # bounds sum_j |A_ij| |x_j|: <= 10 terms of |A_d|/h < R, |x| <= 1/2, sigma_t <= 100
    assert np.max(np.abs(got - ref)) <= 1e-5 * scale
    b = np.zeros(len(rows))
    b[[i for i, (k, *_r) in enumerate(rows) if k == 0]] = [
        p.Q00[iz, iy, ix] for (k, iz, iy, ix) in rows if k == 0]
    gotr = np.array([parts_r[k][iz, iy, ix] for (k, iz, iy, ix) in rows], dtype=np.float64)
    assert np.max(np.abs(gotr - (b - ref))) <= 1e-5 * scale
    # padding written as zero
    mask = np.ones(lay.n_elems, bool)
    for q in range(lay.K):
        nz, ny, nx = lay.active_shape(q)
        box = mask[q * lay.plane_stride: q * lay.plane_stride + lay.pitch_y * (R + 1)].reshape(R + 1, R + 1, lay.pitch_x)
        box[:nz, :ny, :nx] = False
    assert not np.any(yh[mask])
    gpu.close()
    del x, y, r
    torch.cuda.empty_cache()


@pytest.mark.parametrize("ortho", ["cgs2", "cgs1"])
def test_ir_with_each_orthogonalisation_meets_oracle_residual(ortho):
    """Both Gram-Schmidt variants of the FP32 inner GMRES give an FP64-refined
    solution whose oracle residual is <= 1e-6."""
    from paper_1807_00410_gb300 import System
    N, R = 5, 12
    p = pn_inputs.fbm_point(N, R, 7, 0.5, 40.0, 0.95, 0.3)
    med = opn.Medium(p.sigma_t, p.albedo, p.g, p.Q00)
    S = opn.assemble(N, R, med)
    gpu = System(N, R, p.sigma_t, p.albedo, p.g, p.Q00)
    u = gpu.zeros(torch.float64)
    st = gpu.solve(u, solver="ir", tol=1e-6, restart=20, ortho=ortho, profile=True)
    assert st["rel_residual"] <= 1e-6
    assert opn.relative_residual(S.A, S.b, S.layout.join(gpu.to_planes(u))) <= 1.0001e-6
    prof = gpu.profile()
    assert prof["apply"]["launches"] >= st["iterations"]
    assert prof["mdot"]["launches"] > 0 and prof["apply"]["ms"] > 0
    assert st["launches"] > prof["apply"]["launches"]
    gpu.close()


@pytest.mark.parametrize("N,R,restart", [(5, 12, 15), (1, 20, 16), (3, 17, 8)])
def test_ir_with_fp16_basis_meets_oracle_residual(N, R, restart):
    """The FP16-stored Krylov basis (FP32 arithmetic, FP64 refinement) gives a
    solution with oracle residual <= 1e-6 that agrees with the FP32-basis
    solve to the accuracy the residual allows (relative L2 of L00 <= 1e-5)."""
    from paper_1807_00410_gb300 import System
    p = pn_inputs.fbm_point(N, R, 11, 0.5, 40.0, 0.95, 0.3)
    med = opn.Medium(p.sigma_t, p.albedo, p.g, p.Q00)
    S = opn.assemble(N, R, med)
    gpu = System(N, R, p.sigma_t, p.albedo, p.g, p.Q00)
    u16 = gpu.zeros(torch.float64)
    st16 = gpu.solve(u16, solver="ir", tol=1e-6, restart=restart, ortho="cgs1", basis="f16", profile=True)
    assert gpu.profile()["mdot"]["launches"] > 0  # the profile of the last (FP16-basis) solve
    u32 = gpu.zeros(torch.float64)
    st32 = gpu.solve(u32, solver="ir", tol=1e-6, restart=restart, ortho="cgs1")
    assert st16["rel_residual"] <= 1e-6
    assert opn.relative_residual(S.A, S.b, S.layout.join(gpu.to_planes(u16))) <= 1.0001e-6
    a, b = gpu.to_planes(u16)[0], gpu.to_planes(u32)[0]
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-5
    assert st16["iterations"] <= 1.5 * st32["iterations"] + 2 * restart
    gpu.close()


@pytest.mark.parametrize("N,R,restart,augment", [(5, 12, 13, 2), (1, 20, 12, 4), (3, 12, 8, 1), (7, 8, 14, 2),
                                                  (3, 33, 13, 3)])
def test_ir_lgmres_meets_oracle_residual(N, R, restart, augment):
    """LGMRES(m, k): each restart cycle of the FP16-basis inner GMRES appends the
    corrections of up to k earlier cycles (kept across refinement steps) to its
    m Krylov directions.  The solution meets the oracle residual <= 1e-6, and
    (where the oracle's sparse LU is quick) L^{0,0} within 1e-5 of the direct
    solution; the iteration count stays within the plain GMRES(m + k) solve's
    plus a margin."""
    from paper_1807_00410_gb300 import System
    p = pn_inputs.fbm_point(N, R, 21, 0.5, 40.0, 0.95, 0.3)
    S = opn.assemble(N, R, opn.Medium(p.sigma_t, p.albedo, p.g, p.Q00))
    gpu = System(N, R, p.sigma_t, p.albedo, p.g, p.Q00)
    ua = gpu.zeros(torch.float64)
    sta = gpu.solve(ua, solver="ir", tol=1e-6, restart=restart, ortho="cgs1", basis="f16", augment=augment)
    up = gpu.zeros(torch.float64)
    stp = gpu.solve(up, solver="ir", tol=1e-6, restart=restart + augment, ortho="cgs1", basis="f16")
    assert sta["rel_residual"] <= 1e-6
    uo = S.layout.join(gpu.to_planes(ua))
    assert opn.relative_residual(S.A, S.b, uo) <= 1.0001e-6
    if S.A.shape[0] <= 70000:
        ref = S.layout.split(opn.solve_direct(S))[0]
        assert np.linalg.norm(S.layout.split(uo)[0] - ref) / np.linalg.norm(ref) <= 1e-5
    assert sta["iterations"] <= 1.5 * stp["iterations"] + 2 * (restart + augment)
    gpu.close()


def test_solve_orders_after_the_callers_stream_and_l2_residency_changes_no_bit():
    """pn_solve runs on the handle's own stream, joined to the caller's: an
    initial guess written on the caller's stream behind a long fill is seen
    (a converged guess needs no iteration).  Keeping the step vectors resident
    in L2 changes no bit of the solution."""
    from paper_1807_00410_gb300 import System
    p = pn_inputs.fbm_point(5, 20, 4, 0.5, 40.0, 0.95, 0.3)
    gpu = System(5, 20, p.sigma_t, p.albedo, p.g, p.Q00)
    opts = dict(solver="ir", tol=1e-6, restart=12, ortho="cgs1", basis="f16", augment=4)
    u_on = gpu.zeros(torch.float64)
    st_on = gpu.solve(u_on, **opts)
    gpu.set_l2_residency(False)
    u_off = gpu.zeros(torch.float64)
    st_off = gpu.solve(u_off, **opts)
    gpu.set_l2_residency(True)
    assert torch.equal(u_on, u_off) and st_on["iterations"] == st_off["iterations"]
    s = torch.cuda.Stream()
    u = gpu.zeros(torch.float64)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        big = torch.empty(1 << 28, dtype=torch.float32, device="cuda")
        for _ in range(4):
            big.fill_(1.0)
        u.copy_(u_on)
        st = gpu.solve(u, stream=s, **opts)
    assert st["iterations"] == 0 and st["rel_residual"] <= 1e-6
    gpu.close()


def test_staged_and_direct_vector_kernels_agree():
    """The FP16-basis GMRES's multi-dot and multi-axpy staged by bulk copies
    (mask 3) and with direct loads (mask 0): both solutions meet the oracle
    residual and agree to the accuracy the residual allows; masks outside
    [0, 3] are refused."""
    from paper_1807_00410_gb300 import PnError, System
    N, R = 3, 24
    p = pn_inputs.fbm_point(N, R, 8, 0.5, 40.0, 0.95, 0.3)
    S = opn.assemble(N, R, opn.Medium(p.sigma_t, p.albedo, p.g, p.Q00))
    gpu = System(N, R, p.sigma_t, p.albedo, p.g, p.Q00)
    opts = dict(solver="ir", tol=1e-6, restart=12, ortho="cgs1", basis="f16", augment=4)
    sols = []
    for mask in (3, 0, 1, 2):
        gpu.set_stream_kernels(mask)
        u = gpu.zeros(torch.float64)
        st = gpu.solve(u, **opts)
        uo = S.layout.join(gpu.to_planes(u))
        assert st["rel_residual"] <= 1e-6 and opn.relative_residual(S.A, S.b, uo) <= 1.0001e-6
        sols.append(S.layout.split(uo)[0])
    for a in sols[1:]:
        assert np.linalg.norm(a - sols[0]) / np.linalg.norm(sols[0]) <= 2e-5
    with pytest.raises(PnError):
        gpu.set_stream_kernels(4)
    gpu.close()


def test_lgmres_option_limits():
    from paper_1807_00410_gb300 import PnError, System
    p = pn_inputs.fbm_point(3, 8, 2, 0.5, 40.0, 0.95, 0.3)
    gpu = System(3, 8, p.sigma_t, p.albedo, p.g, p.Q00)
    for kw in ({"basis": "f32", "augment": 2}, {"basis": "f16", "restart": 15, "augment": 2},
               {"basis": "f16", "restart": 8, "augment": 9}, {"basis": "f16", "restart": 8, "augment": -1}):
        with pytest.raises(PnError):
            gpu.solve(gpu.zeros(torch.float64), solver="ir", **{"restart": 10, **kw})
    gpu.close()


def test_apply_tiling_plans_give_identical_outputs_and_tuner_picks_one():
    """Every z-chunking of the tiled FP32 operator computes each output with the
    same operands in the same order: apply and residual vectors are bitwise
    equal across plans; the autotuner keeps one of its candidates."""
    from paper_1807_00410_gb300 import System
    N, R = 5, 29
    p = pn_inputs.fbm_point(N, R, 13, 0.5, 40.0, 0.95, 0.3)
    gpu = System(N, R, p.sigma_t, p.albedo, p.g, p.Q00)
    g = torch.Generator(device="cpu").manual_seed(3)
    lay_o = opn.Layout(N, R)
    x = gpu.from_planes([torch.rand(sh, generator=g, dtype=torch.float64).numpy() for sh in lay_o.shapes],
                        dtype=torch.float32)
    ref_y, ref_r = gpu.zeros(torch.float32), gpu.zeros(torch.float32)
    gpu.apply(x, ref_y)
    gpu.residual(x, ref_r)
    for c in (1, 2, 8, 16):
        gpu.set_apply_tiling(c)
        y, r = gpu.zeros(torch.float32), gpu.zeros(torch.float32)
        gpu.apply(x, y)
        gpu.residual(x, r)
        assert torch.equal(y, ref_y) and torch.equal(r, ref_r)
    t = gpu.tune_apply()
    assert t["ctas_per_sm"] in (1, 2, 4, 8) and t["ms"] > 0 and t["kernel"] in ("tma", "register")
    y = gpu.zeros(torch.float32)
    gpu.apply(x, y)
    assert torch.equal(y, ref_y)
    gpu.close()


@pytest.mark.parametrize("N,R", [(0, 5), (1, 2), (1, 33), (2, 9), (3, 17), (4, 12), (5, 29), (6, 6), (7, 11),
                                 (3, 64), (7, 35)])
def test_tma_and_register_operator_kernels_agree_bitwise(N, R):
    """The TMA-staged and the register-staged tiled kernels compute every output
    with the same operands in the same order: apply, transpose and residual
    vectors are bitwise equal, for every z-chunking (chunks of one slice up to
    the whole column), with NaN in every padding slot of the input; the
    residual norm agrees to the rounding of its FP32 partial sums."""
    from paper_1807_00410_gb300 import System
    p = pn_inputs.fbm_point(N, R, 17 + N, 0.5, 40.0, 0.95, 0.3)
    gpu = System(N, R, p.sigma_t, p.albedo, p.g, p.Q00)
    lay_o = opn.Layout(N, R)
    rng = np.random.Generator(np.random.PCG64(N * 1000 + R))
    x = gpu.from_planes([rng.uniform(-1, 1, sh) for sh in lay_o.shapes], dtype=torch.float32)
    pad = gpu.from_planes([np.ones(sh) for sh in lay_o.shapes], dtype=torch.float32) == 0
    x[pad] = float("nan")
    out = {}
    for kern in ("register", "tma"):
        gpu.set_apply_kernel(kern)
        assert gpu.apply_kernel == kern
        for c in (1, 4, 16):
            gpu.set_apply_tiling(c)
            y, yt, r = gpu.zeros(torch.float32), gpu.zeros(torch.float32), gpu.zeros(torch.float32)
            gpu.apply(x, y)
            gpu.apply_t(x, yt)
            rel = gpu.residual(x, r)
            assert torch.isfinite(y).all() and torch.isfinite(r).all()
            out[(kern, c)] = (y, yt, r, rel)
    ref = out[("register", 4)]
    for key, (y, yt, r, rel) in out.items():
        assert torch.equal(y, ref[0]) and torch.equal(yt, ref[1]) and torch.equal(r, ref[2]), key
        # ||r|| adds each thread's FP32 partial sums of r^2 (over other rows in
        # the two kernels) in FP64: equal to FP32 rounding of those sums
        assert abs(rel - ref[3]) <= 1e-6 * ref[3], key
    gpu.close()


@pytest.mark.parametrize("N,R,basis", [(7, 8, "f16"), (7, 7, "f32"), (3, 2, "f16"), (1, 2, "f32")])
def test_ir_solves_at_p7_and_at_the_smallest_grid(N, R, basis):
    """P7 (the tiled kernel's largest classes; its residual mode loads the
    right-hand side in place) and R = 2 (one tile, every slot on the
    boundary) solve to the oracle's 1e-6."""
    from paper_1807_00410_gb300 import System
    p = pn_inputs.fbm_point(N, R, 17, 0.5, 40.0, 0.95, 0.3)
    med = opn.Medium(p.sigma_t, p.albedo, p.g, p.Q00)
    S = opn.assemble(N, R, med)
    gpu = System(N, R, p.sigma_t, p.albedo, p.g, p.Q00)
    u = gpu.zeros(torch.float64)
    st = gpu.solve(u, solver="ir", tol=1e-6, restart=15, ortho="cgs1", basis=basis)
    assert st["rel_residual"] <= 1e-6
    assert opn.relative_residual(S.A, S.b, S.layout.join(gpu.to_planes(u))) <= 1.0001e-6
    gpu.close()


def test_fp16_basis_rejected_outside_refinement():
    from paper_1807_00410_gb300 import System
    from paper_1807_00410_gb300.pn import PnError
    N, R = 3, 8
    p = pn_inputs.fbm_point(N, R, 12, 0.5, 40.0, 0.95, 0.3)
    gpu = System(N, R, p.sigma_t, p.albedo, p.g, p.Q00)
    with pytest.raises(PnError):
        gpu.solve(gpu.zeros(torch.float32), solver="gmres", basis="f16")
    with pytest.raises(PnError):
        gpu.solve(gpu.zeros(torch.float64), solver="ir", restart=20, basis="f16")
    gpu.close()


@pytest.mark.parametrize("N,R", [(1, 6), (3, 7), (5, 5)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_periodic_apply_transpose_residual_match_oracle(N, R, dtype):
    """The periodic test mode (every axis wraps, R slots per axis for every
    class) against the oracle's periodic assembly."""
    from paper_1807_00410_gb300 import System
    rng = np.random.default_rng(100 + 10 * N + R)
    st = rng.uniform(0.5, 20.0, (R, R, R))
    al = rng.uniform(0.2, 0.95, (R, R, R))
    q = rng.uniform(0.0, 1.0, (R, R, R))
    med = opn.Medium(st, al, 0.35, q)
    S = opn.assemble(N, R, med, periodic=True)
    gpu = System(N, R, st, al, 0.35, q, periodic=True)
    assert gpu.layout.n_active == S.layout.n
    tdt = torch.float64 if dtype == "f64" else torch.float32
    parts = [rng.uniform(-1, 1, sh) for sh in S.layout.shapes]
    x = gpu.from_planes(parts, dtype=tdt)
    xu = S.layout.join(gpu.to_planes(x))
    y = gpu.zeros(tdt)
    tol = 1e-12 if dtype == "f64" else 3e-6
    for op, ref in (("apply", S.A @ xu), ("apply_t", S.A.T @ xu), ("residual", S.b - S.A @ xu)):
        getattr(gpu, op)(x, y)
        got = S.layout.join(gpu.to_planes(y))
        np.testing.assert_allclose(got, ref, rtol=0, atol=tol * np.abs(ref).max() * 4)
    gpu.close()


@pytest.mark.parametrize("N,g", [(1, 0.0), (3, 0.4), (5, 0.7)])
def test_periodic_homogeneous_uniform_source_closed_form_on_gpu(N, g):
    """Homogeneous medium, uniform isotropic source, periodic box: transport
    vanishes, so L00 = Q / sigma_a everywhere and every other moment is 0
    (the exact solution of the continuous and the discrete system)."""
    from paper_1807_00410_gb300 import System
    R, st, al, Q0 = 8, 3.0, 0.8, 2.5
    gpu = System(N, R, np.full((R, R, R), st), al, g, np.full((R, R, R), Q0), periodic=True)
    L00 = Q0 / (st * (1.0 - al))
    # the first Krylov vector is an exact eigenvector (a breakdown in every variant)
    for kw in ({"ortho": "cgs1"}, {"ortho": "cgs1", "basis": "f16"}, {"ortho": "cgs2"}):
        u = gpu.zeros(torch.float64)
        s = gpu.solve(u, solver="ir", tol=1e-12, restart=15, **kw)
        assert s["rel_residual"] <= 1e-12
        planes = gpu.to_planes(u)
        np.testing.assert_allclose(planes[0], L00, rtol=1e-10)
        for k in range(1, len(planes)):
            assert np.abs(planes[k]).max() <= 1e-10 * L00
    u = gpu.zeros(torch.float64)
    s = gpu.solve(u, solver="gmres", tol=1e-12, restart=15, ortho="cgs1")
    np.testing.assert_allclose(gpu.to_planes(u)[0], L00, rtol=1e-10)
    gpu.close()


# --- source building and unstaggering ---------------------------------------------

@pytest.mark.parametrize("dtype,axis,sign", [("f64", 0, 1), ("f64", 2, -1), ("f32", 1, 1)])
def test_single_scatter_beam_matches_oracle(dtype, axis, sign):
    from oracle import source as osrc
    from paper_1807_00410_gb300 import pn as ppn
    N, R = 5, 13
    st = 40.0 * pn_inputs.value_noise_fbm(R, 2)
    al = pn_inputs.random_field((R, R, R), 3, 0.5, 0.99)
    ref = osrc.single_scatter_beam(st, al, 0.6, N, axis, sign, 0.3, (0.45, 0.55))
    tdt = torch.float64 if dtype == "f64" else torch.float32
    got = ppn.single_scatter_beam(N, torch.tensor(st, dtype=tdt).cuda(), torch.tensor(al, dtype=tdt).cuda(), 0.6,
                                  axis, sign, 0.3, (0.45, 0.55)).cpu().double().numpy()
    tol = 1e-12 if dtype == "f64" else 1e-5
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    assert (ref != 0).sum() > 0


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_unstagger_matches_oracle(dtype):
    from oracle import source as osrc
    N, R = 3, 9
    med, gpu = _system(N, R, 12)
    lay_o = opn.Layout(N, R)
    planes = _rand_planes(lay_o, 5)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    out = gpu.unstagger(gpu.from_planes(planes, dtype=tdt)).cpu().double().numpy()
    if dtype == "f32":
        planes = [p.astype(np.float32).astype(np.float64) for p in planes]
    ref = osrc.unstagger(lay_o, planes)
    np.testing.assert_allclose(out, ref, atol=1e-12 if dtype == "f64" else 1e-6)
    gpu.close()


def test_beam_source_solve_end_to_end():
    """Beam single-scatter moments built on the GPU feed pn_create as centre
    moments; the FP64-refined solve meets the oracle's residual on the same Q."""
    from oracle import source as osrc
    from paper_1807_00410_gb300 import System
    from paper_1807_00410_gb300 import pn as ppn
    N, R = 3, 12
    p = pn_inputs.cloud_point(N, R, 4, sig_max=30.0, albedo=0.9, g=0.5, sigma_t_min=0.5)
    st_d = torch.tensor(p.sigma_t, dtype=torch.float64).cuda()
    Q = ppn.single_scatter_beam(N, st_d, p.albedo, p.g, 0, 1, 0.25)
    gpu = System(N, R, st_d, p.albedo, p.g, Q, sigma_t_min=p.sigma_t_min)
    u = gpu.zeros(torch.float64)
    st = gpu.solve(u, solver="ir", tol=1e-6, restart=30)
    Qo = osrc.single_scatter_beam(p.sigma_t, p.albedo, p.g, N, 0, 1, 0.25)
    S = opn.assemble(N, R, opn.Medium(p.sigma_t, p.albedo, p.g, Qo, p.sigma_t_min))
    assert st["rel_residual"] <= 1e-6
    assert opn.relative_residual(S.A, S.b, S.layout.join(gpu.to_planes(u))) <= 1.001e-6
    gpu.close()
