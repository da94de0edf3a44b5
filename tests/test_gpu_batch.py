"""The batched solver (pn_batch_*): one launch per phase over instances of
different orders, grid sizes and dimensions.  The batched operator equals
the single-system operator bit for bit in FP64 and the oracle within FP32
rounding; every instance of a batched solve meets its tolerance by the
oracle's own residual and agrees with its single-system solve."""
import numpy as np
import pytest

import pn_inputs
from oracle import pn as opn
from oracle import pn2d

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# (N, R, dims, seed)
MIXED = [(1, 12, 3, 1), (3, 17, 3, 2), (5, 9, 3, 3), (3, 20, 2, 4), (7, 8, 3, 5), (1, 33, 2, 6)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available()
    from paper_1807_00410_gb300 import build
    build.build()


def _instance(N, R, dims, seed, source=True):
    from paper_1807_00410_gb300 import System
    if dims == 3:
        p = pn_inputs.fbm_point(N, R, seed, 0.5, 30.0, 0.9, 0.3)
        Q = p.Q00 if source else np.zeros_like(p.Q00)
        med = opn.Medium(p.sigma_t, p.albedo, p.g, Q)
        return System(N, R, p.sigma_t, p.albedo, p.g, Q), ("3d", N, R, med)
    rng = np.random.default_rng(seed)
    st = rng.uniform(0.5, 30.0, (R, R))
    al = rng.uniform(0.3, 0.95, (R, R))
    q = np.zeros((R, R))
    if source:
        q[R // 2, R // 3] = float(R * R)
    return System(N, R, st, al, 0.3, q, dims=2), ("2d", N, R, (st, al, 0.3, q))


def _oracle(desc):
    kind, N, R, data = desc
    if kind == "3d":
        S = opn.assemble(N, R, data)
        return S.layout, S.A, S.b
    st, al, g, q = data
    return pn2d.assemble_2d(N, R, st, al, g, q)


@pytest.mark.parametrize("tiling", [None, (256, 1024, 1, 1), (65536, 262144, 8, 8)])
def test_batched_apply_equals_single_and_oracle(tiling):
    from paper_1807_00410_gb300 import Batch
    systems, descs = zip(*[_instance(*c) for c in MIXED])
    batch = Batch(systems, restart=4)
    if tiling:
        batch.set_tiling(*tiling)
        t = batch.tiling()
        assert {k: t[k] for k in ("op_chunk", "vec_chunk", "op_ctas_per_sm", "vec_ctas_per_sm")} == dict(
            zip(("op_chunk", "vec_chunk", "op_ctas_per_sm", "vec_ctas_per_sm"), tiling))
    g = torch.Generator(device="cpu").manual_seed(11)
    x64 = []
    for s in systems:
        parts = [torch.rand(sh, generator=g, dtype=torch.float64).numpy() * 2 - 1
                 for sh in [p.shape for p in s.to_planes(s.zeros(torch.float64))]]
        x64.append(s.from_planes(parts, dtype=torch.float64))
    y64 = [s.zeros(torch.float64) for s in systems]
    batch.apply(x64, y64)
    for s, x, y in zip(systems, x64, y64):
        ref = s.zeros(torch.float64)
        s.apply(x, ref)
        assert torch.equal(y, ref)  # same per-point arithmetic, same order
    x32 = [x.float() for x in x64]
    y32 = [s.zeros(torch.float32) for s in systems]
    batch.apply(x32, y32)
    for s, d, x, y in zip(systems, descs, x32, y32):
        lay, A, _ = _oracle(d)
        xr = lay.join(s.to_planes(x))
        ref = A @ xr
        got = lay.join(s.to_planes(y))
        np.testing.assert_allclose(got, ref, rtol=0, atol=4e-6 * np.abs(ref).max())
        # padding and inactive slots are zero
        assert abs(np.abs(y.double().cpu().numpy()).sum() - np.abs(got).sum()) <= 1e-9 * np.abs(got).sum()
    batch.close()
    for s in systems:
        s.close()


def test_batched_solve_meets_oracle_residual_and_matches_single():
    from paper_1807_00410_gb300 import Batch
    cases = [(1, 12, 3, 21), (3, 16, 3, 22), (5, 10, 3, 23), (3, 24, 2, 24), (1, 9, 3, 25)]
    systems, descs = zip(*[_instance(*c) for c in cases])
    batch = Batch(systems, restart=15)
    us = [s.zeros(torch.float64) for s in systems]
    stats = batch.solve(us, tol=1e-6)
    for s, d, u, st in zip(systems, descs, us, stats):
        assert st["status"] == 0 and st["rel_residual"] <= 1e-6 and st["iterations"] > 0
        lay, A, b = _oracle(d)
        uh = lay.join(s.to_planes(u))
        assert np.linalg.norm(b - A @ uh) / np.linalg.norm(b) <= 1.0001e-6
        ref = s.zeros(torch.float64)
        s.solve(ref, solver="ir", tol=1e-6, restart=15, ortho="cgs1")
        assert float((u - ref).norm() / ref.norm()) <= 1e-5
    # a second solve from zero is bitwise identical (fixed reduction order)
    us2 = [s.zeros(torch.float64) for s in systems]
    batch.solve(us2, tol=1e-6)
    assert all(torch.equal(a, b) for a, b in zip(us, us2))
    batch.close()
    for s in systems:
        s.close()


def test_tiled_and_generic_operator_paths_both_meet_the_oracle():
    """Graph mode with per-instance tiled operator launches on concurrent
    branches, and with the one generic launch: both solve every instance to
    the oracle's 1e-6 and agree with each other to what that allows."""
    from paper_1807_00410_gb300 import Batch
    cases = [(1, 16, 3, 61), (3, 14, 3, 62), (5, 12, 3, 63), (3, 18, 2, 64), (7, 8, 3, 65)]
    systems, descs = zip(*[_instance(*c) for c in cases])
    batch = Batch(systems, restart=12)
    out = {}
    for tiled in (True, False):
        batch.set_op_path(tiled)
        assert batch.tiling()["tiled_operator"] == tiled
        us = [s.zeros(torch.float64) for s in systems]
        stats = batch.solve(us, tol=1e-6)
        for s, d, u, st in zip(systems, descs, us, stats):
            lay, A, b = _oracle(d)
            assert st["status"] == 0
            assert np.linalg.norm(b - A @ lay.join(s.to_planes(u))) / np.linalg.norm(b) <= 1.0001e-6
        out[tiled] = us
    for a, b in zip(out[True], out[False]):
        assert float((a - b).norm() / b.norm()) <= 1e-5
    batch.close()
    for s in systems:
        s.close()


def test_batched_zero_source_and_iteration_cap():
    from paper_1807_00410_gb300 import Batch
    s0, _ = _instance(3, 10, 3, 31, source=False)
    s1, d1 = _instance(3, 12, 3, 32)
    batch = Batch([s0, s1], restart=8)
    us = [s0.zeros(torch.float64), s1.zeros(torch.float64)]
    stats = batch.solve(us, tol=1e-6)
    assert stats[0]["status"] == 0 and stats[0]["iterations"] == 0 and float(us[0].abs().max()) == 0.0
    assert stats[1]["status"] == 0 and stats[1]["rel_residual"] <= 1e-6
    # an inner-iteration cap every instance hits: not converged, finite iterates
    capped = [s0.zeros(torch.float64), s1.zeros(torch.float64)]
    stats = batch.solve(capped, tol=1e-12, max_iter=5, raise_on_error=False)
    assert stats[1]["status"] == -4 and stats[1]["iterations"] <= 8 + 5
    assert bool(torch.isfinite(capped[1]).all())
    batch.close()
    s0.close()
    s1.close()


def test_autotuner_keeps_a_valid_tiling_and_solves():
    from paper_1807_00410_gb300 import Batch
    systems, descs = zip(*[_instance(*c) for c in MIXED[:4]])
    batch = Batch(systems, restart=10, tune=True)
    t = batch.tiling()
    assert t["op_chunk"] in (4096, 16384, 65536) and t["vec_chunk"] in (16384, 65536, 262144)
    assert t["op_ctas_per_sm"] in (2, 4, 8) and t["vec_ctas_per_sm"] in (2, 4, 8)
    us = [s.zeros(torch.float64) for s in systems]
    stats = batch.solve(us, tol=1e-6)
    for s, d, u, st in zip(systems, descs, us, stats):
        lay, A, b = _oracle(d)
        uh = lay.join(s.to_planes(u))
        assert st["status"] == 0
        assert np.linalg.norm(b - A @ uh) / np.linalg.norm(b) <= 1.0001e-6
    batch.close()
    for s in systems:
        s.close()


def test_persistent_mode_equals_graph_mode():
    """One cooperative launch per cycle (phases separated by bounded grid
    barriers) computes exactly what the captured graph computes: the same
    work items, partials and reduction order."""
    from paper_1807_00410_gb300 import Batch
    cases = [(1, 12, 3, 41), (3, 14, 3, 42), (5, 8, 3, 43), (3, 16, 2, 44)]
    systems, descs = zip(*[_instance(*c) for c in cases])
    batch = Batch(systems, restart=10)
    batch.set_op_path(False)  # the persistent cycle uses the generic batched operator
    ug = [s.zeros(torch.float64) for s in systems]
    sg = batch.solve(ug, tol=1e-6)
    batch.set_mode(True)
    up = [s.zeros(torch.float64) for s in systems]
    sp = batch.solve(up, tol=1e-6)
    assert [a["iterations"] for a in sg] == [a["iterations"] for a in sp]
    assert all(torch.equal(a, b) for a, b in zip(ug, up))
    assert sp[0]["launches"] < sg[0]["launches"]
    for s, d, u in zip(systems, descs, up):
        lay, A, b = _oracle(d)
        uh = lay.join(s.to_planes(u))
        assert np.linalg.norm(b - A @ uh) / np.linalg.norm(b) <= 1.0001e-6
    batch.close()
    for s in systems:
        s.close()


def test_grid_barrier_completes_and_its_bounded_wait_runs_out():
    """A barrier that every CTA reaches completes; one that expects a CTA
    which does not exist gives up after its poll limit (a few ms here),
    reports PN_ERR_TIMEOUT, and the context stays usable."""
    from paper_1807_00410_gb300.pn import barrier_test
    assert barrier_test(16, 16, 1 << 22) == (0, 0)
    assert barrier_test(16, 17, 20000) == (-7, 1)
    s, d = _instance(3, 10, 3, 51)
    x = s.zeros(torch.float32) + 1.0
    y = s.zeros(torch.float32)
    s.apply(x, y)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(y).all())
    s.close()


def test_batched_exact_eigenvector_breakdown():
    """A homogeneous periodic instance whose first Krylov vector is an exact
    eigenvector (happy breakdown) beside an ordinary one: both converge."""
    from paper_1807_00410_gb300 import Batch, System
    R = 8
    s0 = System(3, R, np.full((R, R, R), 3.0), 0.8, 0.4, np.full((R, R, R), 2.5), periodic=True)
    s1, d1 = _instance(3, 10, 3, 71)
    batch = Batch([s0, s1], restart=10)
    us = [s0.zeros(torch.float64), s1.zeros(torch.float64)]
    st = batch.solve(us, tol=1e-10)
    assert all(x["status"] == 0 for x in st)
    np.testing.assert_allclose(s0.to_planes(us[0])[0], 2.5 / (3.0 * 0.2), rtol=1e-9)
    batch.close()
    s0.close()
    s1.close()


def test_solo_instances_solved_one_by_one_inside_the_batch():
    """With a solo threshold between the instances' sizes, the larger ones are
    solved one after another by pn_solve inside pn_batch_solve and the rest by
    the batched launches: every instance meets the oracle residual 1e-6, and a
    solo instance's solution is bitwise the single-system solve with the same
    options (FP64 refinement around FP32 GMRES(m), one Gram-Schmidt pass)."""
    from paper_1807_00410_gb300 import Batch
    systems, descs = zip(*[_instance(*c) for c in MIXED])
    sizes = [s.layout.n_active for s in systems]
    thr = sorted(sizes)[len(sizes) // 2]
    batch = Batch(systems, restart=8)
    batch.set_solo(thr)
    us = [s.zeros(torch.float64) for s in systems]
    stats = batch.solve(us, tol=1e-6, max_iter=20000)
    for s, d, u, st in zip(systems, descs, us, stats):
        assert st["status"] == 0
        lay, A, b = _oracle(d)
        assert opn.relative_residual(A, b, lay.join(s.to_planes(u))) <= 1.0001e-6
    for s, u, n in zip(systems, us, sizes):
        if n >= thr:
            ref = s.zeros(torch.float64)
            s.solve(ref, solver="ir", tol=1e-6, restart=8, ortho="cgs1", max_iter=20000)
            assert torch.equal(u, ref)
    # the solve's work lists left the solo instances out: a batched apply
    # afterwards still covers every instance
    ys = [s.zeros(torch.float64) for s in systems]
    batch.apply(us, ys)
    for s, u, y in zip(systems, us, ys):
        ref = s.zeros(torch.float64)
        s.apply(u, ref)
        assert torch.equal(y, ref)
    # and a solve with every instance batched again meets the target
    batch.set_solo(0)
    us2 = [s.zeros(torch.float64) for s in systems]
    for st in batch.solve(us2, tol=1e-6, max_iter=20000):
        assert st["status"] == 0 and st["rel_residual"] <= 1e-6
    batch.close()
    for s in systems:
        s.close()
