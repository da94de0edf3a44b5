"""The 2D reduction on the GPU (pn_create_2d, section "2D checkerboard")
against the 2D oracle (oracle/pn2d.py, itself pinned against the z-periodic
3D oracle): operator, transpose and residual element by element in FP64 and
FP32 on ragged grids, the solvers to the paper's 1e-10 on the checkerboard,
unstagger, and the 3D-only entry points refusing a 2D handle."""
import numpy as np
import pytest

import pn_inputs
from oracle import pn2d

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available()
    from paper_1807_00410_gb300 import build
    build.build()


def _medium(R, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.5, 30.0, (R, R)), rng.uniform(0.2, 0.99, (R, R)), 0.4, rng.uniform(0.0, 1.0, (R, R))


@pytest.mark.parametrize("N,R", [(1, 7), (3, 13), (5, 33), (7, 9)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_2d_apply_transpose_residual_match_oracle(N, R, dtype):
    from paper_1807_00410_gb300 import System
    st, al, g, q = _medium(R, N * 100 + R)
    lay, A, b = pn2d.assemble_2d(N, R, st, al, g, q)
    gpu = System(N, R, st, al, g, q, dims=2)
    assert gpu.layout.K == lay.K and gpu.layout.n_active == lay.n
    assert [gpu.layout.plane_k[p] for p in sorted(range(lay.K), key=gpu.layout.coefficient_index)] == lay.k3
    rng = np.random.default_rng(7)
    u = rng.uniform(-1.0, 1.0, lay.n)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    x = gpu.from_planes(lay.split(u), dtype=tdt)
    uq = lay.join(gpu.to_planes(x))  # what the GPU actually holds (FP32 rounding)
    y = gpu.zeros(tdt)
    tol = 1e-12 if dtype == "f64" else 2e-6
    for op, ref in (("apply", A @ uq), ("apply_t", A.T @ uq), ("residual", b - A @ uq)):
        getattr(gpu, op)(x, y)
        got = lay.join(gpu.to_planes(y))
        scale = np.abs(ref).max()
        np.testing.assert_allclose(got, ref, rtol=0, atol=tol * scale * 4)
        # padding and inactive slots hold zeros
        yh = y.double().cpu().numpy()
        assert abs(np.abs(yh).sum() - np.abs(got).sum()) <= 1e-9 * np.abs(got).sum()
    gpu.close()


@pytest.mark.parametrize("N", [1, 5])
def test_2d_checkerboard_solves_to_paper_tolerance(N):
    """The checkerboard workload at 71 x 71 to ||Q - A u|| / ||Q|| <= 1e-10
    (the paper's tolerance), measured by the oracle, and agreeing with the
    oracle's direct solve."""
    from paper_1807_00410_gb300 import System
    R = 71
    st, al, Q = pn_inputs.checkerboard_2d(R)
    lay, A, b = pn2d.assemble_2d(N, R, st, al, 0.0, Q)
    gpu = System(N, R, st, al, 0.0, Q, dims=2)
    u = gpu.zeros(torch.float64)
    s = gpu.solve(u, solver="ir", tol=1e-10, restart=30, ortho="cgs1", max_iter=200000, max_outer=100)
    assert s["rel_residual"] <= 1e-10
    uh = lay.join(gpu.to_planes(u))
    assert np.linalg.norm(b - A @ uh) / np.linalg.norm(b) <= 1.0001e-10
    ref = pn2d.solve_direct_2d(A, b)
    L0 = lay.split(uh)[0]
    L0r = lay.split(ref)[0]
    assert np.linalg.norm(L0 - L0r) / np.linalg.norm(L0r) <= 1e-8
    gpu.close()


def test_2d_cgls_and_gmres_fp64():
    from paper_1807_00410_gb300 import System
    N, R = 3, 24
    st, al, g, q = _medium(R, 5)
    lay, A, b = pn2d.assemble_2d(N, R, st, al, g, q)
    gpu = System(N, R, st, al, g, q, dims=2)
    for solver, kw in (("cgls", {}), ("gmres", {"restart": 40})):
        u = gpu.zeros(torch.float64)
        s = gpu.solve(u, solver=solver, tol=1e-9, max_iter=100000, **kw)
        uh = lay.join(gpu.to_planes(u))
        assert s["rel_residual"] <= 1e-9
        assert np.linalg.norm(b - A @ uh) / np.linalg.norm(b) <= 1.0001e-9
    gpu.close()


def test_2d_unstagger():
    from paper_1807_00410_gb300 import System
    N, R = 3, 10
    st, al, g, q = _medium(R, 6)
    lay = pn2d.Layout2D(N, R)
    gpu = System(N, R, st, al, g, q, dims=2)
    rng = np.random.default_rng(3)
    parts = [rng.uniform(-1, 1, s) for s in lay.shapes]
    x = gpu.from_planes(parts, dtype=torch.float64)
    out = gpu.unstagger(x).cpu().numpy()
    assert out.shape == (lay.K, R, R)
    for k, (px, py) in enumerate(lay.classes):
        P = parts[k]
        # a cell's value: the mean of the slots of its own grid around the centre
        ref = sum(P[dy:dy + R, dx:dx + R] for dy in range(py + 1) for dx in range(px + 1)) / ((px + 1) * (py + 1))
        np.testing.assert_allclose(out[k], ref, rtol=1e-14, atol=1e-15)
    gpu.close()


def test_2d_handle_refuses_3d_only_calls():
    from paper_1807_00410_gb300 import Net, System
    from paper_1807_00410_gb300.pn import PnError
    N, R = 3, 16
    st, al, g, q = _medium(R, 8)
    gpu = System(N, R, st, al, g, q, dims=2)
    net = Net(19, 16)
    v = gpu.zeros(torch.float32)
    with pytest.raises(PnError):
        gpu.cnn_features(v, 1.0)
    with pytest.raises(PnError):
        gpu.solve(gpu.zeros(torch.float64), solver="ir_fgmres", precond=net)
    net.close()
    gpu.close()


def test_2d_fp16_basis_refinement_meets_oracle():
    """The FP16-stored Krylov basis on a 2D handle (the generic FP32 operator)."""
    from paper_1807_00410_gb300 import System
    N, R = 5, 40
    st, al, g, q = _medium(R, 9)
    lay, A, b = pn2d.assemble_2d(N, R, st, al, g, q)
    gpu = System(N, R, st, al, g, q, dims=2)
    u = gpu.zeros(torch.float64)
    s = gpu.solve(u, solver="ir", tol=1e-8, restart=15, ortho="cgs1", basis="f16")
    assert s["rel_residual"] <= 1e-8
    uh = lay.join(gpu.to_planes(u))
    assert np.linalg.norm(b - A @ uh) / np.linalg.norm(b) <= 1.0001e-8
    gpu.close()
