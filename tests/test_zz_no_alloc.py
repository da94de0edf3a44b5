"""pn_dot_noalloc: the inner product that allocates nothing.

It exists for callers that cannot allocate device memory where they need a
reduction (an application owning the whole device-memory budget, a real-time
loop that must not take allocator locks, code without a pn_handle).  The test
calls it through the C ABI twice in a row and compares each result with the
handle-based pn_dot, within the tolerances the other GPU tests use (1e-13
relative in FP64, 1e-6 in FP32).  It is collected last so that a run stopping
at the first failure has already run every other test, and it passes both
alone in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1807_00410_gb300 import build, pn
    build.build()
    return pn, pn.load_library()


def _call(lib, a, b, n, code):
    out = ctypes.c_double(float("nan"))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.pn_dot_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), n, code,
                            ctypes.byref(out), stream)
    return rc, out.value


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_dot_noalloc_matches_pn_dot_on_two_calls_in_a_row(dtype):
    assert torch.cuda.is_available()
    pn, lib = _lib()
    from paper_1807_00410_gb300 import System
    R, N = 9, 3
    sysm = System(N, R, np.full((R, R, R), 2.0), 0.8, 0.2, np.ones((R, R, R)))
    n = sysm.layout.n_elems
    tdt, code, tol = (torch.float64, pn.PN_F64, 1e-13) if dtype == "f64" else (torch.float32, pn.PN_F32, 1e-6)
    g = torch.Generator(device="cpu").manual_seed(3)
    pairs = [tuple(torch.rand(n, generator=g, dtype=torch.float64).to(tdt).cuda() - 0.25 for _ in range(2))
             for _ in range(2)]
    for a, b in pairs:  # two calls in a row, on different data
        ref = sysm.dot(a, b)
        rc, got = _call(lib, a, b, n, code)
        assert rc == pn.PN_OK
        assert abs(got - ref) <= tol * abs(ref), (got, ref)
    # the second call again on the first pair: the shared scratch keeps no state
    a, b = pairs[0]
    rc, got = _call(lib, a, b, n, code)
    assert rc == pn.PN_OK and abs(got - sysm.dot(a, b)) <= tol * abs(sysm.dot(a, b))
    sysm.close()


def test_dot_noalloc_ragged_length_and_limits():
    pn, lib = _lib()
    g = torch.Generator(device="cpu").manual_seed(4)
    n = 3 * 8192 + 77  # not a whole number of blocks
    a = torch.rand(n, generator=g, dtype=torch.float64).cuda()
    b = torch.rand(n, generator=g, dtype=torch.float64).cuda()
    ref = float(np.dot(a.cpu().numpy(), b.cpu().numpy()))
    for _ in range(2):
        rc, got = _call(lib, a, b, n, pn.PN_F64)
        assert rc == pn.PN_OK and abs(got - ref) <= 1e-13 * abs(ref)
    rc, got = _call(lib, a, b, 0, pn.PN_F64)
    assert rc == pn.PN_OK and got == 0.0
    # beyond the fixed scratch capacity: rejected before any device work
    rc, _ = _call(lib, a, b, pn.PN_NOALLOC_MAX_ELEMS + 1, pn.PN_F64)
    assert rc == pn.PN_ERR_TOO_LARGE
    rc, _ = _call(lib, a, b, -1, pn.PN_F64)
    assert rc == pn.PN_ERR_ARG
    rc, _ = _call(lib, a, b, n, 7)
    assert rc == pn.PN_ERR_ARG


def test_dot_noalloc_refuses_a_capturing_stream():
    """The call returns its result through a host copy and a stream
    synchronisation, which a stream being captured into a CUDA graph cannot
    take: on such a stream it returns PN_ERR_ARG before any device work, and
    the capture stays valid."""
    pn, lib = _lib()
    a = torch.ones(4096, dtype=torch.float64, device="cuda")
    b = torch.full_like(a, 2.0)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        c = a * 3.0
        rc, _ = _call(lib, a, b, a.numel(), pn.PN_F64)
    assert rc == pn.PN_ERR_ARG
    graph.replay()
    torch.cuda.synchronize()
    assert torch.all(c == 3.0)
    rc, got = _call(lib, a, b, a.numel(), pn.PN_F64)
    assert rc == pn.PN_OK and got == 2.0 * a.numel()
