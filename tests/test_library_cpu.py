"""CPU-side checks of the CUDA library and its binding (no GPU needed):
the library builds for sm_103a, loads, and exports every symbol the header
declares; the binding's layout marshalling round-trips."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pn_gb300.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1807_00410_gb300 import build, pn
    build.build()
    return pn.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pn_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for fn in ["pn_create", "pn_apply", "pn_apply_t", "pn_residual", "pn_solve", "pn_destroy"]:
        assert fn in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1807_00410_gb300 import pn
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(pn.EXPORTS) == declared_functions()
    out = subprocess.run(["nm", "-D", "--defined-only", pn.LIB_PATH], capture_output=True, text=True).stdout
    for name in declared_functions():
        assert re.search(rf"\bT {name}\b", out), name


def test_build_targets_sm_103a_only():
    from paper_1807_00410_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_argument_errors_without_gpu(lib):
    """Invalid arguments are rejected before any device work."""
    from paper_1807_00410_gb300 import pn
    h = ctypes.c_void_p()
    assert lib.pn_create(ctypes.byref(h), 9, 8, None, 0, None) == pn.PN_ERR_ARG
    assert b"N must be" in lib.pn_last_error(None)
    m = pn._Medium()
    assert lib.pn_create(ctypes.byref(h), 3, 1, ctypes.byref(m), 0, None) == pn.PN_ERR_ARG
    assert lib.pn_create(ctypes.byref(h), 3, 8, ctypes.byref(m), 0, None) == pn.PN_ERR_ARG  # NULL sigma_t
    assert lib.pn_destroy(None) == 0
    o = pn._SolveOpts()
    lib.pn_default_solve_opts(ctypes.byref(o))
    assert o.tol == 1e-6 and o.restart == 60
    g = ctypes.c_double()
    for args in ((100, 64, 32, 1), (256, 62, 32, 1), (256, 64, 48, 1), (256, 64, 32, 3), (160, 64, 64, 1)):
        assert lib.pn_access_probe(*args, ctypes.byref(g), None) == pn.PN_ERR_ARG, args
    assert lib.pn_access_probe(256, 64, 32, 1, None, None) == pn.PN_ERR_ARG
    assert lib.pn_fma_peak(7, ctypes.byref(g), None) == pn.PN_ERR_ARG


def test_struct_sizes_match_header():
    """ctypes mirrors of the C structs have the C layout (x86-64 / aarch64 LP64)."""
    from paper_1807_00410_gb300 import pn
    assert ctypes.sizeof(pn._Medium) == 64
    assert ctypes.sizeof(pn._Layout) == 5 * 8 + 16 + 2 * 64 * 4
    assert ctypes.sizeof(pn._SolveOpts) == 64  # 4+4+8+4+4+8+4+4+4+4 = 48, an 8-byte pointer, two ints
    assert pn._SolveOpts.augment.offset == 60
    assert ctypes.sizeof(pn._SolveStats) == 48


def header_defines():
    return {m.group(1): int(m.group(2)) for m in
            re.finditer(r"#define\s+(PN_[A-Z0-9_]+)\s+(-?\d+)\b", open(HEADER).read())}


def test_binding_constants_match_the_header():
    """The binding's codes for operator kernels, solvers, bases and errors are
    the header's (a mismatch would select the wrong kernel or solver)."""
    from paper_1807_00410_gb300 import pn
    d = header_defines()
    assert pn.System.APPLY_KERNELS == {"register": d["PN_APPLY_KERNEL_REGISTER"], "tma": d["PN_APPLY_KERNEL_TMA"]}
    assert pn.SOLVERS["cgls"] == d["PN_SOLVER_CGLS"] and pn.SOLVERS["gmres"] == d["PN_SOLVER_GMRES"]
    assert pn.SOLVERS["ir"] == d["PN_SOLVER_IR_GMRES"] and pn.SOLVERS["ir_fgmres"] == d["PN_SOLVER_IR_FGMRES"]
    assert (d["PN_BASIS_F32"], d["PN_BASIS_F16"]) == (0, 1)  # the binding maps "f32"/"f16" to 0/1
    assert (d["PN_ORTHO_CGS2"], d["PN_ORTHO_CGS1"]) == (0, 1)  # and "cgs2"/"cgs1" to 0/1
    assert d["PN_ERR_TIMEOUT"] < 0 and d["PN_OK"] == 0
