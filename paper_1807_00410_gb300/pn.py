"""Python binding of libpn_gb300.so (argument marshalling only).

Every computation runs in the library's CUDA kernels; this module only
converts arguments (numpy arrays or torch tensors) to the C ABI declared in
include/pn_gb300.h, allocates caller-owned vectors with torch, and slices the
padded vector layout into per-coefficient views.  There is no CPU fallback:
if the library is missing or fails to load, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpn_gb300.so")

PN_OK = 0
PN_ERR_ARG = -1
PN_ERR_ALLOC = -2
PN_ERR_CUDA = -3
PN_ERR_NOT_CONVERGED = -4
PN_ERR_BREAKDOWN = -5
PN_ERR_NONFINITE = -6
PN_ERR_UNSUPPORTED = -8
PN_ERR_TOO_LARGE = -9
PN_NOALLOC_MAX_ELEMS = 1 << 31
PN_F32, PN_F64 = 0, 1
PN_BC_VACUUM = 0
PN_BC_PERIODIC_TEST = 1
PN_Q_CENTRE_00, PN_Q_CENTRE_MOMENTS = 0, 1
SOLVERS = {"cgls": 0, "gmres": 1, "ir": 2, "ir_fgmres": 3}

ERROR_NAMES = {
    PN_ERR_ARG: "PN_ERR_ARG", PN_ERR_ALLOC: "PN_ERR_ALLOC", PN_ERR_CUDA: "PN_ERR_CUDA",
    PN_ERR_NOT_CONVERGED: "PN_ERR_NOT_CONVERGED", PN_ERR_BREAKDOWN: "PN_ERR_BREAKDOWN",
    PN_ERR_NONFINITE: "PN_ERR_NONFINITE", PN_ERR_UNSUPPORTED: "PN_ERR_UNSUPPORTED",
    PN_ERR_TOO_LARGE: "PN_ERR_TOO_LARGE",
}

# Every symbol the header declares (checked by the CPU test-suite).
EXPORTS = ["pn_create", "pn_create_2d", "pn_destroy", "pn_get_layout", "pn_last_error", "pn_apply", "pn_apply_t",
           "pn_residual", "pn_dot", "pn_axpby", "pn_default_solve_opts", "pn_solve", "pn_profile_get",
           "pn_dot_noalloc", "pn_single_scatter_beam", "pn_unstagger", "pn_cnn_create", "pn_cnn_destroy",
           "pn_cnn_last_error", "pn_cnn_num_params", "pn_cnn_set_params", "pn_cnn_get_params", "pn_cnn_get_grads",
           "pn_cnn_forward", "pn_cnn_backward", "pn_cnn_adam_step", "pn_cnn_train_step", "pn_cnn_features",
           "pn_cnn_targets", "pn_cnn_output", "pn_cnn_precondition", "pn_batch_create", "pn_batch_destroy",
           "pn_batch_last_error", "pn_batch_apply", "pn_batch_solve", "pn_batch_set_tiling", "pn_batch_get_tiling",
           "pn_batch_tune", "pn_batch_set_mode", "pn_batch_barrier_test", "pn_tune_apply",
           "pn_set_apply_tiling", "pn_batch_set_op_path", "pn_batch_get_op_path", "pn_set_apply_kernel",
           "pn_get_apply_kernel", "pn_set_l2_residency", "pn_get_apply_plan", "pn_set_stream_kernels",
           "pn_get_workspace", "pn_wait_timeout_test", "pn_set_pdl", "pn_cnn_set_conv_kernel",
           "pn_cnn_take_error", "pn_fma_peak", "pn_batch_set_solo", "pn_access_probe"]
PROFILE_KINDS = ["apply", "residual", "mdot", "maxpy", "dot", "vector", "scalar", "precond"]


class PnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class _Medium(ctypes.Structure):
    _fields_ = [("sigma_t", ctypes.c_void_p), ("albedo", ctypes.c_void_p), ("albedo_const", ctypes.c_double),
                ("g", ctypes.c_double), ("Q", ctypes.c_void_p), ("q_mode", ctypes.c_int),
                ("dtype", ctypes.c_int), ("on_device", ctypes.c_int), ("sigma_t_min", ctypes.c_double)]


class _Layout(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("K", ctypes.c_int), ("R", ctypes.c_int), ("pitch_x", ctypes.c_int64),
                ("pitch_y", ctypes.c_int64), ("plane_stride", ctypes.c_int64), ("n_elems", ctypes.c_int64),
                ("n_active", ctypes.c_int64), ("plane_k", ctypes.c_int * 64), ("plane_class", ctypes.c_int * 64)]


class _SolveOpts(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("precision", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("restart", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int), ("check_every", ctypes.c_int), ("profile", ctypes.c_int),
                ("ortho", ctypes.c_int), ("precond", ctypes.c_void_p), ("basis", ctypes.c_int),
                ("augment", ctypes.c_int)]


class _SolveStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("outer_iterations", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double), ("launches", ctypes.c_int64),
                ("precond_applications", ctypes.c_int), ("fallback", ctypes.c_int)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1807_00410_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sig = {
        "pn_create": (i, [ctypes.POINTER(vp), i, i, ctypes.POINTER(_Medium), i, vp]),
        "pn_create_2d": (i, [ctypes.POINTER(vp), i, i, ctypes.POINTER(_Medium), i, vp]),
        "pn_destroy": (i, [vp]),
        "pn_get_layout": (i, [vp, ctypes.POINTER(_Layout)]),
        "pn_last_error": (ctypes.c_char_p, [vp]),
        "pn_apply": (i, [vp, vp, vp, i, vp]),
        "pn_apply_t": (i, [vp, vp, vp, i, vp]),
        "pn_residual": (i, [vp, vp, vp, ctypes.POINTER(d), i, vp]),
        "pn_dot": (i, [vp, vp, vp, ctypes.POINTER(d), i, vp]),
        "pn_axpby": (i, [vp, d, vp, d, vp, i, vp]),
        "pn_default_solve_opts": (None, [ctypes.POINTER(_SolveOpts)]),
        "pn_solve": (i, [vp, vp, ctypes.POINTER(_SolveOpts), ctypes.POINTER(_SolveStats), vp]),
        "pn_profile_get": (i, [vp, i, ctypes.POINTER(d), ctypes.POINTER(i64), ctypes.POINTER(d)]),
        "pn_get_workspace": (i, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "pn_wait_timeout_test": (i, [vp, i, ctypes.c_longlong, ctypes.POINTER(i), vp]),
        "pn_dot_noalloc": (i, [vp, vp, i64, i, ctypes.POINTER(d), vp]),
        "pn_single_scatter_beam": (i, [i, i, vp, vp, d, d, i, i, d, d, d, vp, i, vp]),
        "pn_unstagger": (i, [vp, vp, vp, i, vp]),
        "pn_cnn_create": (i, [ctypes.POINTER(vp), i, i, ctypes.POINTER(ctypes.c_int * 4)]),
        "pn_cnn_destroy": (i, [vp]),
        "pn_cnn_last_error": (ctypes.c_char_p, [vp]),
        "pn_cnn_num_params": (i64, [vp]),
        "pn_cnn_set_params": (i, [vp, vp, i64]),
        "pn_cnn_get_params": (i, [vp, vp, i64]),
        "pn_cnn_get_grads": (i, [vp, vp, i64]),
        "pn_cnn_forward": (i, [vp, vp, vp, i, i, i, i, vp]),
        "pn_cnn_backward": (i, [vp, vp, vp]),
        "pn_cnn_adam_step": (i, [vp, d, vp]),
        "pn_cnn_train_step": (i, [vp, vp, vp, i, i, i, i, d, ctypes.POINTER(d), vp]),
        "pn_cnn_features": (i, [vp, vp, d, vp, vp]),
        "pn_cnn_targets": (i, [vp, vp, vp, d, vp, vp]),
        "pn_cnn_output": (i, [vp, vp, d, vp, vp, vp]),
        "pn_cnn_precondition": (i, [vp, vp, vp, vp, vp]),
        "pn_batch_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(vp), i, i, vp]),
        "pn_batch_destroy": (i, [vp]),
        "pn_batch_last_error": (ctypes.c_char_p, [vp]),
        "pn_batch_apply": (i, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), i, vp]),
        "pn_batch_solve": (i, [vp, ctypes.POINTER(vp), ctypes.POINTER(_SolveOpts), ctypes.POINTER(_SolveStats), vp]),
        "pn_batch_set_tiling": (i, [vp, i64, i64, i, i]),
        "pn_batch_get_tiling": (i, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i),
                                    ctypes.POINTER(i)]),
        "pn_batch_tune": (i, [vp, vp]),
        "pn_tune_apply": (i, [vp, vp, ctypes.POINTER(i), ctypes.POINTER(d)]),
        "pn_set_apply_tiling": (i, [vp, i]),
        "pn_set_apply_kernel": (i, [vp, i]),
        "pn_get_apply_kernel": (i, [vp, ctypes.POINTER(i)]),
        "pn_set_l2_residency": (i, [vp, i]),
        "pn_set_stream_kernels": (i, [vp, i]),
        "pn_set_pdl": (i, [vp, i]),
        "pn_cnn_set_conv_kernel": (i, [vp, i]),
        "pn_cnn_take_error": (i, [vp]),
        "pn_fma_peak": (i, [i, ctypes.POINTER(d), vp]),
        "pn_access_probe": (i, [i, i, i, i, ctypes.POINTER(d), vp]),
        "pn_batch_set_solo": (i, [vp, ctypes.c_longlong]),
        "pn_get_apply_plan": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]),
        "pn_batch_set_op_path": (i, [vp, i]),
        "pn_batch_get_op_path": (i, [vp, ctypes.POINTER(i)]),
        "pn_batch_set_mode": (i, [vp, i, ctypes.c_longlong]),
        "pn_batch_barrier_test": (i, [i, i, ctypes.c_longlong, ctypes.POINTER(i), vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _ = i64
    _lib = lib
    return lib


@dataclass
class Layout:
    N: int
    K: int
    R: int
    pitch_x: int
    pitch_y: int
    plane_stride: int
    n_elems: int
    n_active: int
    plane_k: list
    plane_class: list
    dims: int = 3   # 2: the z-independent reduction (one z-slice per plane, l + m even)
    periodic: bool = False  # periodic test mode: R slots per axis for every class

    def plane_of_k(self, k: int) -> int:
        return self.plane_k.index(k)

    @property
    def nz_box(self) -> int:
        """z-slices of a plane box."""
        return self.R + 1 if self.dims == 3 else 1

    def active_shape(self, p: int):
        c = self.plane_class[p]
        R = self.R
        e = 0 if self.periodic else 1
        nz = R + e * ((c >> 2) & 1) if self.dims == 3 else 1
        return (nz, R + e * ((c >> 1) & 1), R + e * (c & 1))  # (z, y, x)

    def coefficient_index(self, p: int) -> int:
        """Position of plane p's coefficient in the handle's coefficient list
        (3D: k; 2D: among the l + m even coefficients in increasing k)."""
        return self.plane_k[p] if self.dims == 3 else sorted(self.plane_k).index(self.plane_k[p])


def _torch():
    import torch
    return torch


def _is_torch(a) -> bool:
    try:
        import torch
        return isinstance(a, torch.Tensor)
    except ImportError:
        return False


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float32:
        return PN_F32
    if t.dtype == torch.float64:
        return PN_F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _stream_ptr(stream):
    if stream is None:
        torch = _torch()
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def single_scatter_beam(N: int, sigma_t, albedo, g: float, axis: int, sign: int, radius: float,
                        centre=(0.5, 0.5), stream=None):
    """Voxel-centre moments (K, R, R, R) of the single-scattered light of a
    collimated beam (pn_single_scatter_beam).  sigma_t (and albedo, unless a
    scalar) are CUDA tensors of shape (R, R, R); the result has their dtype."""
    torch = _torch()
    lib = load_library()
    st = sigma_t.contiguous()
    if not (st.is_cuda and st.dim() == 3 and st.shape[0] == st.shape[1] == st.shape[2]):
        raise TypeError("sigma_t must be a cubic CUDA tensor")
    R = st.shape[0]
    K = (N + 1) ** 2
    al_p, al_c = None, 0.0
    if np.isscalar(albedo):
        al_c = float(albedo)
    else:
        al = albedo.to(st.dtype).contiguous()
        al_p = ctypes.c_void_p(al.data_ptr())
    out = torch.empty((K, R, R, R), dtype=st.dtype, device=st.device)
    rc = lib.pn_single_scatter_beam(int(N), int(R), ctypes.c_void_p(st.data_ptr()), al_p, al_c, float(g), int(axis),
                                    int(sign), float(radius), float(centre[0]), float(centre[1]),
                                    ctypes.c_void_p(out.data_ptr()), _dtype_code(st), _stream_ptr(stream))
    if rc != PN_OK:
        raise PnError(rc, "pn_single_scatter_beam failed")
    return out


def dot_noalloc(x, y, stream=None) -> float:
    """sum(x * y) over two CUDA tensors through pn_dot_noalloc, which uses a
    fixed scratch array inside the library and allocates nothing (for callers
    that cannot allocate device memory where they need the reduction)."""
    lib = load_library()
    if not (_is_torch(x) and _is_torch(y) and x.is_cuda and y.is_cuda and x.is_contiguous() and y.is_contiguous()):
        raise TypeError("expected contiguous CUDA tensors")
    if x.numel() != y.numel() or x.dtype != y.dtype:
        raise ValueError("x and y must have the same length and dtype")
    out = ctypes.c_double()
    rc = lib.pn_dot_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), x.numel(),
                            _dtype_code(x), ctypes.byref(out), _stream_ptr(stream))
    if rc != PN_OK:
        raise PnError(rc, "pn_dot_noalloc failed")
    return out.value


class System:
    """One P_N system (order N, R^3 cells, medium) living on the current GPU.

    sigma_t, albedo (array or scalar) and Q are voxel-centre fields indexed
    [z][y][x]; Q is either an (R, R, R) field of Q^{0,0} or a (K, R, R, R)
    array of centre moments.  numpy inputs are passed as host arrays (the
    library copies them); torch CUDA tensors are passed as device pointers.

    periodic=True builds the periodic test mode (every axis wraps; the exact
    closed forms of a homogeneous medium hold in it).
    dims=2 builds the z-independent 2D reduction (pn_create_2d): fields are
    (R, R) arrays [y][x], K = (N+1)(N+2)/2 coefficients with l + m even, and
    moment sources are (K, R, R) in increasing k.
    """

    def __init__(self, N: int, R: int, sigma_t, albedo, g: float, Q=None, sigma_t_min: float = 0.0,
                 stream=None, dims: int = 3, periodic: bool = False):
        if dims not in (2, 3):
            raise ValueError("dims must be 2 or 3")
        self._lib = load_library()
        self._h = ctypes.c_void_p()
        keep = []

        def arr(a):
            if a is None:
                return None, None, 0
            if _is_torch(a):
                t = a.detach().contiguous()
                if t.dtype not in (_torch().float32, _torch().float64):
                    t = t.double()
                keep.append(t)
                return ctypes.c_void_p(t.data_ptr()), _dtype_code(t), 1 if t.is_cuda else 0
            n = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
            keep.append(n)
            return ctypes.c_void_p(n.ctypes.data), PN_F64, 0

        st_p, st_dt, st_dev = arr(sigma_t)
        m = _Medium()
        m.sigma_t = st_p
        if np.isscalar(albedo):
            m.albedo = None
            m.albedo_const = float(albedo)
        else:
            al = albedo
            if _is_torch(sigma_t) and not _is_torch(al):
                al = _torch().as_tensor(np.asarray(al), dtype=keep[0].dtype, device=keep[0].device)
            if not _is_torch(sigma_t) and _is_torch(al):
                al = al.detach().cpu().double().numpy()
            if _is_torch(al):
                al = al.to(keep[0].dtype)
            al_p, _, _ = arr(al)
            m.albedo = al_p
        m.g = float(g)
        K = (N + 1) ** 2 if dims == 3 else (N + 1) * (N + 2) // 2
        cells = (R,) * dims
        if Q is not None:
            q = Q
            if _is_torch(sigma_t) and not _is_torch(q):
                q = _torch().as_tensor(np.asarray(q), dtype=keep[0].dtype, device=keep[0].device)
            if not _is_torch(sigma_t) and _is_torch(q):
                q = q.detach().cpu().double().numpy()
            if _is_torch(q):
                q = q.to(keep[0].dtype)
            shape = tuple(q.shape)
            if shape == cells:
                m.q_mode = PN_Q_CENTRE_00
            elif shape == (K,) + cells:
                m.q_mode = PN_Q_CENTRE_MOMENTS
            else:
                raise ValueError(f"Q must have shape {cells} or {(K,) + cells}, got {shape}")
            q_p, _, _ = arr(q)
            m.Q = q_p
        m.dtype = st_dt
        m.on_device = st_dev
        m.sigma_t_min = float(sigma_t_min)
        if tuple(np.shape(sigma_t)) != cells:
            raise ValueError(f"sigma_t must have shape {cells}")
        create = self._lib.pn_create if dims == 3 else self._lib.pn_create_2d
        rc = create(ctypes.byref(self._h), int(N), int(R), ctypes.byref(m),
                    PN_BC_PERIODIC_TEST if periodic else PN_BC_VACUUM,
                    _stream_ptr(stream) if (st_dev or stream is not None) else ctypes.c_void_p(0))
        if rc != PN_OK:
            raise PnError(rc, self._lib.pn_last_error(None).decode())
        lay = _Layout()
        self._check(self._lib.pn_get_layout(self._h, ctypes.byref(lay)))
        self.layout = Layout(lay.N, lay.K, lay.R, lay.pitch_x, lay.pitch_y, lay.plane_stride, lay.n_elems,
                             lay.n_active, list(lay.plane_k)[:lay.K], list(lay.plane_class)[:lay.K], dims,
                             bool(periodic))
        self.N, self.R, self.K, self.dims = N, R, K, dims

    # -- plumbing -------------------------------------------------------------
    def _check(self, rc):
        if rc != PN_OK:
            raise PnError(rc, self._lib.pn_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.pn_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _vec(self, t):
        if not _is_torch(t) or not t.is_cuda or not t.is_contiguous():
            raise TypeError("expected a contiguous CUDA tensor")
        if t.numel() != self.layout.n_elems:
            raise ValueError(f"vector has {t.numel()} elements, layout needs {self.layout.n_elems}")
        return ctypes.c_void_p(t.data_ptr()), _dtype_code(t)

    def zeros(self, dtype=None, device="cuda"):
        torch = _torch()
        return torch.zeros(self.layout.n_elems, dtype=dtype or torch.float32, device=device)

    # -- operator and vector calls ---------------------------------------------
    def apply(self, x, y, stream=None):
        """y = A x."""
        xp, dt = self._vec(x)
        yp, dt2 = self._vec(y)
        if dt != dt2:
            raise TypeError("x and y must share a dtype")
        self._check(self._lib.pn_apply(self._h, xp, yp, dt, _stream_ptr(stream)))
        return y

    def apply_t(self, x, y, stream=None):
        """y = A^T x."""
        xp, dt = self._vec(x)
        yp, dt2 = self._vec(y)
        if dt != dt2:
            raise TypeError("x and y must share a dtype")
        self._check(self._lib.pn_apply_t(self._h, xp, yp, dt, _stream_ptr(stream)))
        return y

    def residual(self, x, r, stream=None) -> float:
        """r = Q - A x; returns ||r|| / ||Q|| (FP64 accumulation)."""
        xp, dt = self._vec(x)
        rp, dt2 = self._vec(r)
        if dt != dt2:
            raise TypeError("x and r must share a dtype")
        out = ctypes.c_double()
        self._check(self._lib.pn_residual(self._h, xp, rp, ctypes.byref(out), dt, _stream_ptr(stream)))
        return out.value

    def dot(self, x, y, stream=None) -> float:
        xp, dt = self._vec(x)
        yp, _ = self._vec(y)
        out = ctypes.c_double()
        self._check(self._lib.pn_dot(self._h, xp, yp, ctypes.byref(out), dt, _stream_ptr(stream)))
        return out.value

    def axpby(self, alpha, x, beta, y, stream=None):
        xp, dt = self._vec(x)
        yp, _ = self._vec(y)
        self._check(self._lib.pn_axpby(self._h, float(alpha), xp, float(beta), yp, dt, _stream_ptr(stream)))
        return y

    def solve(self, u, solver: str = "cgls", tol: float = 1e-6, max_iter: int = 100000, restart: int = 60,
              inner_tol: float = 1e-2, max_outer: int = 50, check_every: int = 10, stream=None,
              raise_on_error: bool = True, profile: bool = False, ortho: str = "cgs2", precond=None,
              basis: str = "f32", augment: int = 0) -> dict:
        """Solve A u = Q in place (u is the initial guess).  Returns the stats.
        augment: LGMRES corrections appended per restart cycle (FP16 basis)."""
        up, dt = self._vec(u)
        o = _SolveOpts()
        self._lib.pn_default_solve_opts(ctypes.byref(o))
        o.solver = SOLVERS[solver]
        o.precision = dt
        if solver in ("ir", "ir_fgmres") and dt != PN_F64:
            raise TypeError("iterative refinement keeps u in FP64")
        if precond is not None:
            o.precond = precond._h
        o.tol, o.max_iter, o.restart = float(tol), int(max_iter), int(restart)
        o.inner_tol, o.max_outer, o.check_every = float(inner_tol), int(max_outer), int(check_every)
        o.profile = 1 if profile else 0
        o.ortho = {"cgs2": 0, "cgs1": 1}[ortho]
        o.basis = {"f32": 0, "f16": 1}[basis]
        o.augment = int(augment)
        st = _SolveStats()
        rc = self._lib.pn_solve(self._h, up, ctypes.byref(o), ctypes.byref(st), _stream_ptr(stream))
        stats = {"status": rc, "iterations": st.iterations, "outer_iterations": st.outer_iterations,
                 "rel_residual": st.rel_residual, "seconds": st.seconds, "launches": st.launches,
                 "precond_applications": st.precond_applications, "fallback": st.fallback}
        if rc != PN_OK and raise_on_error:
            raise PnError(rc, self._lib.pn_last_error(self._h).decode() + f" (stats {stats})")
        return stats

    def profile(self) -> dict:
        """Per-kernel-class totals of the last profiled solve:
        {kind: {"ms": ..., "launches": ..., "bytes": ...}}."""
        out = {}
        for i, name in enumerate(PROFILE_KINDS):
            ms, n, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
            self._check(self._lib.pn_profile_get(self._h, i, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b)))
            out[name] = {"ms": ms.value, "launches": n.value, "bytes": b.value}
        return out

    def workspace(self) -> dict:
        """Solver workspace held by the handle (pn_get_workspace): device bytes
        and the number of device allocations made for it so far."""
        b, n = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.pn_get_workspace(self._h, ctypes.byref(b), ctypes.byref(n)))
        return {"bytes": b.value, "allocations": n.value}

    def tune_apply(self, stream=None) -> dict:
        """The operator autotuner (pn_tune_apply): keeps the fastest main kernel
        and z-chunking."""
        c, ms = ctypes.c_int(), ctypes.c_double()
        self._check(self._lib.pn_tune_apply(self._h, _stream_ptr(stream), ctypes.byref(c), ctypes.byref(ms)))
        return {"ctas_per_sm": c.value, "ms": ms.value, "kernel": self.apply_kernel,
                "face_serial": self.apply_plan["face_serial"]}

    @property
    def apply_plan(self) -> dict:
        c, k, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.pn_get_apply_plan(self._h, ctypes.byref(c), ctypes.byref(k), ctypes.byref(f)))
        return {"ctas_per_sm": c.value, "kernel": {0: "register", 1: "tma"}[k.value], "face_serial": bool(f.value)}

    def set_apply_tiling(self, ctas_per_sm: int):
        self._check(self._lib.pn_set_apply_tiling(self._h, int(ctas_per_sm)))

    APPLY_KERNELS = {"register": 0, "tma": 1}

    def set_apply_kernel(self, kernel: str):
        """Main kernel of the tiled FP32 operator: "tma" or "register"."""
        self._check(self._lib.pn_set_apply_kernel(self._h, self.APPLY_KERNELS[kernel]))

    def set_stream_kernels(self, mask: int):
        """FP16-basis GMRES: bit 0 bulk-copy (TMA) staged multi-dot, bit 1 multi-axpy."""
        self._check(self._lib.pn_set_stream_kernels(self._h, int(mask)))

    def set_pdl(self, on: bool):
        """Chain the FP16-basis GMRES's Arnoldi-step kernels by programmatic
        dependent launch (default on; results unchanged)."""
        self._check(self._lib.pn_set_pdl(self._h, 1 if on else 0))

    def set_l2_residency(self, on: bool):
        """Keep the FP16-basis GMRES's two FP32 step vectors resident in L2."""
        self._check(self._lib.pn_set_l2_residency(self._h, 1 if on else 0))

    @property
    def apply_kernel(self) -> str:
        k = ctypes.c_int()
        self._check(self._lib.pn_get_apply_kernel(self._h, ctypes.byref(k)))
        return {v: n for n, v in self.APPLY_KERNELS.items()}[k.value]

    def cnn_features(self, v, scale: float = 1.0, stream=None):
        """Network input features of a padded FP32 vector: (R, R, R, K + 3)."""
        torch = _torch()
        R, K = self.layout.R, self.layout.K
        out = torch.empty((R, R, R, K + 3), dtype=torch.float32, device=v.device)
        self._check(self._lib.pn_cnn_features(self._h, ctypes.c_void_p(v.data_ptr()), float(scale),
                                              ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def cnn_targets(self, e, r, scale: float, stream=None):
        """scale * (e - P r) at the cells' own slots: (R, R, R, K); r None:
        scale * e (P = diag(1 / (D + 1/h)), the preconditioner's fixed part)."""
        torch = _torch()
        R, K = self.layout.R, self.layout.K
        out = torch.empty((R, R, R, K), dtype=torch.float32, device=e.device)
        rp = ctypes.c_void_p(r.data_ptr()) if r is not None else ctypes.c_void_p(0)
        self._check(self._lib.pn_cnn_targets(self._h, ctypes.c_void_p(e.data_ptr()), rp, float(scale),
                                             ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def cnn_output(self, net_out, scale: float, v=None, z=None, stream=None):
        """z = scale * net_out (R, R, R, K) at the cells' own slots + P v (v
        optional; net_out None: P v alone), a padded FP32 vector."""
        torch = _torch()
        if z is None:
            z = self.zeros(torch.float32)
        no = ctypes.c_void_p(net_out.data_ptr()) if net_out is not None else ctypes.c_void_p(0)
        vp_ = ctypes.c_void_p(v.data_ptr()) if v is not None else ctypes.c_void_p(0)
        self._check(self._lib.pn_cnn_output(self._h, no, float(scale), vp_, ctypes.c_void_p(z.data_ptr()),
                                            _stream_ptr(stream)))
        return z

    def precondition(self, net, v, stream=None):
        """z = M(v) with the learned network (padded FP32 vectors)."""
        z = _torch().empty_like(v)
        self._check(self._lib.pn_cnn_precondition(self._h, net._h, ctypes.c_void_p(v.data_ptr()),
                                                  ctypes.c_void_p(z.data_ptr()), _stream_ptr(stream)))
        return z

    def unstagger(self, x, stream=None):
        """Padded vector -> (K, R, R, R) tensor of voxel-centre values."""
        torch = _torch()
        xp, dt = self._vec(x)
        R = self.layout.R
        out = torch.empty((self.layout.K,) + (R,) * self.dims, dtype=x.dtype, device=x.device)
        self._check(self._lib.pn_unstagger(self._h, xp, ctypes.c_void_p(out.data_ptr()), dt, _stream_ptr(stream)))
        return out

    # -- layout marshalling -------------------------------------------------
    def to_planes(self, vec):
        """Padded vector -> list of K numpy arrays in coefficient order (3D: k;
        2D: the l + m even coefficients in increasing k), each the active
        (z, y, x) region of its staggered grid ((y, x) in 2D)."""
        lay = self.layout
        v = vec.detach().cpu().numpy() if _is_torch(vec) else np.asarray(vec)
        R, nzb = lay.R, lay.nz_box
        out = [None] * lay.K
        for p in range(lay.K):
            box = v[p * lay.plane_stride: p * lay.plane_stride + lay.pitch_y * nzb]
            box = box.reshape(nzb, R + 1, lay.pitch_x)
            nz, ny, nx = lay.active_shape(p)
            a = box[:nz, :ny, :nx].copy()
            out[lay.coefficient_index(p)] = a if lay.dims == 3 else a[0]
        return out

    def from_planes(self, planes, dtype=None, device="cuda"):
        """List of K per-coefficient arrays (order of to_planes) -> padded vector."""
        torch = _torch()
        lay = self.layout
        R, nzb = lay.R, lay.nz_box
        host = np.zeros(lay.n_elems, dtype=np.float64)
        for p in range(lay.K):
            nz, ny, nx = lay.active_shape(p)
            box = host[p * lay.plane_stride: p * lay.plane_stride + lay.pitch_y * nzb].reshape(nzb, R + 1, lay.pitch_x)
            box[:nz, :ny, :nx] = np.asarray(planes[lay.coefficient_index(p)], dtype=np.float64).reshape(nz, ny, nx)
        return torch.as_tensor(host, dtype=dtype or torch.float32).to(device)


class Batch:
    """Many systems solved together (pn_batch_*): one launch per phase over
    every instance, the restart cycle replayed as a CUDA graph.  The systems
    are borrowed and must stay open while the batch lives."""

    def __init__(self, systems, restart: int = 15, tune: bool = False, stream=None):
        self._lib = load_library()
        self.systems = list(systems)
        self._h = ctypes.c_void_p()
        n = len(self.systems)
        hs = (ctypes.c_void_p * n)(*[s_._h.value for s_ in self.systems])
        rc = self._lib.pn_batch_create(ctypes.byref(self._h), hs, n, int(restart), _stream_ptr(stream))
        if rc != PN_OK:
            raise PnError(rc, "pn_batch_create failed")
        self.restart = int(restart)
        if tune:
            self.tune(stream)

    def _check(self, rc):
        if rc != PN_OK:
            raise PnError(rc, self._lib.pn_batch_last_error(self._h).decode())

    def close(self):
        if self._h:
            self._lib.pn_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tune(self, stream=None) -> dict:
        self._check(self._lib.pn_batch_tune(self._h, _stream_ptr(stream)))
        return self.tiling()

    def tiling(self) -> dict:
        oc, vc = ctypes.c_int64(), ctypes.c_int64()
        om, vm = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.pn_batch_get_tiling(self._h, ctypes.byref(oc), ctypes.byref(vc), ctypes.byref(om),
                                                  ctypes.byref(vm)))
        t = ctypes.c_int()
        self._check(self._lib.pn_batch_get_op_path(self._h, ctypes.byref(t)))
        return {"op_chunk": oc.value, "vec_chunk": vc.value, "op_ctas_per_sm": om.value, "vec_ctas_per_sm": vm.value,
                "tiled_operator": bool(t.value)}

    def set_op_path(self, tiled: bool):
        self._check(self._lib.pn_batch_set_op_path(self._h, 1 if tiled else 0))

    def set_solo(self, min_unknowns: int):
        """Instances with at least min_unknowns unknowns are solved by pn_solve,
        three at a time on three streams, inside solve(); <= 0: every instance batched.  tune()
        chooses the tiling for the batched instances under this threshold:
        call it again after changing the threshold."""
        self._check(self._lib.pn_batch_set_solo(self._h, int(min_unknowns)))

    def set_mode(self, persistent: bool, spin_limit: int = 1 << 24):
        """persistent=True: one cooperative launch per restart cycle with
        bounded grid barriers; False: the captured CUDA graph (default)."""
        self._check(self._lib.pn_batch_set_mode(self._h, 1 if persistent else 0, int(spin_limit)))

    def set_tiling(self, op_chunk: int, vec_chunk: int, op_ctas_per_sm: int, vec_ctas_per_sm: int):
        self._check(self._lib.pn_batch_set_tiling(self._h, int(op_chunk), int(vec_chunk), int(op_ctas_per_sm),
                                                  int(vec_ctas_per_sm)))

    def apply(self, xs, ys, stream=None):
        """y_i = A_i x_i for every instance, one launch (FP32 or FP64)."""
        n = len(self.systems)
        dt = _dtype_code(xs[0])
        xa = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        ya = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
        self._check(self._lib.pn_batch_apply(self._h, xa, ya, dt, _stream_ptr(stream)))

    def solve(self, us, tol: float = 1e-6, max_iter: int = 100000, inner_tol: float = 1e-2, max_outer: int = 50,
              stream=None, raise_on_error: bool = True):
        """Solve every A_i u_i = Q_i in place (FP64 u_i, initial guesses).
        Returns one stats dict per instance."""
        torch = _torch()
        n = len(self.systems)
        for u in us:
            if u.dtype != torch.float64 or not u.is_cuda:
                raise TypeError("batched refinement keeps every u in FP64 on the GPU")
        o = _SolveOpts()
        self._lib.pn_default_solve_opts(ctypes.byref(o))
        o.solver = SOLVERS["ir"]
        o.precision = PN_F64
        o.tol, o.max_iter, o.restart = float(tol), int(max_iter), self.restart
        o.inner_tol, o.max_outer = float(inner_tol), int(max_outer)
        st = (_SolveStats * n)()
        ua = (ctypes.c_void_p * n)(*[u.data_ptr() for u in us])
        rc = self._lib.pn_batch_solve(self._h, ua, ctypes.byref(o), st, _stream_ptr(stream))
        out = [{"status": st[i].status, "iterations": st[i].iterations, "outer_iterations": st[i].outer_iterations,
                "rel_residual": st[i].rel_residual, "seconds": st[i].seconds, "launches": st[i].launches}
               for i in range(n)]
        if rc != PN_OK and raise_on_error:
            raise PnError(rc, self._lib.pn_batch_last_error(self._h).decode() + f" (stats {out})")
        return out


def wait_timeout_test(system=None, deliver: bool = False, limit_ns: int = 2_000_000, stream=None):
    """pn_wait_timeout_test: arm one mbarrier and wait on it with a limit of
    limit_ns (deliver = False: a phase that never completes).  Returns
    (return code, timed_out)."""
    lib = load_library()
    t = ctypes.c_int(-1)
    h = system._h if system is not None else None
    rc = lib.pn_wait_timeout_test(h, 1 if deliver else 0, int(limit_ns), ctypes.byref(t), _stream_ptr(stream))
    return rc, t.value


def fma_peak(dtype="f64", stream=None) -> float:
    """pn_fma_peak: measured FMA throughput of the GPU in GFLOP/s."""
    lib = load_library()
    out = ctypes.c_double()
    rc = lib.pn_fma_peak(PN_F64 if dtype == "f64" else PN_F32, ctypes.byref(out), _stream_ptr(stream))
    if rc != PN_OK:
        raise PnError(rc, "pn_fma_peak failed")
    return out.value


def access_probe(R: int, planes: int, tile_x: int, slices: int, stream=None) -> float:
    """pn_access_probe: GB/s of a copy with the tiled operator's access pattern
    (tile_x x 128/tile_x column tiles marching in z over `planes` planes,
    `slices` z-slices of loads in flight per thread)."""
    lib = load_library()
    out = ctypes.c_double()
    rc = lib.pn_access_probe(int(R), int(planes), int(tile_x), int(slices), ctypes.byref(out), _stream_ptr(stream))
    if rc != PN_OK:
        raise PnError(rc, "pn_access_probe failed")
    return out.value


def barrier_test(blocks: int, expected: int, spin_limit: int, stream=None):
    """(return code, timed_out) of pn_batch_barrier_test."""
    lib = load_library()
    t = ctypes.c_int(-1)
    rc = lib.pn_batch_barrier_test(int(blocks), int(expected), int(spin_limit), ctypes.byref(t), _stream_ptr(stream))
    return rc, t.value


class Net:
    """The learned preconditioner's 3D convolutional encoder-decoder
    (pn_cnn_*): BF16 tensor-core forward and backward kernels with FP32
    accumulation, FP32 master weights trained by Adam on the GPU.  Tensors
    are float32 CUDA tensors shaped (B, Z, Y, X, C)."""

    def __init__(self, c_in: int, c_out: int, widths=(16, 32, 48, 64)):
        self._lib = load_library()
        self._h = ctypes.c_void_p()
        w = (ctypes.c_int * 4)(*[int(v) for v in widths])
        rc = self._lib.pn_cnn_create(ctypes.byref(self._h), int(c_in), int(c_out), ctypes.byref(w))
        if rc != PN_OK:
            raise PnError(rc, "pn_cnn_create failed")
        self.c_in, self.c_out, self.widths = c_in, c_out, tuple(widths)
        self.n_params = int(self._lib.pn_cnn_num_params(self._h))

    def _check(self, rc):
        if rc != PN_OK:
            raise PnError(rc, self._lib.pn_cnn_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.pn_cnn_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        a = np.ascontiguousarray(np.asarray(flat, dtype=np.float32))
        self._check(self._lib.pn_cnn_set_params(self._h, ctypes.c_void_p(a.ctypes.data), a.size))

    def get_params(self) -> np.ndarray:
        a = np.empty(self.n_params, dtype=np.float32)
        self._check(self._lib.pn_cnn_get_params(self._h, ctypes.c_void_p(a.ctypes.data), a.size))
        return a

    def get_grads(self) -> np.ndarray:
        a = np.empty(self.n_params, dtype=np.float32)
        self._check(self._lib.pn_cnn_get_grads(self._h, ctypes.c_void_p(a.ctypes.data), a.size))
        return a

    CONV_KERNELS = {"mma_sync": 0, "tcgen05": 1}

    def set_conv_kernel(self, kernel: str):
        """Kernel of the 3x3x3 convolutions: "tcgen05" (default) or "mma_sync"."""
        self._check(self._lib.pn_cnn_set_conv_kernel(self._h, self.CONV_KERNELS[kernel]))

    def take_error(self):
        """Raise if a bounded wait of a tcgen05 convolution ran out (clears it)."""
        self._check(self._lib.pn_cnn_take_error(self._h))

    def forward(self, x, stream=None):
        torch = _torch()
        B, Z, Y, X, C = x.shape
        assert C == self.c_in and x.dtype == torch.float32 and x.is_cuda
        x = x.contiguous()
        out = torch.empty((B, Z, Y, X, self.c_out), dtype=torch.float32, device=x.device)
        self._check(self._lib.pn_cnn_forward(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                             B, Z, Y, X, _stream_ptr(stream)))
        return out

    def backward(self, grad_out, stream=None):
        g = grad_out.contiguous()
        self._check(self._lib.pn_cnn_backward(self._h, ctypes.c_void_p(g.data_ptr()), _stream_ptr(stream)))

    def adam_step(self, lr: float, stream=None):
        self._check(self._lib.pn_cnn_adam_step(self._h, float(lr), _stream_ptr(stream)))

    def train_step(self, x, target, lr: float, stream=None) -> float:
        B, Z, Y, X, C = x.shape
        x, t = x.contiguous(), target.contiguous()
        loss = ctypes.c_double()
        self._check(self._lib.pn_cnn_train_step(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                                B, Z, Y, X, float(lr), ctypes.byref(loss), _stream_ptr(stream)))
        return loss.value


def flatten_cnn_params(params: dict, layer_names) -> np.ndarray:
    """{name: (W[o][c][27], b[o])} -> the host parameter order of pn_cnn."""
    parts = []
    for name in layer_names:
        W, b = params[name]
        parts += [np.asarray(W, dtype=np.float64).ravel(), np.asarray(b, dtype=np.float64).ravel()]
    return np.concatenate(parts)


CNN_LAYERS = ["e0a", "e0b", "e1a", "e1b", "e2a", "e2b", "e3a", "e3b", "d2", "d1", "d0", "out"]
