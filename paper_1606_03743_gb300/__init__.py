"""GB300 (sm_103a) library for the potential phi and field E of charged BEM
triangles and rectangles by Gaussian cubature (arXiv:1606.03743).

This module is the thin Python binding of the C ABI in include/bem.h: the
``bem_*`` functions below marshal arguments to the same-named C entry points
(every step of the computation runs in the library's CUDA kernels), and
``Mesh`` wraps a ``bem_mesh*`` handle.  Arrays may be numpy arrays (host) or
torch tensors (CPU or CUDA); results come back as the same kind.  PyTorch is
only used for device memory and the current CUDA stream.

There is no CPU fallback: if libbem.so is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = ["Mesh", "BemError", "load_library", "bem_create", "bem_destroy", "bem_eval", "bem_assemble",
           "bem_matvec", "bem_set_sigma", "bem_centroids", "bem_rule", "bem_num_elements", "bem_last_error",
           "bem_version", "bem_set_stats", "bem_last_stats", "bem_set_timing", "bem_last_times",
           "bem_kernel_launches", "bem_eval_noalloc", "bem_solve", "bem_eval_grad", "bem_set_sigma_linear", "bem_set_sigma_quadratic", "linear_coef_from_corner_values", "bem_peak_rate", "bem_default_limits", "PEAK_FFMA", "PEAK_FFMA2", "PEAK_RSQRT", "PEAK_DFMA", "SOLVE_X0", "SOLVE_REFINE", "FLAG_NODE_TABLE", "NOALLOC_MAX_POINTS", "NOALLOC_MAX_NEAR", "Server", "FP64", "MIXED", "TRIANGLE", "RECTANGLE"]

FP64, MIXED = 0, 1
TRIANGLE, RECTANGLE = 0, 1
STATUS = {0: "BEM_OK", -1: "BEM_ERR_INVALID", -2: "BEM_ERR_OOM", -3: "BEM_ERR_CAPACITY", -4: "BEM_ERR_CUDA",
          -5: "BEM_ERR_TIMEOUT", -6: "BEM_ERR_NOT_FOUND", -7: "BEM_ERR_NOT_CONVERGED"}
SOLVE_X0, SOLVE_REFINE = 1, 2
FLAG_NODE_TABLE = 1


class BemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class bem_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("flags", C.c_int32), ("limits", C.POINTER(C.c_double)),
                ("eps0", C.c_double), ("device_mem_budget", C.c_size_t)]


class bem_solve_options(C.Structure):
    _fields_ = [("restart", C.c_int32), ("max_iter", C.c_int32), ("tol", C.c_double), ("flags", C.c_int32)]


class bem_server_options(C.Structure):
    _fields_ = [("max_points_per_tick", C.c_int64), ("max_near_pairs_per_tick", C.c_int64),
                ("device_mem_budget", C.c_size_t), ("flags", C.c_int32)]


_lib = None


def load_library(build_if_missing: bool = True):
    """Load the in-tree libbem.so (building it first if needed).  With
    BEM_CHECKED=1 in the environment, the checked build (bounds-checked
    kernels, see build.py) is loaded instead."""
    global _lib
    if _lib is not None:
        return _lib
    checked = os.environ.get("BEM_CHECKED", "0") == "1"
    path = _build.lib_path(checked)
    if not os.path.exists(path) or _build._stale(checked):
        if not build_if_missing:
            raise ImportError(f"libbem.so not built: {path}")
        _build.build(checked=checked)
    lib = C.CDLL(path)
    vp, d, i32, i64 = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
    lib.bem_create.argtypes = [vp, vp, vp, C.c_int64, C.POINTER(bem_options), vp, C.POINTER(vp)]
    lib.bem_destroy.argtypes = [vp]
    lib.bem_destroy.restype = None
    lib.bem_num_elements.argtypes = [vp]
    lib.bem_num_elements.restype = C.c_int64
    lib.bem_set_sigma.argtypes = [vp, vp, vp]
    lib.bem_eval.argtypes = [vp, vp, C.c_int64, vp, vp, vp]
    lib.bem_assemble.argtypes = [vp, vp, C.c_int64, vp, vp]
    lib.bem_matvec.argtypes = [vp, vp, vp, vp]
    lib.bem_centroids.argtypes = [vp, vp, vp]
    lib.bem_rule.argtypes = [C.c_int32, C.c_int32, d]
    lib.bem_last_stats.argtypes = [vp, i64]
    lib.bem_set_stats.argtypes = [vp, C.c_int32]
    lib.bem_set_timing.argtypes = [vp, C.c_int32]
    lib.bem_last_times.argtypes = [vp, d]
    lib.bem_kernel_launches.restype = C.c_int64
    lib.bem_eval_noalloc.argtypes = [vp, vp, C.c_int64, vp, vp, vp]
    lib.bem_eval_noalloc.restype = C.c_int
    lib.bem_server_create.argtypes = [vp, C.POINTER(bem_server_options), C.POINTER(vp)]
    lib.bem_server_destroy.argtypes = [vp]
    lib.bem_server_destroy.restype = None
    lib.bem_submit.argtypes = [vp, vp, C.c_int64, C.POINTER(C.c_uint64)]
    lib.bem_poll.argtypes = [vp, C.c_uint64, vp, vp, C.POINTER(C.c_int32)]
    lib.bem_wait.argtypes = [vp, C.c_uint64, C.c_double, vp, vp]
    lib.bem_cancel.argtypes = [vp, C.c_uint64]
    lib.bem_server_pause.argtypes = [vp, C.c_int32]
    lib.bem_server_stats.argtypes = [vp, C.c_int32, d]
    lib.bem_server_latencies.argtypes = [vp, C.c_int64, d, i64, i64]
    lib.bem_set_sigma_linear.argtypes = [vp, vp, vp]
    lib.bem_set_sigma_linear.restype = C.c_int
    lib.bem_set_sigma_quadratic.argtypes = [vp, vp, vp]
    lib.bem_set_sigma_quadratic.restype = C.c_int
    lib.bem_eval_grad.argtypes = [vp, vp, C.c_int64, vp, vp]
    lib.bem_eval_grad.restype = C.c_int
    lib.bem_solve.argtypes = [vp, vp, vp, C.POINTER(bem_solve_options), d, vp]
    lib.bem_solve.restype = C.c_int
    lib.bem_linear_coef_from_corners.argtypes = [vp, vp, C.c_int64, vp]
    lib.bem_linear_coef_from_corners.restype = C.c_int
    lib.bem_default_limits.argtypes = [d]
    lib.bem_default_limits.restype = C.c_int
    lib.bem_peak_rate.argtypes = [C.c_int32, d]
    lib.bem_peak_rate.restype = C.c_int
    for name in ("bem_server_create", "bem_submit", "bem_poll", "bem_wait", "bem_cancel", "bem_server_pause",
                 "bem_server_stats", "bem_server_latencies"):
        getattr(lib, name).restype = C.c_int
    lib.bem_last_error.restype = C.c_char_p
    lib.bem_version.restype = C.c_char_p
    for name in ("bem_create", "bem_set_sigma", "bem_eval", "bem_assemble", "bem_matvec", "bem_centroids",
                 "bem_rule", "bem_last_stats", "bem_set_stats", "bem_set_timing", "bem_last_times"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(rc: int) -> int:
    if rc < 0:
        raise BemError(rc, bem_last_error())
    return rc


# ---------------------------------------------------------------- array marshalling
def _torch():
    try:
        import torch
        return torch
    except ImportError:  # pragma: no cover
        return None


def _is_torch(x) -> bool:
    t = _torch()
    return t is not None and isinstance(x, t.Tensor)


def _stream(stream=None) -> int:
    if stream is not None:
        return int(stream)
    t = _torch()
    if t is not None and t.cuda.is_available() and t.cuda.is_initialized():
        return int(t.cuda.current_stream().cuda_stream)
    return 0


def _prep(x, dtype, shape=None):
    """Contiguous array of the given dtype; returns (object keeping it alive, pointer)."""
    if _is_torch(x):
        t = _torch()
        tdt = {np.float64: t.float64, np.int32: t.int32}[dtype]
        x = x.to(tdt).contiguous()
        if shape is not None:
            x = x.reshape(shape)
        return x, x.data_ptr()
    a = np.ascontiguousarray(np.asarray(x, dtype=dtype))
    if shape is not None:
        a = a.reshape(shape)
    return a, a.ctypes.data


def _empty_like_kind(ref, shape):
    if _is_torch(ref):
        t = _torch()
        return t.empty(shape, dtype=t.float64, device=ref.device)
    return np.empty(shape, dtype=np.float64)


def _ptr(x) -> int:
    return x.data_ptr() if _is_torch(x) else x.ctypes.data


# ---------------------------------------------------------------- C-ABI mirrors
def bem_version() -> str:
    return load_library().bem_version().decode()


def bem_last_error() -> str:
    return load_library().bem_last_error().decode()


def bem_rule(type_: int, r: int) -> np.ndarray:
    """Expanded nodes (alpha, beta, w) of rule r (0..4) of an element type."""
    out = np.zeros((33, 3))
    n = _check(load_library().bem_rule(type_, r, out.ctypes.data_as(C.POINTER(C.c_double))))
    return out[:n].copy()


def bem_default_limits() -> np.ndarray:
    """(2, 5) default DR band limits (triangles, rectangles) of bem_create."""
    out = np.zeros(10)
    _check(load_library().bem_default_limits(out.ctypes.data_as(C.POINTER(C.c_double))))
    return out.reshape(2, 5)


def bem_create(types, verts, sigma, precision: int = FP64, limits=None, eps0: float = 0.0,
               device_mem_budget: int = 0, stream=None, flags: int = 0) -> int:
    lib = load_library()
    t, tp = _prep(types, np.int32)
    n = int(t.shape[0])
    v, vp_ = _prep(verts, np.float64, (n, 4, 3))
    s, sp = _prep(sigma, np.float64, (n,))
    opt = bem_options()
    opt.precision = int(precision)
    opt.flags = int(flags)
    lim_keep = None
    if limits is not None:
        lim_keep = np.ascontiguousarray(np.asarray(limits, np.float64).reshape(10))
        opt.limits = lim_keep.ctypes.data_as(C.POINTER(C.c_double))
    opt.eps0 = float(eps0)
    opt.device_mem_budget = int(device_mem_budget)
    h = C.c_void_p()
    _check(lib.bem_create(tp, vp_, sp, n, C.byref(opt), _stream(stream), C.byref(h)))
    return h.value


def bem_destroy(mesh: int) -> None:
    load_library().bem_destroy(mesh)


def bem_num_elements(mesh: int) -> int:
    return int(load_library().bem_num_elements(mesh))


def bem_set_sigma(mesh: int, sigma, stream=None) -> None:
    s, sp = _prep(sigma, np.float64, (bem_num_elements(mesh),))
    _check(load_library().bem_set_sigma(mesh, sp, _stream(stream)))


def _check_out(name: str, x, n: int, per: int) -> None:
    """An output array the library writes n * per doubles into: float64,
    contiguous and large enough (a short array would get writes past its end)."""
    if x is None:
        return
    if _is_torch(x):
        t = _torch()
        ok_type, ok_contig, size = x.dtype == t.float64, x.is_contiguous(), x.numel()
    else:
        ok_type, ok_contig, size = x.dtype == np.float64, x.flags["C_CONTIGUOUS"], x.size
    if not ok_type or not ok_contig:
        raise ValueError(f"{name} must be a contiguous float64 array")
    if size < n * per:
        raise ValueError(f"{name} holds {size} doubles; {n * per} are written")


def bem_eval(mesh: int, points, phi=None, E=None, stream=None) -> None:
    p, pp = _prep(points, np.float64)
    n = p.numel() // 3 if _is_torch(p) else p.size // 3
    _check_out("phi", phi, n, 1)
    _check_out("E", E, n, 3)
    _check(load_library().bem_eval(mesh, pp, n, _ptr(phi) if phi is not None else None,
                                   _ptr(E) if E is not None else None, _stream(stream)))


# limits of bem_eval_noalloc (include/bem.h)
NOALLOC_MAX_POINTS = 16384
NOALLOC_MAX_NEAR = 262144


def bem_eval_noalloc(mesh: int, points, phi=None, E=None, stream=None) -> None:
    """bem_eval with all scratch in a fixed device array (no allocation);
    points, phi and E must be CUDA tensors, at most NOALLOC_MAX_POINTS points."""
    p, pp = _prep(points, np.float64)
    n = p.numel() // 3 if _is_torch(p) else p.size // 3
    _check_out("phi", phi, n, 1)
    _check_out("E", E, n, 3)
    _check(load_library().bem_eval_noalloc(mesh, pp, n, _ptr(phi) if phi is not None else None,
                                           _ptr(E) if E is not None else None, _stream(stream)))


def bem_assemble(mesh: int, colloc, A, stream=None) -> None:
    p, pp = _prep(colloc, np.float64)
    m = p.numel() // 3 if _is_torch(p) else p.size // 3
    _check_out("A", A, m, bem_num_elements(mesh))
    _check(load_library().bem_assemble(mesh, pp, m, _ptr(A), _stream(stream)))


def bem_matvec(mesh: int, x, y, stream=None) -> None:
    xx, xp = _prep(x, np.float64, (bem_num_elements(mesh),))
    _check_out("y", y, bem_num_elements(mesh), 1)
    _check(load_library().bem_matvec(mesh, xp, _ptr(y), _stream(stream)))


def bem_set_sigma_linear(mesh: int, coef, stream=None) -> None:
    """Linear densities: coef (n_el, 3) = (sigma at the centroid, d sigma / d alpha, d sigma / d beta)."""
    cc, cp = _prep(coef, np.float64, (bem_num_elements(mesh), 3))
    _check(load_library().bem_set_sigma_linear(mesh, cp, _stream(stream)))


def bem_set_sigma_quadratic(mesh: int, coef, stream=None) -> None:
    """Quadratic densities: coef (n_el, 6), sigma = c0 + c1 alpha + c2 beta + c3 alpha^2
    + c4 alpha beta + c5 beta^2 in the element's frame coordinates."""
    cc, cp = _prep(coef, np.float64, (bem_num_elements(mesh), 6))
    _check(load_library().bem_set_sigma_quadratic(mesh, cp, _stream(stream)))


def linear_coef_from_corner_values(types, values):
    """(n, 3) coefficients of bem_set_sigma_linear from density values at the
    corners (n, 3 or 4): bem_linear_coef_from_corners (host arrays; a
    triangle's fourth value is ignored)."""
    t = np.ascontiguousarray(np.asarray(types), dtype=np.int32)
    n = int(t.shape[0])
    v = np.asarray(values, np.float64).reshape(n, -1)
    v4 = np.zeros((n, 4))
    v4[:, : v.shape[1]] = v
    out = np.zeros((n, 3))
    _check(load_library().bem_linear_coef_from_corners(t.ctypes.data, v4.ctypes.data, n, out.ctypes.data))
    return out


# arithmetic pipes of bem_peak_rate
PEAK_FFMA, PEAK_FFMA2, PEAK_RSQRT, PEAK_DFMA = 0, 1, 2, 3


def bem_peak_rate(kind: int) -> dict:
    """Measured throughput of one arithmetic pipe of the current device:
    {ops_per_s (lane operations, an FMA counts once), ms, sm_mhz}."""
    out = np.zeros(3)
    _check(load_library().bem_peak_rate(int(kind), out.ctypes.data_as(C.POINTER(C.c_double))))
    return {"ops_per_s": float(out[0]), "ms": float(out[1]), "sm_mhz": float(out[2])}


def bem_eval_grad(mesh: int, points, G, stream=None) -> None:
    """Field gradient (n, 6) = (dEx/dx, dEy/dy, dEz/dz, dEx/dy, dEx/dz, dEy/dz) at the points."""
    pp, ptr = _prep(points, np.float64)
    n = (pp.numel() if _is_torch(pp) else pp.size) // 3
    _check_out("G", G, n, 6)
    _check(load_library().bem_eval_grad(mesh, ptr, n, _ptr(G), _stream(stream)))


def bem_solve(mesh: int, rhs, sigma, restart: int = 0, max_iter: int = 0, tol: float = 0.0, x0: bool = False,
              refine: bool = False, stream=None) -> dict:
    """Charge densities sigma with A sigma = rhs at the centroids (restarted,
    Jacobi-preconditioned GMRES on bem_matvec; refine: mixed-precision inner
    solves with FP64 residuals on an FP64 mesh).  sigma is written in place
    (and read as the initial guess when x0).  Returns {products, residual,
    converged}; raises BemError (BEM_ERR_NOT_CONVERGED included) on failure."""
    n = bem_num_elements(mesh)
    rr, rp = _prep(rhs, np.float64, (n,))
    opt = bem_solve_options(restart, max_iter, tol, (SOLVE_X0 if x0 else 0) | (SOLVE_REFINE if refine else 0))
    info = np.zeros(3)
    rc = load_library().bem_solve(mesh, rp, _ptr(sigma), C.byref(opt), info.ctypes.data_as(C.POINTER(C.c_double)),
                                  _stream(stream))
    out = {"products": int(info[0]), "residual": float(info[1]), "converged": bool(info[2])}
    if rc < 0:
        err = BemError(rc, bem_last_error())
        err.info = out
        raise err
    return out


def bem_centroids(mesh: int, out, stream=None) -> None:
    _check(load_library().bem_centroids(mesh, _ptr(out), _stream(stream)))


def bem_set_stats(mesh: int, enable: bool) -> None:
    _check(load_library().bem_set_stats(mesh, 1 if enable else 0))


def bem_set_timing(mesh: int, enable: bool) -> None:
    _check(load_library().bem_set_timing(mesh, 1 if enable else 0))


def bem_last_times(mesh: int) -> np.ndarray:
    """(sort, far, near, finalise) milliseconds of the last call with timing on."""
    out = np.zeros(4)
    _check(load_library().bem_last_times(mesh, out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def bem_kernel_launches() -> int:
    return int(load_library().bem_kernel_launches())


def bem_last_stats(mesh: int) -> np.ndarray:
    out = np.zeros(16, np.int64)
    _check(load_library().bem_last_stats(mesh, out.ctypes.data_as(C.POINTER(C.c_int64))))
    return out


# ---------------------------------------------------------------- object API
class Mesh:
    """A device-resident mesh of constant-density triangles and rectangles.

    types (n,) int32, verts (n, 4, 3) float64, sigma (n,) float64 -- numpy
    arrays or torch tensors; precision FP64 or MIXED (see include/bem.h)."""

    def __init__(self, types, verts, sigma, precision: int = FP64, limits=None, eps0: float = 0.0,
                 device_mem_budget: int = 0, stream=None, node_table: bool = False):
        self._h = bem_create(types, verts, sigma, precision, limits, eps0, device_mem_budget, stream,
                             FLAG_NODE_TABLE if node_table else 0)
        self.n = bem_num_elements(self._h)
        self.precision = precision

    @property
    def handle(self) -> int:
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            bem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def eval(self, points, want_phi: bool = True, want_E: bool = True, stream=None):
        """(phi (n,), E (n, 3)) at the field points (same array kind as points)."""
        n = (points.numel() if _is_torch(points) else np.asarray(points).size) // 3
        phi = _empty_like_kind(points, (n,)) if want_phi else None
        E = _empty_like_kind(points, (n, 3)) if want_E else None
        bem_eval(self._h, points, phi, E, stream)
        return phi, E

    def eval_grad(self, points, stream=None):
        """Field gradient (n, 6) at the points (bem_eval_grad), same array kind as points."""
        n = (points.numel() if _is_torch(points) else np.asarray(points).size) // 3
        G = _empty_like_kind(points, (n, 6))
        bem_eval_grad(self._h, points, G, stream)
        return G

    def assemble(self, colloc, stream=None):
        m = (colloc.numel() if _is_torch(colloc) else np.asarray(colloc).size) // 3
        A = _empty_like_kind(colloc, (m, self.n))
        bem_assemble(self._h, colloc, A, stream)
        return A

    def matvec(self, x, stream=None):
        y = _empty_like_kind(x, (self.n,))
        bem_matvec(self._h, x, y, stream)
        return y

    def set_sigma(self, sigma, stream=None):
        bem_set_sigma(self._h, sigma, stream)

    def set_sigma_linear(self, coef, stream=None):
        bem_set_sigma_linear(self._h, coef, stream)

    def set_sigma_quadratic(self, coef, stream=None):
        bem_set_sigma_quadratic(self._h, coef, stream)

    def solve(self, rhs, x0=None, restart: int = 0, max_iter: int = 0, tol: float = 0.0, refine: bool = False,
              stream=None):
        """(sigma, info) with A sigma = rhs at the centroids (bem_solve); sigma
        is the same array kind as rhs."""
        sigma = _empty_like_kind(rhs, (self.n,))
        if x0 is not None:
            sigma[:] = x0
        info = bem_solve(self._h, rhs, sigma, restart, max_iter, tol, x0 is not None, refine, stream)
        return sigma, info

    def centroids(self, like=None, stream=None):
        out = _empty_like_kind(like if like is not None else np.zeros(0), (self.n, 3))
        bem_centroids(self._h, out, stream)
        return out

    def set_stats(self, enable: bool):
        bem_set_stats(self._h, enable)

    def last_stats(self) -> np.ndarray:
        return bem_last_stats(self._h)

    def set_timing(self, enable: bool):
        bem_set_timing(self._h, enable)

    def last_times(self) -> np.ndarray:
        return bem_last_times(self._h)


# ---------------------------------------------------------------- serving
SERVER_STAT_NAMES = ("completed", "p50_ms", "p99_ms", "mean_ms", "ticks", "points", "fallback_ticks",
                     "points_per_tick", "device_bytes", "graph_launches")


class Server:
    """Continuous-batching server of field-point queries on a mesh (see
    bem_server_* in include/bem.h).  Requests are host arrays of points;
    results come back as numpy arrays.  While the server lives it owns the
    mesh."""

    def __init__(self, mesh: "Mesh", max_points_per_tick: int = 0, max_near_pairs_per_tick: int = 0,
                 device_mem_budget: int = 0):
        lib = load_library()
        opt = bem_server_options(int(max_points_per_tick), int(max_near_pairs_per_tick), int(device_mem_budget), 0)
        h = C.c_void_p()
        _check(lib.bem_server_create(mesh.handle, C.byref(opt), C.byref(h)))
        self._h = h.value
        self._mesh = mesh  # keep the mesh alive
        self._sizes = {}

    def close(self):
        if getattr(self, "_h", None):
            load_library().bem_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, points) -> int:
        p = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 3))
        t = C.c_uint64()
        _check(load_library().bem_submit(self._h, p.ctypes.data, p.shape[0], C.byref(t)))
        self._sizes[t.value] = p.shape[0]
        return t.value

    def poll(self, ticket: int):
        """(done, phi, E): phi and E are None until the request has finished."""
        n = self._sizes.get(ticket, 0)  # unknown tickets: the library reports BEM_ERR_NOT_FOUND
        phi, E = np.empty(n), np.empty((n, 3))
        done = C.c_int32()
        _check(load_library().bem_poll(self._h, ticket, phi.ctypes.data, E.ctypes.data, C.byref(done)))
        if not done.value:
            return False, None, None
        self._sizes.pop(ticket, None)
        return True, phi, E

    def wait(self, ticket: int, timeout: float = 60.0):
        n = self._sizes.get(ticket, 0)
        phi, E = np.empty(n), np.empty((n, 3))
        _check(load_library().bem_wait(self._h, ticket, float(timeout), phi.ctypes.data, E.ctypes.data))
        self._sizes.pop(ticket, None)
        return phi, E

    def cancel(self, ticket: int):
        _check(load_library().bem_cancel(self._h, ticket))
        self._sizes.pop(ticket, None)

    def pause(self, paused: bool = True):
        _check(load_library().bem_server_pause(self._h, 1 if paused else 0))

    def stats(self, reset: bool = False) -> dict:
        out = np.zeros(10)
        _check(load_library().bem_server_stats(self._h, 1 if reset else 0,
                                               out.ctypes.data_as(C.POINTER(C.c_double))))
        return dict(zip(SERVER_STAT_NAMES, out.tolist()))

    def latencies(self):
        """(ms, points) of every request completed since creation or the last
        stats reset: latency from submission to results on the host, and size."""
        lib = load_library()
        count = C.c_int64()
        _check(lib.bem_server_latencies(self._h, 0, None, None, C.byref(count)))
        n = count.value
        ms, pts = np.zeros(n), np.zeros(n, np.int64)
        _check(lib.bem_server_latencies(self._h, n, ms.ctypes.data_as(C.POINTER(C.c_double)),
                                        pts.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(count)))
        k = min(n, count.value)
        return ms[:k], pts[:k]
