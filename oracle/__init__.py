"""FP64 CPU oracle for phi and E of charged BEM triangles and rectangles.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, the smoke check in
``__graft_entry__`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may import this package.  It shares no code with the CUDA
library; see ``oracle.c`` for the formulas and their citations.

This module is a thin ctypes wrapper around ``oracle.c`` (built with gcc on
first use, or by ``build()``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

METHOD_PAPER = 0
METHOD_GL2 = 1
METHOD_ANALYTIC = 2
METHOD_RULE = 3
METHOD_SUBDIV = 4

RULE_SIZES = {0: (4, 7, 12, 19, 33), 1: (4, 7, 12, 17, 33)}


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (no -march flags and no FMA
    contraction, so x86 and Arm hosts produce the same arithmetic)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = C.CDLL(_LIB)
        d, i32, i64 = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
        lib.oracle_rule.argtypes = [C.c_int, C.c_int, d]
        lib.oracle_rule.restype = C.c_int
        lib.oracle_gauss_legendre.argtypes = [C.c_int, d, d]
        lib.oracle_default_limits.argtypes = [d]
        lib.oracle_element_geometry.argtypes = [C.c_int, d, d]
        lib.oracle_element.argtypes = [C.c_int, d, d, C.c_int, C.c_int, d, d, C.POINTER(C.c_int)]
        lib.oracle_element.restype = C.c_int
        lib.oracle_eval.argtypes = [C.c_int64, i32, d, d, d, C.c_double, C.c_int64, d, d, d,
                                    C.c_int, C.c_int, C.c_int, i64, d, d]
        lib.oracle_eval.restype = C.c_int
        lib.oracle_assemble.argtypes = [C.c_int64, i32, d, d, C.c_double, C.c_int64, C.c_int64, d, d, C.c_int]
        lib.oracle_assemble.restype = C.c_int
        lib.oracle_max_threads.restype = C.c_int
        lib.oracle_element_batch.argtypes = [C.c_int64, i32, d, d, C.c_int, C.c_int, d, d, i32, C.c_int]
        lib.oracle_element_batch.restype = C.c_int
        lib.oracle_element_grad_var.argtypes = [C.c_int, d, d, d, C.c_int, C.c_int, d, d, C.POINTER(C.c_int)]
        lib.oracle_element_grad_var.restype = C.c_int
        lib.oracle_eval_grad_var.argtypes = [C.c_int64, i32, d, d, d, C.c_double, C.c_int64, d, d, d, C.c_int]
        lib.oracle_eval_grad_var.restype = C.c_int
        lib.oracle_element_quad.argtypes = [C.c_int, d, d, d, C.c_int, C.c_int, d, d, C.POINTER(C.c_int)]
        lib.oracle_element_quad.restype = C.c_int
        lib.oracle_eval_quad.argtypes = [C.c_int64, i32, d, d, d, C.c_double, C.c_int64, d, d, d, C.c_int]
        lib.oracle_eval_quad.restype = C.c_int
        lib.oracle_element_linear.argtypes = [C.c_int, d, d, d, C.c_int, C.c_int, d, d, C.POINTER(C.c_int)]
        lib.oracle_element_linear.restype = C.c_int
        lib.oracle_eval_linear.argtypes = [C.c_int64, i32, d, d, d, C.c_double, C.c_int64, d, d, d, C.c_int]
        lib.oracle_eval_linear.restype = C.c_int
        lib.oracle_element_grad.argtypes = [C.c_int, d, d, C.c_int, C.c_int, d, d, C.POINTER(C.c_int)]
        lib.oracle_element_grad.restype = C.c_int
        lib.oracle_eval_grad.argtypes = [C.c_int64, i32, d, d, d, C.c_double, C.c_int64, d, d, d, C.c_int]
        lib.oracle_eval_grad.restype = C.c_int
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def rule(type_: int, index: int) -> np.ndarray:
    """Expanded nodes of one rule: (N, 4) = (lambda_A, lambda_B, lambda_C, w)
    for triangles or (x, y, 0, w) for rectangles."""
    buf = np.zeros((33, 4))
    n = _load().oracle_rule(type_, index, _dp(buf))
    if n < 0:
        raise ValueError("bad rule")
    return buf[:n].copy()


def gauss_legendre(n: int):
    x, w = np.zeros(n), np.zeros(n)
    _load().oracle_gauss_legendre(n, _dp(x), _dp(w))
    return x, w


def default_limits() -> np.ndarray:
    out = np.zeros(10)
    _load().oracle_default_limits(_dp(out))
    return out.reshape(2, 5)


def element_geometry(type_: int, verts) -> dict:
    v = _f64(verts, (4, 3)) if np.asarray(verts).size == 12 else _f64(np.vstack([np.asarray(verts, float).reshape(3, 3), np.zeros(3)]))
    out = np.zeros(5)
    _load().oracle_element_geometry(type_, _dp(v), _dp(out))
    return {"centroid": out[:3].copy(), "L": float(out[3]), "area": float(out[4])}


def element(type_: int, verts, P, method: int = METHOD_PAPER, param: int = 0, limits=None):
    """phi, E of one element with sigma = 1, WITHOUT the 1/(4 pi eps0) factor.
    Returns (out[4], band) where band 0 = analytic, 1 + r = cubature rule r
    (band is -1 unless method = METHOD_PAPER)."""
    v = np.zeros((4, 3))
    vv = np.asarray(verts, float).reshape(-1, 3)
    v[: vv.shape[0]] = vv
    P = _f64(P, (3,))
    lim = None if limits is None else _f64(limits, (10,))
    out = np.zeros(4)
    band = C.c_int(-1)
    rc = _load().oracle_element(type_, _dp(v), _dp(P), method, param, _dp(lim), _dp(out), C.byref(band))
    if rc != 0:
        raise ValueError("oracle_element: bad arguments")
    return out, band.value


def element_linear(type_: int, verts, coef, P, method: int = METHOD_PAPER, param: int = 0, limits=None):
    """phi, E of one element with the linear density sigma = coef[0] + coef[1]
    alpha + coef[2] beta (the element's frame coordinates), WITHOUT the
    1/(4 pi eps0) factor.  Returns (out[4], band)."""
    v = np.zeros((4, 3))
    vv = np.asarray(verts, float).reshape(-1, 3)
    v[: vv.shape[0]] = vv
    P = _f64(P, (3,))
    cf = _f64(coef, (3,))
    lim = None if limits is None else _f64(limits, (10,))
    out = np.zeros(4)
    band = C.c_int(-1)
    rc = _load().oracle_element_linear(type_, _dp(v), _dp(cf), _dp(P), method, param, _dp(lim), _dp(out),
                                       C.byref(band))
    if rc != 0:
        raise ValueError("oracle_element_linear: bad arguments")
    return out, band.value


def eval_linear(types, verts, coef, pts, limits=None, eps0: float = 0.0, nthreads: int | None = None):
    """phi (n,), E (n, 3) of elements with linear densities coef (n_el, 3), by
    the method, including 1/(4 pi eps0)."""
    types = np.ascontiguousarray(types, dtype=np.int32)
    verts = _f64(verts, (types.shape[0], 4, 3))
    coef = _f64(coef, (types.shape[0], 3))
    pts = _f64(pts).reshape(-1, 3)
    phi = np.zeros(pts.shape[0])
    E = np.zeros((pts.shape[0], 3))
    lim = None if limits is None else _f64(limits, (10,))
    rc = _load().oracle_eval_linear(types.shape[0], types.ctypes.data_as(C.POINTER(C.c_int32)), _dp(verts),
                                    _dp(coef), _dp(lim), eps0, pts.shape[0], _dp(pts), _dp(phi), _dp(E),
                                    nthreads or max_threads())
    if rc != 0:
        raise ValueError("oracle_eval_linear: bad arguments")
    return phi, E


def element_quad(type_: int, verts, coef, P, method: int = METHOD_PAPER, param: int = 0, limits=None):
    """phi, E of one element with the quadratic density sigma = c0 + c1 alpha + c2 beta
    + c3 alpha^2 + c4 alpha beta + c5 beta^2 (coef = c0..c5), WITHOUT 1/(4 pi eps0)."""
    v = np.zeros((4, 3))
    vv = np.asarray(verts, float).reshape(-1, 3)
    v[: vv.shape[0]] = vv
    P = _f64(P, (3,))
    cf = _f64(coef, (6,))
    lim = None if limits is None else _f64(limits, (10,))
    out = np.zeros(4)
    band = C.c_int(-1)
    rc = _load().oracle_element_quad(type_, _dp(v), _dp(cf), _dp(P), method, param, _dp(lim), _dp(out),
                                     C.byref(band))
    if rc != 0:
        raise ValueError("oracle_element_quad: bad arguments")
    return out, band.value


def eval_quad(types, verts, coef, pts, limits=None, eps0: float = 0.0, nthreads: int | None = None):
    """phi (n,), E (n, 3) of elements with quadratic densities coef (n_el, 6), by the
    method, including 1/(4 pi eps0)."""
    types = np.ascontiguousarray(types, dtype=np.int32)
    verts = _f64(verts, (types.shape[0], 4, 3))
    coef = _f64(coef, (types.shape[0], 6))
    pts = _f64(pts).reshape(-1, 3)
    phi = np.zeros(pts.shape[0])
    E = np.zeros((pts.shape[0], 3))
    lim = None if limits is None else _f64(limits, (10,))
    rc = _load().oracle_eval_quad(types.shape[0], types.ctypes.data_as(C.POINTER(C.c_int32)), _dp(verts),
                                  _dp(coef), _dp(lim), eps0, pts.shape[0], _dp(pts), _dp(phi), _dp(E),
                                  nthreads or max_threads())
    if rc != 0:
        raise ValueError("oracle_eval_quad: bad arguments")
    return phi, E


def _coef6(coef, n):
    c = np.asarray(coef, float).reshape(n, -1)
    if c.shape[1] == 3:
        c = np.concatenate([c, np.zeros((n, 3))], axis=1)
    return _f64(c, (n, 6))


def element_grad_var(type_: int, verts, coef, P, method: int = METHOD_PAPER, param: int = 0, limits=None):
    """Field gradient (6,) of one element with a linear (3 coefficients) or
    quadratic (6) density, WITHOUT 1/(4 pi eps0); returns (g, band)."""
    v = np.zeros((4, 3))
    vv = np.asarray(verts, float).reshape(-1, 3)
    v[: vv.shape[0]] = vv
    cf = _coef6(coef, 1)[0].copy()
    P = _f64(P, (3,))
    lim = None if limits is None else _f64(limits, (10,))
    out = np.zeros(6)
    band = C.c_int(-1)
    rc = _load().oracle_element_grad_var(type_, _dp(v), _dp(cf), _dp(P), method, param, _dp(lim), _dp(out),
                                         C.byref(band))
    if rc != 0:
        raise ValueError("oracle_element_grad_var: bad arguments")
    return out, band.value


def eval_grad_var(types, verts, coef, pts, limits=None, eps0: float = 0.0, nthreads: int | None = None,
                  return_gsum: bool = False):
    """Field gradient (n, 6) for elements with linear (n_el, 3) or quadratic
    (n_el, 6) densities, by the method, including 1/(4 pi eps0)."""
    types = np.ascontiguousarray(types, dtype=np.int32)
    verts = _f64(verts, (types.shape[0], 4, 3))
    cf = _coef6(coef, types.shape[0])
    pts = _f64(pts).reshape(-1, 3)
    G = np.zeros((pts.shape[0], 6))
    gs = np.zeros(pts.shape[0]) if return_gsum else None
    lim = None if limits is None else _f64(limits, (10,))
    rc = _load().oracle_eval_grad_var(types.shape[0], types.ctypes.data_as(C.POINTER(C.c_int32)), _dp(verts),
                                      _dp(cf), _dp(lim), eps0, pts.shape[0], _dp(pts), _dp(G), _dp(gs),
                                      nthreads or max_threads())
    if rc != 0:
        raise ValueError("oracle_eval_grad_var: bad arguments")
    return (G, gs) if return_gsum else G


def element_grad(type_: int, verts, P, method: int = METHOD_PAPER, param: int = 0, limits=None):
    """Field gradient dE_i/dx_j of one element with sigma = 1, WITHOUT the
    1/(4 pi eps0) factor, as (xx, yy, zz, xy, xz, yz).  Returns (out[6], band)."""
    v = np.zeros((4, 3))
    vv = np.asarray(verts, float).reshape(-1, 3)
    v[: vv.shape[0]] = vv
    P = _f64(P, (3,))
    lim = None if limits is None else _f64(limits, (10,))
    out = np.zeros(6)
    band = C.c_int(-1)
    rc = _load().oracle_element_grad(type_, _dp(v), _dp(P), method, param, _dp(lim), _dp(out), C.byref(band))
    if rc != 0:
        raise ValueError("oracle_element_grad: bad arguments")
    return out, band.value


def eval_grad(types, verts, sigma, pts, limits=None, eps0: float = 0.0, nthreads: int | None = None,
              return_gsum: bool = False):
    """Field gradient (n, 6) = (xx, yy, zz, xy, xz, yz) of dE_i/dx_j at the
    field points, summed over all elements in index order by the method,
    including 1/(4 pi eps0).  return_gsum: also the sum over elements of each
    contribution's largest |component| (the scale of the cancellation in G)."""
    types = np.ascontiguousarray(types, dtype=np.int32)
    verts = _f64(verts, (types.shape[0], 4, 3))
    sigma = _f64(sigma, (types.shape[0],))
    pts = _f64(pts).reshape(-1, 3)
    G = np.zeros((pts.shape[0], 6))
    gs = np.zeros(pts.shape[0]) if return_gsum else None
    lim = None if limits is None else _f64(limits, (10,))
    rc = _load().oracle_eval_grad(types.shape[0], types.ctypes.data_as(C.POINTER(C.c_int32)), _dp(verts),
                                  _dp(sigma), _dp(lim), eps0, pts.shape[0], _dp(pts), _dp(G), _dp(gs),
                                  nthreads or max_threads())
    if rc != 0:
        raise ValueError("oracle_eval_grad: bad arguments")
    return (G, gs) if return_gsum else G


def element_batch(types, verts, P, method: int = METHOD_PAPER, param: int = 0, limits=None,
                  nthreads: int | None = None):
    """element() for n independent (element, point) pairs; returns (out (n, 4), band (n,))."""
    types = np.ascontiguousarray(types, dtype=np.int32)
    n = types.shape[0]
    verts = _f64(verts, (n, 4, 3))
    P = _f64(P, (n, 3))
    out = np.zeros((n, 4))
    band = np.zeros(n, np.int32)
    lim = None if limits is None else _f64(limits, (10,))
    rc = _load().oracle_element_batch(n, types.ctypes.data_as(C.POINTER(C.c_int32)), _dp(verts), _dp(P), method,
                                      param, _dp(lim), _dp(out), band.ctypes.data_as(C.POINTER(C.c_int32)),
                                      nthreads or max_threads())
    if rc != 0:
        raise ValueError("oracle_element_batch: bad arguments")
    return out, band


def eval_field(types, verts, sigma, pts, method: int = METHOD_PAPER, param: int = 16, limits=None,
               eps0: float = 0.0, nthreads: int | None = None, return_hist: bool = False,
               return_min_dr: bool = False, return_esum: bool = False):
    """phi (n,) and E (n, 3) at the field points, summed over all elements in
    index order, including 1/(4 pi eps0) (eps0 <= 0 selects the SI value).
    Optional extras, in this order: the (2, 6) band histogram, the per-point
    minimum distance ratio, the per-point sum of |E_j| over elements."""
    types = np.ascontiguousarray(types, dtype=np.int32)
    verts = _f64(verts, (types.shape[0], 4, 3))
    sigma = _f64(sigma, (types.shape[0],))
    pts = _f64(pts).reshape(-1, 3)
    n = pts.shape[0]
    phi = np.zeros(n)
    E = np.zeros((n, 3))
    hist = np.zeros(12, np.int64)
    mdr = np.zeros(n) if return_min_dr else None
    esum = np.zeros(n) if return_esum else None
    lim = None if limits is None else _f64(limits, (10,))
    nt = nthreads or max_threads()
    rc = _load().oracle_eval(types.shape[0], types.ctypes.data_as(C.POINTER(C.c_int32)), _dp(verts), _dp(sigma),
                             _dp(lim), eps0, n, _dp(pts), _dp(phi), _dp(E), method, param, nt,
                             hist.ctypes.data_as(C.POINTER(C.c_int64)), _dp(mdr), _dp(esum))
    if rc != 0:
        raise ValueError("oracle_eval: bad arguments")
    out = [phi, E]
    if return_hist:
        out.append(hist.reshape(2, 6))
    if return_min_dr:
        out.append(mdr)
    if return_esum:
        out.append(esum)
    return tuple(out)


def assemble(types, verts, colloc, rows=None, limits=None, eps0: float = 0.0, nthreads: int | None = None):
    """Rows [r0, r1) of the collocation matrix A[i, j] = potential at colloc
    point i of element j with sigma = 1 (including 1/(4 pi eps0))."""
    types = np.ascontiguousarray(types, dtype=np.int32)
    n_el = types.shape[0]
    verts = _f64(verts, (n_el, 4, 3))
    colloc = _f64(colloc).reshape(-1, 3)
    r0, r1 = (0, colloc.shape[0]) if rows is None else rows
    A = np.zeros((r1 - r0, n_el))
    lim = None if limits is None else _f64(limits, (10,))
    nt = nthreads or max_threads()
    rc = _load().oracle_assemble(n_el, types.ctypes.data_as(C.POINTER(C.c_int32)), _dp(verts), _dp(lim), eps0,
                                 r0, r1 - r0, _dp(colloc), _dp(A), nt)
    if rc != 0:
        raise ValueError("oracle_assemble: bad arguments")
    return A


EPS0_SI = 8.8541878128e-12


def coulomb_k(eps0: float = 0.0) -> float:
    e = eps0 if eps0 > 0 else EPS0_SI
    return 1.0 / (4.0 * np.pi * e)
