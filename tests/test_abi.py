"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/bem.h declares; host-only queries (rule tables, error strings)
work without a device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import paper_1606_03743_gb300 as bem
from paper_1606_03743_gb300 import build as bem_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as f:
                txt = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
            names |= set(re.findall(r"\b(bem_\w+)\s*\(", txt))
    return names


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("bem_create", "bem_destroy", "bem_eval", "bem_assemble", "bem_matvec", "bem_set_sigma",
                 "bem_last_error"):
        assert name in d


def test_library_exports_every_declared_symbol():
    lib_path = bem_build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = _declared() - exported
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name)


def test_version_and_error_strings():
    assert "sm_103a" in bem.bem_version()
    assert isinstance(bem.bem_last_error(), str)


def test_bad_rule_query_sets_error():
    with pytest.raises(bem.BemError) as e:
        bem.bem_rule(2, 0)
    assert e.value.code == -1
    assert "bem_rule" in bem.bem_last_error()


@pytest.mark.parametrize("type_,sizes,degrees", [(0, (4, 7, 12, 19, 33), (3, 5, 7, 9, 12)),
                                                 (1, (4, 7, 12, 17, 33), (3, 5, 7, 9, 13))])
def test_library_rules_exact_to_degree(type_, sizes, degrees):
    """The library's own node tables (alpha, beta, w): right node counts,
    weights summing to one and exactness on monomials up to the degree
    (App. A, App. B), checked in the library's coordinates: for a triangle
    with corners e0 = (1, 0), e1 = (0, 1), e2 = (-1, -1) about its centroid,
    and for the square [-1, 1]^2 (e0 = (1, 0), e1 = (0, 1))."""
    for r in range(5):
        nodes = bem.bem_rule(type_, r)
        assert nodes.shape[0] == sizes[r]
        assert abs(nodes[:, 2].sum() - 1.0) < 1e-15
        x, y, w = nodes[:, 0], nodes[:, 1], nodes[:, 2]
        # exact moments by a high-order product rule on the same region
        if type_ == 1:
            g, gw = np.polynomial.legendre.leggauss(20)
            X, Y = np.meshgrid(g, g, indexing="ij")
            W = np.outer(gw, gw) / 4.0
        else:
            # collapsed map of the triangle (1,0), (0,1), (-1,-1), Jacobian u
            g, gw = np.polynomial.legendre.leggauss(20)
            u, v = (g + 1) / 2, (g + 1) / 2
            U, V = np.meshgrid(u, v, indexing="ij")
            A, B, Cc = np.array([1.0, 0.0]), np.array([0.0, 1.0]), np.array([-1.0, -1.0])
            X = A[0] + U * (B[0] - A[0]) + U * V * (Cc[0] - B[0])
            Y = A[1] + U * (B[1] - A[1]) + U * V * (Cc[1] - B[1])
            W = np.outer(gw, gw) / 4.0 * U * 2.0  # normalised to unit mass
        tol = 5e-14 if (type_ == 0 and sizes[r] == 12) else 5e-15
        for n in range(degrees[r] + 1):
            for m in range(degrees[r] + 1 - n):
                ex = np.sum(W * X ** n * Y ** m)
                val = np.sum(w * x ** n * y ** m)
                assert abs(val - ex) <= tol * max(1.0, abs(ex)), (r, n, m, val, ex)


def test_library_rules_match_oracle_tables():
    """Both sides typed the appendix tables independently: the same nodes
    (up to order) after mapping the oracle's barycentric rows to (alpha, beta)."""
    for type_ in (0, 1):
        for r in range(5):
            lib = bem.bem_rule(type_, r)
            orc = oracle.rule(type_, r)
            if type_ == 0:
                o = np.stack([orc[:, 0] - orc[:, 2], orc[:, 1] - orc[:, 2], orc[:, 3]], 1)
            else:
                o = np.stack([orc[:, 0], orc[:, 1], orc[:, 3]], 1)
            key = lambda a: a[np.lexsort((a[:, 1], a[:, 0]))]
            assert np.allclose(key(lib), key(o), rtol=0, atol=1e-15)


def test_rectangle_rules_centrally_symmetric():
    """The mixed far kernel evaluates the rectangle rules' nodes in pairs o, -o
    of equal weight (plus the centre node), so every rectangle rule of App. B
    must map onto itself under (x, y) -> (-x, -y): exactly in the library's
    tables (the kernel pairs nodes by exact equality), and in the oracle's
    independently typed tables up to rounding."""
    for r in range(5):
        lib = bem.bem_rule(1, r)
        centre = (lib[:, 0] == 0.0) & (lib[:, 1] == 0.0)
        assert centre.sum() <= 1
        mirrored = np.stack([-lib[:, 0], -lib[:, 1], lib[:, 2]], 1)
        key = lambda a: a[np.lexsort((a[:, 2], a[:, 1], a[:, 0]))]
        assert np.array_equal(key(lib) + 0.0, key(mirrored) + 0.0)
        orc = oracle.rule(1, r)
        o = np.stack([orc[:, 0], orc[:, 1], orc[:, 3]], 1)
        om = np.stack([-orc[:, 0], -orc[:, 1], orc[:, 3]], 1)
        assert np.allclose(key(o), key(om), rtol=0, atol=1e-15)


def _rule_records(type_, r, precision):
    lib = ctypes.CDLL(bem_build.build())
    lib.bem_test_rule_records.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]
    lib.bem_test_rule_records.restype = ctypes.c_int32
    out = np.zeros((33, 4))
    shape = ctypes.c_int32(0)
    n = lib.bem_test_rule_records(type_, r, precision, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  ctypes.byref(shape))
    assert n > 0
    return out[:n], shape.value


@pytest.mark.parametrize("type_", [0, 1])
@pytest.mark.parametrize("r", range(5))
def test_rule_records_reproduce_the_rules(type_, r):
    """The far kernels' node records (host-built, no GPU): expanded (a pair
    record stands for o and -o) they are the rule's nodes -- exactly in FP64,
    to FP32 rounding in the mixed path; the centre node comes first; the
    mixed path's FP32 weights, pairs counted twice, sum to one as closely as
    single-ulp changes of the weights allow (Eq. 4.1 keeps each element's
    charge)."""
    rule = bem.bem_rule(type_, r)
    key = lambda a: a[np.lexsort((a[:, 2], a[:, 1], a[:, 0]))]
    for prec in (0, 1):
        rec, shape = _rule_records(type_, r, prec)
        c = shape & 1
        assert len(rec) == c + (shape >> 1)
        if c:
            assert rec[0, 0] == 0.0 and rec[0, 1] == 0.0 and rec[0, 3] == 1.0
        assert set(rec[c:, 3]) == ({2.0} if type_ == 1 else {1.0})
        nodes = [rec[:, :3]] + [np.stack([-rec[k:k + 1, 0], -rec[k:k + 1, 1], rec[k:k + 1, 2]], 1)
                                for k in range(len(rec)) if rec[k, 3] == 2.0]
        nodes = key(np.concatenate(nodes) + 0.0)
        assert len(nodes) == len(rule)
        tol = 0.0 if prec == 0 else 1e-7
        assert np.allclose(nodes, key(rule + 0.0), rtol=tol, atol=tol)
        if prec == 1:
            total = float(np.sum(rec[:, 2] * rec[:, 3]))  # exact: FP32 weights summed in FP64
            assert abs(total - 1.0) <= 2 * np.spacing(np.float32(np.abs(rec[:, 2]).min()))


def test_library_default_limits_match_oracle():
    """The library's default DR band limits (bem_default_limits) are the
    oracle's frozen table, which tests/test_oracle_field.py pins against the
    2e-15 criterion of Sec. 4."""
    assert np.array_equal(bem.bem_default_limits(), oracle.default_limits())


def test_corner_value_coefficients():
    """bem_linear_coef_from_corners: a density linear in space, sampled at the
    corners, is reproduced at every corner by the coefficients in the frame
    coordinates of Eq. 3.2 / Eq. 3.3; a triangle takes the mean of its three
    values at its centroid; an unknown type is rejected."""
    import synth
    mesh = synth.plate_mesh(seed=1, n=3)
    rng = np.random.default_rng(5)
    a, c0 = rng.normal(size=3), 1.3
    vals = c0 + mesh.verts @ a
    coef = bem.linear_coef_from_corner_values(mesh.types, vals)
    for t, cf, val in zip(mesh.types, coef, vals):
        if t == bem.TRIANGLE:  # (alpha, beta) at A, B, C = (1, 0), (0, 1), (-1, -1)
            ab, want = np.array([[1, 0], [0, 1], [-1, -1]]), val[:3]
        else:  # natural coordinates of P0..P3
            ab, want = np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]]), val
        assert np.allclose(cf[0] + ab @ cf[1:], want, rtol=1e-14, atol=1e-14)
    one = bem.linear_coef_from_corner_values(np.array([0], np.int32), np.array([[0.3, 1.9, -0.4, 0.0]]))
    m = (0.3 + 1.9 - 0.4) / 3
    assert np.allclose(one, [[m, 0.3 - m, 1.9 - m]], rtol=1e-15)
    with pytest.raises(bem.BemError):
        bem.linear_coef_from_corner_values(np.array([2], np.int32), np.zeros((1, 4)))
