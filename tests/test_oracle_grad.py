"""Pins of the oracle's field gradient dE_i/dx_j (point charges, Sec. 7, and
the analytic near-field branch): finite differences of the already-pinned
field, the closed form on the axis of a square, Laplace's equation (zero
trace), symmetry, the point-charge limit and continuity at the near limit."""
import math

import numpy as np
import pytest

import oracle
import synth

TRI, RECT = 0, 1
SQUARE = np.array([[-0.5, -0.5, 0.0], [0.5, -0.5, 0.0], [0.5, 0.5, 0.0], [-0.5, 0.5, 0.0]])


def full(g):
    xx, yy, zz, xy, xz, yz = g
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def fd_gradient(t, verts, P, method, param, h):
    """4th-order central differences of the oracle's field; column j = dE/dx_j."""
    G = np.zeros((3, 3))
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        f = [oracle.element(t, verts, P + k * e, method, param)[0][1:] for k in (-2, -1, 1, 2)]
        G[:, j] = (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * h)
    return G


def points_at(t, verts, drs, seed):
    g = oracle.element_geometry(t, verts)
    dirs = synth.random_directions(len(drs), seed=seed)
    return g["centroid"] + (np.asarray(drs) * g["L"])[:, None] * dirs, g


@pytest.mark.parametrize("t", [TRI, RECT])
def test_analytic_gradient_is_derivative_of_field(t):
    verts = synth.random_elements(t, 3, seed=20 + t)
    for k, v in enumerate(verts):
        pts, g = points_at(t, v, [0.2, 0.6, 1.3, 2.9], seed=30 + k)
        for P in pts:
            G = full(oracle.element_grad(t, v, P, oracle.METHOD_ANALYTIC)[0])
            Gfd = fd_gradient(t, v, P, oracle.METHOD_ANALYTIC, 0, 2e-4 * np.linalg.norm(P - g["centroid"]))
            # both triangles of the full matrix: the finite differences are not symmetric by construction
            assert np.abs(G - Gfd).max() <= 1e-7 * np.abs(Gfd).max()


@pytest.mark.parametrize("t", [TRI, RECT])
@pytest.mark.parametrize("rule", [0, 2, 4])
def test_cubature_gradient_is_derivative_of_field(t, rule):
    v = synth.random_elements(t, 1, seed=40 + t)[0]
    pts, g = points_at(t, v, [4.0, 20.0, 300.0], seed=41)
    for P in pts:
        G = full(oracle.element_grad(t, v, P, oracle.METHOD_RULE, rule)[0])
        Gfd = fd_gradient(t, v, P, oracle.METHOD_RULE, rule, 1e-3 * np.linalg.norm(P - g["centroid"]))
        assert np.abs(G - Gfd).max() <= 1e-8 * np.abs(Gfd).max()


@pytest.mark.parametrize("z", [0.02, 0.3, 1.0, 4.0, -0.7])
def test_square_axis_closed_form(z):
    """d/dz of E_z = 4 sign(z) atan(a^2 / (|z| R)), R = sqrt(2 a^2 + z^2), and by
    the square's symmetry and Laplace's equation G_xx = G_yy = -G_zz / 2."""
    a, az = 0.5, abs(z)
    R = math.sqrt(2 * a * a + z * z)
    f = a * a / (az * R)
    dfdz = -a * a * (R * R + z * z) / (z * z * R ** 3)  # d f / d|z|
    gzz = 4 * dfdz / (1 + f * f)
    for method in (oracle.METHOD_ANALYTIC, oracle.METHOD_PAPER):
        g, _ = oracle.element_grad(RECT, SQUARE, [0, 0, z], method)
        assert g[2] == pytest.approx(gzz, rel=1e-12)
        assert g[0] == pytest.approx(-gzz / 2, rel=1e-12) and g[1] == pytest.approx(-gzz / 2, rel=1e-12)
        assert np.abs(g[3:]).max() <= 1e-13 * abs(gzz)


@pytest.mark.parametrize("t", [TRI, RECT])
def test_laplace_trace_zero(t):
    """Off the element the field is divergence-free.  (The analytic branch is
    checked where the method uses it: far away its edge terms cancel, the loss
    of accuracy that motivates the cubature, Sec. 1.)"""
    v = synth.random_elements(t, 1, seed=50 + t)[0]
    drs = np.geomspace(0.1, 5000, 40)
    pts, _ = points_at(t, v, drs, seed=51)
    for dr, P in zip(drs, pts):
        for method in (oracle.METHOD_ANALYTIC, oracle.METHOD_PAPER):
            if method == oracle.METHOD_ANALYTIC and dr > 10:
                continue
            g, _ = oracle.element_grad(t, v, P, method)
            assert abs(g[0] + g[1] + g[2]) <= 1e-13 * np.abs(g).max()


@pytest.mark.parametrize("t", [TRI, RECT])
def test_point_charge_limit(t):
    """Far away the element is a point charge q = area at the centroid (the
    dipole moment about the centroid vanishes): error O(DR^-2)."""
    v = synth.random_elements(t, 1, seed=60 + t)[0]
    errs = []
    for dr in (100.0, 1000.0):
        pts, g = points_at(t, v, [dr], seed=61)
        d = pts[0] - g["centroid"]
        D = np.linalg.norm(d)
        ref = g["area"] * (np.eye(3) / D ** 3 - 3 * np.outer(d, d) / D ** 5)
        G = full(oracle.element_grad(t, v, pts[0], oracle.METHOD_PAPER)[0])
        errs.append(np.abs(G - ref).max() / np.abs(ref).max())
    assert errs[0] < 1e-3 and errs[1] < errs[0] / 50  # second order in 1/DR


@pytest.mark.parametrize("t", [TRI, RECT])
def test_gl2_agrees_with_analytic(t):
    v = synth.random_elements(t, 1, seed=70 + t)[0]
    pts, _ = points_at(t, v, [2.0, 5.0], seed=71)
    for P in pts:
        ga = oracle.element_grad(t, v, P, oracle.METHOD_ANALYTIC)[0]
        gg = oracle.element_grad(t, v, P, oracle.METHOD_GL2, 32)[0]
        assert np.abs(ga - gg).max() <= 1e-10 * np.abs(ga).max()


def test_continuity_at_the_near_limit():
    """Just above and below DR = 3 the cubature (33 points) and analytic
    gradients agree (the rule limits were calibrated for phi and E; the
    gradient, one derivative higher, is met to about 1e-11)."""
    for t in (TRI, RECT):
        v = synth.random_elements(t, 1, seed=80 + t)[0]
        pts, _ = points_at(t, v, [3.0] * 5, seed=81)
        for P in pts:
            ga = oracle.element_grad(t, v, P, oracle.METHOD_ANALYTIC)[0]
            gc = oracle.element_grad(t, v, P, oracle.METHOD_RULE, 4)[0]
            assert np.abs(ga - gc).max() <= 1e-10 * np.abs(ga).max()


def test_field_sum_traceless_on_plate():
    mesh = synth.plate_mesh(seed=1, n=4)
    pts = synth.plate_points(seed=1, n=64)
    G = oracle.eval_grad(mesh.types, mesh.verts, mesh.sigma, pts)
    assert np.abs(G[:, 0] + G[:, 1] + G[:, 2]).max() <= 1e-12 * np.abs(G).max()


def test_gsum_bounds_the_gradient():
    """The element-scale sum is the triangle-inequality bound of the largest
    component, and equals it for a single element."""
    mesh = synth.plate_mesh(seed=1, n=4)
    pts = synth.plate_points(seed=2, n=64)
    G, gs = oracle.eval_grad(mesh.types, mesh.verts, mesh.sigma, pts, return_gsum=True)
    assert np.array_equal(G, oracle.eval_grad(mesh.types, mesh.verts, mesh.sigma, pts))
    assert (np.abs(G).max(axis=1) <= gs * (1 + 1e-12)).all()
    G1, gs1 = oracle.eval_grad(mesh.types[:1], mesh.verts[:1], mesh.sigma[:1], pts, return_gsum=True)
    assert np.allclose(np.abs(G1).max(axis=1), gs1, rtol=1e-15, atol=0)
