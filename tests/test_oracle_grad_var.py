"""Pins of the oracle's field gradient for linear and quadratic densities
(point charges w_i area sigma(Q_i) in the cubature branch; the in-plane
derivative moved onto the density in the analytic branch): finite differences
of the already-pinned field of the same density, reduction to the constant
density, product Gauss-Legendre, Laplace's equation (zero trace), continuity
at the near limit, and the sum over a mesh."""
import numpy as np
import pytest

import oracle
import synth

TRI, RECT = 0, 1


def full(g):
    xx, yy, zz, xy, xz, yz = g
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def points_at(t, verts, drs, seed):
    g = oracle.element_geometry(t, verts)
    dirs = synth.random_directions(len(drs), seed=seed)
    return g["centroid"] + (np.asarray(drs) * g["L"])[:, None] * dirs, g


def fd_gradient(t, verts, coef, P, method, param, h):
    """4th-order central differences of the oracle's quadratic-density field; column j = dE/dx_j."""
    G = np.zeros((3, 3))
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        f = [oracle.element_quad(t, verts, coef, P + k * e, method, param)[0][1:] for k in (-2, -1, 1, 2)]
        G[:, j] = (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * h)
    return G


@pytest.mark.parametrize("t", [TRI, RECT])
@pytest.mark.parametrize("order", [1, 2])
def test_analytic_gradient_is_derivative_of_field(t, order):
    rng = np.random.default_rng(400 + 10 * t + order)
    for k, v in enumerate(synth.random_elements(t, 2, seed=401 + t)):
        coef = rng.normal(size=6)
        if order == 1:
            coef[3:] = 0.0
        drs = [0.2, 0.6, 1.3, 2.9]
        pts, g = points_at(t, v, drs, seed=402 + k)
        for dr, P in zip(drs, pts):
            # finite differences of the brute-force subdivided field (smooth in P; 2^6 x 2^6
            # pieces where the point may lie close to the element)
            G = full(oracle.element_grad_var(t, v, coef, P, oracle.METHOD_ANALYTIC)[0])
            Gfd = fd_gradient(t, v, coef, P, oracle.METHOD_SUBDIV, 6 if dr < 0.5 else 4,
                              2e-4 * np.linalg.norm(P - g["centroid"]))
            assert np.abs(G - Gfd).max() <= 1e-8 * np.abs(Gfd).max()


@pytest.mark.parametrize("t", [TRI, RECT])
@pytest.mark.parametrize("rule", [0, 2, 4])
def test_cubature_gradient_is_derivative_of_field(t, rule):
    rng = np.random.default_rng(410 + t)
    v = synth.random_elements(t, 1, seed=411 + t)[0]
    coef = rng.normal(size=6)
    pts, g = points_at(t, v, [4.0, 20.0, 300.0], seed=412)
    for P in pts:
        G = full(oracle.element_grad_var(t, v, coef, P, oracle.METHOD_RULE, rule)[0])
        Gfd = fd_gradient(t, v, coef, P, oracle.METHOD_RULE, rule, 1e-3 * np.linalg.norm(P - g["centroid"]))
        assert np.abs(G - Gfd).max() <= 1e-8 * np.abs(Gfd).max()


@pytest.mark.parametrize("t", [TRI, RECT])
def test_constant_density_reduces_to_the_constant_gradient(t):
    v = synth.random_elements(t, 1, seed=420 + t)[0]
    pts, _ = points_at(t, v, [0.3, 1.0, 2.5, 10.0, 500.0], seed=421)
    for dr, P in zip([0.3, 1.0, 2.5, 10.0, 500.0], pts):
        # the analytic branch only where it stays well conditioned (far away its terms cancel)
        for method in (oracle.METHOD_PAPER,) + ((oracle.METHOD_ANALYTIC,) if dr <= 10 else ()):
            a = oracle.element_grad_var(t, v, [1.7, 0, 0, 0, 0, 0], P, method)[0]
            b = 1.7 * oracle.element_grad(t, v, P, method)[0]
            assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


@pytest.mark.parametrize("t", [TRI, RECT])
def test_analytic_agrees_with_gl2_and_is_traceless(t):
    rng = np.random.default_rng(430 + t)
    v = synth.random_elements(t, 1, seed=431 + t)[0]
    coef = rng.normal(size=6)
    pts, _ = points_at(t, v, [2.0, 3.5, 6.0], seed=432)
    for P in pts:
        ga = oracle.element_grad_var(t, v, coef, P, oracle.METHOD_ANALYTIC)[0]
        gg = oracle.element_grad_var(t, v, coef, P, oracle.METHOD_GL2, 32)[0]
        assert np.abs(ga - gg).max() <= 1e-10 * np.abs(ga).max()
        assert abs(ga[0] + ga[1] + ga[2]) <= 1e-13 * np.abs(ga).max()


def test_continuity_at_the_near_limit():
    rng = np.random.default_rng(440)
    for t in (TRI, RECT):
        v = synth.random_elements(t, 1, seed=441 + t)[0]
        coef = rng.normal(size=6)
        pts, _ = points_at(t, v, [3.0] * 4, seed=442)
        for P in pts:
            ga = oracle.element_grad_var(t, v, coef, P, oracle.METHOD_ANALYTIC)[0]
            gc = oracle.element_grad_var(t, v, coef, P, oracle.METHOD_RULE, 4)[0]
            assert np.abs(ga - gc).max() <= 1e-9 * np.abs(ga).max()


def test_mesh_sum_and_linear_coefficients():
    mesh = synth.plate_mesh(seed=3, n=3)
    rng = np.random.default_rng(450)
    coef = rng.normal(size=(mesh.n, 6))
    pts = synth.plate_points(seed=4, n=10)
    G, gs = oracle.eval_grad_var(mesh.types, mesh.verts, coef, pts, return_gsum=True)
    kc = 1.0 / (4 * np.pi * oracle.EPS0_SI)
    for p in range(len(pts)):
        f = sum(oracle.element_grad_var(int(t), v, c, pts[p])[0] for t, v, c in zip(mesh.types, mesh.verts, coef))
        assert np.allclose(G[p], kc * f, rtol=1e-12, atol=1e-13 * np.abs(kc * f).max())
    assert (np.abs(G).max(axis=1) <= gs * (1 + 1e-12)).all()
    # three coefficients mean a linear density
    G3 = oracle.eval_grad_var(mesh.types, mesh.verts, coef[:, :3], pts)
    G6 = oracle.eval_grad_var(mesh.types, mesh.verts, np.concatenate([coef[:, :3], np.zeros((mesh.n, 3))], 1), pts)
    assert np.array_equal(G3, G6)
