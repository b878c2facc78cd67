"""Pins of the oracle's quadratic charge density sigma = c0 + c1 alpha + c2 beta
+ c3 alpha^2 + c4 alpha beta + c5 beta^2 (the cubature with sigma(Q_i) at the
nodes, and the analytic near field for the quadratic density): reduction to the
linear case, brute-force subdivision, E = -grad phi, closed-form axis values of
sigma = x^2 on a square against adaptive quadrature, a direct product-Gauss sum
of the density written in natural coordinates, the rules against GL2 inside
their bands and Gauss's law with the textbook moments of alpha and beta."""
import numpy as np
import pytest
from scipy import integrate

import oracle
import synth

TRI, RECT = 0, 1
SQUARE = np.array([[-0.5, -0.5, 0.0], [0.5, -0.5, 0.0], [0.5, 0.5, 0.0], [-0.5, 0.5, 0.0]])


def points_at(t, verts, drs, seed):
    g = oracle.element_geometry(t, verts)
    dirs = synth.random_directions(len(drs), seed=seed)
    return g["centroid"] + (np.asarray(drs) * g["L"])[:, None] * dirs, g


@pytest.mark.parametrize("t", [TRI, RECT])
def test_linear_coefficients_reduce_to_the_linear_case(t):
    """c3 = c4 = c5 = 0: the cubature is the linear one term for term; the
    quadratic analytic branch arranges the linear terms differently, so near
    the element (where the method uses it) it agrees to rounding."""
    rng = np.random.default_rng(300 + t)
    v = synth.random_elements(t, 1, seed=301 + t)[0]
    coef = rng.normal(size=3)
    drs = [0.3, 1.0, 2.0, 2.9, 10.0, 100.0, 5000.0]
    pts, _ = points_at(t, v, drs, seed=302)
    for dr, P in zip(drs, pts):
        q = oracle.element_quad(t, v, [*coef, 0.0, 0.0, 0.0], P)[0]
        lin = oracle.element_linear(t, v, coef, P)[0]
        if dr >= 3:
            assert np.array_equal(q, lin)
        else:
            assert np.abs(q - lin).max() <= 1e-11 * np.abs(lin).max()


@pytest.mark.parametrize("t", [TRI, RECT])
def test_analytic_branch_against_brute_force(t):
    rng = np.random.default_rng(310 + t)
    for k, v in enumerate(synth.random_elements(t, 2, seed=311 + t)):
        coef = rng.normal(size=6)
        pts, _ = points_at(t, v, [0.15, 0.5, 1.2, 2.9], seed=312 + k)
        for P in pts:
            a = oracle.element_quad(t, v, coef, P, oracle.METHOD_ANALYTIC)[0]
            b = oracle.element_quad(t, v, coef, P, oracle.METHOD_SUBDIV, 5)[0]
            assert abs(a[0] - b[0]) <= 1e-10 * np.abs(b).max()
            assert np.linalg.norm(a[1:] - b[1:]) <= 1e-10 * np.linalg.norm(b[1:])


@pytest.mark.parametrize("t", [TRI, RECT])
def test_field_is_minus_gradient_of_potential(t):
    rng = np.random.default_rng(320 + t)
    v = synth.random_elements(t, 1, seed=321 + t)[0]
    coef = rng.normal(size=6)
    pts, g = points_at(t, v, [0.4, 2.0, 6.0, 40.0], seed=322)
    for P in pts:
        h = 2e-4 * np.linalg.norm(P - g["centroid"])
        E = oracle.element_quad(t, v, coef, P)[0][1:]
        fd = np.zeros(3)
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            f = [oracle.element_quad(t, v, coef, P + k * e)[0][0] for k in (-2, -1, 1, 2)]
            fd[j] = -(f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * h)
        assert np.linalg.norm(E - fd) <= 1e-8 * np.linalg.norm(E)


@pytest.mark.parametrize("z", [0.05, 0.4, 1.5])
def test_x_squared_density_on_square_axis(z):
    """sigma = x^2 on the square [-1/2, 1/2]^2 (c3 = 1/4 in natural coordinates,
    alpha = 2x): on the axis phi = int x^2 / R dA, E_z = z int x^2 / R^3 dA and
    E_x = E_y = 0 by symmetry."""
    out, _ = oracle.element_quad(RECT, SQUARE, [0.0, 0.0, 0.0, 0.25, 0.0, 0.0], [0, 0, z], oracle.METHOD_ANALYTIC)
    phi, _ = integrate.dblquad(lambda y, x: x * x / np.sqrt(x * x + y * y + z * z), -0.5, 0.5, -0.5, 0.5,
                               epsabs=0, epsrel=1e-13)
    ez, _ = integrate.dblquad(lambda y, x: z * x * x / (x * x + y * y + z * z) ** 1.5, -0.5, 0.5, -0.5, 0.5,
                              epsabs=0, epsrel=1e-13)
    assert out[0] == pytest.approx(phi, rel=1e-11)
    assert out[3] == pytest.approx(ez, rel=1e-11)
    assert abs(out[1]) <= 1e-14 * abs(ez) and abs(out[2]) <= 1e-14 * abs(ez)


def natural_gl2(t, v, coef, P, n=24):
    """Product Gauss-Legendre over the element with sigma written in its natural
    coordinates: a triangle through barycentric coordinates (alpha = lA - lC,
    beta = lB - lC), a rectangle through alpha, beta in [-1, 1] along its sides."""
    x, wq = np.polynomial.legendre.leggauss(n)
    c0, c1, c2, c3, c4, c5 = coef
    acc = np.zeros(4)
    for i in range(n):
        for j in range(n):
            if t == TRI:
                u, w = 0.5 * (x[i] + 1), 0.5 * (x[j] + 1)
                lA, lB, lC = 1 - u, u - u * w, u * w
                Q = lA * v[0] + lB * v[1] + lC * v[2]
                al, be = lA - lC, lB - lC
                area = 0.5 * np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0]))
                wt = 0.25 * wq[i] * wq[j] * 2 * area * u
            else:
                al, be = x[i], x[j]
                Q = 0.25 * ((1 - al) * (1 - be) * v[0] + (1 + al) * (1 - be) * v[1] + (1 + al) * (1 + be) * v[2]
                            + (1 - al) * (1 + be) * v[3])
                area = np.linalg.norm(v[1] - v[0]) * np.linalg.norm(v[3] - v[0])
                wt = 0.25 * wq[i] * wq[j] * area
            s = c0 + c1 * al + c2 * be + c3 * al * al + c4 * al * be + c5 * be * be
            d = P - Q
            r = np.linalg.norm(d)
            acc += wt * s * np.array([1 / r, *(d / r ** 3)])
    return acc


@pytest.mark.parametrize("t", [TRI, RECT])
def test_coefficients_mean_natural_coordinates(t):
    """The oracle's map from (c0..c5) to the density in space agrees with the
    density written in natural coordinates, summed by a product rule of its own."""
    rng = np.random.default_rng(330 + t)
    v = synth.random_elements(t, 1, seed=331 + t)[0]
    coef = rng.normal(size=6)
    g = oracle.element_geometry(t, v)
    for P in (g["centroid"] + np.array([0.3, -0.2, 0.9]) * g["L"], g["centroid"] + np.array([2.0, 1.0, -1.5]) * g["L"]):
        a = oracle.element_quad(t, v, coef, P, oracle.METHOD_GL2, 24)[0]
        b = natural_gl2(t, v, coef, P)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-14 * np.abs(b).max())


@pytest.mark.parametrize("t", [TRI, RECT])
def test_rules_agree_with_gl2_where_the_method_uses_them(t):
    """Each rule just inside its band (the constant-density limits): a quadratic
    density costs two polynomial degrees of the rule's margin, so the method's
    error rises to ~1e-9 (phi) and ~1e-8 (E) at the band edges."""
    rng = np.random.default_rng(340 + t)
    v = synth.random_elements(t, 1, seed=341 + t)[0]
    coef = rng.normal(size=6)
    lim = np.asarray(oracle.default_limits()).reshape(10)[5 * t: 5 * t + 5]
    for rule, dr in zip(range(4, -1, -1), lim * 1.05):
        pts, _ = points_at(t, v, [dr], seed=342)
        a = oracle.element_quad(t, v, coef, pts[0], oracle.METHOD_RULE, rule)[0]
        b = oracle.element_quad(t, v, coef, pts[0], oracle.METHOD_GL2, 32)[0]
        assert abs(a[0] - b[0]) <= 5e-9 * np.abs(b).max()
        assert np.linalg.norm(a[1:] - b[1:]) <= 5e-8 * np.linalg.norm(b[1:])


def test_gauss_law_quadratic_density():
    """The flux through a sphere around the plate is the total charge / eps0,
    with the textbook moments: on a triangle alpha = l0 - l2, beta = l1 - l2
    (barycentric l), int l_i^2 = area / 6 and int l_i l_j = area / 12, so
    int alpha^2 = int beta^2 = area / 6 and int alpha beta = area / 12; on a
    rectangle int alpha^2 = int beta^2 = area / 3 and int alpha beta = 0."""
    mesh = synth.plate_mesh(seed=1, n=6)
    coef = np.random.default_rng(350).normal(size=(mesh.n, 6))
    nt, nphi, R = 48, 96, 3.0
    ct, wt = np.polynomial.legendre.leggauss(nt)
    ph = np.arange(nphi) * 2 * np.pi / nphi
    st = np.sqrt(1 - ct ** 2)
    n = np.stack([st[:, None] * np.cos(ph)[None], st[:, None] * np.sin(ph)[None],
                  np.broadcast_to(ct[:, None], (nt, nphi))], -1).reshape(-1, 3)
    w = (wt[:, None] * np.full(nphi, 2 * np.pi / nphi)[None]).ravel() * R * R
    _, E = oracle.eval_quad(mesh.types, mesh.verts, coef, R * n)
    flux = np.sum(w * (E * n).sum(1))
    area = np.array([oracle.element_geometry(int(t), v)["area"] for t, v in zip(mesh.types, mesh.verts)])
    tri = mesh.types == TRI
    q = area * (coef[:, 0] + (coef[:, 3] + coef[:, 5]) * np.where(tri, 1.0 / 6.0, 1.0 / 3.0)
                + coef[:, 4] * np.where(tri, 1.0 / 12.0, 0.0))
    assert (mesh.types == TRI).any() and (mesh.types == RECT).any()
    assert flux == pytest.approx(q.sum() / oracle.EPS0_SI, rel=1e-12)


def test_eval_sums_elements():
    mesh = synth.plate_mesh(seed=2, n=3)
    coef = np.random.default_rng(360).normal(size=(mesh.n, 6))
    pts = synth.plate_points(seed=2, n=12)
    phi, E = oracle.eval_quad(mesh.types, mesh.verts, coef, pts)
    kc = 1.0 / (4 * np.pi * oracle.EPS0_SI)
    for p in range(len(pts)):
        f = sum(oracle.element_quad(int(t), v, c, pts[p])[0] for t, v, c in zip(mesh.types, mesh.verts, coef))
        assert phi[p] == pytest.approx(kc * f[0], rel=1e-13)
        assert np.allclose(E[p], kc * f[1:], rtol=1e-13, atol=1e-13 * np.abs(kc * f[1:]).max())
