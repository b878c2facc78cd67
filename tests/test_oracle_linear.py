"""Pins of the oracle's linear charge density sigma = s_c + s_a alpha + s_b beta
(the cubature with sigma(Q_i) at the nodes, and the analytic near field for
the linear density): reduction to the constant case, brute-force subdivision,
E = -grad phi, an antisymmetric density's closed-form axis behaviour against
adaptive quadrature, the rules against GL2 inside their bands and Gauss's law."""
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
def test_constant_density_reduces_to_the_constant_case(t):
    v = synth.random_elements(t, 1, seed=200 + t)[0]
    pts, _ = points_at(t, v, [0.3, 2.0, 10.0, 100.0, 5000.0], seed=201)
    for P in pts:
        for method in (oracle.METHOD_PAPER, oracle.METHOD_ANALYTIC):
            lin = oracle.element_linear(t, v, [1.7, 0.0, 0.0], P, method)[0]
            ref = 1.7 * oracle.element(t, v, P, method)[0]
            assert np.allclose(lin, ref, rtol=1e-15, atol=0)


@pytest.mark.parametrize("t", [TRI, RECT])
def test_analytic_branch_against_brute_force(t):
    rng = np.random.default_rng(210 + t)
    for k, v in enumerate(synth.random_elements(t, 2, seed=211 + t)):
        coef = rng.normal(size=3)
        pts, _ = points_at(t, v, [0.15, 0.5, 1.2, 2.9], seed=212 + k)
        for P in pts:
            a = oracle.element_linear(t, v, coef, P, oracle.METHOD_ANALYTIC)[0]
            b = oracle.element_linear(t, v, coef, P, oracle.METHOD_SUBDIV, 5)[0]
            assert abs(a[0] - b[0]) <= 1e-11 * abs(b[0])
            assert np.linalg.norm(a[1:] - b[1:]) <= 1e-10 * np.linalg.norm(b[1:])


@pytest.mark.parametrize("t", [TRI, RECT])
def test_field_is_minus_gradient_of_potential(t):
    rng = np.random.default_rng(220 + t)
    v = synth.random_elements(t, 1, seed=221 + t)[0]
    coef = rng.normal(size=3)
    pts, g = points_at(t, v, [0.4, 2.0, 6.0, 40.0], seed=222)
    for P in pts:
        h = 2e-4 * np.linalg.norm(P - g["centroid"])
        E = oracle.element_linear(t, v, coef, P)[0][1:]
        fd = np.zeros(3)
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            f = [oracle.element_linear(t, v, coef, P + k * e)[0][0] for k in (-2, -1, 1, 2)]
            fd[j] = -(f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * h)
        assert np.linalg.norm(E - fd) <= 1e-8 * np.linalg.norm(E)


@pytest.mark.parametrize("z", [0.05, 0.4, 1.5])
def test_odd_density_on_square_axis(z):
    """sigma = x on the square [-1/2, 1/2]^2 (s_a = 1/2 in natural coordinates):
    on the axis phi = E_y = E_z = 0 by symmetry and E_x = -int x^2 / R^3 dA."""
    out, _ = oracle.element_linear(RECT, SQUARE, [0.0, 0.5, 0.0], [0, 0, z], oracle.METHOD_ANALYTIC)
    ex, _ = integrate.dblquad(lambda y, x: -x * x / (x * x + y * y + z * z) ** 1.5, -0.5, 0.5, -0.5, 0.5,
                              epsabs=0, epsrel=1e-13)
    assert abs(out[0]) <= 1e-15 and abs(out[2]) <= 1e-15 and abs(out[3]) <= 1e-15
    assert out[1] == pytest.approx(ex, rel=1e-11)


@pytest.mark.parametrize("t", [TRI, RECT])
def test_rules_agree_with_gl2_where_the_method_uses_them(t):
    """Each rule just inside its band (the constant-density limits): a linear
    density costs one polynomial degree of the rule's margin, so the method's
    error rises from ~1e-15 to ~1e-11 (phi) and ~1e-10 (E) at the band edges."""
    rng = np.random.default_rng(230 + t)
    v = synth.random_elements(t, 1, seed=231 + t)[0]
    coef = rng.normal(size=3)
    lim = np.asarray(oracle.default_limits()).reshape(10)[5 * t: 5 * t + 5]
    for rule, dr in zip(range(4, -1, -1), lim * 1.05):  # 33-point at its lower limit ... 4-point at its
        pts, _ = points_at(t, v, [dr], seed=232)
        a = oracle.element_linear(t, v, coef, pts[0], oracle.METHOD_RULE, rule)[0]
        b = oracle.element_linear(t, v, coef, pts[0], oracle.METHOD_GL2, 32)[0]
        assert abs(a[0] - b[0]) <= 5e-11 * abs(b[0])
        assert np.linalg.norm(a[1:] - b[1:]) <= 5e-10 * np.linalg.norm(b[1:])


def test_gauss_law_linear_density():
    """The linear part integrates to zero about the centroid: the flux through
    a sphere around the plate is sum_j s_c,j area_j / eps0."""
    mesh = synth.plate_mesh(seed=1, n=6)
    coef = np.random.default_rng(240).normal(size=(mesh.n, 3))
    nt, nphi, R = 48, 96, 3.0
    ct, wt = np.polynomial.legendre.leggauss(nt)
    ph = np.arange(nphi) * 2 * np.pi / nphi
    st = np.sqrt(1 - ct ** 2)
    n = np.stack([st[:, None] * np.cos(ph)[None], st[:, None] * np.sin(ph)[None],
                  np.broadcast_to(ct[:, None], (nt, nphi))], -1).reshape(-1, 3)
    w = (wt[:, None] * np.full(nphi, 2 * np.pi / nphi)[None]).ravel() * R * R
    _, E = oracle.eval_linear(mesh.types, mesh.verts, coef, R * n)
    flux = np.sum(w * (E * n).sum(1))
    area = np.array([oracle.element_geometry(int(t), v)["area"] for t, v in zip(mesh.types, mesh.verts)])
    assert flux == pytest.approx(np.sum(coef[:, 0] * area) / oracle.EPS0_SI, rel=1e-12)


def test_vertex_values_of_a_triangle():
    """s_c, s_a, s_b from vertex values: sigma(A) = s_c + s_a, sigma(B) = s_c + s_b,
    sigma(C) = s_c - s_a - s_b.  A density that is linear in space gives the
    same field whichever vertex values describe it: check against GL2 with the
    plane density evaluated directly."""
    v = synth.random_elements(TRI, 1, seed=250)[0]
    sA, sB, sC = 0.3, 1.9, -0.4
    sc = (sA + sB + sC) / 3
    coef = [sc, sA - sc, sB - sc]
    P = v[:3].mean(0) + np.array([0.3, -0.2, 0.9])
    a = oracle.element_linear(TRI, v, coef, P, oracle.METHOD_GL2, 24)[0]
    # direct GL2: the same collapsed map, sigma by barycentric interpolation
    x, wq = np.polynomial.legendre.leggauss(24)
    A, B, Cv = v[0], v[1], v[2]
    area = 0.5 * np.linalg.norm(np.cross(B - A, Cv - A))
    acc = np.zeros(4)
    for i in range(24):
        for j in range(24):
            u, vv = 0.5 * (x[i] + 1), 0.5 * (x[j] + 1)
            lA, lB, lC = 1 - u, u - u * vv, u * vv
            Q = lA * A + lB * B + lC * Cv
            wt = 0.25 * wq[i] * wq[j] * 2 * area * u * (lA * sA + lB * sB + lC * sC)
            d = P - Q
            r = np.linalg.norm(d)
            acc += wt * np.array([1 / r, *(d / r ** 3)])
    assert np.allclose(a, acc, rtol=1e-13, atol=0)
