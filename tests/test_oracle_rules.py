"""Pins of the oracle's cubature rules (App. A, App. B) and of its GL2
reference (Sec. 2) against closed-form integrals and a library routine."""
import json
import os
from math import factorial

import numpy as np
import pytest

import oracle


def _degrees(golden_dir):
    with open(os.path.join(golden_dir, "paper_rule_degrees.json")) as f:
        g = json.load(f)
    return {0: g["triangle"], 1: g["rectangle"]}


def _tri_moment(i, j, k):
    """Exact mean of lambda_A^i lambda_B^j lambda_C^k over a triangle
    (Dirichlet integral): 2 i! j! k! / (i + j + k + 2)!"""
    return 2.0 * factorial(i) * factorial(j) * factorial(k) / factorial(i + j + k + 2)


def _rect_moment(n, m):
    """Exact mean of x^n y^m over [-1, 1]^2."""
    if n % 2 or m % 2:
        return 0.0
    return (2.0 / (n + 1)) * (2.0 / (m + 1)) / 4.0


def _monomial_errors(type_, nodes, degree):
    """max error over monomials of total degree == degree"""
    worst = 0.0
    if type_ == 0:
        for i in range(degree + 1):
            for j in range(degree + 1 - i):
                k = degree - i - j
                ex = _tri_moment(i, j, k)
                val = np.sum(nodes[:, 3] * nodes[:, 0] ** i * nodes[:, 1] ** j * nodes[:, 2] ** k)
                worst = max(worst, abs(val - ex) / ex)
    else:
        for n in range(degree + 1):
            m = degree - n
            ex = _rect_moment(n, m)
            val = np.sum(nodes[:, 3] * nodes[:, 0] ** n * nodes[:, 1] ** m)
            worst = max(worst, abs(val - ex) / (abs(ex) if ex else 1.0))
    return worst


@pytest.mark.parametrize("type_", [0, 1])
def test_node_counts_and_weight_sum(type_, golden_dir):
    for r, (n, _) in enumerate(_degrees(golden_dir)[type_]):
        nodes = oracle.rule(type_, r)
        assert nodes.shape[0] == n
        # Eq. 3.1: weights sum to one
        assert abs(nodes[:, 3].sum() - 1.0) < 1e-15
        # distinct nodes
        assert len({tuple(np.round(x[:3], 12)) for x in nodes}) == n


@pytest.mark.parametrize("type_", [0, 1])
def test_rules_exact_up_to_degree(type_, golden_dir):
    """Sec. 3: a rule of degree d integrates every monomial x^n y^m with
    n + m <= d exactly.  The 12-point triangle rule carries 16-digit
    decimals (Table A3), hence its looser bound."""
    for r, (n, d) in enumerate(_degrees(golden_dir)[type_]):
        nodes = oracle.rule(type_, r)
        tol = 5e-14 if (type_ == 0 and n == 12) else 5e-15
        for deg in range(d + 1):
            assert _monomial_errors(type_, nodes, deg) < tol, (type_, n, deg)


@pytest.mark.parametrize("type_", [0, 1])
def test_rules_not_exact_above_degree(type_, golden_dir):
    """The stated degrees are tight: every rule fails at degree d + 1."""
    for r, (n, d) in enumerate(_degrees(golden_dir)[type_]):
        nodes = oracle.rule(type_, r)
        assert _monomial_errors(type_, nodes, d + 1) > 1e-6, (type_, n)


def test_nodes_inside_elements():
    """Sec. 3 prefers nodes inside the element; all printed rules have them."""
    for r in range(5):
        t = oracle.rule(0, r)
        assert (t[:, :3] > 0).all() and np.allclose(t[:, :3].sum(1), 1.0, atol=2e-16 * 4)
        q = oracle.rule(1, r)
        assert (np.abs(q[:, :2]) < 1).all()


def test_triangle4_negative_centroid_weight():
    """Table A1 prints a negative centroid weight, -9/16."""
    t = oracle.rule(0, 0)
    assert t[0, 3] == -9.0 / 16.0
    assert np.allclose(t[0, :3], 1.0 / 3.0)


@pytest.mark.parametrize("n", [1, 2, 5, 16, 32])
def test_gauss_legendre_matches_numpy(n):
    x, w = oracle.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(np.sort(x), xr, atol=1e-15, rtol=0)
    assert np.allclose(w[np.argsort(x)], wr, atol=2e-15, rtol=0)


def test_gl2_integrates_polynomials_on_triangle():
    """The collapsed-map GL2 (16 x 16) integrates polynomials exactly: check
    the area and the first moments of a triangle through phi-free means,
    via a far field point where 1/R is smooth: compare to the 33-point rule
    far away (DR ~ 1e4), where both are at the double-precision floor."""
    v = np.array([[0.1, 0.2, 0.3], [0.9, 0.1, 0.2], [0.4, 0.8, 0.6]])
    g = oracle.element_geometry(0, v)
    P = g["centroid"] + np.array([1.0, 2.0, 2.0]) / 3.0 * 1e4 * g["L"]
    a, _ = oracle.element(0, v, P, oracle.METHOD_GL2, 16)
    b, _ = oracle.element(0, v, P, oracle.METHOD_RULE, 4)
    assert np.allclose(a, b, rtol=2e-15, atol=0)
