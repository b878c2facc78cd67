"""Pins of the oracle's potential and field: the analytic near field, the
point-charge cubature (Eq. 4.1), the rule bands (Sec. 4) and the element
sum (Sec. 5), each against something other than the oracle itself."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

TRI, RECT = 0, 1
SQUARE = np.array([[-0.5, -0.5, 0.0], [0.5, -0.5, 0.0], [0.5, 0.5, 0.0], [-0.5, 0.5, 0.0]])
SOME_TRI = np.array([[0.1, 0.2, 0.3], [0.9, 0.1, 0.2], [0.4, 0.8, 0.6], [0, 0, 0]])
SOME_RECT = synth.random_elements(RECT, 1, seed=3)[0]


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("z", [1e-3, 0.05, 0.3, 1.0, 4.0, -0.7])
def test_square_axis_closed_form(z):
    """Uniform square of side 2a on its axis (textbook closed form):
    phi = 4 [2a ln((a + R) / sqrt(a^2 + z^2)) - |z| atan(a^2 / (|z| R))],
    E_z = 4 sign(z) atan(a^2 / (|z| R)), R = sqrt(2 a^2 + z^2)."""
    a, az = 0.5, abs(z)
    R = math.sqrt(2 * a * a + z * z)
    phi = 4 * (2 * a * math.log((a + R) / math.sqrt(a * a + z * z)) - az * math.atan(a * a / (az * R)))
    Ez = 4 * math.copysign(1.0, z) * math.atan(a * a / (az * R))
    out, _ = oracle.element(RECT, SQUARE, [0, 0, z], oracle.METHOD_ANALYTIC)
    assert out[0] == pytest.approx(phi, rel=1e-14)
    assert out[3] == pytest.approx(Ez, rel=1e-14)
    assert abs(out[1]) < 1e-15 and abs(out[2]) < 1e-15


def test_square_in_plane_limit():
    """phi at the centre of the square itself: 8 a ln(1 + sqrt 2)."""
    out, _ = oracle.element(RECT, SQUARE, [0, 0, 0], oracle.METHOD_ANALYTIC)
    assert out[0] == pytest.approx(8 * 0.5 * math.log(1 + math.sqrt(2)), rel=1e-14)
    assert out[3] == 0.0  # mean of both sides of the sheet


@pytest.mark.parametrize("z", [0.02, 0.4, 2.5])
def test_equilateral_triangle_axis_closed_form(z):
    """Regular n-gon of inradius rho on its axis, n = 3: with
    G(t) = rho asinh(rho tan t / sqrt(rho^2 + z^2))
           + z atan(z tan t / sqrt(rho^2 sec^2 t + z^2)),
    phi = n [G(pi/n) - G(-pi/n) - 2 (pi/n) z]  (z > 0)."""
    n, rho = 3, 0.4
    Rc = rho / math.cos(math.pi / n)
    v = np.zeros((4, 3))
    for k in range(3):
        v[k] = (Rc * math.cos(2 * math.pi * k / 3), Rc * math.sin(2 * math.pi * k / 3), 0.0)

    def G(t):
        return (rho * math.asinh(rho * math.tan(t) / math.sqrt(rho * rho + z * z))
                + z * math.atan(z * math.tan(t) / math.sqrt(rho * rho / math.cos(t) ** 2 + z * z)))

    phi = n * (G(math.pi / n) - G(-math.pi / n) - 2 * (math.pi / n) * z)
    out, _ = oracle.element(TRI, v, [0, 0, z], oracle.METHOD_ANALYTIC)
    assert out[0] == pytest.approx(phi, rel=1e-13)


def _quad_field(type_, verts, P):
    """phi and E by scipy's adaptive 2-D quadrature (QUADPACK), over the
    parameter square of the element."""
    from scipy import integrate
    V = [np.asarray(verts[k], float) for k in range(4)]
    P = np.asarray(P, float)
    res = []
    for comp in range(4):
        def f(v, u, comp=comp):
            if type_ == TRI:
                Q = V[0] + u * (V[1] - V[0]) + u * v * (V[2] - V[1])
                jac = u
            else:
                Q = V[0] + u * (V[1] - V[0]) + v * (V[3] - V[0])
                jac = 1.0
            d = P - Q
            r = math.sqrt(d @ d)
            return jac * (1.0 / r if comp == 0 else d[comp - 1] / r ** 3)
        val, _ = integrate.dblquad(f, 0.0, 1.0, 0.0, 1.0, epsabs=1e-15, epsrel=1e-14)
        res.append(val)
    if type_ == TRI:
        jac = np.linalg.norm(np.cross(V[1] - V[0], V[2] - V[0]))  # 2 * area
    else:
        jac = np.linalg.norm(V[1] - V[0]) * np.linalg.norm(V[3] - V[0])
    return np.array(res) * jac


@pytest.mark.parametrize("type_,verts,P", [
    (TRI, SOME_TRI, [0.45, 0.35, 0.55]),
    (TRI, SOME_TRI, [0.2, 1.0, -0.3]),
    (RECT, SOME_RECT, None),
])
def test_analytic_vs_adaptive_quadrature(type_, verts, P):
    if P is None:
        g = oracle.element_geometry(type_, verts)
        P = g["centroid"] + np.array([0.3, -0.2, 0.25])
    out, _ = oracle.element(type_, verts, P, oracle.METHOD_ANALYTIC)
    ref = _quad_field(type_, verts, P)
    assert np.allclose(out, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


# ------------------------------------------------------------ brute force
@pytest.mark.parametrize("type_", [TRI, RECT])
def test_analytic_vs_subdivision_near_field(type_):
    """O-PIN 5: brute-force fine subdivision (GL2 on 2^k x 2^k pieces)
    converges to the analytic value for near-field points, DR in [0.1, 3]."""
    verts = synth.random_elements(type_, 6, seed=5)
    dirs = synth.random_directions(6, seed=5)
    for i, dr in enumerate([0.1, 0.3, 0.7, 1.2, 2.0, 3.0]):
        g = oracle.element_geometry(type_, verts[i])
        P = g["centroid"] + dr * g["L"] * dirs[i]
        a, _ = oracle.element(type_, verts[i], P, oracle.METHOD_ANALYTIC)
        b, _ = oracle.element(type_, verts[i], P, oracle.METHOD_SUBDIV, 5)
        c, _ = oracle.element(type_, verts[i], P, oracle.METHOD_SUBDIV, 6)
        scale = np.abs(c).max()
        assert np.abs(b - c).max() < 1e-12 * scale  # subdivision converged
        assert np.allclose(a, c, rtol=0, atol=1e-12 * scale), (dr, a, c)


# ------------------------------------------------------------ E = -grad phi
def _fd_grad(type_, verts, P, method, param, h):
    g = np.zeros(3)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        f = [oracle.element(type_, verts, np.asarray(P) + s * e, method, param)[0][0] for s in (2, 1, -1, -2)]
        g[k] = (-f[0] + 8 * f[1] - 8 * f[2] + f[3]) / (12 * h)
    return g


@pytest.mark.parametrize("type_", [TRI, RECT])
@pytest.mark.parametrize("method,param,dr", [
    (oracle.METHOD_ANALYTIC, 0, 0.4), (oracle.METHOD_ANALYTIC, 0, 2.5),
    (oracle.METHOD_RULE, 1, 30.0), (oracle.METHOD_RULE, 4, 4.0), (oracle.METHOD_PAPER, 0, 50.0),
])
def test_field_is_minus_gradient(type_, method, param, dr):
    """O-PIN 4: E = -grad phi (fourth-order central differences)."""
    verts = synth.random_elements(type_, 1, seed=9)[0]
    g = oracle.element_geometry(type_, verts)
    P = g["centroid"] + dr * g["L"] * synth.random_directions(1, seed=9)[0]
    out, _ = oracle.element(type_, verts, P, method, param)
    grad = _fd_grad(type_, verts, P, method, param, 2e-4 * dr * g["L"])
    assert np.allclose(out[1:], -grad, rtol=0, atol=1e-8 * np.linalg.norm(out[1:]))


@pytest.mark.parametrize("type_", [TRI, RECT])
def test_continuity_at_near_limit(type_):
    """Across the DR = 3 switch (Sec. 4) the analytic and 33-point values
    agree to the 33-point rule's accuracy at DR = 3 (about 1e-13 for phi and
    a few 1e-12 for E, Sec. 4 experiment)."""
    verts = synth.random_elements(type_, 20, seed=12)
    dirs = synth.random_directions(20, seed=12)
    for i in range(20):
        g = oracle.element_geometry(type_, verts[i])
        P = g["centroid"] + 3.0 * g["L"] * dirs[i]
        a, _ = oracle.element(type_, verts[i], P, oracle.METHOD_ANALYTIC)
        c, _ = oracle.element(type_, verts[i], P, oracle.METHOD_RULE, 4)
        assert abs(a[0] - c[0]) < 2e-11 * abs(a[0])
        assert np.abs(a[1:] - c[1:]).sum() < 2e-9 * np.linalg.norm(a[1:])


# ------------------------------------------------------------ far field
@pytest.mark.parametrize("type_", [TRI, RECT])
def test_point_charge_limit(type_):
    """O-PIN 3: far away the element acts as its total charge at the
    centroid; the dipole term vanishes about the centroid, so
    phi D / q - 1 falls off as DR^-2 and E -> q (P - C) / D^3."""
    verts = synth.random_elements(type_, 1, seed=21)[0]
    g = oracle.element_geometry(type_, verts)
    d = synth.random_directions(1, seed=21)[0]
    devs = []
    drs = [20.0, 40.0, 80.0, 160.0]
    for dr in drs:
        D = dr * g["L"]
        out, _ = oracle.element(type_, verts, g["centroid"] + D * d, oracle.METHOD_PAPER)
        devs.append(abs(out[0] * D / g["area"] - 1.0))
        Ept = g["area"] * d / D ** 2
        assert np.linalg.norm(out[1:] - Ept) < 10 * np.linalg.norm(Ept) / dr ** 2
    slope = np.polyfit(np.log(drs), np.log(devs), 1)[0]
    assert slope == pytest.approx(-2.0, abs=0.1)


@pytest.mark.parametrize("type_", [TRI, RECT])
def test_rules_agree_far_away(type_):
    """O-PIN 8: at DR >= 2000 all five rules of a type agree to the double
    precision floor (Sec. 4)."""
    verts = synth.random_elements(type_, 50, seed=31)
    dirs = synth.random_directions(50, seed=31)
    for i in range(50):
        g = oracle.element_geometry(type_, verts[i])
        P = g["centroid"] + 3000.0 * g["L"] * dirs[i]
        vals = np.array([oracle.element(type_, verts[i], P, oracle.METHOD_RULE, r)[0] for r in range(5)])
        assert np.ptp(vals[:, 0]) < 4e-15 * abs(vals[4, 0])
        assert np.abs(vals[:, 1:] - vals[4, 1:]).sum(1).max() < 2e-14 * np.linalg.norm(vals[4, 1:])


@pytest.mark.slow
def test_paper_triangle_bands_reproduced(golden_dir):
    """Sec. 4 prints, for a 2e-15 triangle potential, the lower DR limit of
    each rule.  The oracle's rules, geometry and GL2 reference reproduce
    them: at each printed limit the mean err(phi) of that rule over random
    unit-cube triangles is at the 2e-15 level, and at half the limit it is
    clearly above it."""
    from oracle import dr_experiment
    with open(os.path.join(golden_dir, "paper_bands.json")) as f:
        g = json.load(f)
    idx = {"4": 0, "7": 1, "12": 2, "19": 3, "33": 4}
    for N, lim in g["triangle_phi_lower_limit_by_N"].items():
        r = idx[N]
        at = dr_experiment.errors(TRI, float(lim), n_el=1000, seed=41)[r, 0]
        below = dr_experiment.errors(TRI, float(lim) / 2.0, n_el=1000, seed=43)[r, 0]
        assert at <= 1.5 * g["target"], (N, at)
        assert below > g["target"], (N, below)


TARGET = 2e-15  # Sec. 4: the relative accuracy the printed limits are chosen for


@pytest.mark.slow
@pytest.mark.parametrize("type_", [TRI, RECT])
def test_default_limits_meet_the_field_target(type_):
    """Sec. 4: with potential and field computed together, each rule serves
    from the DR at which the field (the stricter of the two) reaches the
    2e-15 level.  The frozen default table (reading 1) is pinned by the
    paper's own experiment on fresh random elements: at every limit, the
    near limit included, the rule of the band above it meets 2e-15 in both
    mean err(phi) and mean err(E); at 0.7 x the limit it misses in one of
    them (the limit was not rounded up by more than that)."""
    from oracle import dr_experiment
    lim = oracle.default_limits()[type_]
    for k in range(5):
        r = 4 - k  # the rule of the band [lim[k], lim[k+1]): 33 points above lim[0] ... 4 above lim[4]
        at = dr_experiment.errors(type_, float(lim[k]), n_el=2000, seed=901 + k)[r]
        below = dr_experiment.errors(type_, 0.7 * float(lim[k]), n_el=2000, seed=911 + k)[r]
        assert at[0] <= TARGET and at[1] <= TARGET, (k, lim[k], at)
        assert max(below) > TARGET, (k, lim[k], below)


@pytest.mark.slow
def test_potential_only_limits_fail_the_field_target(golden_dir):
    """The check above catches a table calibrated on the potential alone: the
    paper's printed triangle-potential limits (Sec. 4) give mean field errors
    above 2e-15 at their lower ends, while their potential errors meet it."""
    from oracle import dr_experiment
    with open(os.path.join(golden_dir, "paper_bands.json")) as f:
        g = json.load(f)
    idx = {"4": 0, "7": 1, "12": 2, "19": 3, "33": 4}
    worst_E = 0.0
    for N, lim in g["triangle_phi_lower_limit_by_N"].items():
        e = dr_experiment.errors(TRI, float(lim), n_el=2000, seed=921 + idx[N])[idx[N]]
        assert e[0] <= 1.5 * TARGET, (N, e)
        worst_E = max(worst_E, e[1])
    assert worst_E > 2 * TARGET, worst_E


def test_gl2_accurate_above_dr2(golden_dir):
    """Sec. 2: GL2 with 16 x 16 nodes is accurate to ~1e-15 above DR = 2;
    checked against brute-force subdivision."""
    for type_ in (TRI, RECT):
        verts = synth.random_elements(type_, 5, seed=51)
        dirs = synth.random_directions(5, seed=51)
        for i, dr in enumerate([2.0, 3.0, 5.0, 10.0, 100.0]):
            g = oracle.element_geometry(type_, verts[i])
            P = g["centroid"] + dr * g["L"] * dirs[i]
            a, _ = oracle.element(type_, verts[i], P, oracle.METHOD_GL2, 16)
            b, _ = oracle.element(type_, verts[i], P, oracle.METHOD_SUBDIV, 3)
            tol = 1e-12 if dr < 3 else 1e-14
            assert abs(a[0] - b[0]) < tol * abs(b[0])


# ------------------------------------------------------------ dispatch
@pytest.mark.parametrize("type_", [TRI, RECT])
def test_band_dispatch(type_):
    """Sec. 4: analytic below the first limit, then 33, 19|17, 12, 7, 4 points
    as DR grows; the chosen branch's value is returned unchanged."""
    lim = oracle.default_limits()[type_]
    verts = synth.random_elements(type_, 1, seed=61)[0]
    g = oracle.element_geometry(type_, verts)
    d = synth.random_directions(1, seed=61)[0]
    probes = [0.5 * lim[0]] + [0.5 * (lim[k] + lim[k + 1]) for k in range(4)] + [2 * lim[4]]
    for k, dr in enumerate(probes):
        P = g["centroid"] + dr * g["L"] * d
        out, band = oracle.element(type_, verts, P, oracle.METHOD_PAPER)
        assert band == (0 if k == 0 else 1 + (5 - k))
        if band == 0:
            ref, _ = oracle.element(type_, verts, P, oracle.METHOD_ANALYTIC)
        else:
            ref, _ = oracle.element(type_, verts, P, oracle.METHOD_RULE, band - 1)
        assert np.array_equal(out, ref)


def test_custom_limits_are_used():
    lim = np.array([[0.5, 1, 2, 3, 4], [0.5, 1, 2, 3, 4]], float)
    P = SOME_TRI[:3].mean(0) + np.array([0, 0, 10.0])
    _, band = oracle.element(TRI, SOME_TRI, P, oracle.METHOD_PAPER, limits=lim)
    assert band == 1  # DR >> 4: the 4-point rule


# ------------------------------------------------------------ many elements
def test_eval_is_sigma_weighted_sum_times_k():
    mesh = synth.plate_mesh(seed=1, n=2)
    pts = synth.plate_points(seed=1, n=5)
    phi, E = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts)
    k = oracle.coulomb_k()
    for p in range(5):
        tot = np.zeros(4)
        for j in range(mesh.n):
            out, _ = oracle.element(int(mesh.types[j]), mesh.verts[j], pts[p])
            tot += mesh.sigma[j] * out
        assert np.allclose([phi[p], *E[p]], k * tot, rtol=1e-14, atol=0)


def test_eval_thread_count_does_not_change_result():
    mesh = synth.plate_mesh(seed=1, n=4)
    pts = synth.plate_points(seed=1, n=64)
    a = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts, nthreads=1)
    b = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts, nthreads=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_plate_symmetry():
    """O-PIN 7: the plate lies in z = 0, so phi(x, y, -z) = phi(x, y, z),
    E_z is odd and E_x, E_y are even in z."""
    mesh = synth.plate_mesh(seed=1)
    pts = synth.plate_points(seed=1, n=200)
    mirr = pts * np.array([1, 1, -1])
    a_phi, a_E = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts)
    b_phi, b_E = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, mirr)
    assert np.allclose(a_phi, b_phi, rtol=1e-14, atol=0)
    assert np.allclose(a_E[:, :2], b_E[:, :2], rtol=0, atol=1e-13 * np.abs(a_E).max())
    assert np.allclose(a_E[:, 2], -b_E[:, 2], rtol=0, atol=1e-13 * np.abs(a_E).max())


def test_gauss_law_plate():
    """O-PIN 6: the flux of E through a sphere of radius 3 enclosing the
    plate equals Q / eps0 (Gauss-Legendre in cos(theta) x trapezoid in phi)."""
    mesh = synth.plate_mesh(seed=1)
    nt, nphi, R = 48, 96, 3.0
    ct, wt = np.polynomial.legendre.leggauss(nt)
    ph = np.arange(nphi) * 2 * np.pi / nphi
    st = np.sqrt(1 - ct ** 2)
    n = np.stack([st[:, None] * np.cos(ph)[None], st[:, None] * np.sin(ph)[None],
                  np.broadcast_to(ct[:, None], (nt, nphi))], -1).reshape(-1, 3)
    w = (wt[:, None] * np.full(nphi, 2 * np.pi / nphi)[None]).ravel() * R * R
    _, E = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, R * n)
    flux = np.sum(w * (E * n).sum(1))
    area = np.array([oracle.element_geometry(int(t), v)["area"] for t, v in zip(mesh.types, mesh.verts)])
    Q = np.sum(mesh.sigma * area)
    assert flux == pytest.approx(Q / oracle.EPS0_SI, rel=1e-12)


def test_assembly_times_sigma_is_potential():
    """The collocation matrix applied to sigma gives the potential at the
    collocation points (linearity of Eq. 2.1 in sigma)."""
    mesh = synth.sphere_cylinder_mesh(seed=3, freq=2, n_phi=4, n_z=3)
    col = synth.collocation_points(mesh)
    A = oracle.assemble(mesh.types, mesh.verts, col)
    phi, _ = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, col)
    assert np.allclose(A @ mesh.sigma, phi, rtol=1e-13, atol=0)
    # self terms use the analytic branch: a field point on its own element
    rows = oracle.assemble(mesh.types, mesh.verts, col, rows=(0, 3))
    assert np.array_equal(rows, A[:3])


@pytest.mark.parametrize("type_", [TRI, RECT])
def test_potential_continuous_onto_an_edge(type_):
    """A field point on an element edge (or corner) has a finite potential,
    the limit of points approaching it; the oracle returns that limit."""
    verts = synth.random_elements(type_, 1, seed=71)[0]
    nv = 3 if type_ == TRI else 4
    a, b = verts[0], verts[1]
    cen = verts[:nv].mean(0)
    for P in (0.3 * a + 0.7 * b, a.copy()):
        on, _ = oracle.element(type_, verts, P, oracle.METHOD_ANALYTIC)
        assert np.isfinite(on).all()
        for eps in (1e-9, 1e-11):
            near, _ = oracle.element(type_, verts, P + eps * (cen - P), oracle.METHOD_ANALYTIC)
            assert abs(near[0] - on[0]) < 1e-7 * abs(on[0])


def test_esum_is_sum_of_element_field_norms():
    mesh = synth.plate_mesh(seed=1, n=2)
    pts = synth.plate_points(seed=2, n=4)
    _, E, es = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts, return_esum=True)
    k = oracle.coulomb_k()
    for p in range(4):
        ref = sum(abs(mesh.sigma[j]) * np.linalg.norm(oracle.element(int(mesh.types[j]), mesh.verts[j], pts[p])[0][1:])
                  for j in range(mesh.n))
        assert es[p] == pytest.approx(k * ref, rel=1e-13)
        assert es[p] >= np.linalg.norm(E[p]) * (1 - 1e-12)  # triangle inequality


@pytest.mark.parametrize("t", [0, 1])
def test_centroid_of_a_tilted_element_takes_the_mean_of_both_sides(t):
    """The centroid of an element in general position lies on it only up to the
    rounding of its coordinates (h of order 1e-17): it still counts as on the
    element, so its normal field is the mean of the two one-sided limits."""
    for k, v in enumerate(synth.random_elements(t, 4, seed=470 + t)):
        g = oracle.element_geometry(t, v)
        C = g["centroid"]
        n = np.cross(v[1] - v[0], v[2] - v[0])
        n /= np.linalg.norm(n)
        delta = 1e-8 * g["L"]
        on = oracle.element(t, v, C, oracle.METHOD_ANALYTIC)[0]
        up = oracle.element(t, v, C + delta * n, oracle.METHOD_ANALYTIC)[0]
        dn = oracle.element(t, v, C - delta * n, oracle.METHOD_ANALYTIC)[0]
        assert abs(up[1:] @ n - dn[1:] @ n) == pytest.approx(4 * math.pi, rel=1e-6)  # the jump
        assert np.abs(on[1:] - 0.5 * (up[1:] + dn[1:])).max() <= 1e-6 * np.abs(up[1:]).max()
