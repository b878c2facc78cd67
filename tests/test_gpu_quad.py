"""Parity of quadratic charge densities (bem_set_sigma_quadratic) with the FP64
oracle: the far field with sigma at the nodes and the analytic near field of
the quadratic density, both precisions, through bem_eval, bem_eval_noalloc
and the server; switching between constant, linear and quadratic densities."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bem():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1606_03743_gb300 as b
    b.load_library()
    return b


def rel_phi(a, b):
    return np.abs(a - b) / np.abs(b)


def rel_E(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


@pytest.fixture(scope="module")
def case():
    mesh = synth.plate_mesh(seed=1)
    coef = (np.random.default_rng(400).normal(size=(mesh.n, 6)) * [1.0, 0.3, 0.3, 0.15, 0.15, 0.15]
            + [1.0, 0, 0, 0, 0, 0])
    pts = synth.plate_points(seed=8, n=3000)
    rphi, rE = oracle.eval_quad(mesh.types, mesh.verts, coef, pts)
    _, _, mdr = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts, return_min_dr=True)
    return mesh, coef, pts, rphi, rE, mdr


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
def test_quadratic_density_parity(bem, case, prec, tol):
    mesh, coef, pts, rphi, rE, mdr = case
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=prec) as m:
        m.set_sigma_quadratic(coef)
        phi, E = m.eval(pts)
    far = mdr >= 3.0
    assert far.sum() > 1000 and (~far).sum() >= 10
    near_tol = tol if prec == 0 else 1e-5
    assert rel_phi(phi, rphi)[far].max() <= tol and rel_E(E, rE)[far].max() <= tol
    assert rel_phi(phi, rphi)[~far].max() <= near_tol and rel_E(E, rE)[~far].max() <= near_tol


def test_every_band_and_ragged_batch(bem):
    """Points from DR 0.02 to 700 (every rule band and the near field) on a
    small plate; a point count that is not a multiple of the tile."""
    mesh = synth.plate_mesh(seed=2, n=4)
    rng = np.random.default_rng(2)
    pts = synth.random_directions(2999, seed=2) * np.geomspace(0.02, 700.0, 2999)[:, None]
    pts += rng.uniform(-0.5, 0.5, (2999, 3)) * [1, 1, 0]
    pts[np.abs(pts[:, 2]) < 0.01, 2] = 0.01
    coef = rng.normal(size=(mesh.n, 6)) * 0.2 + [1.0, 0, 0, 0, 0, 0]
    rphi, rE = oracle.eval_quad(mesh.types, mesh.verts, coef, pts)
    _, _, hist = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts, return_hist=True)
    assert (hist > 0).all()
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.FP64) as m:
        m.set_sigma_quadratic(coef)
        phi, E = m.eval(pts)
    assert rel_phi(phi, rphi).max() <= 1e-12 and rel_E(E, rE).max() <= 1e-12


def test_zero_second_order_equals_linear_and_reset(bem, case):
    """c3 = c4 = c5 = 0 gives the linear result far away bit for bit (the same
    node charges) and to rounding near the elements (another arrangement of
    the same integrals); bem_set_sigma_linear and bem_set_sigma switch back."""
    mesh, coef, pts, _, _, mdr = case
    lin = coef[:, :3]
    q0 = np.concatenate([lin, np.zeros((mesh.n, 3))], axis=1)
    far = mdr >= oracle.default_limits()[:, 0].max()  # points with no near (analytic) pair
    for prec in (0, 1):
        with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=prec) as m:
            m.set_sigma_linear(lin)
            phi1, E1 = m.eval(pts)
            m.set_sigma_quadratic(q0)
            phi2, E2 = m.eval(pts)
            m.set_sigma_quadratic(coef)
            m.set_sigma_linear(lin)
            phi3, E3 = m.eval(pts)
            m.set_sigma_quadratic(coef)
            m.set_sigma(mesh.sigma)
            phi4, E4 = m.eval(pts)
            m.set_sigma_quadratic(np.concatenate([mesh.sigma[:, None], np.zeros((mesh.n, 5))], axis=1))
            phi5, E5 = m.eval(pts)
        assert np.array_equal(phi1, phi3) and np.array_equal(E1, E3)
        # the constant-density kernel sums a rectangle rule's nodes o and -o together, the
        # varying-density kernel one by one: the same to rounding (FP64) or within the mixed
        # path's tolerance
        t5 = 1e-13 if prec == 0 else 1e-6
        assert rel_phi(phi5, phi4)[far].max() <= t5 and rel_E(E5, E4)[far].max() <= t5
        assert rel_phi(phi5, phi4).max() <= 10 * t5 and rel_E(E5, E4).max() <= 10 * t5
        assert rel_phi(phi2, phi1).max() <= 1e-11 and rel_E(E2, E1).max() <= 1e-11
        # the far sums take the same node charges: only the near pairs can differ
        assert np.array_equal(phi2[far], phi1[far]) and np.array_equal(E2[far], E1[far])


def test_noalloc_and_server_use_quadratic_density(bem, case):
    import torch
    mesh, coef, pts, *_ = case
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=1) as m:
        m.set_sigma_quadratic(coef)
        phi, E = m.eval(pts)
        p_d = torch.from_numpy(pts).cuda()
        phi_d = torch.empty(len(pts), dtype=torch.float64, device="cuda")
        E_d = torch.empty((len(pts), 3), dtype=torch.float64, device="cuda")
        bem.bem_eval_noalloc(m.handle, p_d, phi_d, E_d)
        torch.cuda.synchronize()
        assert np.array_equal(phi_d.cpu().numpy(), phi) and np.array_equal(E_d.cpu().numpy(), E)
        with bem.Server(m) as srv:
            t = srv.submit(pts[:500])
            sphi, sE = srv.wait(t, timeout=60)
        assert np.array_equal(sphi, phi[:500]) and np.array_equal(sE, E[:500])


def test_device_coefficients(bem, case):
    import torch
    mesh, coef, pts, *_ = case
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=0) as m:
        m.set_sigma_quadratic(coef)
        phi, E = m.eval(pts[:300])
        m.set_sigma(mesh.sigma)
        m.set_sigma_quadratic(torch.from_numpy(coef).cuda())
        phi2, E2 = m.eval(pts[:300])
        assert np.array_equal(phi, phi2) and np.array_equal(E, E2)


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-6)])
def test_gradient_of_quadratic_density(bem, case, prec, tol):
    """bem_eval_grad on a quadratic mesh against the oracle's gradient for the
    quadratic density, near points included."""
    mesh, coef, pts, _, _, mdr = case
    sub = np.concatenate([np.where(mdr < 3)[0], np.arange(0, len(pts), 5)])
    P = pts[sub]
    ref = oracle.eval_grad_var(mesh.types, mesh.verts, coef, P)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=prec) as m:
        m.set_sigma_quadratic(coef)
        G = m.eval_grad(P)
        m.set_sigma(mesh.sigma)
        G0 = m.eval_grad(P)
    err = np.abs(G - ref).max(axis=1) / np.abs(ref).max(axis=1)
    far = mdr[sub] >= 3
    assert err[far].max() <= tol
    assert err[~far].max() <= (1e-11 if prec == 0 else 1e-5)
    # back to constant densities: the constant gradient again
    ref0 = oracle.eval_grad(mesh.types, mesh.verts, mesh.sigma, P)
    assert (np.abs(G0 - ref0).max(axis=1) / np.abs(ref0).max(axis=1))[far].max() <= tol


def test_gradient_every_band_quadratic(bem):
    """Quadratic densities, points from DR 0.02 to 700, FP64 kernel."""
    mesh = synth.plate_mesh(seed=2, n=4)
    rng = np.random.default_rng(5)
    pts = synth.random_directions(1500, seed=5) * np.geomspace(0.02, 700.0, 1500)[:, None]
    pts += rng.uniform(-0.5, 0.5, (1500, 3)) * [1, 1, 0]
    pts[np.abs(pts[:, 2]) < 0.01, 2] = 0.01
    coef = rng.normal(size=(mesh.n, 6)) * 0.2 + [1.0, 0, 0, 0, 0, 0]
    ref = oracle.eval_grad_var(mesh.types, mesh.verts, coef, pts)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.FP64) as m:
        m.set_sigma_quadratic(coef)
        G = m.eval_grad(pts)
    assert (np.abs(G - ref).max(axis=1) / np.abs(ref).max(axis=1)).max() <= 1e-11


def test_node_table_mesh_takes_varying_densities(bem, case):
    """A mesh created with the node table (constant densities only) evaluates
    quadratic densities by the on-the-fly expansion: the same results as a
    mesh without the table."""
    mesh, coef, pts, *_ = case
    out = []
    for nt in (False, True):
        with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.MIXED, node_table=nt) as m:
            m.set_sigma_quadratic(coef)
            out.append(m.eval(pts[:1000]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("prec", [0, 1])
def test_points_on_the_elements(bem, prec):
    """Field and gradient at the element centroids (points on the elements: the
    normal field of the element itself taken as the mean of both sides) with
    quadratic densities, against the oracle's same convention."""
    mesh = synth.sphere_cylinder_mesh(seed=3, freq=4, n_phi=8, n_z=6)
    coef = np.random.default_rng(460).normal(size=(mesh.n, 6)) * 0.2 + [1.0, 0, 0, 0, 0, 0]
    cen = synth.collocation_points(mesh)
    rphi, rE = oracle.eval_quad(mesh.types, mesh.verts, coef, cen)
    rG = oracle.eval_grad_var(mesh.types, mesh.verts, coef, cen)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=prec) as m:
        m.set_sigma_quadratic(coef)
        phi, E = m.eval(cen)
        G = m.eval_grad(cen)
    tol = 1e-12 if prec == 0 else 1e-5
    assert np.isfinite(phi).all() and np.isfinite(E).all() and np.isfinite(G).all()
    assert rel_phi(phi, rphi).max() <= tol
    assert (np.abs(E - rE).max(axis=1) / np.abs(rE).max(axis=1)).max() <= tol
    assert (np.abs(G - rG).max(axis=1) / np.abs(rG).max(axis=1)).max() <= (1e-11 if prec == 0 else 1e-5)
