"""Parity of linear charge densities (bem_set_sigma_linear) with the FP64
oracle: the far field with sigma at the nodes and the analytic near field of
the linear density, both precisions, through bem_eval, bem_eval_noalloc and
the server."""
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
    coef = np.random.default_rng(300).normal(size=(mesh.n, 3)) * [1.0, 0.3, 0.3] + [1.0, 0.0, 0.0]
    pts = synth.plate_points(seed=8, n=3000)
    rphi, rE = oracle.eval_linear(mesh.types, mesh.verts, coef, pts)
    _, _, mdr = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts, return_min_dr=True)
    return mesh, coef, pts, rphi, rE, mdr


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
def test_linear_density_parity(bem, case, prec, tol):
    mesh, coef, pts, rphi, rE, mdr = case
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=prec) as m:
        m.set_sigma_linear(coef)
        phi, E = m.eval(pts)
    far = mdr >= 3.0
    near_tol = tol if prec == 0 else 1e-5
    assert rel_phi(phi, rphi)[far].max() <= tol and rel_E(E, rE)[far].max() <= tol
    assert rel_phi(phi, rphi)[~far].max() <= near_tol and rel_E(E, rE)[~far].max() <= near_tol


def test_zero_slopes_equal_constant_and_reset(bem, case):
    """Zero slopes give the constant-density result to rounding (FP64) or
    within the mixed path's tolerance: the constant-density kernel sums a
    rectangle rule's nodes o and -o together (their charges are equal), the
    varying-density kernel one by one.  Going back to constant densities gives
    the first result bit for bit."""
    mesh, coef, pts, rphi, rE, mdr = case
    c0 = np.stack([mesh.sigma, np.zeros(mesh.n), np.zeros(mesh.n)], axis=1)
    far = mdr >= 3.0
    for prec in (0, 1):
        with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=prec) as m:
            phi0, E0 = m.eval(pts)
            m.set_sigma_linear(c0)
            phi1, E1 = m.eval(pts)
            m.set_sigma_linear(coef)
            m.set_sigma(mesh.sigma)  # back to constant densities
            phi2, E2 = m.eval(pts)
        if prec == 0:
            assert rel_phi(phi1, phi0).max() <= 1e-13 and rel_E(E1, E0).max() <= 1e-13
        else:
            assert rel_phi(phi1, phi0)[far].max() <= 1e-6 and rel_E(E1, E0)[far].max() <= 1e-6
            assert rel_phi(phi1, phi0)[~far].max() <= 1e-5 and rel_E(E1, E0)[~far].max() <= 1e-5
        assert np.array_equal(phi0, phi2) and np.array_equal(E0, E2)


def test_corner_values_helper(bem):
    """Corner values that lie on a plane in space give the same field as that
    plane's density evaluated by the oracle from the fitted coefficients."""
    mesh = synth.plate_mesh(seed=1, n=4)
    a = np.array([0.4, -0.7, 0.2])
    vals = 1.0 + mesh.verts @ a  # density linear in space, sampled at the corners
    coef = bem.linear_coef_from_corner_values(mesh.types, vals)
    pts = synth.plate_points(seed=9, n=200)
    rphi, rE = oracle.eval_linear(mesh.types, mesh.verts, coef, pts)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=0) as m:
        m.set_sigma_linear(coef)
        phi, E = m.eval(pts)
    assert rel_phi(phi, rphi).max() <= 1e-12 and rel_E(E, rE).max() <= 1e-12
    # the fitted density reproduces the plane at every element's centroid
    cen = synth.collocation_points(mesh)
    assert np.allclose(coef[:, 0], 1.0 + cen @ a, rtol=1e-14)


def test_noalloc_and_server_use_linear_density(bem, case):
    import torch
    mesh, coef, pts, rphi, rE, mdr = case
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=1) as m:
        m.set_sigma_linear(coef)
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


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-6)])
def test_gradient_of_linear_density(bem, case, prec, tol):
    """bem_eval_grad on a linear mesh against the oracle's gradient for the
    linear density (largest component error over the largest component)."""
    mesh, coef, pts, _, _, mdr = case
    sub = np.concatenate([np.where(mdr < 3)[0], np.arange(0, len(pts), 5)])
    P = pts[sub]
    ref = oracle.eval_grad_var(mesh.types, mesh.verts, coef, P)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=prec) as m:
        m.set_sigma_linear(coef)
        G = m.eval_grad(P)
    err = np.abs(G - ref).max(axis=1) / np.abs(ref).max(axis=1)
    far = mdr[sub] >= 3
    assert err[far].max() <= tol
    assert err[~far].max() <= (1e-11 if prec == 0 else 1e-5)
