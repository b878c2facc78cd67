"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times: the 150 000-element coaxial mesh with 1 000 000 points and the
500 000-element mesh with 4 000 000 points (evaluated in slices), compared with
the oracle on sampled points; plus degenerate elements (long, thin
triangles and rectangles) against the oracle."""
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


def sampled_check(mesh, pts, phi, E, idx, tol, kappa_max, bands=False):
    rphi, rE, mdr, esum = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts[idx], return_min_dr=True,
                                            return_esum=True)
    if bands:  # the sample reaches every band of the nearest element (near, 33, 19|17, 12 points)
        lim = oracle.default_limits()[0]
        hist = np.histogram(mdr, bins=[0, lim[0], lim[1], lim[2], lim[3], np.inf])[0]
        assert (hist[:4] > 0).all(), hist
    kappa = esum / np.linalg.norm(rE, axis=1)
    gate = (mdr >= 3) & (kappa <= kappa_max)
    assert gate.sum() >= len(idx) // 2
    assert rel_phi(phi[idx], rphi)[gate].max() <= tol
    assert rel_E(E[idx], rE)[gate].max() <= tol
    # every sampled point, gated or not, within 1e-4 of the terms' size
    assert (np.linalg.norm(E[idx] - rE, axis=1) / esum).max() <= 1e-4 * tol / 1e-6


@pytest.mark.parametrize("prec,tol,kmax", [(1, 1e-6, 100.0), (0, 1e-12, 1e9)])
def test_coax_150k_1M(bem, prec, tol, kmax):
    """512 sampled points against the oracle.  Every band of the nearest
    element is among them, and the run sends a share of its (warp, element)
    pairs through the per-point band path of straddling tiles; the same
    points evaluated on their own (other tiles, other straddling pairs) give
    the same bits, so both paths agree for them."""
    import torch
    mesh = synth.coax_mesh(seed=2)
    pts = synth.coax_points(seed=2, n=1_000_000)
    dev = torch.device("cuda")
    n = len(pts) if prec == 1 else 65536  # the FP64 kernel on a batch that still spans many tiles
    idx = np.random.default_rng(11).choice(n, 512, replace=False)
    with bem.Mesh(torch.from_numpy(mesh.types).to(dev), torch.from_numpy(mesh.verts).to(dev),
                  torch.from_numpy(mesh.sigma).to(dev), precision=prec) as m:
        p_d = torch.from_numpy(pts[:n]).to(dev)
        phi = torch.empty(n, dtype=torch.float64, device=dev)
        E = torch.empty((n, 3), dtype=torch.float64, device=dev)
        m.set_stats(True)
        bem.bem_eval(m.handle, p_d, phi, E)
        stats = m.last_stats()
        m.set_stats(False)
        torch.cuda.synchronize()
        phi, E = phi.cpu().numpy(), E.cpu().numpy()
        phi1, E1 = m.eval(pts[idx])
    assert stats[14] > 0.05 * (stats[13] + stats[14])  # straddling (warp, element) pairs took the per-point path
    assert np.array_equal(phi[idx], phi1) and np.array_equal(E[idx], E1)
    sampled_check(mesh, pts[:n], phi, E, idx, tol, kmax, bands=True)


def test_coax_500k_4M_sliced(bem):
    """4 000 000 points: more than one evaluation slice (2^21 points)."""
    import torch
    mesh = synth.coax_mesh_large(seed=4)
    pts = synth.coax_points(seed=4, n=4_000_000)
    dev = torch.device("cuda")
    with bem.Mesh(torch.from_numpy(mesh.types).to(dev), torch.from_numpy(mesh.verts).to(dev),
                  torch.from_numpy(mesh.sigma).to(dev), precision=bem.MIXED) as m:
        p_d = torch.from_numpy(pts).to(dev)
        phi = torch.empty(len(pts), dtype=torch.float64, device=dev)
        E = torch.empty((len(pts), 3), dtype=torch.float64, device=dev)
        bem.bem_eval(m.handle, p_d, phi, E)
        torch.cuda.synchronize()
        # a point's result does not depend on its slice: re-evaluate a few alone
        idx = np.array([0, 2_097_151, 2_097_152, 3_999_999])
        phi1, E1 = m.eval(pts[idx])
        phi, E = phi.cpu().numpy(), E.cpu().numpy()
    assert np.array_equal(phi[idx], phi1) and np.array_equal(E[idx], E1)
    sidx = np.random.default_rng(12).choice(len(pts), 256, replace=False)
    sampled_check(mesh, pts, phi, E, sidx, 1e-6, 100.0)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
def test_degenerate_thin_elements(bem, prec, tol):
    """Triangles and rectangles with side ratios up to 1:200, points from DR 0.2 to 1e4."""
    rng = np.random.default_rng(13)
    verts, types = [], []
    for k in range(40):
        ratio = 10.0 ** rng.uniform(1, 2.3)
        c = rng.uniform(-1, 1, 3)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        w = np.cross(u, rng.normal(size=3))
        w /= np.linalg.norm(w)
        a, b = 0.2, 0.2 / ratio
        if k % 2:
            types.append(1)
            verts.append([c, c + a * u, c + a * u + b * w, c + b * w])
        else:
            types.append(0)
            verts.append([c, c + a * u, c + 0.5 * a * u + b * w, np.zeros(3)])
    types = np.array(types, np.int32)
    verts = np.array(verts)
    sigma = rng.uniform(0.5, 1.5, len(types))
    pts = rng.normal(size=(3000, 3)) * np.geomspace(0.01, 50.0, 3000)[:, None]
    rphi, rE, mdr = oracle.eval_field(types, verts, sigma, pts, return_min_dr=True)
    with bem.Mesh(types, verts, sigma, precision=prec) as m:
        phi, E = m.eval(pts)
    far = mdr >= 3
    assert rel_phi(phi, rphi)[far].max() <= tol and rel_E(E, rE)[far].max() <= tol
    near_tol = tol if prec == 0 else 1e-5
    assert rel_phi(phi, rphi)[~far].max() <= near_tol and rel_E(E, rE)[~far].max() <= near_tol


def test_coax_150k_gradient_mixed(bem):
    """The mixed gradient at the size bench.py times it (262 144 points of the
    150 000-element mesh), sampled against the oracle.  Its bar: FP32 rounding
    of each element's tensor, |dG| <= 1e-7 sum_j max|G_j| at every sampled
    point, and <= 2e-6 max|G| where min DR >= 3 and kappa_G <= 100."""
    import torch
    mesh = synth.coax_mesh(seed=2)
    pts = synth.coax_points(seed=2, n=1_000_000)[:262_144]
    dev = torch.device("cuda")
    with bem.Mesh(torch.from_numpy(mesh.types).to(dev), torch.from_numpy(mesh.verts).to(dev),
                  torch.from_numpy(mesh.sigma).to(dev), precision=bem.MIXED) as m:
        p_d = torch.from_numpy(pts).to(dev)
        G = torch.empty((len(pts), 6), dtype=torch.float64, device=dev)
        bem.bem_eval_grad(m.handle, p_d, G)
        torch.cuda.synchronize()
        G = G.cpu().numpy()
    idx = np.random.default_rng(14).choice(len(pts), 32, replace=False)
    ref, gsum = oracle.eval_grad(mesh.types, mesh.verts, mesh.sigma, pts[idx], return_gsum=True)
    _, _, mdr = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts[idx], return_min_dr=True)
    d = np.abs(G[idx] - ref).max(axis=1)
    assert (d / gsum).max() <= 1e-7
    kap = gsum / np.abs(ref).max(axis=1)
    gate = (mdr >= 3) & (kap <= 100)
    assert gate.sum() >= 16
    assert (d / np.abs(ref).max(axis=1))[gate].max() <= 2e-6


def test_coax_150k_1M_quadratic(bem):
    """Quadratic densities on the full 150 000 x 1 000 000 workload, sampled."""
    import torch
    mesh = synth.coax_mesh(seed=2)
    pts = synth.coax_points(seed=2, n=1_000_000)
    rng = np.random.default_rng(31)
    coef = np.concatenate([mesh.sigma[:, None], (rng.normal(0.0, 0.15, (2, mesh.n)) * mesh.sigma).T,
                           (rng.normal(0.0, 0.05, (3, mesh.n)) * mesh.sigma).T], axis=1)
    dev = torch.device("cuda")
    with bem.Mesh(torch.from_numpy(mesh.types).to(dev), torch.from_numpy(mesh.verts).to(dev),
                  torch.from_numpy(mesh.sigma).to(dev), precision=bem.MIXED) as m:
        m.set_sigma_quadratic(coef)
        p_d = torch.from_numpy(pts).to(dev)
        phi = torch.empty(len(pts), dtype=torch.float64, device=dev)
        E = torch.empty((len(pts), 3), dtype=torch.float64, device=dev)
        bem.bem_eval(m.handle, p_d, phi, E)
        torch.cuda.synchronize()
        phi, E = phi.cpu().numpy(), E.cpu().numpy()
    idx = np.random.default_rng(15).choice(len(pts), 32, replace=False)
    rphi, rE = oracle.eval_quad(mesh.types, mesh.verts, coef, pts[idx])
    _, cE, mdr, esum = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts[idx], return_min_dr=True,
                                         return_esum=True)
    gate = (mdr >= 3) & (esum / np.linalg.norm(cE, axis=1) <= 100)
    assert gate.sum() >= 16
    assert rel_phi(phi[idx], rphi)[gate].max() <= 1e-6
    assert rel_E(E[idx], rE)[gate].max() <= 1e-6


def test_sphere_cylinder_20k_assembly_matvec_solve(bem):
    """The 20 000-element collocation workload bench.py times: the dense
    20 000 x 20 000 matrix (both precisions) on sampled rows, the matrix-free
    product on the same rows, and the refined and mixed solves checked by the
    oracle's own rows."""
    import torch
    mesh = synth.sphere_cylinder_mesh(seed=3)
    col = synth.collocation_points(mesh)
    dev = torch.device("cuda")
    rows = [0, 9_999, 17_999, 18_000, 19_999]
    ref = np.concatenate([oracle.assemble(mesh.types, mesh.verts, col, rows=(r, r + 1)) for r in rows])
    x = mesh.sigma
    rhs = np.where(mesh.types == 0, 1.0, 0.0)
    for prec, tol in ((bem.FP64, 1e-12), (bem.MIXED, 1e-6)):
        with bem.Mesh(torch.from_numpy(mesh.types).to(dev), torch.from_numpy(mesh.verts).to(dev),
                      torch.from_numpy(mesh.sigma).to(dev), precision=prec) as m:
            A = torch.empty((mesh.n, mesh.n), dtype=torch.float64, device=dev)
            bem.bem_assemble(m.handle, torch.from_numpy(col).to(dev), A)
            torch.cuda.synchronize()
            Ar = A[rows].cpu().numpy()
            del A
            assert (np.abs(Ar - ref) / np.abs(ref)).max() <= tol
            y = m.matvec(x)
            assert (np.abs(y[rows] - ref @ x) / np.abs(ref @ x)).max() <= tol
            if prec == bem.FP64:
                sig, info = m.solve(rhs, refine=True)
                bar = 1e-9  # relative residual ~1e-12 of |rhs| = 134, plus the FP64 parity of the rows
            else:
                sig, info = m.solve(rhs)
                bar = 2e-4  # relative residual 1e-6 of |rhs|, plus 1e-6 of each row's terms
            assert info["converged"]
            # the oracle's rows of A sigma reproduce the prescribed potentials
            assert np.abs(ref @ sig - rhs[rows]).max() <= bar
