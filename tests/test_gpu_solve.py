"""Parity of bem_solve (restarted GMRES on bem_matvec) with a direct solve of
the oracle's collocation matrix, on an electrode problem: a sphere at 1 V
around an inner cylinder at 0 V."""
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


@pytest.fixture(scope="module")
def problem():
    mesh = synth.sphere_cylinder_mesh(seed=3, freq=6, n_phi=8, n_z=10)  # 720 triangles + 80 rectangles
    col = synth.collocation_points(mesh)
    A = oracle.assemble(mesh.types, mesh.verts, col)
    rhs = np.where(mesh.types == 0, 1.0, 0.0)  # sphere (triangles) at 1 V, cylinder at 0 V
    ref = np.linalg.solve(A, rhs)
    return mesh, A, rhs, ref


def test_fp64_solve_matches_direct_solve(bem, problem):
    mesh, A, rhs, ref = problem
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.FP64) as m:
        sigma, info = m.solve(rhs)
    assert info["converged"] and info["residual"] <= 1e-12
    assert np.abs(sigma - ref).max() / np.abs(ref).max() <= 1e-10
    # the residual against the oracle's own matrix
    assert np.linalg.norm(A @ sigma - rhs) / np.linalg.norm(rhs) <= 1e-11


def test_refined_solve_matches_direct_solve(bem, problem):
    """Mixed-precision inner solves with FP64 residuals reach the FP64 answer."""
    mesh, A, rhs, ref = problem
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.FP64) as m:
        sigma, info = m.solve(rhs, refine=True)
        plain, pinfo = m.solve(rhs)
    assert info["converged"] and info["residual"] <= 1e-12
    assert np.abs(sigma - ref).max() / np.abs(ref).max() <= 1e-10
    assert np.linalg.norm(A @ sigma - rhs) / np.linalg.norm(rhs) <= 1e-11
    assert np.abs(sigma - plain).max() / np.abs(ref).max() <= 1e-10


def test_mixed_solve_reaches_its_tolerance(bem, problem):
    mesh, A, rhs, ref = problem
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.MIXED) as m:
        sigma, info = m.solve(rhs)
    assert info["converged"] and info["residual"] <= 1e-6
    assert np.linalg.norm(A @ sigma - rhs) / np.linalg.norm(rhs) <= 2e-6
    assert np.abs(sigma - ref).max() / np.abs(ref).max() <= 1e-4


def test_device_arrays_and_repeatability(bem, problem):
    import torch
    mesh, A, rhs, ref = problem
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.FP64) as m:
        r_d = torch.from_numpy(rhs).cuda()
        s1, i1 = m.solve(r_d)
        s2, i2 = m.solve(r_d)
    assert s1.is_cuda and i1 == i2
    assert torch.equal(s1, s2)  # fixed-order reductions: the same bits
    assert np.abs(s1.cpu().numpy() - ref).max() / np.abs(ref).max() <= 1e-10


def test_initial_guess_and_iteration_limit(bem, problem):
    mesh, A, rhs, ref = problem
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.FP64) as m:
        # starting from the solution: converged at the first residual check
        sigma, info = m.solve(rhs, x0=ref, tol=1e-9)
        assert info["converged"] and info["products"] == 1
        # too few products for the tolerance: BEM_ERR_NOT_CONVERGED with the last iterate
        with pytest.raises(bem.BemError) as e:
            m.solve(rhs, max_iter=3, tol=1e-14)
        assert e.value.code == -7
        assert not e.value.info["converged"] and e.value.info["products"] <= 4
        # zero potentials: zero charge, no products
        sigma, info = m.solve(np.zeros(mesh.n))
        assert info["converged"] and not sigma.any()
        with pytest.raises(bem.BemError):
            m.solve(rhs, restart=1000)


def test_solution_reproduces_the_potentials(bem, problem):
    """Evaluating the solved densities at the centroids gives back the
    prescribed electrode potentials."""
    mesh, A, rhs, ref = problem
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.FP64) as m:
        sigma, info = m.solve(rhs)
        m.set_sigma(sigma)
        phi, _ = m.eval(synth.collocation_points(mesh), want_E=False)
    assert np.abs(phi - rhs).max() <= 1e-11
