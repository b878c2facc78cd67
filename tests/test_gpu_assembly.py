"""Parity of the collocation matrix (bem_assemble) and of the matrix-free
product (bem_matvec) with the FP64 oracle."""
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
def mesh():
    # 720 triangles on a sphere + 80 rectangles on an inner cylinder
    return synth.sphere_cylinder_mesh(seed=3, freq=6, n_phi=8, n_z=10)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
def test_assembly_parity(bem, mesh, prec, tol):
    col = synth.collocation_points(mesh)
    ref = oracle.assemble(mesh.types, mesh.verts, col)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=prec) as m:
        A = m.assemble(col)
    assert A.shape == ref.shape
    # entrywise relative error (every entry is a positive potential coefficient)
    err = np.abs(A - ref) / np.abs(ref)
    assert err.max() <= tol, err.max()
    # the self terms (analytic, point on its own element) are the row maxima
    assert np.array_equal(np.argmax(A, axis=1), np.arange(mesh.n))


def test_assembly_rows_subset_and_device_output(bem, mesh):
    import torch
    col = synth.collocation_points(mesh)
    rows = np.array([5, 77, 400, 799])
    ref = oracle.assemble(mesh.types, mesh.verts, col[rows])
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma) as m:
        A = m.assemble(torch.from_numpy(col[rows]).cuda())
        assert A.is_cuda
        A = A.cpu().numpy()
    assert np.max(np.abs(A - ref) / np.abs(ref)) <= 1e-12


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
def test_matvec_parity(bem, mesh, prec, tol):
    rng = np.random.default_rng(17)
    x = rng.normal(1.0, 0.2, mesh.n)
    col = synth.collocation_points(mesh)
    ref, _ = oracle.eval_field(mesh.types, mesh.verts, x, col)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=prec) as m:
        y = m.matvec(x)
        # the mesh's own sigma is untouched by a matvec
        phi_mesh, _ = m.eval(col[:3])
    assert np.max(np.abs(y - ref) / np.abs(ref)) <= tol
    ref_mesh, _ = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, col[:3])
    assert np.max(np.abs(phi_mesh - ref_mesh) / np.abs(ref_mesh)) <= tol


def test_matvec_equals_assembled_matrix_times_x(bem, mesh):
    rng = np.random.default_rng(18)
    x = rng.normal(1.0, 0.2, mesh.n)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=0) as m:
        A = m.assemble(synth.collocation_points(mesh))
        y = m.matvec(x)
    assert np.max(np.abs(A @ x - y) / np.abs(y)) <= 1e-12


def test_set_sigma_changes_eval(bem, mesh):
    col = synth.collocation_points(mesh)[:50]
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=0) as m:
        phi1, _ = m.eval(col)
        m.set_sigma(2.0 * mesh.sigma)
        phi2, _ = m.eval(col)
    assert np.allclose(phi2, 2.0 * phi1, rtol=1e-14, atol=0)
