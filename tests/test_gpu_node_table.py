"""The precomputed-node variant (BEM_FLAG_NODE_TABLE, the precomputed
Gaussian points of the paper's Sec. 6, Table 4): the same parity bar as the
on-the-fly mixed path, bit-for-bit batch independence, agreement with the
on-the-fly path to FP32 rounding, and assembly / matrix-free product."""
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


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    if a.ndim == 1:
        return np.abs(a - b) / np.abs(b)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


@pytest.mark.parametrize("case", ["plate", "bands", "ragged"])
def test_parity(bem, case):
    if case == "plate":
        mesh, pts = synth.plate_mesh(seed=1), synth.plate_points(seed=1)
    elif case == "bands":
        mesh = synth.plate_mesh(seed=2, n=4)
        rng = np.random.default_rng(2)
        pts = synth.random_directions(3000, seed=2) * np.geomspace(0.02, 700.0, 3000)[:, None]
        pts += rng.uniform(-0.5, 0.5, (3000, 3)) * [1, 1, 0]
        pts[np.abs(pts[:, 2]) < 0.01, 2] = 0.01
    else:
        mesh, pts = synth.plate_mesh(seed=3, n=5), synth.plate_points(seed=3, n=1000)
    rphi, rE, hist, mdr = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts, return_hist=True,
                                            return_min_dr=True)
    if case == "bands":
        assert (hist > 0).all()
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.MIXED, node_table=True) as m:
        phi, E = m.eval(pts)
    far = mdr >= 3.0
    assert rel(phi, rphi)[far].max() <= 1e-6 and rel(E, rE)[far].max() <= 1e-6
    assert rel(phi, rphi)[~far].max(initial=0) <= 1e-5 and rel(E, rE)[~far].max(initial=0) <= 1e-5


def test_batch_independence_and_agreement_with_on_the_fly(bem):
    mesh = synth.plate_mesh(seed=1)
    pts = synth.plate_points(seed=5, n=3000)
    idx = np.array([0, 17, 1234, 2999])
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.MIXED, node_table=True) as m:
        phi, E = m.eval(pts)
        phi2, E2 = m.eval(pts[idx])
        phi3, E3 = m.eval(pts)
    assert np.array_equal(phi[idx], phi2) and np.array_equal(E[idx], E2)
    assert np.array_equal(phi, phi3) and np.array_equal(E, E3)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.MIXED) as m:
        fphi, fE = m.eval(pts)
    assert rel(phi, fphi).max() <= 1e-6 and rel(E, fE).max() <= 1e-6


def test_assembly_and_matvec(bem):
    mesh = synth.sphere_cylinder_mesh(seed=3, freq=6, n_phi=8, n_z=10)
    col = synth.collocation_points(mesh)
    ref = oracle.assemble(mesh.types, mesh.verts, col)
    x = mesh.sigma
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.MIXED, node_table=True) as m:
        A = m.assemble(col)
        y = m.matvec(x)
    assert (np.abs(A - ref) / np.abs(ref)).max() <= 1e-6
    assert rel(y, ref @ x).max() <= 1e-6


def test_flag_on_fp64_mesh_changes_nothing(bem):
    mesh = synth.plate_mesh(seed=1, n=8)
    pts = synth.plate_points(seed=6, n=500)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.FP64, node_table=True) as m:
        phi, E = m.eval(pts)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.FP64) as m:
        phi2, E2 = m.eval(pts)
    assert np.array_equal(phi, phi2) and np.array_equal(E, E2)


def test_unknown_flag_rejected(bem):
    mesh = synth.plate_mesh(seed=1, n=2)
    with pytest.raises(bem.BemError):
        bem.bem_create(mesh.types, mesh.verts, mesh.sigma, bem.MIXED, flags=4)
