"""Parity of bem_eval_grad (field gradient dE_i/dx_j, FP64 far kernel in its
gradient mode + analytic near-field gradient) with the FP64 oracle."""
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


def rel(G, R):
    """per point: largest component error over the largest component"""
    return np.abs(G - R).max(axis=1) / np.abs(R).max(axis=1)


@pytest.mark.parametrize("case", ["plate", "bands"])
def test_gradient_parity(bem, case):
    if case == "plate":
        mesh, pts = synth.plate_mesh(seed=1), synth.plate_points(seed=1, n=2048)
    else:
        mesh = synth.plate_mesh(seed=2, n=4)
        rng = np.random.default_rng(2)
        pts = synth.random_directions(2000, seed=2) * np.geomspace(0.02, 700.0, 2000)[:, None]
        pts += rng.uniform(-0.5, 0.5, (2000, 3)) * [1, 1, 0]
        pts[np.abs(pts[:, 2]) < 0.01, 2] = 0.01
    ref = oracle.eval_grad(mesh.types, mesh.verts, mesh.sigma, pts)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.FP64) as m:
        G = m.eval_grad(pts)
    assert G.shape == (len(pts), 6)
    assert rel(G, ref).max() <= 1e-11
    # Laplace: traceless off the elements
    assert (np.abs(G[:, 0] + G[:, 1] + G[:, 2]) / np.abs(G).max(axis=1)).max() <= 1e-11


def test_gradient_is_derivative_of_field(bem):
    """Central differences of the library's own E (FP64) agree with its gradient."""
    mesh = synth.plate_mesh(seed=1, n=8)
    pts = synth.plate_points(seed=7, n=200, zmin=0.2)
    h = 1e-5
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.FP64) as m:
        G = m.eval_grad(pts)
        for j, (a, b) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
            e = np.zeros(3)
            e[b] = h
            Ep = m.eval(pts + e)[1][:, a]
            Em = m.eval(pts - e)[1][:, a]
            fd = (Ep - Em) / (2 * h)
            assert (np.abs(G[:, j] - fd) / np.abs(G).max(axis=1)).max() <= 1e-6


def test_batch_independence(bem):
    mesh = synth.plate_mesh(seed=1)
    pts = synth.plate_points(seed=5, n=1500)
    idx = np.array([0, 17, 999, 1499])
    for prec in (bem.FP64, bem.MIXED):
        with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=prec) as m:
            G = m.eval_grad(pts)
            G2 = m.eval_grad(pts[idx])
            G3 = m.eval_grad(pts)
        assert np.array_equal(G[idx], G2) and np.array_equal(G, G3)


@pytest.mark.parametrize("case", ["plate", "bands", "ragged"])
def test_mixed_gradient_parity(bem, case):
    """The mixed far sums (FP32 node terms, frame-form rebuild, hi + lo running
    sums) against the FP64 oracle: 1e-6 of the largest component where every
    element is beyond the near limit; near pairs are FP64."""
    if case == "plate":
        mesh, pts = synth.plate_mesh(seed=1), synth.plate_points(seed=1, n=2048)
    elif case == "bands":
        mesh = synth.plate_mesh(seed=2, n=4)
        rng = np.random.default_rng(2)
        pts = synth.random_directions(2000, seed=2) * np.geomspace(0.02, 700.0, 2000)[:, None]
        pts += rng.uniform(-0.5, 0.5, (2000, 3)) * [1, 1, 0]
        pts[np.abs(pts[:, 2]) < 0.01, 2] = 0.01
    else:
        mesh, pts = synth.plate_mesh(seed=3, n=5), synth.plate_points(seed=3, n=999)
    ref = oracle.eval_grad(mesh.types, mesh.verts, mesh.sigma, pts)
    _, _, hist, mdr = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts, return_hist=True,
                                        return_min_dr=True)
    if case == "bands":
        assert (hist > 0).all()
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.MIXED) as m:
        G = m.eval_grad(pts)
    far = mdr >= 3.0
    err = rel(G, ref)
    assert err[far].max() <= 1e-6
    assert err[~far].max(initial=0) <= 1e-5


def test_device_arrays_and_empty(bem):
    import torch
    mesh = synth.plate_mesh(seed=1, n=4)
    pts = synth.plate_points(seed=6, n=300)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=bem.FP64) as m:
        Gh = m.eval_grad(pts)
        Gd = m.eval_grad(torch.from_numpy(pts).cuda())
        assert Gd.is_cuda and np.array_equal(Gd.cpu().numpy(), Gh)
        assert m.eval_grad(np.zeros((0, 3))).shape == (0, 6)
