"""bem_eval_noalloc: the evaluation entry point for callers that cannot let
the library allocate device memory (an application that pre-reserves all
GPU memory for its own pool, or a tracking loop that must never wait on the
allocator).  Its scratch is a fixed device array, so it must give the same
results as bem_eval, call after call, even though the array keeps the
previous call's contents.

The file name makes pytest collect it last."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1606_03743_gb300 as bem
    bem.load_library()
    return torch, bem


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    if a.ndim == 1:
        return np.abs(a - b) / np.abs(b)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_eval_on_two_calls(env, prec):
    torch, bem = env
    mesh = synth.plate_mesh(seed=1)
    dev = torch.device("cuda", 0)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=prec) as m:
        for call, (seed, n) in enumerate([(11, 4096), (12, 3001)]):  # two calls in a row, different sizes
            pts = torch.from_numpy(synth.plate_points(seed=seed, n=n)).to(dev)
            ref_phi = torch.empty(n, dtype=torch.float64, device=dev)
            ref_E = torch.empty((n, 3), dtype=torch.float64, device=dev)
            bem.bem_eval(m.handle, pts, ref_phi, ref_E)
            phi = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
            E = torch.full((n, 3), float("nan"), dtype=torch.float64, device=dev)
            bem.bem_eval_noalloc(m.handle, pts, phi, E)
            torch.cuda.synchronize()
            ep = _rel(phi.cpu().numpy(), ref_phi.cpu().numpy())
            eE = _rel(E.cpu().numpy(), ref_E.cpu().numpy())
            assert ep.max() <= TOL[prec], (call, ep.max())
            assert eE.max() <= TOL[prec], (call, eE.max())


def test_noalloc_limits_and_host_arrays(env):
    torch, bem = env
    mesh = synth.plate_mesh(seed=1, n=4)
    dev = torch.device("cuda", 0)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma) as m:
        too_many = torch.zeros((bem.NOALLOC_MAX_POINTS + 1, 3), dtype=torch.float64, device=dev)
        with pytest.raises(bem.BemError) as e:
            bem.bem_eval_noalloc(m.handle, too_many, torch.empty(bem.NOALLOC_MAX_POINTS + 1, dtype=torch.float64,
                                                                     device=dev))
        assert e.value.code == -1 and "at most" in str(e.value)
        host = synth.plate_points(seed=3, n=10)
        with pytest.raises(bem.BemError) as e:
            bem.bem_eval_noalloc(m.handle, host, np.empty(10))
        assert e.value.code == -1 and "device arrays" in str(e.value)
        # a full-size call still works after the rejected ones
        pts = torch.from_numpy(synth.plate_points(seed=4, n=bem.NOALLOC_MAX_POINTS)).to(dev)
        phi = torch.empty(bem.NOALLOC_MAX_POINTS, dtype=torch.float64, device=dev)
        bem.bem_eval_noalloc(m.handle, pts, phi, None)
        ref = torch.empty_like(phi)
        bem.bem_eval(m.handle, pts, ref, None)
        assert _rel(phi.cpu().numpy(), ref.cpu().numpy()).max() <= 1e-12


def test_noalloc_near_capacity_overflow_then_recovers(env):
    """More near-field pairs than the fixed array holds (16 384 points hugging
    the plate, a few hundred near pairs each): BEM_ERR_CAPACITY, with every
    write kept inside the array; the next call of normal size matches
    bem_eval again, so the overflow left nothing behind."""
    torch, bem = env
    mesh = synth.plate_mesh(seed=1)
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(21)
    n = bem.NOALLOC_MAX_POINTS
    hug = np.stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.5, 0.5, n), rng.uniform(0.01, 0.05, n)], axis=1)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma) as m:
        ref_phi = torch.empty(n, dtype=torch.float64, device=dev)
        bem.bem_eval(m.handle, torch.from_numpy(hug).to(dev), ref_phi, None)
        assert m.last_stats()[12] > bem.NOALLOC_MAX_NEAR  # the case really overflows
        phi = torch.empty(n, dtype=torch.float64, device=dev)
        E = torch.empty((n, 3), dtype=torch.float64, device=dev)
        with pytest.raises(bem.BemError) as e:
            bem.bem_eval_noalloc(m.handle, torch.from_numpy(hug).to(dev), phi, E)
        assert e.value.code == -3  # BEM_ERR_CAPACITY
        pts = torch.from_numpy(synth.plate_points(seed=22, n=4000)).to(dev)
        ref = torch.empty(4000, dtype=torch.float64, device=dev)
        ref_E = torch.empty((4000, 3), dtype=torch.float64, device=dev)
        bem.bem_eval(m.handle, pts, ref, ref_E)
        phi2 = torch.empty(4000, dtype=torch.float64, device=dev)
        E2 = torch.empty((4000, 3), dtype=torch.float64, device=dev)
        bem.bem_eval_noalloc(m.handle, pts, phi2, E2)
        torch.cuda.synchronize()
    assert _rel(phi2.cpu().numpy(), ref.cpu().numpy()).max() <= 1e-12
    assert _rel(E2.cpu().numpy(), ref_E.cpu().numpy()).max() <= 1e-12
