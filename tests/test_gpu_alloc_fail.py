"""Device-allocation failures, injected on the host (include/bem_test.h).

Every call that allocates must return BEM_ERR_OOM when an allocation fails,
release what it had allocated, and leave the mesh usable: the next call,
with allocation working again, gives the same results as a mesh that never
saw the failure.  No GPU fault is involved: the hook makes the library's
allocation wrapper report cudaErrorMemoryAllocation without calling the
CUDA runtime.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

OOM = -2


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1606_03743_gb300 as bem
    lib = bem.load_library()
    lib.bem_test_fail_alloc_after.argtypes = [ctypes.c_int64]
    lib.bem_test_fail_alloc_after.restype = ctypes.c_int
    lib.bem_test_alloc_count.restype = ctypes.c_int64
    yield torch, bem, lib
    lib.bem_test_fail_alloc_after(-1)


class Inject:
    """Within the block, allocations after the first n fail."""

    def __init__(self, lib, n):
        self.lib, self.n = lib, n

    def __enter__(self):
        self.lib.bem_test_fail_alloc_after(self.n)

    def __exit__(self, *exc):
        self.lib.bem_test_fail_alloc_after(-1)


def _oom(bem, fn, *args, **kw):
    with pytest.raises(bem.BemError) as e:
        fn(*args, **kw)
    assert e.value.code == OOM, e.value
    return e.value


@pytest.mark.parametrize("prec,table", [(0, False), (1, False), (1, True)])
def test_create_fails_cleanly_at_every_allocation(env, prec, table):
    """bem_create with the k-th of its allocations failing, for every k:
    BEM_ERR_OOM each time, and a mesh created afterwards evaluates exactly
    like one created before (FP64, mixed, mixed with the node table)."""
    torch, bem, lib = env
    mesh = synth.plate_mesh(seed=1, n=4)
    pts = synth.plate_points(seed=2, n=300)
    c0 = lib.bem_test_alloc_count()
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=prec, node_table=table) as m:
        n_alloc = lib.bem_test_alloc_count() - c0
        ref = m.eval(pts)
    assert n_alloc >= 10
    for k in range(n_alloc):
        with Inject(lib, k):
            _oom(bem, bem.Mesh, mesh.types, mesh.verts, mesh.sigma, precision=prec, node_table=table)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=prec, node_table=table) as m:
        phi, E = m.eval(pts)
    assert np.array_equal(phi, ref[0]) and np.array_equal(E, ref[1])


@pytest.mark.parametrize("prec", [0, 1])
def test_eval_workspace_growth(env, prec):
    """bem_eval that must grow the point workspace: BEM_ERR_OOM, then the
    same call succeeds and matches the oracle (and the small batch that ran
    before still gives the same bits)."""
    torch, bem, lib = env
    mesh = synth.plate_mesh(seed=1, n=4)
    small = synth.plate_points(seed=3, n=200)
    big = synth.plate_points(seed=4, n=5000)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=prec) as m:
        phi0, E0 = m.eval(small)
        with Inject(lib, 0):
            _oom(bem, m.eval, big)
        phi, E = m.eval(big)
        phi1, E1 = m.eval(small)
    assert np.array_equal(phi0, phi1) and np.array_equal(E0, E1)
    rphi, rE = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, big)
    tol = 1e-12 if prec == 0 else 1e-5
    assert (np.abs(phi - rphi) / np.abs(rphi)).max() <= tol
    assert (np.linalg.norm(E - rE, axis=1) / np.linalg.norm(rE, axis=1)).max() <= tol


def test_assemble_host_output_buffer(env):
    """bem_assemble into a host array stages the matrix in a device buffer of
    its own: failing that allocation gives BEM_ERR_OOM; the retry matches
    the oracle."""
    torch, bem, lib = env
    mesh = synth.plate_mesh(seed=1, n=4)
    col = synth.collocation_points(mesh)[:40]
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma) as m:
        m.assemble(torch.from_numpy(col).cuda())  # sizes the point workspace
        torch.cuda.synchronize()
        with Inject(lib, 0):
            _oom(bem, m.assemble, col)
        A = m.assemble(col)
    ref = oracle.assemble(mesh.types, mesh.verts, col)
    assert np.abs(A - ref).max() <= 1e-12 * np.abs(ref).max()


def test_grad_scratch(env):
    """bem_eval_grad allocates its gradient partial sums per call."""
    torch, bem, lib = env
    mesh = synth.plate_mesh(seed=1, n=4)
    pts = synth.plate_points(seed=5, n=256)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma) as m:
        G0 = m.eval_grad(pts)
        with Inject(lib, 0):
            _oom(bem, m.eval_grad, pts)
        G1 = m.eval_grad(pts)
    assert np.array_equal(G0, G1)


def test_solve_buffers(env):
    """bem_solve allocates its Krylov basis per call."""
    torch, bem, lib = env
    mesh = synth.sphere_cylinder_mesh(seed=3, freq=3, n_phi=8, n_z=4)  # sphere at 1 V, inner cylinder at 0 V
    rhs = np.where(mesh.types == 0, 1.0, 0.0)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma) as m:
        s0, _ = m.solve(rhs)
        with Inject(lib, 0):
            _oom(bem, m.solve, rhs)
        s1, info = m.solve(rhs)
    assert info["converged"] and np.array_equal(s0, s1)


@pytest.mark.parametrize("kind", ["linear", "quadratic"])
def test_varying_density_buffers(env, kind):
    """bem_set_sigma_linear / _quadratic allocate the per-element
    coefficients on first use: on failure the mesh keeps its constant
    densities."""
    torch, bem, lib = env
    mesh = synth.plate_mesh(seed=1, n=4)
    pts = synth.plate_points(seed=6, n=200)
    ncoef = 3 if kind == "linear" else 6
    coef = np.zeros((mesh.n, ncoef))
    coef[:, 0] = mesh.sigma + 0.5
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma) as m:
        ref = m.eval(pts)
        setter = m.set_sigma_linear if kind == "linear" else m.set_sigma_quadratic
        with Inject(lib, 0):
            _oom(bem, setter, coef)
        phi, E = m.eval(pts)
        assert np.array_equal(phi, ref[0]) and np.array_equal(E, ref[1])
        setter(coef)
        phi2, _ = m.eval(pts)
    assert not np.array_equal(phi2, ref[0])


def test_server_create_fails_cleanly_at_every_allocation(env):
    """bem_server_create with the k-th of its device or pinned allocations
    failing, for every k: BEM_ERR_OOM each time; a server created afterwards
    returns bem_eval's results."""
    torch, bem, lib = env
    mesh = synth.plate_mesh(seed=1, n=4)
    pts = synth.plate_points(seed=7, n=300)
    with bem.Mesh(mesh.types, mesh.verts, mesh.sigma, precision=1) as m:
        ref = m.eval(pts)
        c0 = lib.bem_test_alloc_count()
        with bem.Server(m, max_points_per_tick=4096) as srv:
            n_alloc = lib.bem_test_alloc_count() - c0
            t = srv.submit(pts)
            srv.wait(t, timeout=60)
        assert n_alloc >= 10
        for k in range(n_alloc):
            with Inject(lib, k):
                _oom(bem, bem.Server, m, max_points_per_tick=4096)
        with bem.Server(m, max_points_per_tick=4096) as srv:
            t = srv.submit(pts)
            phi, E = srv.wait(t, timeout=60)
    assert np.array_equal(phi, ref[0]) and np.array_equal(E, ref[1])


def test_pointer_location(env):
    """Arrays are classified against the mesh's device: device memory of that
    device is used in place, host memory is staged, and another GPU's memory
    is rejected (checked here by asking about device 0's memory on behalf of
    a mesh on device 1, which needs no second GPU)."""
    torch, bem, lib = env
    lib.bem_test_ptr_location.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    lib.bem_test_ptr_location.restype = ctypes.c_int32
    d = torch.zeros(16, dtype=torch.float64, device="cuda:0")
    h = np.zeros(16)
    pinned = torch.zeros(16, dtype=torch.float64).pin_memory()
    assert lib.bem_test_ptr_location(d.data_ptr(), 0) == 1
    assert lib.bem_test_ptr_location(d.data_ptr(), 1) == 2
    assert lib.bem_test_ptr_location(h.ctypes.data, 0) == 0
    assert lib.bem_test_ptr_location(pinned.data_ptr(), 0) == 0
