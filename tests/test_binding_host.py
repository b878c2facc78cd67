"""Host-side helpers of the Python binding (no GPU): the linear-density
coefficients from corner values reproduce those values at the corners."""
import numpy as np

import paper_1606_03743_gb300 as bem
import synth


def test_linear_coef_from_corner_values_reproduces_corners():
    mesh = synth.plate_mesh(seed=1, n=3)
    rng = np.random.default_rng(5)
    a, c0 = rng.normal(size=3), 1.3
    vals = c0 + mesh.verts @ a  # a density linear in space: planar corner values
    coef = bem.linear_coef_from_corner_values(mesh.types, vals)
    for t, v, cf, val in zip(mesh.types, mesh.verts, coef, vals):
        if t == bem.TRIANGLE:  # (alpha, beta) at A, B, C = (1, 0), (0, 1), (-1, -1)
            ab = np.array([[1, 0], [0, 1], [-1, -1]])
            want = val[:3]
        else:  # natural coordinates of P0..P3
            ab = np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]])
            want = val
        got = cf[0] + ab @ cf[1:]
        assert np.allclose(got, want, rtol=1e-14, atol=1e-14)


def test_linear_coef_triangle_mean():
    coef = bem.linear_coef_from_corner_values(np.array([0], np.int32), np.array([[0.3, 1.9, -0.4, 0.0]]))
    m = (0.3 + 1.9 - 0.4) / 3
    assert np.allclose(coef, [[m, 0.3 - m, 1.9 - m]], rtol=1e-15)
