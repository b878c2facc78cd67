"""Pins of the collocation system that bem_solve solves, on the oracle side:
the oracle's assembled matrix (Sec. 1 / Sec. 5 context: the linear system for
the charge densities) solved by a library routine reproduces the closed-form
capacitance of a sphere, C = 4 pi eps0 R, with the O(h^2) convergence of
flat constant-density elements."""
import math

import numpy as np
import pytest

import oracle
import synth


def _sphere_charge(freq, R=1.0, V=1.0):
    types, verts = synth._concat([synth.icosphere_triangles(R, freq)])
    mesh = synth.Mesh(types, verts, np.ones(types.shape[0]))
    col = synth.collocation_points(mesh)
    A = oracle.assemble(types, verts, col)
    sigma = np.linalg.solve(A, np.full(types.shape[0], V))
    area = np.array([oracle.element_geometry(0, v[:3])["area"] for v in verts])
    return float(sigma @ area)


def test_sphere_capacitance_converges():
    exact = 4.0 * math.pi * oracle.EPS0_SI * 1.0 * 1.0  # Q = C V
    e4 = abs(_sphere_charge(4) - exact) / exact
    e8 = abs(_sphere_charge(8) - exact) / exact
    assert e8 < 1e-2
    assert e8 < e4 / 2.5  # second order in the element size


def test_uniform_density_on_sphere():
    """By symmetry the exact density on a sphere at constant potential is
    uniform, eps0 V / R; the discrete solution's spread shrinks with the mesh."""
    types, verts = synth._concat([synth.icosphere_triangles(1.0, 6)])
    mesh = synth.Mesh(types, verts, np.ones(types.shape[0]))
    A = oracle.assemble(types, verts, synth.collocation_points(mesh))
    sigma = np.linalg.solve(A, np.ones(types.shape[0]))
    ref = oracle.EPS0_SI
    assert abs(np.median(sigma) - ref) / ref < 2e-2
    assert (sigma.max() - sigma.min()) / ref < 0.1
