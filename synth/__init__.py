"""Seeded synthetic inputs: element meshes, charge densities and field points.

This module is shared by the oracle tests, the CUDA parity tests and the
benchmark.  It only lays out geometry and draws random numbers; none of the
method's arithmetic (distance ratios, cubature nodes, potentials) lives here.

The paper measures on the KATRIN main-spectrometer meshes (1.5 M triangles or
rectangles, 3000 field points in a 9 m x 3.5 m cylinder, Sec. 5), which are
not available.  The workloads below stand in for them: mixed triangle and
rectangle meshes of electrode-like surfaces with 1e5-5e5 elements and field
points inside the electrodes.

Mesh arrays (numpy):
  types  int32   (n,)      0 = triangle, 1 = rectangle
  verts  float64 (n, 4, 3) triangle corners A, B, C (4th row zero);
                           rectangle corners P0, P1, P2, P3 around the
                           boundary, side a = P0->P1, side b = P0->P3
  sigma  float64 (n,)      constant charge density per element
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

TRI = 0
RECT = 1


@dataclass
class Mesh:
    types: np.ndarray
    verts: np.ndarray
    sigma: np.ndarray

    @property
    def n(self) -> int:
        return int(self.types.shape[0])

    def subset(self, idx) -> "Mesh":
        return Mesh(self.types[idx].copy(), self.verts[idx].copy(), self.sigma[idx].copy())


def _concat(parts) -> tuple[np.ndarray, np.ndarray]:
    types = np.concatenate([p[0] for p in parts]).astype(np.int32)
    verts = np.concatenate([p[1] for p in parts]).astype(np.float64)
    return types, verts


# ---------------------------------------------------------------- primitives
def plate_rectangles(nx: int, ny: int, x0=-0.5, x1=0.5, y0=-0.5, y1=0.5, z=0.0):
    """nx x ny axis-aligned rectangles tiling [x0,x1] x [y0,y1] at height z."""
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    v = np.zeros((nx * ny, 4, 3))
    k = 0
    for j in range(ny):
        for i in range(nx):
            v[k, 0] = (xs[i], ys[j], z)
            v[k, 1] = (xs[i + 1], ys[j], z)
            v[k, 2] = (xs[i + 1], ys[j + 1], z)
            v[k, 3] = (xs[i], ys[j + 1], z)
            k += 1
    return np.full(nx * ny, RECT, np.int32), v


def plate_triangles(nx: int, ny: int, x0=-0.5, x1=0.5, y0=-0.5, y1=0.5, z=0.0):
    """nx x ny squares, each split along its (x+, y+) diagonal into two right
    triangles (2 nx ny triangles)."""
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    v = np.zeros((2 * nx * ny, 4, 3))
    k = 0
    for j in range(ny):
        for i in range(nx):
            a = (xs[i], ys[j], z)
            b = (xs[i + 1], ys[j], z)
            c = (xs[i + 1], ys[j + 1], z)
            d = (xs[i], ys[j + 1], z)
            v[k, 0], v[k, 1], v[k, 2] = a, b, c
            v[k + 1, 0], v[k + 1, 1], v[k + 1, 2] = a, c, d
            k += 2
    return np.full(2 * nx * ny, TRI, np.int32), v


def cylinder_rectangles(radius: float, n_phi: int, n_z: int, z0: float, z1: float):
    """Flat rectangles with their corners on a cylinder: n_phi azimuthal x n_z
    axial; side a is the chord, side b is along z."""
    ph = np.linspace(0.0, 2.0 * math.pi, n_phi + 1)
    zs = np.linspace(z0, z1, n_z + 1)
    c, s = np.cos(ph), np.sin(ph)
    c[-1], s[-1] = c[0], s[0]
    i, j = np.meshgrid(np.arange(n_phi), np.arange(n_z), indexing="xy")
    i, j = i.ravel(), j.ravel()
    v = np.zeros((n_phi * n_z, 4, 3))
    v[:, 0] = np.stack([radius * c[i], radius * s[i], zs[j]], -1)
    v[:, 1] = np.stack([radius * c[i + 1], radius * s[i + 1], zs[j]], -1)
    v[:, 2] = np.stack([radius * c[i + 1], radius * s[i + 1], zs[j + 1]], -1)
    v[:, 3] = np.stack([radius * c[i], radius * s[i], zs[j + 1]], -1)
    return np.full(n_phi * n_z, RECT, np.int32), v


def disc_triangles(radius: float, n_sector: int, n_ring: int, z: float):
    """Disc of radius `radius` at height z: n_ring rings; the innermost ring
    is n_sector triangles around the centre, every outer ring is n_sector
    trapezoids split into two triangles (n_sector * (2 n_ring - 1) total)."""
    ph = np.linspace(0.0, 2.0 * math.pi, n_sector + 1)
    c, s = np.cos(ph), np.sin(ph)
    c[-1], s[-1] = c[0], s[0]
    rs = np.linspace(0.0, radius, n_ring + 1)
    out = []
    i = np.arange(n_sector)
    # innermost ring: centre + two points on the first circle
    v = np.zeros((n_sector, 4, 3))
    v[:, 0] = (0.0, 0.0, z)
    v[:, 1] = np.stack([rs[1] * c[i], rs[1] * s[i], np.full(n_sector, z)], -1)
    v[:, 2] = np.stack([rs[1] * c[i + 1], rs[1] * s[i + 1], np.full(n_sector, z)], -1)
    out.append(v)
    for k in range(1, n_ring):
        r0, r1 = rs[k], rs[k + 1]
        a = np.stack([r0 * c[i], r0 * s[i], np.full(n_sector, z)], -1)
        b = np.stack([r1 * c[i], r1 * s[i], np.full(n_sector, z)], -1)
        cc = np.stack([r1 * c[i + 1], r1 * s[i + 1], np.full(n_sector, z)], -1)
        d = np.stack([r0 * c[i + 1], r0 * s[i + 1], np.full(n_sector, z)], -1)
        t1 = np.zeros((n_sector, 4, 3))
        t2 = np.zeros((n_sector, 4, 3))
        t1[:, 0], t1[:, 1], t1[:, 2] = a, b, cc
        t2[:, 0], t2[:, 1], t2[:, 2] = a, cc, d
        out.append(t1)
        out.append(t2)
    v = np.concatenate(out)
    return np.full(v.shape[0], TRI, np.int32), v


def icosphere_triangles(radius: float, freq: int):
    """Geodesic icosahedral sphere: each of the 20 faces split into freq^2
    triangles, vertices projected onto the sphere (20 freq^2 triangles)."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    base = np.array([(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
                     (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)], float)
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    tris = []
    for (ia, ib, ic) in faces:
        A, B, C = base[ia], base[ib], base[ic]

        def p(i, j):
            q = A + (B - A) * (i / freq) + (C - A) * (j / freq)
            return radius * q / np.linalg.norm(q)

        for i in range(freq):
            for j in range(freq - i):
                tris.append((p(i, j), p(i + 1, j), p(i, j + 1)))
                if i + j < freq - 1:
                    tris.append((p(i + 1, j), p(i + 1, j + 1), p(i, j + 1)))
    v = np.zeros((len(tris), 4, 3))
    v[:, :3] = np.array(tris)
    return np.full(len(tris), TRI, np.int32), v


# ---------------------------------------------------------------- workloads
def plate_mesh(seed: int = 1, n: int = 16) -> Mesh:
    """Flat unit square plate in z = 0: n x n rectangles plus 2 n^2 right
    triangles (a second n x n grid of the same plate, each square split in
    two); sigma ~ U[0.5, 1.5] per element, rectangles first."""
    rng = np.random.default_rng(seed)
    types, verts = _concat([plate_rectangles(n, n), plate_triangles(n, n)])
    sigma = rng.uniform(0.5, 1.5, types.shape[0])
    return Mesh(types, verts, sigma)


def plate_points(seed: int = 1, n: int = 4096, zmin: float = 0.05) -> np.ndarray:
    """Field points uniform in [-2, 2]^3, resampled until |z| >= zmin."""
    rng = np.random.default_rng(seed + 1000)
    pts = rng.uniform(-2.0, 2.0, (n, 3))
    bad = np.abs(pts[:, 2]) < zmin
    while bad.any():
        pts[bad] = rng.uniform(-2.0, 2.0, (int(bad.sum()), 3))
        bad = np.abs(pts[:, 2]) < zmin
    return pts


def coax_mesh(seed: int = 2, n_phi: int = 200, n_z: int = 250, n_ring: int = 63,
              r_in: float = 1.0, r_out: float = 1.2, half_len: float = 2.0) -> Mesh:
    """Coaxial cylinder electrodes (radii r_in and r_out, length 2 half_len),
    each n_phi x n_z flat rectangles, plus the two end-cap discs closing the
    inner cylinder (n_phi sectors x n_ring rings of triangles each);
    sigma ~ N(1, 0.2).  Defaults: 100 k rectangles + 50 k triangles."""
    rng = np.random.default_rng(seed)
    types, verts = _concat([
        cylinder_rectangles(r_in, n_phi, n_z, -half_len, half_len),
        cylinder_rectangles(r_out, n_phi, n_z, -half_len, half_len),
        disc_triangles(r_in, n_phi, n_ring, -half_len),
        disc_triangles(r_in, n_phi, n_ring, half_len),
    ])
    sigma = rng.normal(1.0, 0.2, types.shape[0])
    return Mesh(types, verts, sigma)


def coax_points(seed: int = 2, n: int = 1_000_000, r_max: float = 0.95, z_max: float = 1.9) -> np.ndarray:
    """Field points area-uniform in the disc r < r_max times z in [-z_max, z_max]."""
    rng = np.random.default_rng(seed + 1000)
    r = r_max * np.sqrt(rng.uniform(0.0, 1.0, n))
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    z = rng.uniform(-z_max, z_max, n)
    return np.stack([r * np.cos(ph), r * np.sin(ph), z], -1)


def coax_mesh_large(seed: int = 4) -> Mesh:
    """The coaxial mesh scaled to 500 k elements: 400 x 500 rectangles per
    cylinder (400 k), end caps of 400 sectors x 63 rings (100 k triangles)."""
    return coax_mesh(seed, n_phi=400, n_z=500, n_ring=63)


def sphere_cylinder_mesh(seed: int = 3, freq: int = 30, n_phi: int = 40, n_z: int = 50) -> Mesh:
    """BEM assembly workload: geodesic sphere of radius 1 (20 freq^2
    triangles) plus an inner coaxial cylinder of radius 0.3, z in [-0.6, 0.6]
    (n_phi x n_z rectangles).  Defaults: 18 000 + 2 000 = 20 000 elements;
    sigma ~ N(1, 0.2) (used by the matrix-free product)."""
    rng = np.random.default_rng(seed)
    types, verts = _concat([
        icosphere_triangles(1.0, freq),
        cylinder_rectangles(0.3, n_phi, n_z, -0.6, 0.6),
    ])
    sigma = rng.normal(1.0, 0.2, types.shape[0])
    return Mesh(types, verts, sigma)


def collocation_points(mesh: Mesh) -> np.ndarray:
    """Collocation points at the element centroids (vertex means): the usual
    choice for constant-density BEM elements."""
    nv = np.where(mesh.types == TRI, 3, 4)[:, None]
    s = mesh.verts.sum(axis=1)
    return s / nv


def helix_requests(seed: int = 5, n_req: int = 10_000, min_size: int = 1, max_size: int = 100_000,
                   r_max: float = 0.95, z_max: float = 1.9):
    """Query batches for the serving workload: sizes floor(10^U[0,5]) clipped
    to [min_size, max_size], each batch the successive positions of one
    charged-particle-like helical track inside r < r_max, |z| < z_max.
    Returns a list of (n_i, 3) float64 arrays."""
    rng = np.random.default_rng(seed)
    sizes = np.clip(np.floor(10.0 ** rng.uniform(0.0, 5.0, n_req)).astype(np.int64), min_size, max_size)
    out = []
    for n in sizes:
        r0 = rng.uniform(0.1, 0.9)
        rc = rng.uniform(0.0, min(r0, r_max - r0))  # gyration radius keeps the track inside
        cx, cy = (r0 - rc) * math.cos(ph0 := rng.uniform(0, 2 * math.pi)), (r0 - rc) * math.sin(ph0)
        omega = rng.uniform(0.5, 5.0) * (1 if rng.uniform() < 0.5 else -1)
        vz = rng.uniform(-1.0, 1.0)
        z0 = rng.uniform(-z_max, z_max)
        t = np.linspace(0.0, 2.0, int(n))
        ph = rng.uniform(0, 2 * math.pi) + omega * t
        z = z0 + vz * t
        # reflect z into [-z_max, z_max]
        span = 2.0 * z_max
        z = np.abs(np.mod(z + z_max, 2 * span) - span) - z_max
        out.append(np.stack([cx + rc * np.cos(ph), cy + rc * np.sin(ph), z], -1))
    return out


def random_elements(type_: int, n: int, seed: int = 0) -> np.ndarray:
    """n random elements with corners inside the unit cube (the element
    generator of the paper's accuracy experiments, Sec. 2 and Sec. 4).
    Triangles: three uniform corners.  Rectangles: P0, P1 uniform; a third
    uniform point X fixes the second side, P3 = P0 + the part of X - P0
    orthogonal to P1 - P0, P2 = P1 + P3 - P0.  Returns verts (n, 4, 3)."""
    rng = np.random.default_rng(seed)
    v = np.zeros((n, 4, 3))
    if type_ == TRI:
        v[:, :3] = rng.uniform(0.0, 1.0, (n, 3, 3))
        return v
    p0 = rng.uniform(0.0, 1.0, (n, 3))
    p1 = rng.uniform(0.0, 1.0, (n, 3))
    x = rng.uniform(0.0, 1.0, (n, 3))
    ux = (p1 - p0) / np.linalg.norm(p1 - p0, axis=1, keepdims=True)
    w = x - p0
    w -= (w * ux).sum(1, keepdims=True) * ux
    v[:, 0], v[:, 1], v[:, 3] = p0, p1, p0 + w
    v[:, 2] = p1 + w
    return v


def random_directions(n: int, seed: int = 0) -> np.ndarray:
    """n unit vectors uniform on the sphere."""
    rng = np.random.default_rng(seed + 7919)
    d = rng.normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)
