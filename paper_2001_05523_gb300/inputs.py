"""Seeded synthetic inputs: surface meshes and right-hand sides.

This module holds no arithmetic of the boundary element method itself. It only
produces the geometry and the random densities that both the CUDA path and the
CPU oracle consume, so that the two see identical inputs.

Meshes (all triangles oriented counter-clockwise seen from outside, so the
normal (b-a)x(c-a) points out of the enclosed body):

* ``sphere(s)``: the eight faces of the double pyramid |x1|+|x2|+|x3| = 1 are
  each split regularly into s*s congruent triangles, then every vertex is
  projected once onto the unit sphere (the construction of the paper's first
  experiment, section 5).  n = 8 s^2 triangles, 4 s^2 + 2 vertices.
* ``ellipsoid(s, axes)``: the sphere mesh scaled by the semi-axes.
* ``cube(s)``: the unit cube [0,1]^3, each face an s*s grid of squares, each
  square split into two triangles along its (0,0)-(1,1) diagonal.
  n = 12 s^2 triangles.
* ``jitter(mesh, frac, seed)``: every vertex moved by an independent uniform
  offset in [-frac*h, frac*h]^3 with h the mean edge length of the mesh.

Right-hand sides: ``rhs(n, nrhs, seed)`` draws N(0,1) samples with numpy's
PCG64 generator, shape (nrhs, n) (one row per right-hand side, i.e. the
column-major n x nrhs layout with leading dimension n).
"""
from __future__ import annotations

import dataclasses

import numpy as np

BASE_SEED = 20010552


@dataclasses.dataclass
class Mesh:
    """Triangulated closed surface: vertices (nv, 3) f64, triangles (nt, 3) i32."""

    vertices: np.ndarray
    triangles: np.ndarray
    name: str = "mesh"

    @property
    def nv(self) -> int:
        return int(self.vertices.shape[0])

    @property
    def nt(self) -> int:
        return int(self.triangles.shape[0])


def _dedupe(keys: np.ndarray, tri_keys: np.ndarray):
    """Map integer lattice keys (m,3) to unique vertex ids (sorted order)."""
    uniq, inv = np.unique(keys, axis=0, return_inverse=True)
    tris = inv.reshape(tri_keys)
    return uniq, tris.astype(np.int32)


def sphere(s: int) -> Mesh:
    """Unit sphere from the double pyramid, s subdivisions per face edge."""
    if s < 1:
        raise ValueError("s must be >= 1")
    ii, jj = np.meshgrid(np.arange(s + 1), np.arange(s + 1), indexing="ij")
    mask = (ii + jj) <= s
    # local triangles on the (i, j) lattice of one face, as (i, j) index pairs
    up = []
    down = []
    for i in range(s):
        for j in range(s - i):
            up.append(((i, j), (i + 1, j), (i, j + 1)))
            if i + j + 1 < s:
                down.append(((i + 1, j), (i + 1, j + 1), (i, j + 1)))
    local = np.array(up + down, dtype=np.int64)  # (s^2, 3, 2)
    all_keys = []
    for sx in (1, -1):
        for sy in (1, -1):
            for sz in (1, -1):
                A = np.array([sx * s, 0, 0])
                B = np.array([0, sy * s, 0])
                C = np.array([0, 0, sz * s])
                if sx * sy * sz < 0:  # keep the outward orientation
                    B, C = C, B
                # integer lattice point: A + i*(B-A)/s + j*(C-A)/s, scaled by s
                pts = (A[None, None, :] * s + local[..., 0:1] * (B - A)[None, None, :]
                       + local[..., 1:2] * (C - A)[None, None, :]) // s
                all_keys.append(pts)
    keys = np.concatenate(all_keys, axis=0)  # (8 s^2, 3, 3) integer coords (sum of |.| = s)
    del mask
    uniq, tris = _dedupe(keys.reshape(-1, 3), keys.shape[:2])
    v = uniq.astype(np.float64)
    v /= np.sqrt((v * v).sum(axis=1))[:, None]
    return Mesh(v, tris, name=f"sphere_s{s}")


def ellipsoid(s: int, axes=(1.0, 0.5, 0.25)) -> Mesh:
    m = sphere(s)
    v = m.vertices * np.asarray(axes, dtype=np.float64)[None, :]
    return Mesh(v, m.triangles, name=f"ellipsoid_s{s}")


def cube(s: int) -> Mesh:
    """Unit cube surface, s x s squares per face, two triangles per square."""
    if s < 1:
        raise ValueError("s must be >= 1")
    e = np.eye(3, dtype=np.int64)
    faces = [  # (origin, du, dv) with du x dv the outward normal
        (e[0], e[1], e[2]), (np.zeros(3, np.int64), e[2], e[1]),
        (e[1], e[2], e[0]), (np.zeros(3, np.int64), e[0], e[2]),
        (e[2], e[0], e[1]), (np.zeros(3, np.int64), e[1], e[0]),
    ]
    u, w = np.meshgrid(np.arange(s), np.arange(s), indexing="ij")
    u = u.ravel()
    w = w.ravel()
    keys = []
    for o, du, dv in faces:
        def P(a, b):
            return o[None, :] * s + a[:, None] * du[None, :] + b[:, None] * dv[None, :]
        p00, p10, p11, p01 = P(u, w), P(u + 1, w), P(u + 1, w + 1), P(u, w + 1)
        keys.append(np.stack([p00, p10, p11], axis=1))
        keys.append(np.stack([p00, p11, p01], axis=1))
    keys = np.concatenate(keys, axis=0)
    uniq, tris = _dedupe(keys.reshape(-1, 3), keys.shape[:2])
    return Mesh(uniq.astype(np.float64) / s, tris, name=f"cube_s{s}")


def mean_edge_length(mesh: Mesh) -> float:
    t = mesh.triangles.astype(np.int64)
    edges = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]], axis=0)
    edges = np.unique(np.sort(edges, axis=1), axis=0)
    d = mesh.vertices[edges[:, 0]] - mesh.vertices[edges[:, 1]]
    return float(np.sqrt((d * d).sum(axis=1)).mean())


def jitter(mesh: Mesh, frac: float, seed: int) -> Mesh:
    h = mean_edge_length(mesh)
    rng = np.random.default_rng(seed)
    off = rng.uniform(-frac * h, frac * h, size=mesh.vertices.shape)
    return Mesh(mesh.vertices + off, mesh.triangles.copy(), name=mesh.name + "_jit")


def rhs(n: int, nrhs: int, seed: int = BASE_SEED) -> np.ndarray:
    """N(0,1) right-hand sides, shape (nrhs, n), float64."""
    x = np.random.default_rng(seed).standard_normal((n, nrhs))
    return np.ascontiguousarray(x.T)


def batch_meshes(count: int = 64, seed: int = BASE_SEED, nmin: int = 2000, nmax: int = 65536):
    """Uneven mesh family: type i mod 3 in (sphere, ellipsoid, cube), size drawn
    uniformly among the s that give nmin <= n <= nmax, vertices jittered by
    +-1% of the mean edge length, each mesh seeded by seed + i."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed + i)
        kind = i % 3
        if kind < 2:
            smin = int(np.ceil(np.sqrt(nmin / 8)))
            smax = int(np.floor(np.sqrt(nmax / 8)))
        else:
            smin = int(np.ceil(np.sqrt(nmin / 12)))
            smax = int(np.floor(np.sqrt(nmax / 12)))
        s = int(rng.integers(smin, smax + 1))
        m = sphere(s) if kind == 0 else ellipsoid(s) if kind == 1 else cube(s)
        out.append(jitter(m, 0.01, seed + 1000 + i))
    return out


def named(name: str) -> Mesh:
    """Meshes of the benchmark workloads, by name."""
    table = {
        "sphere512": lambda: sphere(8),
        "sphere2k": lambda: sphere(16),
        "sphere32k": lambda: sphere(64),
        "ellipsoid131k": lambda: ellipsoid(128),
        "sphere2M": lambda: sphere(512),
    }
    return table[name]()
