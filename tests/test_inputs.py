"""Seeded synthetic inputs: mesh topology, orientation and the paper's sizes."""
import os

import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _closed_oriented(m):
    t = m.triangles.astype(np.int64)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    de = set(map(tuple, e.tolist()))
    return len(de) == len(e) and all((b, a) in de for a, b in de)


def _volume(m):
    v, t = m.vertices, m.triangles
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    return np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6


def test_table1_sizes_are_octahedron_refinements():
    ns = [int(x) for x in open(os.path.join(GOLD, "table1_sphere_n.txt")) if x.strip() and not x.startswith("#")]
    for n in ns:
        s = int(round(np.sqrt(n / 8)))
        assert 8 * s * s == n
    for n in ns[:3]:
        m = I.sphere(int(round(np.sqrt(n / 8))))
        assert m.nt == n and m.nv == n // 2 + 2


@pytest.mark.parametrize("mk", [lambda: I.sphere(5), lambda: I.ellipsoid(4), lambda: I.cube(3),
                                lambda: I.jitter(I.cube(4), 0.01, 1)])
def test_meshes_closed_and_outward(mk):
    m = mk()
    assert _closed_oriented(m) and _volume(m) > 0


def test_sphere_vertices_on_sphere_and_volume():
    m = I.sphere(16)
    assert np.allclose(np.linalg.norm(m.vertices, axis=1), 1.0, atol=1e-15)
    assert abs(_volume(m) - 4 * np.pi / 3) < 0.03  # inscribed polyhedron, O(h^2) deficit
    assert abs(_volume(I.cube(5)) - 1.0) < 1e-14


def test_test_points_outside_unit_ball():
    pts = np.loadtxt(os.path.join(GOLD, "section5_test_points.txt"))
    assert np.all(np.linalg.norm(pts, axis=1) > 1.0)


def test_jitter_and_rhs_seeded():
    m = I.sphere(8)
    a, b = I.jitter(m, 0.01, 3), I.jitter(m, 0.01, 3)
    assert np.array_equal(a.vertices, b.vertices)
    h = I.mean_edge_length(m)
    assert np.abs(a.vertices - m.vertices).max() <= 0.01 * h
    x = I.rhs(100, 3, seed=5)
    assert x.shape == (3, 100) and np.array_equal(x, I.rhs(100, 3, seed=5))


def test_batch_family_sizes():
    ms = I.batch_meshes(6)
    for i, m in enumerate(ms):
        assert 2000 <= m.nt <= 65536 and _closed_oriented(m)
        assert m.nt % (8 if i % 3 < 2 else 12) == 0
