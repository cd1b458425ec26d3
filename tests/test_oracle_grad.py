"""Pin of the oracle's hand-derived shape gradient d/dX sum_r <w_r, A x_r>
(A = G or K; cluster tree and block lists frozen) against central finite
differences of the oracle's own H^2 product, part by part.  The double layer
adds the source triangles' area-normals, the Hessian of the Lagrange
polynomials in its leaf basis W = int n . grad L, and the Sauter-Schwab
points of both orientations of a singular pair."""
import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I


def _fd(orc, H, mesh, w, x, v, d, parts, h=1e-6):
    X = mesh.vertices.copy()
    vals = []
    for sgn in (1.0, -1.0):
        Xp = X.copy()
        Xp[v, d] += sgn * h
        H.update_geometry(Xp)
        vals.append(float((w * H.matvec(x, parts=parts)).sum()))
    H.update_geometry(X)
    return (vals[0] - vals[1]) / (2 * h)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("name", ["sphere", "cube"])
@pytest.mark.parametrize("parts", [1, 2])
def test_gradient_matches_central_differences(orc, name, parts, kernel):
    mesh = I.jitter(I.sphere(5), 0.05, 11) if name == "sphere" else I.jitter(I.cube(4), 0.02, 12)
    H = orc.H2(mesh, kernel, m=3, eta=2.0, leaf=6)
    assert H.nfar > 0
    w = I.rhs(mesh.nt, 2, seed=21)
    x = I.rhs(mesh.nt, 2, seed=22)
    g = H.grad_vertices(w, x, parts=parts)
    rng = np.random.default_rng(5)
    scale = np.abs(g).max()
    worst = 0.0
    for v in rng.choice(mesh.nv, 10, replace=False):
        for d in range(3):
            fd = _fd(orc, H, mesh, w, x, int(v), d, parts)
            worst = max(worst, abs(fd - g[v, d]) / scale)
    assert worst < 1e-5, worst


@pytest.mark.parametrize("kernel", [0, 1])
def test_gradient_total_is_sum_of_parts(orc, kernel):
    mesh = I.jitter(I.sphere(4), 0.05, 3)
    H = orc.H2(mesh, kernel, m=3, leaf=6)
    w, x = I.rhs(mesh.nt, 1, seed=1), I.rhs(mesh.nt, 1, seed=2)
    g = H.grad_vertices(w, x)
    assert np.allclose(g, H.grad_vertices(w, x, parts=1) + H.grad_vertices(w, x, parts=2), rtol=0, atol=1e-15)


def test_double_layer_gradient_of_a_rigid_motion_vanishes(orc):
    """<w, K x> is invariant under translations and rotations of the whole
    mesh (the tree and blocks move with it; boxes are axis-parallel, so only
    translations keep the H^2 form exactly invariant): the gradient sums to
    zero over the vertices along every axis."""
    mesh = I.jitter(I.sphere(5), 0.05, 4)
    H = orc.H2(mesh, orc.DLP, m=3, leaf=6)
    w, x = I.rhs(mesh.nt, 2, seed=3), I.rhs(mesh.nt, 2, seed=4)
    g = H.grad_vertices(w, x)
    assert np.abs(g.sum(0)).max() < 1e-9 * np.abs(g).max()


def test_gradient_of_the_hessian_of_the_leaf_basis(orc):
    """The double layer's farfield gradient uses second derivatives of the
    Lagrange polynomials: with x = 1 on one leaf and w = 1 on a far leaf the
    farfield part alone matches central differences (a planted sign error in
    the Hessian or the area-normal term fails it)."""
    mesh = I.jitter(I.ellipsoid(5), 0.03, 9)
    H = orc.H2(mesh, orc.DLP, m=4, eta=2.0, leaf=8)
    x = I.rhs(mesh.nt, 1, seed=31)
    w = I.rhs(mesh.nt, 1, seed=32)
    g = H.grad_vertices(w, x, parts=1)
    scale = np.abs(g).max()
    rng = np.random.default_rng(2)
    for v in rng.choice(mesh.nv, 6, replace=False):
        for d in range(3):
            fd = _fd(orc, H, mesh, w, x, int(v), d, 1)
            assert abs(fd - g[v, d]) < 1e-5 * scale
