"""Pins for the oracle's dense Galerkin matrices G and K (section 1, eq. (slp),
eq. (dlp)) against closed forms on the sphere and invariants of the operators.
"""
import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I
from tests import _brute as B


def areas(mesh):
    v, t = mesh.vertices, mesh.triangles
    return 0.5 * np.linalg.norm(np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]]), axis=1)


def centroids(mesh):
    return mesh.vertices[mesh.triangles].mean(1)


def harmonic(l, p):
    """Homogeneous harmonic polynomial r^l Y_l (zonal), evaluated at p (N,3)."""
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    r2 = x * x + y * y + z * z
    return {0: np.ones_like(z), 1: z, 2: 3 * z * z - r2, 3: z * (5 * z * z - 3 * r2),
            4: 35 * z**4 - 30 * z * z * r2 + 3 * r2 * r2}[l]


@pytest.fixture(scope="module")
def sph():
    return {s: I.sphere(s) for s in (4, 8, 16)}


@pytest.fixture(scope="module")
def G512(orc, sph):
    return orc.dense_matrix(0, sph[8])


def test_single_layer_symmetric_positive_definite(orc, sph, G512):
    # regular pairs: symmetric up to the summation order of the 7 x 7 rule
    assert np.abs(G512 - G512.T).max() <= 1e-15 * np.abs(G512).max()
    # singular pairs: computed once in the canonical orientation, exactly symmetric
    m = sph[8]
    t = m.triangles
    for i in range(0, m.nt, 37):
        for j in range(m.nt):
            if len(set(t[i]) & set(t[j])) > 0:
                assert G512[i, j] == G512[j, i]
    np.linalg.cholesky(G512)
    assert np.linalg.eigvalsh(G512).min() > 0


def test_V1_equals_1_on_sphere(orc, sph):
    errs = []
    for s in (4, 8, 16):
        m = sph[s]
        y = orc.dense_matvec(0, m, np.ones((1, m.nt)))[0]
        errs.append(np.abs(y / areas(m) - 1).max())
    assert errs[-1] < 3e-3
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0  # O(h^2)


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4])
def test_single_layer_eigenvalues(orc, sph, l):
    """V Y_l = Y_l / (2l+1) on the unit sphere: the Galerkin Rayleigh quotient."""
    errs = []
    for s in (8, 16):
        m = sph[s]
        x = harmonic(l, centroids(m) / np.linalg.norm(centroids(m), axis=1)[:, None])
        y = orc.dense_matvec(0, m, x[None, :])[0]
        rq = (x @ y) / (x @ (areas(m) * x))
        errs.append(abs(rq * (2 * l + 1) - 1))
    # converges to the closed form at O(h^2)
    assert errs[-1] < 4e-3 * (l + 1) and errs[0] / errs[1] > 3.3


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4])
def test_double_layer_on_harmonics(orc, sph, l):
    """K Y_l = -Y_l / (2(2l+1)), from Green's boundary formula (section 1,
    eq. (dirichlet_to_neumann)) with u = r^l Y_l."""
    errs = []
    for s in (8, 16):
        m = sph[s]
        a = areas(m)
        x = harmonic(l, centroids(m) / np.linalg.norm(centroids(m), axis=1)[:, None])
        y = orc.dense_matvec(1, m, x[None, :])[0]
        want = -a * x / (2 * (2 * l + 1))
        errs.append(np.linalg.norm(y - want) / np.linalg.norm(want))
    assert errs[-1] < 1.2e-2 * (l + 0.1) and errs[0] / errs[1] > 3.3


@pytest.mark.parametrize("name", ["sphere", "cube", "ellipsoid"])
def test_double_layer_row_sums(orc, name):
    """sum_j k_ij = -1/2 |tau_i| on a closed polyhedron (solid angle of the
    whole surface seen from a face point, section 1 with u = 1); the residual
    is pure quadrature error."""
    m = {"sphere": I.sphere(6), "cube": I.cube(4), "ellipsoid": I.ellipsoid(6)}[name]
    r5 = np.abs(orc.dense_matvec(1, m, np.ones((1, m.nt)), q_ss=5)[0] / areas(m) + 0.5)
    r8 = np.abs(orc.dense_matvec(1, m, np.ones((1, m.nt)), q_ss=8)[0] / areas(m) + 0.5)
    assert r5.max() < 1e-3 and np.median(r5) < 2e-5
    if name == "ellipsoid":  # worst rows are limited by the singular rule: shrink with q
        assert r8.max() < 0.5 * r5.max()


def _proj(mesh, f):
    """Piecewise-constant L2 projection (triangle means) by a high-order rule."""
    v, t = mesh.vertices, mesh.triangles
    return np.array([B.tri_integral(v[tt], f, q=8) for tt in t]) / areas(mesh)


@pytest.mark.parametrize("y0", [(1.2, 1.2, 1.2), (1.0, 0.25, 1.0)])
def test_green_identity(orc, sph, y0):
    """Green's boundary formula (section 1) for u = g(., y0), y0 outside (the
    test data of section 5): G N - K D = 1/2 M D with D, N the projections of
    u and du/dn; the residual is the discretisation error and shrinks with h."""
    y0 = np.asarray(y0)
    res = []
    for s in (4, 8):
        m = sph[s]
        v, t = m.vertices, m.triangles
        nrm = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])
        nrm /= np.linalg.norm(nrm, axis=1)[:, None]
        u = lambda p: 1.0 / (4 * np.pi * np.linalg.norm(p - y0, axis=1))  # noqa: E731
        D = _proj(m, u)
        N = np.zeros(m.nt)
        for i, tt in enumerate(t):
            du = lambda p, n=nrm[i]: -((p - y0) @ n) / (4 * np.pi * np.linalg.norm(p - y0, axis=1) ** 3)  # noqa: E731
            N[i] = B.tri_integral(v[tt], du, q=8) / areas(m)[i]
        lhs = orc.dense_matvec(0, m, N[None])[0] - orc.dense_matvec(1, m, D[None])[0]
        rhs = 0.5 * areas(m) * D
        res.append(np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs))
    assert res[1] < res[0] and res[1] < 2e-2


def test_dense_rows_and_transpose(orc, sph):
    m = sph[4]
    x = I.rhs(m.nt, 3, seed=11)
    for k in (0, 1):
        A = orc.dense_matrix(k, m)
        y = orc.dense_matvec(k, m, x)
        assert np.allclose(y, (A @ x.T).T, rtol=0, atol=1e-15 * np.abs(y).max() * 10)
        rows = np.array([0, 3, 127])
        assert np.allclose(orc.dense_rows(k, m, rows, x), y[:, rows], rtol=0, atol=1e-16)
        yt = orc.dense_matvec(k, m, x, transpose=True)
        assert np.allclose(yt, (A.T @ x.T).T, rtol=0, atol=1e-15 * np.abs(yt).max() * 10)
