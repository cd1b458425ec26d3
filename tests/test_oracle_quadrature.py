"""Pins for the oracle's quadrature rules and singular-quadrature region maps.

Every check compares against mathematics fixed independently of the code under
test: closed-form monomial integrals, and independent brute-force integrals
(analytic inner potential, subdivided outer rule) for the singular pairs.
"""
from math import factorial

import numpy as np
import pytest

from tests import _brute as B


def simplex_moment(a, b):
    # int over {u,v>=0,u+v<=1} of u^a v^b = a! b! / (a+b+2)!, normalised by the area 1/2
    return 2.0 * factorial(a) * factorial(b) / factorial(a + b + 2)


def tri_moment(a, b):
    # int over T = {0 <= x2 <= x1 <= 1} of x1^a x2^b
    return 1.0 / ((b + 1) * (a + b + 2))


@pytest.mark.parametrize("q", [1, 2, 3, 5, 8, 13, 20])
def test_gauss_legendre_exact_to_degree_2q_minus_1(orc, q):
    x, w = orc.gauss_legendre01(q)
    for d in range(2 * q):
        assert abs((w * x**d).sum() - 1.0 / (d + 1)) < 1e-14
    # and not exact at degree 2q (the rule is a genuine q-point rule)
    assert abs((w * x ** (2 * q)).sum() - 1.0 / (2 * q + 1)) > 1e-16
    assert np.all(np.diff(x) > 0) and np.all((x > 0) & (x < 1))


def test_radon7_degree5(orc):
    uv, w = orc.radon7()
    assert abs(w.sum() - 1) < 1e-15
    for a in range(6):
        for b in range(6 - a):
            assert abs((w * uv[:, 0] ** a * uv[:, 1] ** b).sum() - simplex_moment(a, b)) < 1e-15
    # degree 6 is not integrated exactly
    errs = [abs((w * uv[:, 0] ** a * uv[:, 1] ** (6 - a)).sum() - simplex_moment(a, 6 - a)) for a in range(7)]
    assert max(errs) > 1e-6
    # fully symmetric (invariant under permutations of the barycentric coordinates)
    bary = np.column_stack([1 - uv.sum(1), uv])
    for perm in ([1, 0, 2], [2, 1, 0], [0, 2, 1]):
        pb = bary[:, perm]
        idx = [int(np.argmin(np.abs(bary - p).sum(1))) for p in pb]
        assert np.allclose(bary[idx], pb, atol=1e-15) and np.allclose(w[idx], w, atol=1e-16)


@pytest.mark.parametrize("q", [2, 5, 6, 7])
def test_collapsed_rule_degree(orc, q):
    uv, w = orc.collapsed_rule(q)
    for a in range(2 * q - 1):
        for b in range(2 * q - 1 - a):
            assert abs((w * uv[:, 0] ** a * uv[:, 1] ** b).sum() - simplex_moment(a, b)) < 1e-14


def test_tri_geom(orc):
    area, n = orc.tri_geom([0, 0, 0], [2, 0, 0], [0, 3, 0])
    assert area == 3.0 and np.allclose(n, [0, 0, 1])
    area, n = orc.tri_geom([0, 0, 0], [0, 3, 0], [2, 0, 0])
    assert np.allclose(n, [0, 0, -1])


@pytest.mark.parametrize("kind", [3, 2, 1])
def test_ss_regions_cover_TxT_once(orc, kind):
    """The region maps with their Jacobians are a change of variables of T x T:
    every moment x1^a x2^b y1^c y2^d of total degree <= 6 is reproduced."""
    worst = 0.0
    for a in range(4):
        for b in range(4 - a):
            for c in range(4 - a - b):
                for d in range(4 - a - b - c):
                    got = orc.ss_moment(kind, 8, a, b, c, d)
                    want = tri_moment(a, b) * tri_moment(c, d)
                    worst = max(worst, abs(got - want) / want)
    assert worst < 1e-13


@pytest.fixture(scope="module")
def jmesh():
    from paper_2001_05523_gb300 import inputs as I

    return I.jitter(I.sphere(3), 0.05, 3)


def _first_pair(orc, mesh, ns):
    for j in range(mesh.nt):
        if orc.shared_vertices(mesh, 0, j) == ns:
            return j
    raise AssertionError


@pytest.mark.parametrize("ns", [3, 2, 1])
def test_singular_slp_vs_brute_force(orc, jmesh, ns):
    j = _first_pair(orc, jmesh, ns)
    kind, P, Q = orc.orient_pair(jmesh, 0, j)
    assert kind == ns
    X = jmesh.vertices[jmesh.triangles[0]]
    Y = jmesh.vertices[jmesh.triangles[j]]
    ref = B.pair_brute(X, Y, 0, L=5)
    q16 = orc.ss_pair(0, kind, P, Q, 16)
    q5 = orc.ss_pair(0, kind, P, Q, 5)
    assert abs(q16 / ref - 1) < 2e-9
    assert abs(q5 / ref - 1) < 5e-5
    # the dense entry uses q = 5 and is symmetric by construction
    e = orc.entry(0, jmesh, 0, j, 5)
    assert e == q5 and orc.entry(0, jmesh, j, 0, 5) == e


@pytest.mark.parametrize("ns", [2, 1])
def test_singular_dlp_vs_brute_force(orc, jmesh, ns):
    j = _first_pair(orc, jmesh, ns)
    X = jmesh.vertices[jmesh.triangles[0]]
    Y = jmesh.vertices[jmesh.triangles[j]]
    # k_0j: x in tau_0, y in tau_j, normal of tau_j
    ref = B.pair_brute(X, Y, 1, L=5)
    e5 = orc.entry(1, jmesh, 0, j, 5)
    e16 = orc.entry(1, jmesh, 0, j, 16)
    assert abs(e16 / ref - 1) < 2e-8
    assert abs(e5 / ref - 1) < 1e-4
    # k_j0 (other orientation of the same canonical point set)
    ref2 = B.pair_brute(Y, X, 1, L=5)
    e16b = orc.entry(1, jmesh, j, 0, 16)
    assert abs(e16b / ref2 - 1) < 2e-8


def test_dlp_identical_and_coplanar(orc):
    from paper_2001_05523_gb300 import inputs as I

    cube = I.cube(2)
    A = orc.dense_matrix(1, cube)
    assert np.all(np.diag(A) == 0.0)
    # pairs on the same (flat) face: x - y is orthogonal to n_y, every entry vanishes
    v, t = cube.vertices, cube.triangles
    nrm = np.array([orc.tri_geom(*v[tt])[1] for tt in t])
    ctr = v[t].mean(1)
    same_face = (np.abs(nrm @ nrm.T - 1) < 1e-12) & (np.abs(np.einsum("ik,jk->ij", ctr, nrm) - np.einsum("jk,jk->j", ctr, nrm)[None, :]) < 1e-12)
    assert np.abs(A[same_face]).max() < 1e-17


def test_regular_pair_vs_brute_force(orc):
    rng = np.random.default_rng(7)
    Y = rng.standard_normal((3, 3)) * 0.1
    for dist in (0.5, 1.0, 3.0):
        X = rng.standard_normal((3, 3)) * 0.1 + np.array([dist, 0.2, -0.1])
        for kernel in (0, 1):
            ref = B.pair_brute(X, Y, kernel, L=2)
            got = orc.pair_regular(kernel, X, Y)
            assert abs(got / ref - 1) < 1e-5 * (0.5 / dist) ** 4 * 20


def test_orient_pair_shared_first(orc, jmesh):
    t = jmesh.triangles
    for ns in (2, 1):
        j = _first_pair(orc, jmesh, ns)
        kind, P, Q = orc.orient_pair(jmesh, 0, j)
        shared = set(t[0]) & set(t[j])
        vid = lambda p: int(np.argmin(np.abs(jmesh.vertices - p).sum(1)))  # noqa: E731
        pv = [vid(p) for p in P]
        qv = [vid(q) for q in Q]
        assert set(pv) == set(t[0]) and set(qv) == set(t[j])
        assert set(pv[:ns]) == shared and pv[:ns] == qv[:ns]
        if ns == 2:  # P keeps the orientation of tau_0 (a rotation)
            k = list(t[0]).index(pv[0])
            assert [int(a) for a in np.roll(t[0], -k)] == pv
