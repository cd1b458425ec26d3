"""Pins for the oracle's H^2 approximation (section 2: cluster tree, block tree,
eq. (transfer), eq. (vsw); section 3: eq. (admissibility), tensor Chebyshev
interpolation) against structural invariants, polynomial exactness and the
dense definition.
"""
import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I
from tests import _brute as B


@pytest.fixture(scope="module")
def m2k():
    return I.sphere(16)


@pytest.fixture(scope="module")
def H2k(orc, m2k):
    return orc.H2(m2k, orc.SLP, m=4, eta=2.0, leaf=32)


def test_block_counts_match_independent_probe(orc, m2k):
    """Counts of clusters, leaves, farfield and nearfield blocks at leaf 32,
    eta = 2 reported by an independent probe of the same rules (n = 2,048 and
    8,192 triangles)."""
    H = orc.H2(m2k, orc.SLP, m=2)
    assert (H.nclusters, H.nleaves, H.nfar, H.nnear) == (191, 96, 2240, 1632)
    H = orc.H2(I.sphere(32), orc.SLP, m=2)
    assert (H.nclusters, H.nleaves, H.nfar, H.nnear) == (719, 360, 8688, 6800)


def test_cluster_tree_invariants(H2k, m2k):
    tr = H2k.tree()
    n = m2k.nt
    assert sorted(tr["perm"].tolist()) == list(range(n))
    v, t = m2k.vertices, m2k.triangles
    cen = v[t].mean(1)
    for c in range(H2k.nclusters):
        b, e = tr["begin"][c], tr["end"][c]
        idx = tr["perm"][b:e]
        pts = v[t[idx]].reshape(-1, 3)
        assert np.array_equal(tr["bmin"][c], pts.min(0)) and np.array_equal(tr["bmax"][c], pts.max(0))
        c0, c1 = tr["child0"][c], tr["child1"][c]
        if c0 < 0:
            assert c1 < 0 and e - b <= 32
            continue
        assert e - b > 32 and c0 == c + 1  # depth-first pre-order
        assert tr["begin"][c0] == b and tr["end"][c0] == tr["begin"][c1] and tr["end"][c1] == e
        ext = tr["bmax"][c] - tr["bmin"][c]
        ax = int(np.argmax(ext))
        mid = 0.5 * (tr["bmin"][c][ax] + tr["bmax"][c][ax])
        lo = cen[tr["perm"][b:tr["end"][c0]], ax]
        hi = cen[tr["perm"][tr["begin"][c1]:e], ax]
        all_c = cen[idx, ax]
        if np.any(all_c < mid) and np.any(all_c >= mid):
            assert np.all(lo < mid) and np.all(hi >= mid)
        else:
            assert tr["end"][c0] - b == (e - b) // 2 and lo.max() <= hi.min()


def test_block_tree_partitions_and_admissibility(H2k, m2k):
    tr = H2k.tree()
    (ft, fs), (nt, ns) = H2k.blocks()
    n = m2k.nt
    cover = np.zeros((n, n), dtype=np.int32)
    pos = np.empty(n, dtype=np.int64)
    pos[tr["perm"]] = np.arange(n)

    def diam(c):
        return np.linalg.norm(tr["bmax"][c] - tr["bmin"][c])

    def dist(a, b):
        g = np.maximum(0, np.maximum(tr["bmin"][b] - tr["bmax"][a], tr["bmin"][a] - tr["bmax"][b]))
        return np.linalg.norm(g)

    for t_, s_ in zip(ft, fs):
        cover[tr["begin"][t_]:tr["end"][t_], tr["begin"][s_]:tr["end"][s_]] += 1
        assert dist(t_, s_) > 0 and max(diam(t_), diam(s_)) <= 2.0 * dist(t_, s_)
    leaf = tr["child0"] < 0
    for t_, s_ in zip(nt, ns):
        cover[tr["begin"][t_]:tr["end"][t_], tr["begin"][s_]:tr["end"][s_]] += 1
        assert leaf[t_] and leaf[s_]
        d = dist(t_, s_)
        assert not (d > 0 and max(diam(t_), diam(s_)) <= 2.0 * d)
    assert np.all(cover == 1)
    # symmetric block structure
    assert set(zip(ft.tolist(), fs.tolist())) == set(zip(fs.tolist(), ft.tolist()))
    # every singular pair (shared vertex) lies in a nearfield block
    t = m2k.triangles
    for i in range(0, n, 101):
        for j in np.nonzero((t[:, :, None] == t[i][None, None, :]).any(axis=(1, 2)))[0]:
            a, b = pos[i], pos[j]
            hits = [(t_, s_) for t_, s_ in zip(nt, ns) if tr["begin"][t_] <= a < tr["end"][t_] and tr["begin"][s_] <= b < tr["end"][s_]]
            assert len(hits) == 1


def test_chebyshev_nodes(H2k):
    """The nodes are the roots of T_m on the (floored) cluster box."""
    tr = H2k.tree()
    z = H2k.nodes()
    m = H2k.m
    for c in range(0, H2k.nclusters, 7):
        lo, hi = tr["bmin"][c], tr["bmax"][c]
        ctr, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
        half = np.maximum(half, 1e-2 * half.max())
        for d in range(3):
            u = (z[c, d] - ctr[d]) / half[d]
            Tm = np.polynomial.chebyshev.chebval(u, [0] * m + [1])
            assert np.abs(Tm).max() < 1e-12 and len(np.unique(np.round(u, 12))) == m


def test_flat_cluster_nodes_are_distinct(orc):
    H = orc.H2(I.cube(8), orc.SLP, m=4)
    z = H.nodes()
    assert np.all(np.diff(np.sort(z, axis=2), axis=2) > 0)


def _tensor_poly(p, cx, cy, cz):
    return (np.polynomial.polynomial.polyval(p[:, 0], cx) * np.polynomial.polynomial.polyval(p[:, 1], cy)
            * np.polynomial.polynomial.polyval(p[:, 2], cz))


@pytest.mark.parametrize("kernel", [0, 1])
def test_leaf_bases_reproduce_polynomials(orc, m2k, kernel):
    """sum_nu V_t[i,nu] p(xi_nu) = int_{tau_i} p and, for the double layer,
    sum_mu W_s[j,mu] p(xi_mu) = int_{tau_j} n_j . grad p, for every tensor
    polynomial p of degree <= m-1 per coordinate (interpolation is exact)."""
    H = orc.H2(m2k, kernel, m=4)
    tr = H.tree()
    z = H.nodes()
    rng = np.random.default_rng(3)
    cx, cy, cz = rng.standard_normal((3, 4))
    v, t = m2k.vertices, m2k.triangles
    leaves = np.nonzero(tr["child0"] < 0)[0][:6]
    for c in leaves:
        V, W = H.leaf_basis(c)
        g = np.stack(np.meshgrid(z[c, 0], z[c, 1], z[c, 2], indexing="ij"), -1)
        xi = g.transpose(2, 1, 0, 3).reshape(-1, 3)  # nu = a + m (b + m c)
        pv = _tensor_poly(xi, cx, cy, cz)
        for a, i in enumerate(tr["perm"][tr["begin"][c]:tr["end"][c]]):
            T = v[t[i]]
            want = B.tri_integral(T, lambda p: _tensor_poly(p, cx, cy, cz), q=8)
            assert abs(V[a] @ pv - want) <= 1e-12 * max(1.0, abs(want))
            if kernel == 1:
                n = np.cross(T[1] - T[0], T[2] - T[0])
                n /= np.linalg.norm(n)
                dcx, dcy, dcz = (np.polynomial.polynomial.polyder(cc) for cc in (cx, cy, cz))
                grad = lambda p: (n[0] * _tensor_poly(p, dcx, cy, cz) + n[1] * _tensor_poly(p, cx, dcy, cz)  # noqa: E731
                                  + n[2] * _tensor_poly(p, cx, cy, dcz))
                wantd = B.tri_integral(T, grad, q=8)
                assert abs(W[a] @ pv - wantd) <= 1e-11 * max(1.0, abs(wantd))


def test_transfer_matrices_nest(orc, H2k):
    """E_{t'} maps node values of a polynomial on the parent box to its node
    values on the child box (eq. (transfer) with exact reproduction)."""
    tr = H2k.tree()
    z = H2k.nodes()
    parent = {}
    for c in range(H2k.nclusters):
        for ch in (tr["child0"][c], tr["child1"][c]):
            if ch >= 0:
                parent[ch] = c
    rng = np.random.default_rng(5)
    cx, cy, cz = rng.standard_normal((3, 4))

    def nodes(c):
        g = np.stack(np.meshgrid(z[c, 0], z[c, 1], z[c, 2], indexing="ij"), -1)
        return g.transpose(2, 1, 0, 3).reshape(-1, 3)

    for ch in list(parent)[::9]:
        E = H2k.transfer(ch)
        pp = _tensor_poly(nodes(parent[ch]), cx, cy, cz)
        pc = _tensor_poly(nodes(ch), cx, cy, cz)
        assert np.abs(E @ pp - pc).max() <= 1e-11 * np.abs(pc).max()


def test_polynomial_kernel_farfield_is_exact(orc, m2k):
    """With the test kernel P(x) Q(y) (degree 3 per coordinate) and m = 4, the
    farfield part of the H^2 product equals sum over farfield blocks (t,s) of
    (int_{tau_i} P)(int_{tau_j} Q) x_j exactly: pins the tree, blocks, bases,
    transfers and the up/down passes independently of the quadrature."""
    H = orc.H2(m2k, orc.TEST_POLY, m=4)
    x = I.rhs(m2k.nt, 2, seed=9)
    y = H.matvec(x, parts=orc.PART_FAR)
    v, t = m2k.vertices, m2k.triangles
    Pf = lambda p: orc.test_poly_PQ(p)[0]  # noqa: E731
    Qf = lambda p: orc.test_poly_PQ(p)[1]  # noqa: E731
    iP = np.array([B.tri_integral(v[tt], Pf, q=6) for tt in t])
    iQ = np.array([B.tri_integral(v[tt], Qf, q=6) for tt in t])
    tr = H.tree()
    (ft, fs), _ = H.blocks()
    want = np.zeros_like(x)
    for t_, s_ in zip(ft, fs):
        rows = tr["perm"][tr["begin"][t_]:tr["end"][t_]]
        cols = tr["perm"][tr["begin"][s_]:tr["end"][s_]]
        want[:, rows] += iP[rows][None, :] * (x[:, cols] @ iQ[cols])[:, None]
    assert np.abs(y - want).max() <= 1e-12 * np.abs(want).max()
    yt = H.matvec(x, transpose=True, parts=orc.PART_FAR)
    wantt = np.zeros_like(x)
    for t_, s_ in zip(ft, fs):
        rows = tr["perm"][tr["begin"][t_]:tr["end"][t_]]
        cols = tr["perm"][tr["begin"][s_]:tr["end"][s_]]
        wantt[:, cols] += iQ[cols][None, :] * (x[:, rows] @ iP[rows])[:, None]
    assert np.abs(yt - wantt).max() <= 1e-12 * np.abs(wantt).max()


def test_eta_zero_is_dense(orc, m2k):
    x = I.rhs(m2k.nt, 2)
    for k in (0, 1):
        H = orc.H2(m2k, k, m=3, eta=0.0)
        assert H.nfar == 0
        yd = orc.dense_matvec(k, m2k, x)
        assert np.linalg.norm(H.matvec(x) - yd) <= 1e-14 * np.linalg.norm(yd)


def test_error_decays_geometrically_in_m(orc, m2k):
    """Section 3: interpolation error ~ q^m."""
    x = I.rhs(m2k.nt, 2)
    yd = orc.dense_matvec(0, m2k, x)
    errs = [np.linalg.norm(orc.H2(m2k, 0, m=m).matvec(x) - yd) / np.linalg.norm(yd) for m in (2, 3, 4, 5, 6)]
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 4.0) and errs[2] < 5e-4


def test_rows_transpose_and_symmetry(orc, m2k):
    x = I.rhs(m2k.nt, 2)
    w = I.rhs(m2k.nt, 2, seed=77)
    for k in (0, 1):
        H = orc.H2(m2k, k, m=4)
        y = H.matvec(x)
        rows = np.array([0, 5, 999, m2k.nt - 1])
        assert np.abs(H.rows(rows, x) - y[:, rows]).max() <= 1e-14 * np.abs(y).max()
        yt = H.matvec(w, transpose=True)
        assert abs((w * y).sum() - (yt * x).sum()) <= 1e-13 * np.abs(w * y).sum()
        if k == 0:
            assert np.abs(yt - H.matvec(w)).max() <= 1e-14 * np.abs(yt).max()


def test_double_layer_h2_error(orc, m2k):
    x = I.rhs(m2k.nt, 1)
    yd = orc.dense_matvec(1, m2k, x)
    e4 = np.linalg.norm(orc.H2(m2k, 1, m=4).matvec(x) - yd) / np.linalg.norm(yd)
    e6 = np.linalg.norm(orc.H2(m2k, 1, m=6).matvec(x) - yd) / np.linalg.norm(yd)
    assert e4 < 5e-3 and e6 < e4 / 10


@pytest.mark.parametrize("kernel", [0, 1])
def test_subtree_rows_equal_full_product(orc, kernel):
    """or_h2_matvec_subtree (the bounded sample the benchmark times on the host)
    gives exactly the rows of the full product for the triangles of a cluster,
    and zero elsewhere."""
    mesh = I.jitter(I.sphere(12), 0.01, 2)
    H = orc.H2(mesh, kernel, m=3)
    x = I.rhs(mesh.nt, 2, seed=4)
    full = H.matvec(x)
    tr = H.tree()
    for c0 in (0, 1, 5, int(np.flatnonzero(tr["child0"] < 0)[7])):
        y = H.matvec_subtree(c0, x)
        assert np.array_equal(y, H.matvec_subtree_from(c0, H.upward(x), x))
        rows = tr["perm"][tr["begin"][c0]:tr["end"][c0]]
        assert np.allclose(y[:, rows], full[:, rows], rtol=1e-12, atol=1e-14 * np.abs(full).max())
        others = np.setdiff1d(np.arange(mesh.nt), rows)
        assert np.all(y[:, others] == 0)
