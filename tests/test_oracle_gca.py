"""Pins of the oracle's Green cross approximation (section 4), each against a
fact that does not come from the oracle's own formulas:

  boundary rule      the divergence theorem and closed-form surface moments
                     of a box; outward normals
  Green's formula    g~_grn(x, y) -> g(x, y) for x in B_t, y outside omega_t
                     (error falling with the quadrature order), and -> 0 when
                     y lies inside omega_t too (Green's second identity)
  L = (A C)          reproduces int_tau u for harmonic u (section 4's
                     representation, weights split as w^(1/2) on each side)
  ACA                exact on matrices of known low rank; pivots are the
                     largest entries of the residual (brute force)
  interpolation      V_t is the identity on the pivot rows, for leaves and,
                     through the transfers, for their parents (nesting)
  product            eta = 0 equals the dense matrix; symmetric; the error
                     against the dense matrix falls with the ACA tolerance
"""
import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I


def g(x, y):
    return 1.0 / (4 * np.pi * np.linalg.norm(np.asarray(x) - np.asarray(y)))


def test_boundary_rule_divergence_theorem_and_moments(orc):
    lo, hi = np.array([-0.3, 0.1, 0.2]), np.array([0.5, 0.4, 1.1])
    for q in (2, 3, 4):
        z, w, nz = orc.gca_boundary_rule(lo, hi, q)
        L = hi - lo
        area = 2 * (L[0] * L[1] + L[1] * L[2] + L[0] * L[2])
        assert abs(w.sum() - area) < 1e-13
        # outward: the normal points away from the centre
        assert np.all(np.einsum("kd,kd->k", nz, z - 0.5 * (lo + hi)) > 0)
        # divergence theorem for F = (x^2 y, y z^2, x z): div F = 2 x y + z^2 + x
        F = np.stack([z[:, 0] ** 2 * z[:, 1], z[:, 1] * z[:, 2] ** 2, z[:, 0] * z[:, 2]], 1)
        flux = np.sum(w * np.einsum("kd,kd->k", F, nz))

        def mono(a, b, c):  # int over the box of x^a y^b z^c
            return np.prod([(hi[d] ** (e + 1) - lo[d] ** (e + 1)) / (e + 1) for d, e in enumerate((a, b, c))])

        vol = 2 * mono(1, 1, 0) + mono(0, 0, 2) + mono(1, 0, 0)
        assert abs(flux - vol) < 1e-12 * max(1.0, abs(vol))


def test_green_representation_converges_and_vanishes_inside(orc):
    lo, hi = np.array([-1.0, -1.0, -1.0]), np.array([1.0, 1.0, 1.0])
    x = np.array([0.2, -0.1, 0.3])
    y_out = np.array([2.9, 1.5, -2.2])
    errs = [abs(orc.gca_green(lo, hi, q, x, y_out) - g(x, y_out)) / g(x, y_out) for q in (2, 4, 6, 8)]
    assert errs[-1] < 3e-5 and errs[0] > 1e3 * errs[-1], errs
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    # y inside omega as well: the boundary integral of Green's second identity is 0
    y_in = np.array([-0.5, 0.4, -0.2])
    assert abs(orc.gca_green(lo, hi, 8, x, y_in)) < 1e-4 * g(x, y_in)


@pytest.mark.parametrize("which", ["quadratic", "point_source"])
def test_L_reproduces_harmonic_functions(orc, which):
    """int_tau_i u ~ sum_nu A_i,nu w^(1/2) du/dn(z_nu) - C_i,nu w^(1/2) u(z_nu)
    for u harmonic in omega_t (a harmonic polynomial; a point source outside),
    the discretised Green representation behind L; the error falls
    geometrically with the quadrature order q."""
    mesh = I.sphere(8)
    tr = orc.H2(mesh, 0, m=1).tree()
    leaf = int(np.flatnonzero(tr["child0"] < 0)[3])
    lo, hi = tr["bmin"][leaf], tr["bmax"][leaf]
    delta = np.max(hi - lo)
    y0 = np.array([3.0, -2.0, 2.5])
    if which == "quadratic":
        u = lambda p: p[..., 0] ** 2 - p[..., 2] ** 2  # noqa: E731
        grad = lambda p: np.stack([2 * p[..., 0], 0 * p[..., 1], -2 * p[..., 2]], -1)  # noqa: E731
    else:
        u = lambda p: 1.0 / np.linalg.norm(p - y0, axis=-1)  # noqa: E731
        grad = lambda p: -(p - y0) / np.linalg.norm(p - y0, axis=-1)[..., None] ** 3  # noqa: E731
    errs = []
    for q in (2, 4, 6, 8, 10):
        rows, L = orc.GCA(mesh, q=q, eps=1e-8, kmax=64).L(leaf)
        z, w, nz = orc.gca_boundary_rule(lo - delta, hi + delta, q)
        k = z.shape[0]
        b = np.sqrt(w) * np.einsum("kd,kd->k", grad(z), nz)
        d = np.sqrt(w) * u(z)
        approx = L[:, :k] @ b - L[:, k:] @ d
        # int over each triangle by a fine rule (independent of the 7-point rule)
        uv, wt = orc.collapsed_rule(12)
        exact = []
        for i in rows:
            A, B, C = mesh.vertices[mesh.triangles[i]]
            pts = A + uv[:, :1] * (B - A) + uv[:, 1:] * (C - A)
            exact.append(0.5 * np.linalg.norm(np.cross(B - A, C - A)) * np.sum(wt * u(pts)))
        exact = np.array(exact)
        errs.append(np.max(np.abs(approx - exact)) / np.max(np.abs(exact)))
    assert all(b < 0.3 * a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-5 and errs[0] > 1e4 * errs[-1], errs


def test_aca_exact_on_low_rank_and_pivots_are_maxima(orc):
    rng = np.random.default_rng(5)
    for r in (1, 3, 7):
        M = rng.standard_normal((20, r)) @ rng.standard_normal((r, 30))
        tau, sigma = orc.gca_aca(M, 0.0, 30)
        assert len(tau) >= r
        # the cross approximation with the first r pivots reproduces M
        t, s = tau[:r], sigma[:r]
        R = M[:, s] @ np.linalg.solve(M[np.ix_(t, s)], M[t, :])
        assert np.max(np.abs(R - M)) < 1e-10 * np.max(np.abs(M))
        # brute force: each pivot is the first entry (row-major) within 2^-40 of
        # the largest of the residual of the earlier ones
        Rz = M.copy()
        for i, j in zip(tau[:r], sigma[:r]):
            A = np.abs(Rz)
            first = np.flatnonzero(A.ravel() >= A.max() * (1 - 2.0 ** -40))[0]
            assert (i, j) == divmod(int(first), Rz.shape[1])
            Rz = Rz - np.outer(Rz[:, j], Rz[i, :] / Rz[i, j])
    # exact ties resolve to the first entry in row-major order
    tau, sigma = orc.gca_aca(np.array([[1.0, 2.0], [2.0, -2.0]]), 0.0, 1)
    assert (tau[0], sigma[0]) == (0, 1)
    # tolerance: stops once the pivot falls below eps times the first
    M = np.diag([1.0, 1e-3, 1e-7, 1e-12])
    tau, _ = orc.gca_aca(M, 1e-6, 10)
    assert len(tau) == 2


def test_interpolation_identity_on_pivots_leaf_and_nested(orc):
    mesh = I.jitter(I.sphere(10), 0.01, 2)
    G = orc.GCA(mesh, q=4, eps=1e-7, kmax=48)
    tr = orc.H2(mesh, 0, m=1).tree()
    perm, begin, end, c0, c1 = tr["perm"], tr["begin"], tr["end"], tr["child0"], tr["child1"]
    ranks = G.ranks()

    def V_of(c):  # V_t by the nesting of eq. (transfer)
        if c0[c] < 0:
            return G.leaf_basis(c, int(end[c] - begin[c]))
        a, b = c0[c], c1[c]
        Va, Vb = V_of(a), V_of(b)
        Ea, Eb = G.transfer(a, c), G.transfer(b, c)
        return np.vstack([Va @ Ea, Vb @ Eb])

    checked = 0
    for c in range(1, len(begin)):
        if end[c] - begin[c] > 200 or ranks[c] == 0:
            continue
        V = V_of(c)
        pos = {int(i): a for a, i in enumerate(perm[begin[c]:end[c]])}
        P = G.pivots(c)
        rowsP = V[[pos[int(i)] for i in P]]
        assert np.max(np.abs(rowsP - np.eye(len(P)))) < 1e-9, c
        checked += 1
    assert checked > 10


def test_eta0_equals_dense_and_symmetry(orc):
    mesh = I.sphere(6)
    x = I.rhs(mesh.nt, 2, seed=3)
    G0 = orc.GCA(mesh, q=3, eta=0.0)
    d = orc.dense_matvec(0, mesh, x)
    assert np.linalg.norm(G0.matvec(x) - d) / np.linalg.norm(d) < 1e-14
    mesh = I.jitter(I.sphere(12), 0.01, 4)
    G = orc.GCA(mesh, q=4, eps=1e-6)
    a, b = I.rhs(mesh.nt, 1, seed=1)[0], I.rhs(mesh.nt, 1, seed=2)[0]
    ga, gb = G.matvec(a)[0], G.matvec(b)[0]
    assert abs(ga @ b - a @ gb) < 1e-12 * abs(ga @ b)


def test_error_falls_with_aca_tolerance(orc):
    mesh = I.sphere(16)
    x = I.rhs(mesh.nt, 2, seed=1)
    d = orc.dense_matvec(0, mesh, x)
    errs = []
    for eps in (1e-3, 1e-5, 1e-7, 1e-9):
        G = orc.GCA(mesh, q=5, eps=eps, kmax=128)
        errs.append(np.linalg.norm(G.matvec(x) - d) / np.linalg.norm(d))
    assert all(b < 0.5 * a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-8, errs
