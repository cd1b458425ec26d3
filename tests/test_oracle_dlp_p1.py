"""Pins for the oracle's double layer with continuous piecewise-linear trial
functions (section 1, eq. (dlp) with phi_j the hat functions; the paper's
discretisation of the Dirichlet values, section 5): K1 in R^{n x nv},
K1[i, v] = sum over the triangles j at vertex v of
int_{tau_i} int_{tau_j} dg/dn_y lambda_{j,v}(y) dy dx.

* The three corner values of a pair sum to the piecewise-constant entry k_ij
  (the barycentric coordinates sum to 1), which is pinned on its own; a
  triangle with itself gives 0.
* Pairs far apart agree with brute-force quadrature of the defining integral.
* Green's identity for a linear u = a.x + b: on a polyhedral surface u is
  exactly piecewise linear and its normal derivative a.n exactly piecewise
  constant, so (M1 / 2 + K1) u = G (a.n) holds up to quadrature error only
  (M1: the mixed mass matrix, |tau_i| / 3 per corner).  The same identity with
  the piecewise-constant K on triangle averages of u carries a discretisation
  error two orders larger, and rotating the corner values of every pair (a
  planted mistake) breaks it by as much.
* The Neumann-to-Dirichlet form of the same identity, W u = (M1^T / 2 - K1^T)
  du/dn, with the oracle's hypersingular operator.
"""
import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I
from tests import _brute as B


def geometry(mesh):
    v, t = mesh.vertices, mesh.triangles
    cr = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])
    area = 0.5 * np.linalg.norm(cr, axis=1)
    return area, cr / (2 * area[:, None])


def mass_p0_p1(mesh, area):
    M1 = np.zeros((mesh.nt, mesh.nv))
    for c in range(3):
        np.add.at(M1, (np.arange(mesh.nt), mesh.triangles[:, c]), area / 3)
    return M1


def test_corner_values_sum_to_the_constant_entry(orc):
    mesh = I.jitter(I.sphere(6), 0.02, 3)
    t = mesh.triangles
    rng = np.random.default_rng(0)
    pairs = [tuple(rng.integers(mesh.nt, size=2)) for _ in range(200)]
    pairs += [(i, j) for i in range(0, mesh.nt, 37) for j in range(mesh.nt) if set(t[i]) & set(t[j])]
    for i, j in pairs:
        e3 = orc.entry_dlp_p1(mesh, int(i), int(j))
        e = orc.entry(1, mesh, int(i), int(j))
        if i == j:
            assert np.all(e3 == 0.0)
        else:
            assert abs(e3.sum() - e) <= 1e-13 * abs(e), (i, j, e3, e)
    K1 = orc.dense_dlp_p1(mesh)
    K = orc.dense_matrix(1, mesh)
    assert np.abs(K1.sum(1) - K.sum(1)).max() < 1e-14 * np.abs(K).sum(1).max()


def test_separated_pairs_equal_brute_force(orc):
    mesh = I.jitter(I.sphere(4), 0.02, 5)
    v, t = mesh.vertices, mesh.triangles
    U, V, W = B.tri_rule(12)
    ctr = v[t].mean(1)
    rng = np.random.default_rng(1)
    for _ in range(8):
        i = int(rng.integers(mesh.nt))
        j = int(np.argsort(np.linalg.norm(ctr - ctr[i], axis=1))[-1 - int(rng.integers(40))])
        X, Y = v[t[i]], v[t[j]]
        ax = 0.5 * np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0]))
        cr = np.cross(Y[1] - Y[0], Y[2] - Y[0])
        ay = 0.5 * np.linalg.norm(cr)
        ny = cr / (2 * ay)
        P = X[0] + U[:, None] * (X[1] - X[0]) + V[:, None] * (X[2] - X[0])
        Q = Y[0] + U[:, None] * (Y[1] - Y[0]) + V[:, None] * (Y[2] - Y[0])
        D = P[:, None, :] - Q[None, :, :]
        k = (D @ ny) / (4 * np.pi * np.linalg.norm(D, axis=2) ** 3)
        lam = np.stack([1 - U - V, U, V])
        ref = np.array([((ax * W)[:, None] * (ay * W)[None, :] * k * lam[c][None, :]).sum() for c in range(3)])
        e = orc.entry_dlp_p1(mesh, i, j)
        assert np.abs(e - ref).max() < 1e-5 * np.abs(ref).max(), (i, j, e, ref)


MESHES = {
    "sphere": (lambda: I.sphere(8), 1e-4),
    "cube": (lambda: I.cube(4), 3e-4),
    "jittered ellipsoid": (lambda: I.jitter(I.ellipsoid(6), 0.02, 1), 1e-3),
}


@pytest.mark.parametrize("name", list(MESHES))
def test_green_identity_for_linear_functions(orc, name):
    make, tol = MESHES[name]
    mesh = make()
    v, t = mesh.vertices, mesh.triangles
    area, nrm = geometry(mesh)
    a, b = np.array([0.3, -0.7, 0.5]), 0.2
    u = v @ a + b
    G = orc.dense_matrix(0, mesh)
    rhs = G @ (nrm @ a)
    K1 = orc.dense_dlp_p1(mesh)
    lhs = 0.5 * mass_p0_p1(mesh, area) @ u + K1 @ u
    err = np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs)
    assert err < tol, err
    # the piecewise-constant double layer on triangle averages: discretisation error
    K = orc.dense_matrix(1, mesh)
    ubar = v[t].mean(1) @ a + b
    err0 = np.linalg.norm(0.5 * area * ubar + K @ ubar - rhs) / np.linalg.norm(rhs)
    assert err0 > 30 * err, (err0, err)


def test_planted_corner_rotation_breaks_green_identity(orc):
    mesh = I.sphere(4)
    v, t = mesh.vertices, mesh.triangles
    area, nrm = geometry(mesh)
    a, b = np.array([0.3, -0.7, 0.5]), 0.2
    u = v @ a + b
    rhs = orc.dense_matrix(0, mesh) @ (nrm @ a)
    lhs = 0.5 * area * u[t].mean(1)
    for i in range(mesh.nt):
        for j in range(mesh.nt):
            lhs[i] += np.roll(orc.entry_dlp_p1(mesh, i, j), 1) @ u[t[j]]
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) > 1e-2


@pytest.mark.parametrize("name", list(MESHES))
def test_neumann_to_dirichlet_identity(orc, name):
    """The normal derivative of Green's representation (section 1, eq.
    (neumann_to_dirichlet)) tested with the hat functions: W u =
    (M1^T / 2 - K1^T) du/dn.  For a linear u on a polyhedral surface both sides
    are exact up to quadrature, which ties the hypersingular operator (through
    its single-layer representation), K1 and M1 together, signs included."""
    make, tol = MESHES[name]
    mesh = make()
    v = mesh.vertices
    area, nrm = geometry(mesh)
    a = np.array([0.3, -0.7, 0.5])
    u = v @ a + 0.2
    bn = nrm @ a
    lhs = orc.hypersingular_dense(mesh) @ u
    rhs = 0.5 * mass_p0_p1(mesh, area).T @ bn - orc.dense_dlp_p1(mesh).T @ bn
    assert np.linalg.norm(lhs - rhs) < tol * np.linalg.norm(rhs)


def test_neumann_to_dirichlet_solution_converges_at_order_two(orc):
    """The Neumann-to-Dirichlet problem with the paper's discretisation
    (section 5: Neumann data piecewise constant, Dirichlet values piecewise
    linear; expected O(h^2) for the Dirichlet values in L2): on the unit sphere,
    for the test functions u1 = x1^2 - x3^2, u2 = g(., (1.2, 1.2, 1.2)),
    u3 = g(., (1, 0.25, 1)), b the L2 projection of du/dn onto the triangles,
    W x = (M1^T / 2 - K1^T) b with the constants fixed by the mean of u.  From
    2,048 to 8,192 triangles the L2 error of x against u at the vertices falls
    by 3.3-3.7 (orders 1.7-1.9)."""
    uv, w = orc.radon7()
    y1, y2 = np.array([1.2, 1.2, 1.2]), np.array([1.0, 0.25, 1.0])

    def u_dn(k, p):
        if k == 0:
            return p[..., 0] ** 2 - p[..., 2] ** 2, 2 * p[..., 0] ** 2 - 2 * p[..., 2] ** 2
        d = p - (y1 if k == 1 else y2)
        r = np.linalg.norm(d, axis=-1)
        return 1 / (4 * np.pi * r), -(d * p).sum(-1) / (4 * np.pi * r ** 3)

    errs = {}
    for s in (16, 32):
        mesh = I.sphere(s)
        v, t = mesh.vertices, mesh.triangles
        area, _ = geometry(mesh)
        a, b, c = (v[t[:, k]] for k in range(3))
        pts = a[:, None] + uv[None, :, 0, None] * (b - a)[:, None] + uv[None, :, 1, None] * (c - a)[:, None]
        proj = pts / np.linalg.norm(pts, axis=-1, keepdims=True)
        M1 = mass_p0_p1(mesh, area)
        Mp = np.zeros((mesh.nv, mesh.nv))
        loc = np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]]) / 12.0
        for k in range(3):
            for m in range(3):
                np.add.at(Mp, (t[:, k], t[:, m]), area * loc[k, m])
        W = orc.hypersingular_dense(mesh)
        K1 = orc.dense_dlp_p1(mesh)
        mv = Mp.sum(1)
        for k in range(3):
            bn = (u_dn(k, proj)[1] * w[None, :]).sum(1)
            uI = u_dn(k, v)[0]
            x = np.linalg.solve(W + np.outer(mv, mv), 0.5 * M1.T @ bn - K1.T @ bn + mv * (mv @ uI))
            e = x - uI
            errs[(k, s)] = np.sqrt(e @ Mp @ e / (uI @ Mp @ uI))
    for k in range(3):
        assert errs[(k, 16)] / errs[(k, 32)] > 3.0, errs
        assert errs[(k, 32)] < 3e-4, errs


def test_h2_form_equals_dense_at_eta_zero_and_converges_in_m(orc):
    """K1 in the H^2 form of section 2 (per-corner source basis W1, the same
    transfers, coupling and output basis V as the other operators): with
    eta = 0 it is the dense K1; with eta = 2 its error decays geometrically in
    the interpolation order (section 3)."""
    mesh = I.jitter(I.ellipsoid(8), 0.01, 2)
    x = I.rhs(mesh.nv, 3, seed=4)
    ref = x @ orc.dense_dlp_p1(mesh).T
    y0 = orc.H2(mesh, 1, m=4, eta=0.0).matvec_dlp_p1(x)
    assert np.linalg.norm(y0 - ref) < 1e-13 * np.linalg.norm(ref)
    errs = [np.linalg.norm(orc.H2(mesh, 1, m=m, eta=2.0).matvec_dlp_p1(x) - ref) / np.linalg.norm(ref)
            for m in (2, 3, 4, 5, 6)]
    assert all(errs[q] / errs[q + 1] > 2.5 for q in range(4)), errs
    assert errs[-1] < 1e-4, errs


def test_h2_transpose_equals_dense_and_is_the_adjoint(orc):
    """K1^T in the H^2 form (V on the triangle side, the transposed passes,
    W1 gathered to the vertices): the dense K1^T at eta = 0, and the adjoint
    of the forward H^2 product at eta = 2 to rounding."""
    mesh = I.jitter(I.ellipsoid(8), 0.01, 2)
    K1 = orc.dense_dlp_p1(mesh)
    xt = I.rhs(mesh.nt, 3, seed=5)
    xv = I.rhs(mesh.nv, 3, seed=4)
    y0 = orc.H2(mesh, 1, m=4, eta=0.0).matvec_dlp_p1(xt, transpose=True)
    assert np.linalg.norm(y0 - xt @ K1) < 1e-13 * np.linalg.norm(xt @ K1)
    H = orc.H2(mesh, 1, m=4, eta=2.0)
    yt = H.matvec_dlp_p1(xt, transpose=True)
    y = H.matvec_dlp_p1(xv)
    assert abs((xt * y).sum() - (yt * xv).sum()) < 1e-13 * np.linalg.norm(xt) * np.linalg.norm(y) * 10
    assert np.linalg.norm(yt - xt @ K1) < 3e-3 * np.linalg.norm(xt @ K1)
