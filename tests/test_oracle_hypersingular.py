"""Pins for the oracle's hypersingular operator W (section 1: w_ij =
-int phi_i d/dn_x int dg/dn_y phi_j on continuous piecewise-linear phi, set up
through its single-layer representation W = sum_d C_d^T G C_d with the
constant surface curls C_d of the hat functions).

* W annihilates constants (the curl of a constant vanishes), is symmetric and
  positive semi-definite with a one-dimensional kernel on a closed connected
  surface.
* On the unit sphere W Y_l = l (l + 1) / (2 l + 1) Y_l (closed form of the
  hypersingular operator's spectrum): the Galerkin Rayleigh quotient of the
  piecewise-linear interpolant, with the P1 mass matrix, converges at O(h^2).
* For vertex pairs with disjoint supports the representation's entries equal
  the defining integral -int int phi_i phi_j d/dn_x d/dn_y g evaluated
  directly (brute-force quadrature of the second normal derivatives of g),
  which pins the curls' signs, magnitudes and corner assignment.
"""
import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I
from tests import _brute as B


def harmonic(l, p):
    """Homogeneous harmonic polynomial r^l Y_l (zonal) at p (N, 3)."""
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    r2 = x * x + y * y + z * z
    return {1: z, 2: 3 * z * z - r2, 3: z * (5 * z * z - 3 * r2)}[l]


def mass_p1(mesh):
    """P1 mass matrix: |tau| / 12 [[2, 1, 1], [1, 2, 1], [1, 1, 2]] per triangle."""
    v, t = mesh.vertices, mesh.triangles
    A = 0.5 * np.linalg.norm(np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]]), axis=1)
    M = np.zeros((mesh.nv, mesh.nv))
    loc = np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]]) / 12.0
    for k in range(3):
        for m in range(3):
            np.add.at(M, (t[:, k], t[:, m]), A * loc[k, m])
    return M


@pytest.mark.parametrize("name", ["sphere", "cube", "jitter"])
def test_kernel_symmetry_and_semidefiniteness(orc, name):
    mesh = {"sphere": I.sphere(6), "cube": I.cube(5), "jitter": I.jitter(I.ellipsoid(5), 0.02, 1)}[name]
    W = orc.hypersingular_dense(mesh)
    scale = np.abs(W).max()
    assert np.abs(W @ np.ones(mesh.nv)).max() < 1e-13 * scale
    assert np.abs(W - W.T).max() < 1e-14 * scale
    ev = np.linalg.eigvalsh(0.5 * (W + W.T))
    assert ev[0] > -1e-12 * scale
    assert ev[1] > 1e-3 * ev[-1]  # only the constants in the kernel


@pytest.mark.parametrize("l", [1, 2, 3])
def test_sphere_eigenvalues(orc, l):
    errs = []
    for s in (4, 8, 16):
        mesh = I.sphere(s)
        W = orc.hypersingular_dense(mesh)
        u = harmonic(l, mesh.vertices)
        errs.append(abs((u @ W @ u) / (u @ mass_p1(mesh) @ u) - l * (l + 1) / (2 * l + 1)))
    assert errs[-1] < 5e-3
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0  # O(h^2)


def test_separated_entries_equal_the_defining_integral(orc):
    mesh = I.jitter(I.sphere(6), 0.02, 2)
    v, t = mesh.vertices, mesh.triangles
    rows, cols, vals = orc.curl_p1(mesh)
    nrm = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    star = [np.where((t == j).any(1))[0] for j in range(mesh.nv)]
    U, V, Wq = B.tri_rule(8)

    def rule(tau):
        a, b, c = v[t[tau]]
        area = 0.5 * np.linalg.norm(np.cross(b - a, c - a))
        return a + U[:, None] * (b - a) + V[:, None] * (c - a), area * Wq

    def hat(tau, j, p):
        """Barycentric coordinate of vertex j in triangle tau at points p."""
        k = list(t[tau]).index(j)
        a, b, c = v[t[tau]]
        cr = np.cross(b - a, c - a)
        o1, o2 = v[t[tau][(k + 1) % 3]], v[t[tau][(k + 2) % 3]]
        return np.cross(o1 - p, o2 - p) @ cr / (cr @ cr)

    def curl(tau, j):
        k = list(t[tau]).index(j)
        return np.array([vals[d][3 * tau + k] for d in range(3)])

    W = orc.hypersingular_dense(mesh)
    rng = np.random.default_rng(3)
    checked = 0
    for i in rng.choice(mesh.nv, 12, replace=False):
        j = int(np.argmax(np.linalg.norm(v - v[i], axis=1) - 1e-9 * rng.random(mesh.nv)))
        rep = direct = 0.0
        for tau in star[i]:
            P, wp = rule(tau)
            hi = hat(tau, i, P)
            for sg in star[j]:
                Q, wq = rule(sg)
                hj = hat(sg, j, Q)
                D = P[:, None, :] - Q[None, :, :]
                r = np.linalg.norm(D, axis=2)
                gts = (wp[:, None] * wq[None, :] / (4 * np.pi * r)).sum()
                rep += curl(tau, i) @ curl(sg, j) * gts
                nx, ny = nrm[tau], nrm[sg]
                d2g = ((nx @ ny) / r**3 - 3 * (D @ nx) * (D @ ny) / r**5) / (4 * np.pi)
                direct -= ((wp * hi)[:, None] * (wq * hj)[None, :] * d2g).sum()
        assert abs(rep - direct) < 1e-9 * abs(direct), (i, j, rep, direct)
        # and the oracle's matrix entry (7-point rule for G) agrees to its quadrature error
        assert abs(W[i, j] - direct) < 1e-4 * abs(direct), (i, j, W[i, j], direct)
        checked += 1
    assert checked == 12


def test_matvec_forms_agree(orc):
    mesh = I.ellipsoid(6)
    x = I.rhs(mesh.nv, 3, seed=5)
    W = orc.hypersingular_dense(mesh)
    y = orc.hypersingular_matvec(mesh, x)
    assert np.abs(y - x @ W.T).max() < 1e-13 * np.abs(x @ W.T).max()
    # through the H^2 product with eta = 0 (everything nearfield: the dense matrix)
    y2 = orc.hypersingular_matvec(mesh, x, slp_matvec=orc.H2(mesh, 0, m=4, eta=0.0).matvec)
    assert np.abs(y2 - y).max() < 1e-12 * np.abs(y).max()
