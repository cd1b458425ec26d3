"""The double layer with piecewise-linear trial functions, K1 (section 1, eq.
(dlp) with the hat functions of the vertices), on the GPU against the oracle,
and the Neumann-to-Dirichlet problem (eq. (neumann_to_dirichlet)) solved with
it and the hypersingular operator.

1. h2bem_apply_dlp_p1 against the oracle's H^2 product of the same form
   (per-corner source bases W1_c, the double layer's transfers, coupling and
   output basis V): forward and transposed, several right-hand-side widths,
   1e-10 in FP64 and 1e-6 in MIXED_FP32 (FP32 output basis V; the per-corner
   bases, the nearfield and the Sauter-Schwab pairs are FP64 in every tier).
2. With eta = 0 every block is nearfield and the product is the oracle's
   dense K1; the mass term alpha M1 is the exact P0 x P1 mass matrix.
3. The Neumann-to-Dirichlet solve (W + m m^T) x = (M1^T / 2 - K1^T) b + m (m . u)
   by the library's conjugate gradients: with eta = 0 it matches a dense
   direct solve with the oracle's matrices; on the unit sphere, for the
   paper's test functions (section 5), the L2 error of the Dirichlet values
   falls by more than 3 from 2,048 to 8,192 triangles (order ~1.8, the
   oracle's own rate for the same discretisation).
"""
import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I
from tests._parity import close, rel

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed_fp32": 1e-6}
Y1 = np.array([1.2, 1.2, 1.2])
Y2 = np.array([1.0, 0.25, 1.0])


@pytest.fixture(scope="module")
def H():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_05523_gb300 import build, h2bem

    build.build()
    return h2bem


def areas(mesh):
    a, b, c = (mesh.vertices[mesh.triangles[:, k]] for k in range(3))
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)


def mass_p0_p1(mesh):
    """(M1)_{i v} = |tau_i| / 3 for the corners v of tau_i (nt x nv)."""
    M = np.zeros((mesh.nt, mesh.nv))
    ar = areas(mesh)
    for k in range(3):
        np.add.at(M, (np.arange(mesh.nt), mesh.triangles[:, k]), ar / 3.0)
    return M


def k1_apply(H, op, x, transpose=False, alpha=0.0):
    import torch

    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    nout = op.nv if transpose else op.n
    yd = torch.full((x.shape[0], nout), float("nan"), dtype=torch.float64, device="cuda")
    H.h2bem_apply_dlp_p1(op.op, xd, yd, transpose=transpose, alpha=alpha)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


MESHES = {
    "sphere": lambda: I.sphere(12),
    "jitter_ellipsoid": lambda: I.jitter(I.ellipsoid(10), 0.01, 3),
    "cube": lambda: I.cube(9),
}


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_k1_matches_oracle_h2(H, orc, name, precision):
    mesh = MESHES[name]()
    ref = orc.H2(mesh, 1, m=4)
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=1, m=4, eta=2.0, leaf_size=32, precision=precision)
    xv = I.rhs(mesh.nv, 3, seed=5)
    xt = I.rhs(mesh.nt, 3, seed=6)
    close(k1_apply(H, op, xv), ref.matvec_dlp_p1(xv), TOL[precision], f"K1 {name} {precision}")
    close(k1_apply(H, op, xt, transpose=True), ref.matvec_dlp_p1(xt, transpose=True), TOL[precision],
          f"K1^T {name} {precision}")
    op.close()


@pytest.mark.parametrize("nrhs", [1, 2, 16, 21, 64])
def test_k1_rhs_widths(H, orc, nrhs):
    mesh = I.jitter(I.sphere(10), 0.01, 7)
    ref = orc.H2(mesh, 1, m=4)
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=1, m=4, eta=2.0, precision="fp64")
    xv = I.rhs(mesh.nv, nrhs, seed=nrhs)
    xt = I.rhs(mesh.nt, nrhs, seed=nrhs + 100)
    close(k1_apply(H, op, xv), ref.matvec_dlp_p1(xv), TOL["fp64"], f"K1 nrhs {nrhs}")
    close(k1_apply(H, op, xt, transpose=True), ref.matvec_dlp_p1(xt, transpose=True), TOL["fp64"],
          f"K1^T nrhs {nrhs}")
    op.close()


def test_k1_dense_at_eta_zero_and_mass_term(H, orc):
    mesh = I.jitter(I.ellipsoid(7), 0.02, 4)
    K1 = orc.dense_dlp_p1(mesh)
    M1 = mass_p0_p1(mesh)
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=1, eta=0.0, precision="fp64")
    xv = I.rhs(mesh.nv, 4, seed=1)
    xt = I.rhs(mesh.nt, 4, seed=2)
    close(k1_apply(H, op, xv), xv @ K1.T, 1e-10, "dense K1")
    close(k1_apply(H, op, xt, transpose=True), xt @ K1, 1e-10, "dense K1^T")
    close(k1_apply(H, op, xv, alpha=0.5), xv @ (K1 + 0.5 * M1).T, 1e-10, "K1 + M1/2")
    close(k1_apply(H, op, xt, transpose=True, alpha=-0.5), xt @ (K1 - 0.5 * M1), 1e-10, "K1^T - M1^T/2")
    op.close()


def test_k1_rejects_unsupported(H):
    import torch

    mesh = I.sphere(5)
    x = torch.zeros((1, mesh.nv), dtype=torch.float64, device="cuda")
    y = torch.zeros((1, mesh.nt), dtype=torch.float64, device="cuda")
    for kw in ({"kernel": 0}, {"kernel": 1, "recompute_basis": True}):
        op = H.Operator(mesh.vertices, mesh.triangles, m=4, precision="fp64", **kw)
        with pytest.raises(H.H2bemError) as e:
            H.h2bem_apply_dlp_p1(op.op, x, y)
        assert e.value.code == H.H2BEM_ERR_ARG
        op.close()
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=1, precision="fp64")
    with pytest.raises(H.H2bemError) as e:  # y too short for the forward product
        H.h2bem_apply_dlp_p1(op.op, x, x)
    assert e.value.code == H.H2BEM_ERR_ARG
    with pytest.raises(H.H2bemError) as e:
        H.h2bem_apply_dlp_p1(op.op, x.cpu(), y.cpu())
    assert e.value.code == H.H2BEM_ERR_ARG
    op.close()


# ------------------------------------------------------------ Neumann-to-Dirichlet
def mass_p1(mesh):
    """The P1 mass matrix (nv x nv, scipy.sparse)."""
    import scipy.sparse as sp

    t, ar = mesh.triangles, areas(mesh)
    loc = np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]]) / 12.0
    rows = np.concatenate([t[:, k] for k in range(3) for _ in range(3)])
    cols = np.concatenate([t[:, m] for _ in range(3) for m in range(3)])
    vals = np.concatenate([ar * loc[k, m] for k in range(3) for m in range(3)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(mesh.nv, mesh.nv))


def u_and_dn(k, p):
    """The test functions of section 5 and their normal derivatives on the unit sphere (normal = p)."""
    if k == 0:
        return p[..., 0] ** 2 - p[..., 2] ** 2, 2 * p[..., 0] ** 2 - 2 * p[..., 2] ** 2
    d = p - (Y1 if k == 1 else Y2)
    r = np.linalg.norm(d, axis=-1)
    return 1 / (4 * np.pi * r), -(d * p).sum(-1) / (4 * np.pi * r ** 3)


def neumann_data(orc, mesh):
    """b (3, nt): the 7-point-rule L2 projection of du/dn onto the triangles (points
    projected onto the sphere), uI (3, nv): u at the vertices."""
    uv, w = orc.radon7()
    v, t = mesh.vertices, mesh.triangles
    a, b, c = (v[t[:, k]] for k in range(3))
    pts = a[:, None] + uv[None, :, 0, None] * (b - a)[:, None] + uv[None, :, 1, None] * (c - a)[:, None]
    proj = pts / np.linalg.norm(pts, axis=-1, keepdims=True)
    bn = np.stack([(u_and_dn(k, proj)[1] * w[None, :]).sum(1) for k in range(3)])
    uI = np.stack([u_and_dn(k, v)[0] for k in range(3)])
    return bn, uI


def ntd_solve(H, mesh, bn, uI, m=4, eta=2.0, precision="fp64", rtol=1e-10):
    """(W + mv mv^T) x = (M1^T / 2 - K1^T) b + mv (mv . uI) on the GPU: the right-hand
    side through h2bem_apply_dlp_p1 (transposed, alpha = -1/2 on -b), the solve
    through h2bem_cg_hypersingular.  Returns (x, rhs, iterations, relres)."""
    import torch

    slp = H.Operator(mesh.vertices, mesh.triangles, kernel=0, m=m, eta=eta, precision=precision)
    dlp = H.Operator(mesh.vertices, mesh.triangles, kernel=1, m=m, eta=eta, precision=precision)
    mv = np.asarray(mass_p1(mesh).sum(1)).ravel()
    bd = torch.from_numpy(np.ascontiguousarray(-bn)).cuda()
    rhs = torch.empty((bn.shape[0], mesh.nv), dtype=torch.float64, device="cuda")
    H.h2bem_apply_dlp_p1(dlp.op, bd, rhs, transpose=True, alpha=-0.5)
    mvd = torch.from_numpy(mv).cuda()
    rhs += (torch.from_numpy(uI).cuda() @ mvd)[:, None] * mvd[None, :]
    x = torch.empty_like(rhs)
    it, rr = H.h2bem_cg_hypersingular(slp.op, mvd, rhs, x, rtol=rtol, maxit=2000)
    torch.cuda.synchronize()
    out = x.cpu().numpy(), rhs.cpu().numpy(), it, rr
    slp.close()
    dlp.close()
    return out


def test_ntd_dense_matches_direct_solve(H, orc):
    mesh = I.sphere(8)
    bn, uI = neumann_data(orc, mesh)
    x, rhs, it, rr = ntd_solve(H, mesh, bn, uI, eta=0.0, rtol=1e-12)
    mv = np.asarray(mass_p1(mesh).sum(1)).ravel()
    K1 = orc.dense_dlp_p1(mesh)
    M1 = mass_p0_p1(mesh)
    rhs_ref = bn @ (0.5 * M1 - K1) + np.outer(uI @ mv, mv)
    close(rhs, rhs_ref, 1e-10, "NtD right-hand side")
    A = orc.hypersingular_dense(mesh) + np.outer(mv, mv)
    x_ref = np.linalg.solve(A, rhs_ref.T).T
    print(f"NtD dense: {it} CG iterations, relres {max(rr):.1e}")
    assert max(rr) < 1e-12
    assert rel(x, x_ref) < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_ntd_dirichlet_error_is_order_h2(H, orc, precision):
    errs = {}
    for s in (16, 32):
        mesh = I.sphere(s)
        bn, uI = neumann_data(orc, mesh)
        x, _, it, rr = ntd_solve(H, mesh, bn, uI, m=5, precision=precision, rtol=1e-9)
        assert max(rr) < 1e-9, rr
        Mp = mass_p1(mesh)
        for k in range(3):
            e = x[k] - uI[k]
            errs[(k, s)] = np.sqrt(e @ (Mp @ e) / (uI[k] @ (Mp @ uI[k])))
        print(f"NtD {precision} s={s} (nt {mesh.nt}): {it} iterations, errors "
              + ", ".join(f"{errs[(k, s)]:.2e}" for k in range(3)))
    for k in range(3):
        assert errs[(k, 16)] / errs[(k, 32)] > 3.0, errs
        assert errs[(k, 32)] < 3e-4, errs
