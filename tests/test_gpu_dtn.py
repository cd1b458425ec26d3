"""Dirichlet-to-Neumann problem (section 1, eq. (matrix_dtn)): G x = (M/2 + K) b
with piecewise-constant Dirichlet data b and Neumann data x, solved by the
library's conjugate gradients on the GPU.

1. With eta = 0 (every block nearfield) the operators are the dense Galerkin
   matrices: the right-hand side and the CG solution match a dense direct
   solve with the oracle's matrices.
2. On the unit sphere, for the paper's harmonic test functions (section 5:
   u1 = x1^2 - x3^2, u2 = g(., y1), u3 = g(., y2) with y1 = (1.2, 1.2, 1.2),
   y2 = (1, 0.25, 1)), b the L2 projection of u onto the triangles, the L2
   error of x against the exact Neumann data decreases as O(h) (the paper's
   observation for its Dirichlet-to-Neumann experiment).
3. The condition number of G grows as 1/h, so the matrix accuracy has to grow
   with n to keep the O(h) rate (section 5 raises the interpolation order with
   n).  At a fixed m = 4 the error stops improving past ~32k triangles; with
   m = 5, 6, 6 on 8k, 32k and 131k triangles it halves at each refinement."""
import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I

pytestmark = pytest.mark.gpu

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


def rule_points(mesh, orc):
    """7-point rule points (nt, 7, 3), weights (7,) summing to 1, areas (nt,)."""
    uv, w = orc.radon7()
    u, v = uv[:, 0], uv[:, 1]
    a, b, c = (mesh.vertices[mesh.triangles[:, k]] for k in range(3))
    pts = a[:, None, :] + u[None, :, None] * (b - a)[:, None, :] + v[None, :, None] * (c - a)[:, None, :]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    return pts, w, area


def u_and_dn(name, p):
    """u and its normal derivative at points p on the unit sphere (normal = p)."""
    if name == "u1":
        return p[..., 0] ** 2 - p[..., 2] ** 2, 2 * p[..., 0] ** 2 - 2 * p[..., 2] ** 2
    y = Y1 if name == "u2" else Y2
    d = p - y
    r = np.linalg.norm(d, axis=-1)
    return 1 / (4 * np.pi * r), -(d * p).sum(-1) / (4 * np.pi * r ** 3)


def test_cg_and_rhs_match_dense_direct_solve(H, orc):
    import torch

    mesh = I.jitter(I.sphere(6), 0.02, 3)
    G = orc.dense_matrix(0, mesh)
    K = orc.dense_matrix(1, mesh)
    _, _, area = rule_points(mesh, orc)
    b = I.rhs(mesh.nt, 2, seed=5)
    rhs_ref = (0.5 * area[None, :] * b) + b @ K.T
    x_ref = np.linalg.solve(G, rhs_ref.T).T
    opG = H.Operator(mesh.vertices, mesh.triangles, kernel=0, eta=0.0)
    opK = H.Operator(mesh.vertices, mesh.triangles, kernel=1, eta=0.0)
    bd = torch.from_numpy(b).cuda()
    rhs = torch.empty_like(bd)
    H.h2bem_apply_mass(opK.op, 0.5, bd, rhs)
    x = torch.empty_like(bd)
    it, rel = H.h2bem_cg(opG.op, rhs, x, rtol=1e-13, maxit=2000)
    torch.cuda.synchronize()
    assert np.linalg.norm(rhs.cpu().numpy() - rhs_ref) / np.linalg.norm(rhs_ref) < 1e-12
    assert max(rel) < 1e-12 and it > 0
    assert np.linalg.norm(x.cpu().numpy() - x_ref) / np.linalg.norm(x_ref) < 1e-8
    opG.close()
    opK.close()


NAMES = ("u1", "u2", "u3")


def neumann_errors(H, orc, s, m, precision, rtol):
    """Solves the DtN system on sphere(s) and returns the relative L2 errors
    of the Neumann data for u1, u2, u3."""
    import torch

    mesh = I.sphere(s)
    pts, w, area = rule_points(mesh, orc)
    proj = pts / np.linalg.norm(pts, axis=-1, keepdims=True)
    opG = H.Operator(mesh.vertices, mesh.triangles, kernel=0, m=m, precision=precision)
    opK = H.Operator(mesh.vertices, mesh.triangles, kernel=1, m=m, precision=precision)
    # L2 projection onto the triangles (the rule integrates u over each triangle)
    b = np.stack([(u_and_dn(nm, pts)[0] * w[None, :]).sum(1) for nm in NAMES])
    bd = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    rhs = torch.empty_like(bd)
    H.h2bem_apply_mass(opK.op, 0.5, bd, rhs)
    x = torch.empty_like(bd)
    it, rel = H.h2bem_cg(opG.op, rhs, x, rtol=rtol, maxit=3000)
    torch.cuda.synchronize()
    assert max(rel) < rtol, (s, it, rel)
    xs = x.cpu().numpy()
    errs = {}
    for k, nm in enumerate(NAMES):
        dn = u_and_dn(nm, proj)[1]
        e2 = (area[:, None] * w[None, :] * (xs[k][:, None] - dn) ** 2).sum()
        n2 = (area[:, None] * w[None, :] * dn ** 2).sum()
        errs[nm] = np.sqrt(e2 / n2)
    opG.close()
    opK.close()
    return errs


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_dtn_neumann_error_is_order_h(H, orc, precision):
    errs = {}
    for s in (8, 16, 32):
        for nm, e in neumann_errors(H, orc, s, 4, precision, 1e-9).items():
            errs[(nm, s)] = e
    for nm in NAMES:
        r1 = errs[(nm, 8)] / errs[(nm, 16)]
        r2 = errs[(nm, 16)] / errs[(nm, 32)]
        assert 1.6 < r1 and 1.6 < r2, (nm, errs)
        assert errs[(nm, 32)] < 0.1, (nm, errs)


def test_dtn_order_schedule_keeps_order_h(H, orc):
    """m = 5, 6, 6 on 8,192, 32,768 and 131,072 triangles: the error halves per
    refinement (rate >= 1.8 each step) and ends below 1.5 % for every u."""
    errs = {s: neumann_errors(H, orc, s, m, "mixed_fp32", 1e-8) for s, m in ((32, 5), (64, 6), (128, 6))}
    for nm in NAMES:
        assert errs[32][nm] / errs[64][nm] > 1.8, (nm, errs)
        assert errs[64][nm] / errs[128][nm] > 1.8, (nm, errs)
        assert errs[128][nm] < 0.015, (nm, errs)
