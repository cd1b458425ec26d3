"""Hypersingular operator W (section 1) on the GPU through its single-layer
representation W = sum_d C_d^T G C_d, against the oracle.

Tolerances (relative, 2-norm over all right-hand sides) are those of the
single layer that carries the product: 1e-10 in FP64, 1e-6 in MIXED_FP32
(the curls C_d and their sums are FP64 in every tier).  With eta = 0 the
single layer is the dense Galerkin matrix, so W is the oracle's dense W.
"""
import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed_fp32": 1e-6}


@pytest.fixture(scope="module")
def H():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_05523_gb300 import build, h2bem

    build.build()
    return h2bem


from tests._parity import close, rel  # noqa: E402


def apply_w(H, op, x):
    import torch

    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.full_like(xd, float("nan"))
    H.h2bem_apply_hypersingular(op.op, xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_dense_equals_oracle_matrix(H, orc, precision):
    mesh = I.jitter(I.sphere(7), 0.02, 4)
    x = I.rhs(mesh.nv, 3, seed=2)
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=0, eta=0.0, precision=precision)
    y = apply_w(H, op, x)
    op.close()
    W = orc.hypersingular_dense(mesh)
    close(y, x @ W.T, TOL[precision])


@pytest.mark.parametrize("name", ["sphere", "cube", "ellipsoid"])
@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
@pytest.mark.parametrize("nrhs", [1, 6])
def test_h2_matches_oracle(H, orc, name, precision, nrhs):
    """3 nrhs columns through the single layer: 3 and 18 (a 16 + 2 chunking)."""
    mesh = {"sphere": I.sphere(14), "cube": I.jitter(I.cube(9), 0.01, 3), "ellipsoid": I.ellipsoid(12)}[name]
    x = I.rhs(mesh.nv, nrhs, seed=7)
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=0, precision=precision)
    y = apply_w(H, op, x)
    op.close()
    ref = orc.hypersingular_matvec(mesh, x, slp_matvec=orc.H2(mesh, 0, m=4).matvec)
    close(y, ref, TOL[precision])


def test_constants_and_symmetry(H):
    mesh = I.jitter(I.ellipsoid(10), 0.01, 5)
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=0)
    x = I.rhs(mesh.nv, 2, seed=1)
    ones = np.ones((1, mesh.nv))
    y1 = apply_w(H, op, ones)
    yx = apply_w(H, op, x)
    op.close()
    assert np.abs(y1).max() < 1e-12 * np.abs(yx).max()
    # <W x0, x1> = <x0, W x1> (the H^2 single layer is symmetric to its quadrature's rounding)
    assert abs(x[1] @ yx[0] - x[0] @ yx[1]) < 1e-9 * np.linalg.norm(yx) * np.linalg.norm(x)


def test_sphere_rayleigh_quotient(H):
    """W Y_2 = (6/5) Y_2 on the unit sphere (O(h^2) for the P1 interpolant)."""
    mesh = I.sphere(32)
    v, t = mesh.vertices, mesh.triangles
    u = 3 * v[:, 2] ** 2 - (v ** 2).sum(1)
    A = 0.5 * np.linalg.norm(np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]]), axis=1)
    # u^T M u with the P1 mass matrix |tau|/12 [[2,1,1],[1,2,1],[1,1,2]]
    ut = u[t]
    uMu = (A / 12 * ((ut ** 2).sum(1) + ut.sum(1) ** 2)).sum()
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=0, precision="mixed_fp32")
    y = apply_w(H, op, u[None, :])[0]
    op.close()
    assert abs(u @ y / uMu - 6 / 5) < 2e-3


def test_batch_is_block_diagonal(H, orc):
    meshes = [I.sphere(6), I.jitter(I.cube(5), 0.01, 1)]
    B = H.BatchOperator(meshes, kernel=0, m=4)
    nvs = [m.nv for m in meshes]
    x = I.rhs(sum(nvs), 2, seed=3)
    y = apply_w(H, B, x)
    B.close()
    off = 0
    for mh, nv in zip(meshes, nvs):
        ref = orc.hypersingular_matvec(mh, np.ascontiguousarray(x[:, off:off + nv]),
                                       slp_matvec=orc.H2(mh, 0, m=4).matvec)
        close(y[:, off:off + nv], ref, 1e-10)
        off += nv


def test_rejects_double_layer(H):
    import torch

    mesh = I.sphere(4)
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=1)
    x = torch.zeros((1, mesh.nv), dtype=torch.float64, device="cuda")
    with pytest.raises(H.H2bemError) as err:
        H.h2bem_apply_hypersingular(op.op, x, x.clone())
    assert err.value.code == H.H2BEM_ERR_ARG
    op.close()
