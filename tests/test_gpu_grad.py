"""GPU shape gradient d/dX sum_r <w_r, G x_r> (single layer, FP64, tree and
blocks frozen) against the oracle's hand-derived gradient, which is itself
pinned by central finite differences (tests/test_oracle_grad.py)."""
import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_05523_gb300 import build, h2bem

    build.build()
    return h2bem


CASES = {
    "sphere_m3_leaf6": (lambda: I.jitter(I.sphere(5), 0.05, 11), 3, 6),
    "cube_m3_leaf6": (lambda: I.jitter(I.cube(4), 0.02, 12), 3, 6),
    "ellipsoid_m4_leaf32": (lambda: I.jitter(I.ellipsoid(14), 0.01, 13), 4, 32),
    "sphere_m2_leaf1": (lambda: I.jitter(I.sphere(3), 0.03, 14), 2, 1),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("nrhs", [1, 3])
def test_shape_gradient_matches_oracle(H, orc, name, nrhs):
    import torch

    mk, m, leaf = CASES[name]
    mesh = mk()
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=0, m=m, leaf_size=leaf)
    w = I.rhs(mesh.nt, nrhs, seed=31)
    x = I.rhs(mesh.nt, nrhs, seed=32)
    wd, xd = torch.from_numpy(w).cuda(), torch.from_numpy(x).cuda()
    g = torch.zeros((mesh.nv, 3), dtype=torch.float64, device="cuda")
    dx = torch.zeros_like(xd)
    H.h2bem_grad(op.op, wd, xd, g, dx)
    torch.cuda.synchronize()
    ref = orc.H2(mesh, 0, m=m, leaf=leaf).grad_vertices(w, x)
    gg = g.cpu().numpy()
    assert np.abs(gg - ref).max() <= 1e-10 * np.abs(ref).max()
    refx = orc.H2(mesh, 0, m=m, leaf=leaf).matvec(w, transpose=True)
    assert np.linalg.norm(dx.cpu().numpy() - refx) / np.linalg.norm(refx) < 1e-10
    op.close()


def test_shape_gradient_rejects_double_layer(H):
    import torch

    mesh = I.sphere(3)
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=1, m=2)
    z = torch.zeros((1, mesh.nt), dtype=torch.float64, device="cuda")
    g = torch.zeros((mesh.nv, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(H.H2bemError):
        H.h2bem_grad(op.op, z, z, g)
    op.close()


def test_autograd_shape_and_batch(H, orc):
    """The autograd wrapper returns G^T g and the shape gradient; on a batch of
    meshes (one block-diagonal operator) the gradient equals the per-mesh
    gradients."""
    import torch

    from paper_2001_05523_gb300 import autograd as A

    meshes = [I.jitter(I.sphere(6), 0.02, 41), I.jitter(I.cube(5), 0.02, 42), I.jitter(I.ellipsoid(7), 0.02, 43)]
    B = H.BatchOperator(meshes, kernel=0, m=3, leaf_size=8)
    V = torch.from_numpy(np.concatenate([mm.vertices for mm in meshes])).cuda().requires_grad_(True)
    x = torch.from_numpy(I.rhs(B.n, 2, seed=5)).cuda().requires_grad_(True)
    w = torch.from_numpy(I.rhs(B.n, 2, seed=6)).cuda()
    loss = (w * A.h2_apply_shape(x, V, B)).sum()
    loss.backward()
    gV = V.grad.cpu().numpy()
    gx = x.grad.cpu().numpy()
    voff = 0
    for b, mesh in enumerate(meshes):
        lo, hi = int(B.offsets[b]), int(B.offsets[b + 1])
        Ho = orc.H2(mesh, 0, m=3, leaf=8)
        ref = Ho.grad_vertices(w[:, lo:hi].cpu().numpy(), x[:, lo:hi].detach().cpu().numpy())
        assert np.abs(gV[voff:voff + mesh.nv] - ref).max() <= 1e-10 * np.abs(ref).max()
        refx = Ho.matvec(w[:, lo:hi].cpu().numpy(), transpose=True)
        assert np.linalg.norm(gx[:, lo:hi] - refx) / np.linalg.norm(refx) < 1e-10
        voff += mesh.nv
    B.close()
