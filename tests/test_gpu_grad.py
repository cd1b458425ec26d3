"""GPU shape gradient d/dX sum_r <w_r, A x_r> (A = G or K, FP64, tree and
blocks frozen) against the oracle's hand-derived gradient, which is itself
pinned by central finite differences (tests/test_oracle_grad.py), and
against central differences of the GPU apply."""
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


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("nrhs", [1, 3])
def test_shape_gradient_matches_oracle(H, orc, name, nrhs, kernel):
    import torch

    mk, m, leaf = CASES[name]
    mesh = mk()
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=kernel, m=m, leaf_size=leaf)
    w = I.rhs(mesh.nt, nrhs, seed=31)
    x = I.rhs(mesh.nt, nrhs, seed=32)
    wd, xd = torch.from_numpy(w).cuda(), torch.from_numpy(x).cuda()
    g = torch.zeros((mesh.nv, 3), dtype=torch.float64, device="cuda")
    dx = torch.zeros_like(xd)
    H.h2bem_grad(op.op, wd, xd, g, dx)
    torch.cuda.synchronize()
    ref = orc.H2(mesh, kernel, m=m, leaf=leaf).grad_vertices(w, x)
    gg = g.cpu().numpy()
    err = np.abs(gg - ref).max() / np.abs(ref).max()
    print(f"grad kernel {kernel} {name} nrhs {nrhs}: {err:.2e}")
    # double layer: on the jittered cube's nearly coplanar face pairs the two
    # orientations' terms (k_ij through the points, k_ji through the normal)
    # cancel to a small part of their size, so the two codes' summation orders
    # differ by more (measured 8.9e-11; 4e-13 to 4e-12 on the curved meshes)
    assert err <= (3e-10 if kernel == 1 else 1e-10)
    refx = orc.H2(mesh, kernel, m=m, leaf=leaf).matvec(w, transpose=True)
    assert np.linalg.norm(dx.cpu().numpy() - refx) / np.linalg.norm(refx) < 1e-10
    op.close()


def test_shape_gradient_rejects_stored_cross_approximation_bases(H):
    import torch

    mesh = I.sphere(3)
    for kw in ({"gca": True}, {"hca": True}):
        op = H.Operator(mesh.vertices, mesh.triangles, kernel=0, m=2, **kw)
        z = torch.zeros((1, mesh.nt), dtype=torch.float64, device="cuda")
        g = torch.zeros((mesh.nv, 3), dtype=torch.float64, device="cuda")
        with pytest.raises(H.H2bemError) as e:
            H.h2bem_grad(op.op, z, z, g)
        assert e.value.code == H.H2BEM_ERR_ARG
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


@pytest.mark.parametrize("kernel", [0, 1])
def test_shape_gradient_matches_gpu_central_differences(H, kernel):
    """32 sampled vertex coordinates: the gradient of sum_r <w_r, A(X) x_r>
    against central differences (step 1e-6) of the GPU FP64 apply with the
    cluster tree held fixed (uploaded unchanged; boxes and blocks follow the
    moved vertices, and a coordinate whose move changes the block counts is
    skipped).  Relative to the largest gradient entry: 1e-5."""
    import torch

    mesh = I.jitter(I.sphere(6), 0.03, 41)
    m, leaf, h = 3, 8, 1e-6
    base = H.Operator(mesh.vertices, mesh.triangles, kernel=kernel, m=m, leaf_size=leaf)
    tr = H.h2bem_tree_export(base.tree, mesh.nt)
    counts = (base.stats()["nfar"], base.stats()["nnear"])
    w = I.rhs(mesh.nt, 2, seed=51)
    x = I.rhs(mesh.nt, 2, seed=52)
    wd, xd = torch.from_numpy(w).cuda(), torch.from_numpy(x).cuda()
    g = torch.zeros((mesh.nv, 3), dtype=torch.float64, device="cuda")
    H.h2bem_grad(base.op, wd, xd, g)
    torch.cuda.synchronize()
    g = g.cpu().numpy()
    base.close()

    def f(X):
        ms = H.h2bem_mesh_create(X, mesh.triangles)
        ts = H.h2bem_tree_upload(ms, tr["perm"], tr["begin"], tr["end"], tr["child0"], tr["child1"])
        o = H.h2bem_opts_default()
        op = H.h2bem_operator_create(ms, ts, kernel, m, 2.0, o)
        st = H.h2bem_stats_get(op)
        y = torch.empty_like(xd)
        H.h2bem_apply(op, xd, y)
        torch.cuda.synchronize()
        val = float((wd * y).sum())
        for hd, fn in ((op, H.h2bem_operator_destroy), (ts, H.h2bem_tree_destroy), (ms, H.h2bem_mesh_destroy)):
            fn(hd)
        return val, (st["nfar"], st["nnear"])

    rng = np.random.default_rng(7)
    picks = [(int(v), int(d)) for v, d in zip(rng.choice(mesh.nv, 32, replace=False), rng.integers(0, 3, 32))]
    scale = np.abs(g).max()
    checked = 0
    for v, d in picks:
        Xp, Xm = mesh.vertices.copy(), mesh.vertices.copy()
        Xp[v, d] += h
        Xm[v, d] -= h
        fp, cp = f(Xp)
        fm, cm = f(Xm)
        if cp != counts or cm != counts:
            continue
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[v, d]) <= 1e-5 * scale, (v, d, fd, g[v, d])
        checked += 1
    assert checked >= 24
