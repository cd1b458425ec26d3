"""Stored nearfield (opts.store_near) against the oracle.

The stored blocks hold the same entries the on-the-fly kernels evaluate (the
7 x 7-point rule on regular pairs, Sauter-Schwab on pairs sharing a vertex),
rounded once to the tier's working precision, so the tolerances are those of
the on-the-fly tiers (relative, 2-norm over all right-hand sides):
  FP64        1e-10  (rounding order only)
  MIXED_FP32  1e-6   (entries stored in FP32: one rounding of ~6e-8 each, and
                      FP32 products and row sums)
With eta = 0 every block is nearfield, so the stored blocks are the whole
dense Galerkin matrix: the apply then equals the oracle's dense matrix times x,
and it is bit-for-bit repeatable (each row of y is summed by one CTA, in a
fixed order, without atomics).
"""
import ctypes

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


def apply_np(op, x, transpose=False):
    import torch

    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.full_like(xd, float("nan"))
    op.apply(xd, yd, transpose=transpose)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def stored_apply(H, mesh, x, kernel=0, m=4, eta=2.0, leaf=32, precision="fp64", transpose=False, **kw):
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=kernel, m=m, eta=eta, leaf_size=leaf,
                    precision=precision, store_near=True, **kw)
    y = apply_np(op, x, transpose)
    st = op.stats()
    op.close()
    return y, st


MESHES = {
    "sphere2k": lambda: I.sphere(16),
    "cube": lambda: I.cube(11),
    "jitter": lambda: I.jitter(I.sphere(13), 0.01, 2),
}


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_stored_matches_oracle(H, orc, name, kernel, precision):
    mesh = MESHES[name]()
    x = I.rhs(mesh.nt, 3, seed=11)
    y, st = stored_apply(H, mesh, x, kernel=kernel, precision=precision)
    ref = orc.H2(mesh, kernel, m=4).matvec(x)
    close(y, ref, TOL[precision])
    es = 8 if precision == "fp64" else 4
    # every ordered nearfield pair once, plus the odd leading dimension and 16-byte padding
    assert st["near_pairs"] * es <= st["near_stored_bytes"] <= 1.3 * st["near_pairs"] * es


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_stored_transpose(H, orc, kernel, precision):
    mesh = I.jitter(I.ellipsoid(12), 0.01, 6)
    x = I.rhs(mesh.nt, 2, seed=9)
    y, _ = stored_apply(H, mesh, x, kernel=kernel, precision=precision, transpose=True)
    ref = orc.H2(mesh, kernel, m=4).matvec(x, transpose=True)
    close(y, ref, TOL[precision])


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("transpose", [False, True])
def test_stored_equals_on_the_fly_on_cube(H, orc, kernel, transpose):
    """Jittered cube, both directions: both tiers against the oracle, and the
    mixed tier's stored nearfield against its on-the-fly one (the two differ
    by the FP32 rounding of the stored entries and the order of the sums)."""
    mesh = I.jitter(I.cube(9), 0.01, 3)
    x = I.rhs(mesh.nt, 2, seed=9)
    y, _ = stored_apply(H, mesh, x, kernel=kernel, transpose=transpose)
    close(y, orc.H2(mesh, kernel, m=4).matvec(x, transpose=transpose), TOL["fp64"])
    ys, _ = stored_apply(H, mesh, x, kernel=kernel, precision="mixed_fp32", transpose=transpose)
    a = H.Operator(mesh.vertices, mesh.triangles, kernel=kernel, precision="mixed_fp32")
    yf = apply_np(a, x, transpose)
    a.close()
    close(ys, yf, 3e-7)
    close(ys, orc.H2(mesh, kernel, m=4).matvec(x, transpose=transpose), TOL["mixed_fp32"])


@pytest.mark.parametrize("nrhs", [1, 4, 5, 8, 16, 21])
@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_stored_rhs_widths(H, orc, nrhs, precision):
    """Widths 1, 4, 8, 16 and the padded ones (5 -> 8, 21 -> 16 + 8)."""
    mesh = I.ellipsoid(10)
    x = I.rhs(mesh.nt, nrhs, seed=nrhs)
    y, _ = stored_apply(H, mesh, x, kernel=1, precision=precision)
    ref = orc.H2(mesh, 1, m=4).matvec(x)
    close(y, ref, TOL[precision])


@pytest.mark.parametrize("leaf", [1, 7, 33, 64])
@pytest.mark.parametrize("kernel", [0, 1])
def test_stored_leaf_sizes(H, orc, leaf, kernel):
    """Odd leaves (leading dimension = leaf size), one-triangle leaves, and
    leaves of more than 32 triangles (two rows per lane)."""
    mesh = I.jitter(I.sphere(10), 0.01, 5)
    x = I.rhs(mesh.nt, 4, seed=leaf)
    for tr in (False, True):
        y, _ = stored_apply(H, mesh, x, kernel=kernel, leaf=leaf, transpose=tr)
        ref = orc.H2(mesh, kernel, m=4, leaf=leaf).matvec(x, transpose=tr)
        close(y, ref, 1e-10)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_stored_dense_equals_oracle_matrix_and_repeats_bitwise(H, orc, kernel, precision):
    mesh = I.jitter(I.sphere(7), 0.02, 4)
    x = I.rhs(mesh.nt, 3, seed=1)
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=kernel, eta=0.0, precision=precision, store_near=True)
    y1 = apply_np(op, x)
    y2 = apply_np(op, x)
    yt = apply_np(op, x, transpose=True)
    op.close()
    A = orc.dense_matrix(kernel, mesh)
    close(y1, x @ A.T, TOL[precision])
    close(yt, x @ A, TOL[precision])
    assert np.array_equal(y1, y2)


def test_stored_equals_on_the_fly_with_cache_and_fp64_singular(H):
    """The stored entries are those of the on-the-fly apply; with cached
    singular entries and with FP64 singular points in the mixed tier."""
    mesh = I.jitter(I.sphere(14), 0.01, 8)
    x = I.rhs(mesh.nt, 8, seed=2)
    for kw in ({}, {"cache_singular": True}, {"singular_fp64": True}):
        for kernel in (0, 1):
            a = H.Operator(mesh.vertices, mesh.triangles, kernel=kernel, precision="mixed_fp32", **kw)
            ya = apply_np(a, x)
            a.close()
            yb, _ = stored_apply(H, mesh, x, kernel=kernel, precision="mixed_fp32", **kw)
            close(yb, ya, 5e-7)


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_stored_batch(H, orc, precision):
    meshes = [I.sphere(6), I.jitter(I.cube(5), 0.01, 1), I.ellipsoid(7)]
    B = H.BatchOperator(meshes, kernel=0, m=4, precision=precision, store_near=True)
    x = I.rhs(B.n, 2, seed=3)
    y = apply_np(B, x)
    B.close()
    for k, mh in enumerate(meshes):
        a, b = int(np.sum([m.nt for m in meshes[:k]])), int(np.sum([m.nt for m in meshes[:k + 1]]))
        ref = orc.H2(mh, 0, m=4).matvec(np.ascontiguousarray(x[:, a:b]))
        close(y[:, a:b], ref, TOL[precision])


def test_stored_graph_replay_and_noalloc(H, orc):
    import torch

    mesh = I.ellipsoid(9)
    x = I.rhs(mesh.nt, 4, seed=6)
    ref = orc.H2(mesh, 0, m=4).matvec(x)
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=0, precision="mixed_fp32", store_near=True,
                    use_graph=True)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    s = torch.cuda.Stream()
    for _ in range(3):  # plain, captured, replayed
        yd.fill_(float("nan"))
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            H.h2bem_apply(op.op, xd, yd, s)
        s.synchronize()
        close(yd.cpu().numpy(), ref, 1e-6)
    y2 = torch.full_like(xd, float("nan"))
    rc = H.lib().h2bem_apply_noalloc(op.op, ctypes.c_void_p(xd.data_ptr()), xd.shape[1], xd.shape[0],
                                     ctypes.c_void_p(y2.data_ptr()), y2.shape[1], None)
    torch.cuda.synchronize()
    assert rc == H.H2BEM_OK
    close(y2.cpu().numpy(), ref, 1e-6)
    op.close()


def test_stored_dtn_solve_matches_on_the_fly(H):
    """Conjugate gradients on the stored operators: same solution as on the fly."""
    import torch

    mesh = I.sphere(12)
    b = I.rhs(mesh.nt, 2, seed=4)
    out = []
    for store in (False, True):
        G = H.Operator(mesh.vertices, mesh.triangles, kernel=0, precision="mixed_fp32", store_near=store)
        K = H.Operator(mesh.vertices, mesh.triangles, kernel=1, precision="mixed_fp32", store_near=store)
        bd = torch.from_numpy(b).cuda()
        rhs = torch.empty_like(bd)
        H.h2bem_apply_mass(K.op, 0.5, bd, rhs)
        xd = torch.empty_like(bd)
        it, relres = H.h2bem_cg(G.op, rhs, xd, rtol=1e-9, maxit=2000)
        torch.cuda.synchronize()
        assert max(relres) < 1e-9
        out.append(xd.cpu().numpy())
        G.close()
        K.close()
    close(out[1], out[0], 1e-5)
