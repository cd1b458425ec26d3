"""GCA cluster bases (section 4) on the GPU against the oracle's GCA product.

Both sides build the same bases (the same ranks and pivot triangles, checked
on the host in tests/test_lib_host.py) and the same nearfield, so the
products agree to rounding: FP64 tier 1e-10, MIXED_FP32 1e-6 (FP32 bases,
transfers, coupling matrices and cluster vectors), in the 2-norm and per row.
"""
import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I
from tests._parity import close

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


def gca_apply(H, mesh, x, precision="fp64", q=4, kmax=64, eps=1e-6, eta=2.0, transpose=False, **kw):
    import torch

    op = H.Operator(mesh.vertices, mesh.triangles, kernel=0, m=4, eta=eta, leaf_size=32, precision=precision,
                    gca=True, gca_q=q, gca_kmax=kmax, gca_eps=eps, **kw)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.full_like(xd, float("nan"))
    op.apply(xd, yd, transpose=transpose)
    torch.cuda.synchronize()
    st = op.stats()
    y = yd.cpu().numpy()
    op.close()
    return y, st


MESHES = {
    "sphere": lambda: I.sphere(20),
    "jitter_ellipsoid": lambda: I.jitter(I.ellipsoid(16), 0.01, 3),
    "cube": lambda: I.cube(14),
}


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_gca_matches_oracle(H, orc, name, precision):
    mesh = MESHES[name]()
    x = I.rhs(mesh.nt, 3, seed=11)
    y, st = gca_apply(H, mesh, x, precision=precision)
    G = orc.GCA(mesh, q=4, eps=1e-6, kmax=64)
    close(y, G.matvec(x), TOL[precision], f"gca {name} {precision}")
    assert abs(st["mean_rank"] - G.ranks().mean()) < 1e-12
    assert st["far_stored_bytes"] > 0


@pytest.mark.parametrize("q,kmax,eps", [(2, 16, 1e-4), (5, 64, 1e-8), (3, 33, 0.0)])
def test_gca_parameters(H, orc, q, kmax, eps):
    mesh = I.jitter(I.sphere(14), 0.01, 8)
    x = I.rhs(mesh.nt, 2, seed=q)
    y, _ = gca_apply(H, mesh, x, q=q, kmax=kmax, eps=eps)
    close(y, orc.GCA(mesh, q=q, eps=eps, kmax=kmax).matvec(x), TOL["fp64"], f"gca q{q} kmax{kmax}")


@pytest.mark.parametrize("nrhs", [1, 5, 16, 21])
def test_gca_rhs_widths_and_transpose(H, orc, nrhs):
    mesh = I.jitter(I.sphere(12), 0.01, 5)
    x = I.rhs(mesh.nt, nrhs, seed=nrhs)
    ref = orc.GCA(mesh, q=4, eps=1e-6, kmax=64).matvec(x)
    for tr in (False, True):  # G~ is symmetric: the transposed apply runs the same farfield
        y, _ = gca_apply(H, mesh, x, transpose=tr)
        close(y, ref, TOL["fp64"], f"gca nrhs {nrhs} transpose {tr}")


def test_gca_with_stored_nearfield_and_cached_singular(H, orc):
    mesh = I.jitter(I.cube(10), 0.01, 2)
    x = I.rhs(mesh.nt, 4, seed=2)
    ref = orc.GCA(mesh, q=4, eps=1e-6, kmax=64).matvec(x)
    for kw in ({"store_near": True}, {"cache_singular": True}):
        for prec in ("fp64", "mixed_fp32"):
            y, _ = gca_apply(H, mesh, x, precision=prec, **kw)
            close(y, ref, TOL[prec], f"gca {kw} {prec}")


def test_gca_far_more_accurate_than_chebyshev_at_lower_rank(H, orc):
    """At m = 4 the Chebyshev bases carry k = 64 values per cluster; the GCA
    bases at q = 4, eps = 1e-6 a mean rank below that, and the product is
    closer to the dense Galerkin matrix (eq. (slp))."""
    import torch

    mesh = I.sphere(24)
    x = I.rhs(mesh.nt, 2, seed=1)
    d = orc.dense_matvec(0, mesh, x)
    yg, st = gca_apply(H, mesh, x)
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=0, m=4, eta=2.0, precision="fp64")
    yc = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    op.close()
    eg = np.linalg.norm(yg - d) / np.linalg.norm(d)
    ec = np.linalg.norm(yc - d) / np.linalg.norm(d)
    print(f"dense error: gca {eg:.2e} (mean rank {st['mean_rank']:.1f}), chebyshev m4 {ec:.2e}")
    assert st["mean_rank"] < 64 and eg < 0.01 * ec


def test_gca_rejects_unsupported(H):
    import torch

    mesh = I.sphere(6)
    for kw in ({"kernel": 1}, {"precision": "mixed_tf32"}, {"recompute_basis": True}, {"gca_kmax": 65},
               {"gca_q": 0}):
        args = dict(kernel=0, m=4, eta=2.0, precision="fp64", gca=True)
        args.update(kw)
        with pytest.raises(H.H2bemError) as e:
            H.Operator(mesh.vertices, mesh.triangles, **args)
        assert e.value.code == H.H2BEM_ERR_ARG
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=0, gca=True)
    w = torch.zeros((1, mesh.nt), dtype=torch.float64, device="cuda")
    g = torch.zeros((mesh.nv, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(H.H2bemError) as e:
        H.h2bem_grad(op.op, w, w, g)
    assert e.value.code == H.H2BEM_ERR_ARG
    op.close()
