"""Transfers over the top levels of the tree in one launch each way (section
2, eq. (transfer)) against the oracle's H^2 product, over repeated applies of
one operator.

In the FP32 tiers with m = 4 (up to 8 right-hand sides) the levels with at
most 1,024 parents run as one launch each way (k_up_tree: per-cluster arrival
counts, the last child's warp computes the parent; k_down_top: each cluster
below them walks its ancestor path from the root); the other levels, and the
other tiers and orders, launch per level.  The arrival counts carry over from
one apply to the next, so every apply of the same operator is checked, in
both directions."""
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


from tests._parity import close  # noqa: E402


@pytest.mark.parametrize("m", [4, 5])
@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_repeated_applies_match_oracle(H, orc, precision, kernel, m):
    import torch

    mesh = I.jitter(I.sphere(14), 0.01, 3 + m)
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=kernel, m=m, eta=2.0, precision=precision)
    ref = orc.H2(mesh, kernel, m=m)
    for it, (nrhs, tr) in enumerate(((3, False), (8, True), (1, False), (16, False), (5, True))):
        x = I.rhs(mesh.nt, nrhs, seed=10 * m + it)
        y = op.apply(torch.from_numpy(x).cuda(), transpose=tr).cpu().numpy()
        close(y, ref.matvec(x, transpose=tr), TOL[precision], f"apply {it} (nrhs {nrhs}, transpose {tr})")
    if precision == "mixed_fp32" and m == 4:
        # every level of this tree has at most 1,024 parents: leaf forward,
        # upward, coupling, downward, leaf backward plus the nearfield, the
        # singular pairs and the permutations (18 for the double layer), a
        # fixed count rather than two per tree level
        assert op.stats()["launches"] <= 20
    op.close()


def test_forest_and_leaf_only_trees(H, orc):
    """Mixed tier (the one-launch path): a batch of meshes of different sizes
    (a forest: several roots at the head of the downward list) and a mesh
    whose tree is one leaf."""
    import torch

    meshes = [I.sphere(9), I.jitter(I.cube(6), 0.01, 2), I.sphere(2)]
    B = H.BatchOperator(meshes, kernel=0, m=4, eta=2.0, precision="mixed_fp32")
    nts = [mm.nt for mm in meshes]
    off = np.concatenate([[0], np.cumsum(nts)])
    x = I.rhs(int(off[-1]), 4, seed=5)
    for _ in range(2):
        y = B.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        for i, mm in enumerate(meshes):
            lo, hi = off[i], off[i + 1]
            close(y[:, lo:hi], orc.H2(mm, 0, m=4).matvec(x[:, lo:hi]), TOL["mixed_fp32"], f"mesh {i}")
    B.close()
    tiny = I.sphere(1)
    op = H.Operator(tiny.vertices, tiny.triangles, kernel=0, m=4, leaf_size=32, precision="mixed_fp32")
    x = I.rhs(tiny.nt, 2, seed=1)
    close(op.apply(torch.from_numpy(x).cuda()).cpu().numpy(), orc.H2(tiny, 0, m=4).matvec(x), TOL["mixed_fp32"])
    op.close()
