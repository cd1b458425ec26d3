"""Batched meshes as one block-diagonal operator (every stage one launch over
all meshes) and CUDA-graph replay of the apply sequence."""
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


def _family():
    # uneven sizes and all three shape types, jittered (small members of the batch family)
    return [I.jitter(I.sphere(9), 0.01, 1), I.jitter(I.ellipsoid(13), 0.01, 2), I.jitter(I.cube(7), 0.01, 3),
            I.jitter(I.sphere(17), 0.01, 4), I.jitter(I.cube(11), 0.01, 5), I.sphere(1)]


@pytest.mark.parametrize("kernel,precision", [(0, "fp64"), (1, "fp64"), (0, "mixed_fp32")])
def test_batch_equals_single_operators(H, kernel, precision):
    import torch

    meshes = _family()
    B = H.BatchOperator(meshes, kernel=kernel, m=4, precision=precision)
    x = torch.from_numpy(I.rhs(B.n, 3, seed=7)).cuda()
    y = B.apply(x)
    torch.cuda.synchronize()
    for b, mesh in enumerate(meshes):
        lo, hi = int(B.offsets[b]), int(B.offsets[b + 1])
        op = H.Operator(mesh.vertices, mesh.triangles, kernel=kernel, m=4, precision=precision)
        yb = op.apply(x[:, lo:hi].contiguous())
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(y[:, lo:hi] - yb) / torch.linalg.norm(yb))
        assert err < (1e-12 if precision == "fp64" else 1e-6), (b, err)
        op.close()
    st = B.stats()
    assert st["n"] == B.n
    B.close()


def test_batch_against_oracle(H, orc):
    import torch

    meshes = _family()[:3]
    B = H.BatchOperator(meshes, kernel=1, m=4)
    x = I.rhs(B.n, 2, seed=9)
    y = B.apply(torch.from_numpy(x).cuda(), transpose=True).cpu().numpy()
    for b, mesh in enumerate(meshes):
        lo, hi = int(B.offsets[b]), int(B.offsets[b + 1])
        ref = orc.H2(mesh, 1, m=4).matvec(x[:, lo:hi], transpose=True)
        assert np.linalg.norm(y[:, lo:hi] - ref) / np.linalg.norm(ref) < 1e-10
    B.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_graph_replay_matches_plain_launches(H, precision):
    import torch

    mesh = I.jitter(I.sphere(14), 0.01, 8)
    g = H.Operator(mesh.vertices, mesh.triangles, kernel=0, m=4, precision=precision, use_graph=True)
    p = H.Operator(mesh.vertices, mesh.triangles, kernel=0, m=4, precision=precision)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        x = torch.from_numpy(I.rhs(mesh.nt, 5, seed=2)).cuda()
        ref = p.apply(x)
        y = torch.empty_like(x)
        for it in range(4):  # plain, capture, replay, replay
            x.copy_(torch.from_numpy(I.rhs(mesh.nt, 5, seed=2 + it)).cuda())
            ref = p.apply(x)
            y.zero_()
            H.h2bem_apply(g.op, x, y, s)
            s.synchronize()
            assert float(torch.linalg.norm(y - ref) / torch.linalg.norm(ref)) < 1e-13
        assert g.stats()["launches"] == p.stats()["launches"]
    g.close()
    p.close()
