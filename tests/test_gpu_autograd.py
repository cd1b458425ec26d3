"""Gradients through the torch.autograd wrapper: d<w, A x>/dx = A^T x-gradient
by the hand-written transposed pass, against the oracle's transposed H^2
product and central finite differences (the map is linear, so differences at
any step agree up to rounding)."""
import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_05523_gb300 import autograd, build, h2bem

    build.build()
    return h2bem, autograd


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_grad_wrt_x(mods, orc, kernel, precision):
    import torch

    H, A = mods
    mesh = I.jitter(I.sphere(12), 0.01, 17)
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=kernel, m=4, precision=precision)
    x = torch.from_numpy(I.rhs(mesh.nt, 2, seed=1)).cuda().requires_grad_(True)
    w = torch.from_numpy(I.rhs(mesh.nt, 2, seed=2)).cuda()
    loss = (w * A.h2_apply(x, op)).sum()
    loss.backward()
    g = x.grad.cpu().numpy()
    ref = orc.H2(mesh, kernel, m=4).matvec(w.cpu().numpy(), transpose=True)
    tol = 1e-10 if precision == "fp64" else 1e-6
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < tol
    if precision != "fp64":  # FP32 rounding noise swamps a difference quotient
        op.close()
        return
    # central differences on sampled coordinates
    rng = np.random.default_rng(3)
    with torch.no_grad():
        for _ in range(4):
            r, i = int(rng.integers(0, 2)), int(rng.integers(0, mesh.nt))
            e = torch.zeros_like(x)
            e[r, i] = 1e-6
            fd = ((w * A.h2_apply(x + e, op)).sum() - (w * A.h2_apply(x - e, op)).sum()) / 2e-6
            assert abs(float(fd) - g[r, i]) <= 1e-5 * max(abs(g[r, i]), np.abs(g).max() * 1e-3)
    op.close()
