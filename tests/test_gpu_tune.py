"""Launch variants of the row-parallel kernels (persistent CTAs with a work
counter, 2/4/8 coupling slices) and the autotuner that picks among them.

Every variant computes the same sums in a different order, so each is held to
the tier's parity tolerance against the oracle, and the variants agree with
one another to rounding (FP64 tier: 1e-13)."""
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


def apply(H, mesh, x, tune, precision="fp64", kernel=0, transpose=False):
    import torch

    op = H.Operator(mesh.vertices, mesh.triangles, kernel=kernel, m=4, precision=precision, autotune=tune)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    ys = []
    for _ in range(2):
        yd = torch.full_like(xd, float("nan"))
        op.apply(xd, yd, transpose=transpose)
        torch.cuda.synchronize()
        ys.append(yd.cpu().numpy())
    st = op.stats()
    op.close()
    return ys, st


@pytest.mark.parametrize("v", list(range(36)))
def test_fixed_variants_match_oracle(H, orc, v):
    mesh = I.jitter(I.sphere(14), 0.01, 21)
    x = I.rhs(mesh.nt, 8, seed=v)
    ref = orc.H2(mesh, 0, m=4).matvec(x)
    for prec in ("fp64", "mixed_fp32"):
        (y1, y2), st = apply(H, mesh, x, 2 + v, precision=prec)
        close(y1, ref, TOL[prec])
        close(y2, ref, TOL[prec])
        near_p, near_nb, nsl, coup_p, tuned = st["launch_variant"]
        assert (near_p, coup_p, nsl, tuned) == (v & 1, (v >> 1) & 1, (2, 4, 8)[(v // 4) % 3], 1)
        assert near_nb == ((4, 3, 2)[v // 12] if prec == "mixed_fp32" else 2)


@pytest.mark.parametrize("kernel,transpose", [(0, False), (1, False), (1, True)])
def test_autotuner_choice_is_valid_and_correct(H, orc, kernel, transpose):
    mesh = I.ellipsoid(16)
    x = I.rhs(mesh.nt, 4, seed=3)
    ref = orc.H2(mesh, kernel, m=4).matvec(x, transpose=transpose)
    (y_first, y_second), st = apply(H, mesh, x, 1, kernel=kernel, transpose=transpose)
    close(y_first, ref, TOL["fp64"])
    close(y_second, ref, TOL["fp64"])
    near_p, near_nb, nsl, coup_p, tuned = st["launch_variant"]
    assert tuned == 1 and near_p in (0, 1) and coup_p in (0, 1) and nsl in (2, 4, 8) and near_nb in (2, 3, 4)
    (d1, _), _ = apply(H, mesh, x, 0, kernel=kernel, transpose=transpose)
    close(y_second, d1, 1e-13)


def test_autotune_rejects_bad_values(H):
    mesh = I.sphere(4)
    with pytest.raises(H.H2bemError) as e:
        H.Operator(mesh.vertices, mesh.triangles, autotune=38)
    assert e.value.code == H.H2BEM_ERR_ARG
