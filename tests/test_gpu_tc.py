"""Tensor-core coupling (tcgen05) against the oracle.

Tiers and tolerances (relative, 2-norm over all right-hand sides, against the
oracle's FP64 H^2 product):
  MIXED_TF32  1e-3   operands S and x-hat rounded to TF32 (round to nearest,
                     unit roundoff u = 2^-11): each product of the coupling
                     carries at most 2u ~ 9.8e-4 relative error, and the
                     farfield is a part of y, so the result stays below 2u
  MIXED_BF16  1e-2   the same with BF16 operands (u = 2^-9, 2u ~ 3.9e-3), with
                     a factor 2.5 for the sums
  MIXED_FP32  1e-6   SIMT FP32 coupling (reference point of the ordering test)
The double layer keeps its coupling on the SIMT kernels in every mixed tier
(its differentiated-basis side is FP64), so it is held to the mixed tolerance.
"""
import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"mixed_tf32": 1e-3, "mixed_bf16": 1e-2, "mixed_fp32": 1e-6}


@pytest.fixture(scope="module")
def H():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_05523_gb300 import build, h2bem

    build.build()
    return h2bem


from tests._parity import close, rel  # noqa: E402


def run(H, mesh, x, kernel=0, m=4, precision="mixed_tf32", transpose=False, leaf=32):
    import torch

    op = H.Operator(mesh.vertices, mesh.triangles, kernel=kernel, m=m, eta=2.0, leaf_size=leaf, precision=precision)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.full_like(xd, float("nan"))
    op.apply(xd, yd, transpose=transpose)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    op.close()
    return y


@pytest.mark.parametrize("precision", ["mixed_tf32", "mixed_bf16", "mixed_fp32"])
@pytest.mark.parametrize("nrhs", [1, 4, 8, 16])
def test_slp_tiers_match_oracle(H, orc, precision, nrhs):
    mesh = I.jitter(I.sphere(16), 0.01, 7)
    x = I.rhs(mesh.nt, nrhs, seed=40 + nrhs)
    y = run(H, mesh, x, precision=precision)
    ref = orc.H2(mesh, 0, m=4).matvec(x)
    close(y, ref, TOL[precision])


@pytest.mark.parametrize("precision", ["mixed_tf32", "mixed_bf16"])
@pytest.mark.parametrize("m", [2, 3, 5])
def test_tc_orders(H, orc, precision, m):
    """m = 5: k = 125 rows in two 64-row tiles, K padded to 128; m = 2, 3: one padded tile."""
    mesh = I.ellipsoid(12)
    x = I.rhs(mesh.nt, 3, seed=m)
    y = run(H, mesh, x, m=m, precision=precision)
    ref = orc.H2(mesh, 0, m=m).matvec(x)
    close(y, ref, TOL[precision])


@pytest.mark.parametrize("precision", ["mixed_tf32", "mixed_bf16", "mixed_fp32"])
def test_slp_transpose(H, orc, precision):
    mesh = I.jitter(I.cube(9), 0.01, 3)
    x = I.rhs(mesh.nt, 2, seed=9)
    y = run(H, mesh, x, precision=precision, transpose=True)
    ref = orc.H2(mesh, 0, m=4).matvec(x, transpose=True)
    close(y, ref, TOL[precision])


@pytest.mark.parametrize("precision", ["mixed_tf32", "mixed_bf16"])
@pytest.mark.parametrize("transpose", [False, True])
def test_dlp_keeps_simt_coupling(H, orc, precision, transpose):
    mesh = I.ellipsoid(12)
    x = I.rhs(mesh.nt, 2, seed=5)
    y = run(H, mesh, x, kernel=1, precision=precision, transpose=transpose)
    ref = orc.H2(mesh, 1, m=4).matvec(x, transpose=transpose)
    close(y, ref, TOL["mixed_fp32"])


def test_tiers_ordered_by_operand_precision(H):
    """Against the FP64 tier on the same operator: BF16 error > TF32 error > FP32 error."""
    mesh = I.sphere(24)
    x = I.rhs(mesh.nt, 8, seed=3)
    ref = run(H, mesh, x, precision="fp64")
    e = {p: rel(run(H, mesh, x, precision=p), ref) for p in ("mixed_fp32", "mixed_tf32", "mixed_bf16")}
    assert e["mixed_fp32"] < e["mixed_tf32"] < e["mixed_bf16"], e
    assert e["mixed_fp32"] < 1e-6 and e["mixed_tf32"] < 1e-3 and e["mixed_bf16"] < 1e-2, e


def test_tc_tiers_reject_m6(H):
    mesh = I.sphere(4)
    for p in ("mixed_tf32", "mixed_bf16"):
        with pytest.raises(H.H2bemError) as err:
            H.Operator(mesh.vertices, mesh.triangles, kernel=0, m=6, precision=p)
        assert err.value.code == H.H2BEM_ERR_ARG


def test_tc_timeout_path_reports_and_recovers(H, orc):
    """The bounded waits of the tensor-core coupling: with opts.tc_wait_test the
    first pipeline wait of every CTA with three or more blocks waits on a
    barrier that nothing signals and gives up after about 50 us.  The CTA
    drains the MMAs it issued (normal bound), frees its tensor memory and
    returns; h2bem_stats_get reports H2BEM_ERR_TIMEOUT, the next call finds the
    flag cleared, and an ordinary operator on the same context gives the
    oracle's result."""
    import torch

    mesh = I.jitter(I.sphere(16), 0.01, 7)
    x = I.rhs(mesh.nt, 4, seed=2)
    xd = torch.from_numpy(x).cuda()
    bad = H.Operator(mesh.vertices, mesh.triangles, kernel=0, m=4, eta=2.0, precision="mixed_tf32", tc_wait_test=True)
    yd = torch.empty_like(xd)
    H.h2bem_apply(bad.op, xd, yd)  # device buffers: asynchronous, no status here
    torch.cuda.synchronize()
    with pytest.raises(H.H2bemError) as e:
        bad.stats()
    assert e.value.code == H.H2BEM_ERR_TIMEOUT
    bad.stats()  # the flag was read and cleared
    # host buffers: the synchronous apply reports it itself
    yh = np.zeros_like(x)
    with pytest.raises(H.H2bemError) as e:
        bad.apply(x, yh)
    assert e.value.code == H.H2BEM_ERR_TIMEOUT
    bad.close()
    y = run(H, mesh, x, precision="mixed_tf32")
    close(y, orc.H2(mesh, 0, m=4).matvec(x), TOL["mixed_tf32"], "after the timeout")
