"""The allocation-free apply (h2bem_apply_noalloc) against the ordinary apply.

h2bem_apply_noalloc exists for callers that cannot let the library allocate
device memory when they apply an operator (for example a caller whose device
memory is all handed out by its own pool allocator).  It keeps its work
vectors in a fixed array inside the library.  These tests call it through the
C ABI twice in a row, so that the second call starts from the first call's
leftover work vectors, and compare both results with h2bem_apply's.  The file
is named so that pytest collects it after every other test file.
"""
import ctypes

import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed_fp32": 1e-6, "mixed_tf32": 1e-6, "mixed_bf16": 1e-6}


@pytest.fixture(scope="module")
def H():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_05523_gb300 import build, h2bem

    build.build()
    return h2bem


def _noalloc(H, op, x, y):
    """Call the C entry point directly: (nrhs, n) device tensors."""
    import torch

    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = H.lib().h2bem_apply_noalloc(op.op, ctypes.c_void_p(x.data_ptr()), x.shape[1], x.shape[0],
                                     ctypes.c_void_p(y.data_ptr()), y.shape[1], stream)
    return rc


# Every tier, and the options that change the launch sequence (recomputed
# bases, cached singular entries, FP64 singular points, stored nearfield).
# The tensor-core tiers run the same kernels in both calls, so they are held to
# the FP32 tier's tolerance against each other.
CASES = [(0, "fp64", {}), (1, "fp64", {}), (0, "mixed_fp32", {}), (1, "mixed_fp32", {}), (0, "mixed_tf32", {}),
         (0, "mixed_bf16", {}), (0, "mixed_fp32", {"recompute_basis": True}), (1, "fp64", {"recompute_basis": True}),
         (0, "mixed_fp32", {"cache_singular": True}), (1, "mixed_fp32", {"singular_fp64": True}),
         (0, "mixed_bf16", {"store_near": True}), (1, "fp64", {"store_near": True})]


@pytest.mark.parametrize("kernel,precision,opts", CASES)
def test_noalloc_matches_apply_twice(H, kernel, precision, opts):
    import torch

    mesh = I.jitter(I.sphere(18), 0.01, 21)
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=kernel, m=4, eta=2.0, precision=precision, **opts)
    x = torch.from_numpy(I.rhs(mesh.nt, 5, seed=31)).cuda()
    ref = torch.empty_like(x)
    H.h2bem_apply(op.op, x, ref)
    for _ in range(2):
        y = torch.full_like(x, float("nan"))
        assert _noalloc(H, op, x, y) == H.H2BEM_OK
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(y - ref) / torch.linalg.norm(ref))
        assert err < TOL[precision], err
    op.close()


def test_noalloc_many_rhs_in_chunks(H):
    import torch

    mesh = I.sphere(10)
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=0, m=3)
    x = torch.from_numpy(I.rhs(mesh.nt, 21, seed=5)).cuda()
    ref = op.apply(x)
    y = torch.empty_like(x)
    for _ in range(2):
        assert _noalloc(H, op, x, y) == H.H2BEM_OK
        torch.cuda.synchronize()
        assert float(torch.linalg.norm(y - ref) / torch.linalg.norm(ref)) < TOL["fp64"]
    op.close()


def test_noalloc_rejects_oversize_and_host_buffers(H):
    import torch

    mesh = I.sphere(96)  # 73,728 triangles: FP64 work space for 16 rhs (~120 MiB) exceeds the fixed array
    op = H.Operator(mesh.vertices, mesh.triangles, kernel=0, m=4, precision="fp64")
    x = torch.zeros((16, mesh.nt), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    assert _noalloc(H, op, x, y) == H.H2BEM_ERR_ARG
    buf = ctypes.create_string_buffer(512)
    H.lib().h2bem_last_error(buf, 512)
    assert b"work space" in buf.value
    xs, ys = x[:1].cpu(), y[:1].cpu()
    assert _noalloc(H, op, xs, ys) == H.H2BEM_ERR_ARG
    op.close()
