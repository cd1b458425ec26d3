"""Host-side library logic (no GPU): the C ABI loads and exports every symbol
include/h2bem.h declares; mesh validation; the library's own cluster tree and
block tree agree exactly with the oracle's (integer work: bit-exact)."""
import re

import numpy as np
import pytest

from paper_2001_05523_gb300 import inputs as I


@pytest.fixture(scope="module")
def H():
    from paper_2001_05523_gb300 import build, h2bem

    build.build()
    return h2bem


def test_exports_every_declared_symbol(H):
    import os

    hdr = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "h2bem.h")).read()
    declared = set(re.findall(r"^int (h2bem_\w+)\(", hdr, flags=re.M))
    assert declared and declared == set(H.EXPORTED)
    L = H.lib()
    for name in declared:
        assert hasattr(L, name)


def test_mesh_validation(H):
    m = I.sphere(2)
    h = H.h2bem_mesh_create(m.vertices, m.triangles)
    H.h2bem_mesh_destroy(h)
    with pytest.raises(H.H2bemError) as e:
        H.h2bem_mesh_create(m.vertices, m.triangles[:, ::-1])  # inward
    assert e.value.code == H.H2BEM_ERR_MESH
    bad = m.triangles.copy()
    bad[0, 0] = m.nv
    with pytest.raises(H.H2bemError) as e:
        H.h2bem_mesh_create(m.vertices, bad)
    assert e.value.code == H.H2BEM_ERR_ARG
    deg = m.triangles.copy()
    deg[0, 1] = deg[0, 0]
    with pytest.raises(H.H2bemError) as e:
        H.h2bem_mesh_create(m.vertices, deg)
    assert e.value.code == H.H2BEM_ERR_MESH


@pytest.mark.parametrize("mk,leaf", [(lambda: I.sphere(16), 32), (lambda: I.cube(9), 32),
                                     (lambda: I.ellipsoid(12), 32), (lambda: I.jitter(I.sphere(10), 0.01, 4), 7),
                                     (lambda: I.sphere(1), 32), (lambda: I.cube(3), 1)])
def test_tree_and_blocks_match_oracle(H, orc, mk, leaf):
    m = mk()
    mh = H.h2bem_mesh_create(m.vertices, m.triangles)
    th = H.h2bem_tree_build(mh, leaf)
    tr = H.h2bem_tree_export(th, m.nt)
    oh = orc.H2(m, orc.SLP, m=2, eta=2.0, leaf=leaf)
    otr = oh.tree()
    for k in tr:
        assert np.array_equal(tr[k], otr[k]), k
    for eta in (2.0, 0.0, 0.7):
        (ft, fs), (nt, ns) = H.h2bem_blocks(th, eta)
        oh = orc.H2(m, orc.SLP, m=2, eta=eta, leaf=leaf)
        (oft, ofs), (ont, ons) = oh.blocks()
        assert sorted(zip(ft.tolist(), fs.tolist())) == sorted(zip(oft.tolist(), ofs.tolist()))
        assert sorted(zip(nt.tolist(), ns.tolist())) == sorted(zip(ont.tolist(), ons.tolist()))
    H.h2bem_tree_destroy(th)
    H.h2bem_mesh_destroy(mh)


def test_tree_upload_roundtrip_and_rejects(H):
    m = I.sphere(6)
    mh = H.h2bem_mesh_create(m.vertices, m.triangles)
    tr = H.h2bem_tree_export(H.h2bem_tree_build(mh, 16), m.nt)
    th = H.h2bem_tree_upload(mh, tr["perm"], tr["begin"], tr["end"], tr["child0"], tr["child1"])
    tr2 = H.h2bem_tree_export(th, m.nt)
    for k in tr:
        assert np.array_equal(tr[k], tr2[k])
    bad = tr["perm"].copy()
    bad[0] = bad[1]
    with pytest.raises(H.H2bemError):
        H.h2bem_tree_upload(mh, bad, tr["begin"], tr["end"], tr["child0"], tr["child1"])
    c1 = tr["child1"].copy()
    c1[0] = -1
    with pytest.raises(H.H2bemError):
        H.h2bem_tree_upload(mh, tr["perm"], tr["begin"], tr["end"], tr["child0"], c1)


def test_operator_create_without_gpu_fails_loudly(H):
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    m = I.sphere(4)
    mh = H.h2bem_mesh_create(m.vertices, m.triangles)
    th = H.h2bem_tree_build(mh, 32)
    with pytest.raises(H.H2bemError) as e:
        H.h2bem_operator_create(mh, th, 0, 4, 2.0)
    assert e.value.code == H.H2BEM_ERR_CUDA


def test_operator_argument_checks(H):
    m = I.sphere(4)
    mh = H.h2bem_mesh_create(m.vertices, m.triangles)
    th = H.h2bem_tree_build(mh, 32)
    for args in ((5, 4, 2.0), (0, 0, 2.0), (0, 9, 2.0), (0, 4, -1.0)):
        with pytest.raises(H.H2bemError) as e:
            H.h2bem_operator_create(mh, th, *args)
        assert e.value.code == H.H2BEM_ERR_ARG
    o = H.h2bem_opts_default()
    o.q_ss = 99
    with pytest.raises(H.H2bemError) as e:
        H.h2bem_operator_create(mh, th, 0, 4, 2.0, o)
    assert e.value.code == H.H2BEM_ERR_ARG
    m8 = I.sphere(8)
    mh8 = H.h2bem_mesh_create(m8.vertices, m8.triangles)
    big = H.h2bem_tree_build(mh8, 200)  # leaves of 128 triangles
    with pytest.raises(H.H2bemError) as e:
        H.h2bem_operator_create(mh8, big, 0, 4, 2.0)
    assert e.value.code == H.H2BEM_ERR_ARG


@pytest.mark.parametrize("mk,q,kmax,eps", [(lambda: I.sphere(16), 4, 64, 1e-6), (lambda: I.jitter(I.sphere(12), 0.01, 3), 3, 40, 1e-5),
                                           (lambda: I.cube(9), 4, 64, 1e-7), (lambda: I.ellipsoid(14), 2, 24, 0.0)])
def test_gca_bases_match_oracle(H, orc, mk, q, kmax, eps):
    """The library's host construction of the GCA bases (section 4) picks the
    same ranks and pivot triangles as the oracle's, cluster by cluster: the
    adaptive cross approximation is a sequence of discrete choices, and the
    pivot rule (first entry within 2^-40 of the largest) makes them agree
    although the two compute L with their own Gauss rules and sums."""
    m = mk()
    mh = H.h2bem_mesh_create(m.vertices, m.triangles)
    th = H.h2bem_tree_build(mh, 32)
    tr = H.h2bem_tree_export(th, m.nt)
    nc = len(tr["begin"])
    rank, piv = H.h2bem_gca_bases(mh, th, nc, q=q, kmax=kmax, eps=eps)
    G = orc.GCA(m, q=q, eps=eps, kmax=kmax)
    assert np.array_equal(rank, G.ranks().astype(np.int64))
    off = np.concatenate([[0], np.cumsum(rank)])
    for c in range(nc):
        assert np.array_equal(tr["perm"][piv[off[c]:off[c + 1]]], G.pivots(c)), c
    H.h2bem_tree_destroy(th)
    H.h2bem_mesh_destroy(mh)


@pytest.mark.parametrize("mk,m,eps_aca,eps", [
    (lambda: I.sphere(12), 4, 1e-6, 1e-6),
    (lambda: I.jitter(I.ellipsoid(10), 0.01, 3), 4, 1e-4, 1e-5),
    (lambda: I.cube(8), 3, 1e-6, 1e-8),
])
def test_hca_ranks_match_oracle(H, orc, mk, m, eps_aca, eps):
    """The library's host construction of the HCA blocks and their compression
    (section 3) takes the same discrete decisions as the oracle: the rank of
    every block's cross approximation (pivot rule within 2^-40 of the largest)
    and of every cluster's truncated basis (singular values above eps times
    the largest), although the two compute them with their own QR and Jacobi
    codes."""
    mesh = mk()
    mh = H.h2bem_mesh_create(mesh.vertices, mesh.triangles)
    th = H.h2bem_tree_build(mh, 32)
    tr = H.h2bem_tree_export(th, mesh.nt)
    nc = len(tr["begin"])
    rank, brank = H.h2bem_hca_ranks(mh, th, nc, m=m, eta=2.0, eps_aca=eps_aca, eps=eps)
    (ft, fs), _ = H.h2bem_blocks(th, 2.0)
    Ho = orc.HCA(mesh, m=m, eps_aca=eps_aca, eps_c=eps)
    assert np.array_equal(rank, Ho.ranks().astype(np.int64))
    oft, ofs = Ho.blocks()
    ob = dict(zip(zip(oft.tolist(), ofs.tolist()), Ho.block_ranks().tolist()))
    assert len(ob) == len(brank)
    for t, s, r in zip(ft.tolist(), fs.tolist(), brank.tolist()):
        assert ob[(t, s)] == r, (t, s)
    H.h2bem_tree_destroy(th)
    H.h2bem_mesh_destroy(mh)
