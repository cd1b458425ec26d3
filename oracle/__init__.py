"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_2001_05523_gb300`` never does: it has no CPU fallback.

The arithmetic lives in ``h2oracle.c`` (plain C, FP64, OpenMP over rows);
this module compiles it with gcc and marshals numpy arrays through ctypes.
The specification each function follows is written out in ``h2oracle.h``.
The hypersingular operator at the end of this module is plain numpy on top
of those functions (its curls and the sum over the three components).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "h2oracle.c")
_HDR = os.path.join(_HERE, "h2oracle.h")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

SLP, DLP, TEST_POLY = 0, 1, 2
PART_FAR, PART_NEAR, PART_ALL = 1, 2, 3
IDENTICAL, EDGE, VERTEX = 3, 2, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so that the tree's
    floating-point decisions match the written specification bit for bit)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            d, i32, i64, vp = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
            L.or_gauss_legendre01.argtypes = [i32, vp, vp]
            L.or_radon7.argtypes = [vp, vp]
            L.or_collapsed_rule.argtypes = [i32, vp, vp]
            L.or_collapsed_rule.restype = i32
            L.or_tri_geom.argtypes = [vp, vp, vp, vp, vp]
            L.or_pair_regular.argtypes = [i32, vp, vp]
            L.or_pair_regular.restype = d
            L.or_ss_pair.argtypes = [i32, i32, vp, vp, vp, d, i32]
            L.or_ss_pair.restype = d
            L.or_entry.argtypes = [i32, vp, i64, i64, i32]
            L.or_entry.restype = d
            L.or_shared_vertices.argtypes = [vp, i64, i64]
            L.or_orient_pair.argtypes = [vp, i64, i64, vp, vp, vp]
            L.or_dense_matvec.argtypes = [i32, vp, i32, vp, i32, vp, i32]
            L.or_dense_rows.argtypes = [i32, vp, i32, vp, i64, vp, i32, vp]
            L.or_dense_matrix.argtypes = [i32, vp, i32, vp]
            L.or_ss_pair3.argtypes = [i32, i32, vp, vp, vp, d, i32, i32, vp]
            L.or_entry_dlp_p1.argtypes = [vp, i64, i64, i32, vp]
            L.or_dense_dlp_p1.argtypes = [vp, i32, vp]
            L.or_h2_create.argtypes = [vp, i64, vp, i64, i32, i32, d, i32, i32]
            L.or_h2_create.restype = vp
            L.or_h2_destroy.argtypes = [vp]
            L.or_h2_sizes.argtypes = [vp, vp]
            L.or_h2_tree.argtypes = [vp] * 8
            L.or_h2_blocks.argtypes = [vp] * 5
            L.or_h2_leaf_basis.argtypes = [vp, i64, vp, vp]
            L.or_h2_leaf_basis.restype = i32
            L.or_h2_transfer.argtypes = [vp, i64, vp]
            L.or_h2_transfer.restype = i32
            L.or_h2_nodes.argtypes = [vp, vp]
            L.or_h2_matvec.argtypes = [vp, vp, i32, vp, i32, i32]
            L.or_h2_matvec_dlp_p1.argtypes = [vp, vp, i32, vp, i32, i32]
            L.or_ss_moment.argtypes = [i32, i32, i32, i32, i32, i32]
            L.or_ss_moment.restype = d
            L.or_test_poly_P.argtypes = [vp]
            L.or_test_poly_P.restype = d
            L.or_test_poly_Q.argtypes = [vp]
            L.or_test_poly_Q.restype = d
            L.or_h2_rows.argtypes = [vp, vp, i64, vp, i32, vp]
            L.or_h2_matvec_subtree.argtypes = [vp, i64, vp, i32, vp]
            L.or_h2_upward.argtypes = [vp, vp, i32, vp]
            L.or_h2_matvec_subtree_from.argtypes = [vp, i64, vp, vp, i32, vp]
            L.or_h2_update_geometry.argtypes = [vp, vp]
            L.or_h2_grad.argtypes = [vp, vp, vp, i32, vp, i32]
            L.or_h2_grad.restype = i32
            L.or_num_threads.restype = i32
            L.or_set_threads.argtypes = [i32]
            L.or_gca_boundary_rule.argtypes = [vp, vp, i32, vp, vp, vp]
            L.or_gca_boundary_rule.restype = i32
            L.or_gca_green.argtypes = [vp, vp, i32, vp, vp]
            L.or_gca_green.restype = d
            L.or_gca_aca.argtypes = [vp, i32, i32, d, i32, vp, vp]
            L.or_gca_aca.restype = i32
            L.or_gca_create.argtypes = [vp, i64, vp, i64, i32, d, i32, d, i32, i32]
            L.or_gca_create.restype = vp
            L.or_gca_destroy.argtypes = [vp]
            L.or_gca_sizes.argtypes = [vp, vp]
            L.or_gca_ranks.argtypes = [vp, vp]
            L.or_gca_pivots.argtypes = [vp, i64, vp]
            L.or_gca_basis.argtypes = [vp, i64, vp]
            L.or_gca_basis.restype = i32
            L.or_gca_transfer.argtypes = [vp, i64, vp]
            L.or_gca_transfer.restype = i32
            L.or_gca_L.argtypes = [vp, i64, vp, vp]
            L.or_gca_L.restype = i64
            L.or_gca_rowcount.argtypes = [vp, i64]
            L.or_gca_rowcount.restype = i64
            L.or_gca_matvec.argtypes = [vp, vp, i32, vp, i32]
            L.or_hca_create.argtypes = [vp, i64, vp, i64, i32, d, i32, d, i32, d, i32, i32]
            L.or_hca_create.restype = vp
            L.or_hca_destroy.argtypes = [vp]
            L.or_hca_sizes.argtypes = [vp, vp]
            L.or_hca_ranks.argtypes = [vp, vp, vp]
            L.or_hca_blocks.argtypes = [vp, vp, vp]
            L.or_hca_cluster.argtypes = [vp, i64, vp]
            L.or_hca_cluster.restype = i64
            L.or_hca_block.argtypes = [vp, i64, vp, vp, vp]
            L.or_hca_block.restype = i32
            L.or_hca_node.argtypes = [vp, i64, i32, vp]
            L.or_hca_kernel.argtypes = [vp, i64, vp, vp]
            L.or_hca_kernel.restype = d
            L.or_hca_block_matrix.argtypes = [vp, i64, vp]
            L.or_hca_basis.argtypes = [vp, i64, vp]
            L.or_hca_basis.restype = i32
            L.or_hca_transfer.argtypes = [vp, i64, vp]
            L.or_hca_transfer.restype = i32
            L.or_hca_coupling.argtypes = [vp, i64, vp]
            L.or_hca_coupling.restype = i32
            L.or_hca_matvec.argtypes = [vp, vp, i32, vp, i32, i32]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


# ---------------------------------------------------------------- quadrature
def gauss_legendre01(q: int):
    x = np.zeros(q)
    w = np.zeros(q)
    if lib().or_gauss_legendre01(q, _p(x), _p(w)):
        raise ValueError("bad q")
    return x, w


def radon7():
    uv = np.zeros((7, 2))
    w = np.zeros(7)
    lib().or_radon7(_p(uv), _p(w))
    return uv, w


def collapsed_rule(q: int):
    uv = np.zeros((q * q, 2))
    w = np.zeros(q * q)
    n = lib().or_collapsed_rule(q, _p(uv), _p(w))
    return uv[:n], w[:n]


def tri_geom(a, b, c):
    a, b, c = _f64(a), _f64(b), _f64(c)
    area = np.zeros(1)
    nrm = np.zeros(3)
    lib().or_tri_geom(_p(a), _p(b), _p(c), _p(area), _p(nrm))
    return float(area[0]), nrm


def ss_moment(kind: int, q: int, a: int, b: int, c: int, d: int) -> float:
    return float(lib().or_ss_moment(kind, q, a, b, c, d))


def test_poly_PQ(pts: np.ndarray):
    pts = _f64(pts).reshape(-1, 3)
    P = np.array([lib().or_test_poly_P(_p(np.ascontiguousarray(p))) for p in pts])
    Q = np.array([lib().or_test_poly_Q(_p(np.ascontiguousarray(p))) for p in pts])
    return P, Q


def pair_regular(kernel: int, X, Y) -> float:
    X, Y = _f64(X).reshape(9), _f64(Y).reshape(9)
    return float(lib().or_pair_regular(kernel, _p(X), _p(Y)))


def ss_pair(kernel: int, kind: int, P, Q, q: int, nrm=None, sgn: float = 1.0) -> float:
    P, Q = _f64(P).reshape(9), _f64(Q).reshape(9)
    n = _f64(nrm if nrm is not None else np.zeros(3))
    return float(lib().or_ss_pair(kernel, kind, _p(P), _p(Q), _p(n), sgn, q))


class _MeshC(ctypes.Structure):
    _fields_ = [("xyz", ctypes.c_void_p), ("tri", ctypes.c_void_p), ("nv", ctypes.c_int64), ("nt", ctypes.c_int64)]


class MeshRef:
    """Keeps the numpy buffers alive while C holds pointers to them."""

    def __init__(self, vertices, triangles):
        self.v = _f64(vertices)
        self.t = np.ascontiguousarray(triangles, dtype=np.int32)
        self.c = _MeshC(_p(self.v).value, _p(self.t).value, self.v.shape[0], self.t.shape[0])

    @property
    def ptr(self):
        return ctypes.cast(ctypes.pointer(self.c), ctypes.c_void_p)


def _mesh(mesh) -> MeshRef:
    return MeshRef(mesh.vertices, mesh.triangles)


def entry(kernel: int, mesh, i: int, j: int, q_ss: int = 5) -> float:
    M = _mesh(mesh)
    return float(lib().or_entry(kernel, M.ptr, i, j, q_ss))


def shared_vertices(mesh, i: int, j: int) -> int:
    M = _mesh(mesh)
    return int(lib().or_shared_vertices(M.ptr, i, j))


def orient_pair(mesh, lo: int, hi: int):
    M = _mesh(mesh)
    t = ctypes.c_int(0)
    P = np.zeros(9)
    Q = np.zeros(9)
    lib().or_orient_pair(M.ptr, lo, hi, ctypes.byref(t), _p(P), _p(Q))
    return int(t.value), P.reshape(3, 3), Q.reshape(3, 3)


def dense_matrix(kernel: int, mesh, q_ss: int = 5) -> np.ndarray:
    M = _mesh(mesh)
    A = np.zeros((mesh.nt, mesh.nt))
    lib().or_dense_matrix(kernel, M.ptr, q_ss, _p(A))
    return A


def entry_dlp_p1(mesh, i: int, j: int, q_ss: int = 5) -> np.ndarray:
    """int_{tau_i} int_{tau_j} dg/dn_y lambda_{j,c}(y) for the corners c of tau_j
    (the double layer with piecewise-linear trial functions, per pair)."""
    M = _mesh(mesh)
    out = np.zeros(3)
    lib().or_entry_dlp_p1(M.ptr, i, j, q_ss, _p(out))
    return out


def dense_dlp_p1(mesh, q_ss: int = 5) -> np.ndarray:
    """K1 (nt x nv): the double layer with piecewise-linear trial functions."""
    M = _mesh(mesh)
    A = np.zeros((mesh.nt, mesh.vertices.shape[0]))
    lib().or_dense_dlp_p1(M.ptr, q_ss, _p(A))
    return A


def ss_pair3(kernel: int, kind: int, P, Q, q: int, side: int, nrm=None, sgn: float = 1.0) -> np.ndarray:
    P, Q = _f64(np.asarray(P).reshape(-1)), _f64(np.asarray(Q).reshape(-1))
    n = _f64(np.zeros(3) if nrm is None else np.asarray(nrm))
    out = np.zeros(3)
    lib().or_ss_pair3(kernel, kind, _p(P), _p(Q), _p(n), sgn, q, side, _p(out))
    return out


def dense_matvec(kernel: int, mesh, x: np.ndarray, q_ss: int = 5, transpose: bool = False) -> np.ndarray:
    """x: (nrhs, n) -> y: (nrhs, n)."""
    M = _mesh(mesh)
    x = _f64(x)
    nrhs = x.shape[0]
    y = np.zeros_like(x)
    lib().or_dense_matvec(kernel, M.ptr, q_ss, _p(x), nrhs, _p(y), int(transpose))
    return y


def dense_rows(kernel: int, mesh, rows, x: np.ndarray, q_ss: int = 5) -> np.ndarray:
    """Rows of the dense product: returns (nrhs, len(rows))."""
    M = _mesh(mesh)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    x = _f64(x)
    nrhs = x.shape[0]
    y = np.zeros((nrhs, rows.size))
    lib().or_dense_rows(kernel, M.ptr, q_ss, _p(rows), rows.size, _p(x), nrhs, _p(y))
    return y


class H2:
    """The oracle's H^2 approximation of G (SLP) or K (DLP)."""

    def __init__(self, mesh, kernel: int = SLP, m: int = 4, eta: float = 2.0, leaf: int = 32, q_ss: int = 5):
        self.mesh = mesh
        v = _f64(mesh.vertices)
        t = np.ascontiguousarray(mesh.triangles, dtype=np.int32)
        self._keep = (v, t)
        h = lib().or_h2_create(_p(v), v.shape[0], _p(t), t.shape[0], kernel, m, float(eta), leaf, q_ss)
        if not h:
            raise ValueError("or_h2_create failed")
        self.h = ctypes.c_void_p(h)
        sz = np.zeros(6, dtype=np.int64)
        lib().or_h2_sizes(self.h, _p(sz))
        self.nclusters, self.nfar, self.nnear, self.k, self.nleaves, self.qb = (int(a) for a in sz)
        self.n = mesh.nt
        self.m = m
        self.kernel = kernel

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            lib().or_h2_destroy(h)
            self.h = None

    def tree(self):
        nc = self.nclusters
        out = dict(perm=np.zeros(self.n, np.int64), begin=np.zeros(nc, np.int64), end=np.zeros(nc, np.int64),
                   child0=np.zeros(nc, np.int64), child1=np.zeros(nc, np.int64),
                   bmin=np.zeros((nc, 3)), bmax=np.zeros((nc, 3)))
        lib().or_h2_tree(self.h, *(_p(out[k]) for k in ("perm", "begin", "end", "child0", "child1", "bmin", "bmax")))
        return out

    def blocks(self):
        ft, fs = np.zeros(self.nfar, np.int64), np.zeros(self.nfar, np.int64)
        nt, ns = np.zeros(self.nnear, np.int64), np.zeros(self.nnear, np.int64)
        lib().or_h2_blocks(self.h, _p(ft), _p(fs), _p(nt), _p(ns))
        return (ft, fs), (nt, ns)

    def leaf_basis(self, c: int):
        tr = self.tree()
        sz = int(tr["end"][c] - tr["begin"][c])
        V = np.zeros((sz, self.k))
        W = np.zeros((sz, self.k))
        if lib().or_h2_leaf_basis(self.h, c, _p(V), _p(W)):
            raise ValueError("not a leaf")
        return V, W

    def transfer(self, c: int):
        E = np.zeros((self.k, self.k))
        if lib().or_h2_transfer(self.h, c, _p(E)):
            raise ValueError("bad cluster")
        return E

    def nodes(self):
        z = np.zeros((self.nclusters, 3, self.m))
        lib().or_h2_nodes(self.h, _p(z))
        return z

    def matvec(self, x: np.ndarray, transpose: bool = False, parts: int = PART_ALL) -> np.ndarray:
        """x: (nrhs, n) -> (nrhs, n)."""
        x = _f64(x)
        if x.ndim == 1:
            x = x[None, :]
        y = np.zeros_like(x)
        lib().or_h2_matvec(self.h, _p(x), x.shape[0], _p(y), int(transpose), int(parts))
        return y

    def matvec_dlp_p1(self, x: np.ndarray, transpose: bool = False, parts: int = PART_ALL) -> np.ndarray:
        """K1 x: (nrhs, nv) -> (nrhs, nt), or K1^T x: (nrhs, nt) -> (nrhs, nv)
        (the double layer with piecewise-linear trial functions)."""
        x = _f64(x)
        if x.ndim == 1:
            x = x[None, :]
        nv = self.mesh.vertices.shape[0]
        y = np.zeros((x.shape[0], nv if transpose else self.n))
        lib().or_h2_matvec_dlp_p1(self.h, _p(x), x.shape[0], _p(y), int(transpose), int(parts))
        return y

    def update_geometry(self, vertices) -> None:
        """New vertex positions with the cluster tree and block lists unchanged."""
        v = _f64(vertices)
        self._keep = (v, self._keep[1])
        lib().or_h2_update_geometry(self.h, _p(v))

    def grad_vertices(self, w: np.ndarray, x: np.ndarray, parts: int = PART_ALL) -> np.ndarray:
        """d/dX of sum_r <w_r, A x_r> (single or double layer), shape (nv, 3)."""
        w, x = _f64(w), _f64(x)
        g = np.zeros((self.mesh.nv, 3))
        if lib().or_h2_grad(self.h, _p(w), _p(x), x.shape[0], _p(g), int(parts)):
            raise ValueError("gradient is available for the single and double layer only")
        return g

    def matvec_subtree(self, c0: int, x: np.ndarray) -> np.ndarray:
        """Forward product restricted to the rows of cluster c0: (nrhs, n), other rows 0."""
        x = _f64(x)
        if x.ndim == 1:
            x = x[None, :]
        y = np.zeros_like(x)
        lib().or_h2_matvec_subtree(self.h, int(c0), _p(x), x.shape[0], _p(y))
        return y

    def upward(self, x: np.ndarray) -> np.ndarray:
        """x-hat of every cluster (leaf forward transformation and upward pass)."""
        x = _f64(x)
        if x.ndim == 1:
            x = x[None, :]
        xh = np.zeros((self.nclusters, self.k, x.shape[0]))
        lib().or_h2_upward(self.h, _p(x), x.shape[0], _p(xh))
        return xh

    def matvec_subtree_from(self, c0: int, xh: np.ndarray, x: np.ndarray) -> np.ndarray:
        """As matvec_subtree with x-hat from upward()."""
        x = _f64(x)
        if x.ndim == 1:
            x = x[None, :]
        y = np.zeros_like(x)
        lib().or_h2_matvec_subtree_from(self.h, int(c0), _p(xh), _p(x), x.shape[0], _p(y))
        return y

    def rows(self, rows, x: np.ndarray) -> np.ndarray:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        x = _f64(x)
        y = np.zeros((x.shape[0], rows.size))
        lib().or_h2_rows(self.h, _p(rows), rows.size, _p(x), x.shape[0], _p(y))
        return y


# ---------------------------------------------------------------------------
# Green cross approximation of the single layer (section 4); the arithmetic is
# in h2oracle.c (or_gca_*), whose comment block states each step.
# ---------------------------------------------------------------------------
def gca_boundary_rule(lo, hi, q: int):
    """Composite Gauss rule on the boundary of the box [lo, hi]: points (k, 3),
    weights (k,), outward normals (k, 3), k = 6 q^2."""
    k = 6 * q * q
    z, w, nz = np.zeros((k, 3)), np.zeros(k), np.zeros((k, 3))
    if lib().or_gca_boundary_rule(_p(_f64(lo)), _p(_f64(hi)), q, _p(z), _p(w), _p(nz)) != k:
        raise ValueError("bad q")
    return z, w, nz


def gca_green(lo, hi, q: int, x, y) -> float:
    """g~_grn(x, y): Green's representation formula on the box [lo, hi] with the rule above."""
    return float(lib().or_gca_green(_p(_f64(lo)), _p(_f64(hi)), q, _p(_f64(x)), _p(_f64(y))))


def gca_aca(L: np.ndarray, eps: float, kmax: int):
    """Full-pivot cross approximation of L: (tau, sigma) pivot lists."""
    L = _f64(L)
    rows, cols = L.shape
    tau = np.zeros(kmax + 1, np.int32)
    sigma = np.zeros(kmax + 1, np.int32)
    k = lib().or_gca_aca(_p(L), rows, cols, float(eps), int(kmax), _p(tau), _p(sigma))
    return tau[:k].copy(), sigma[:k].copy()


class GCA:
    """The oracle's GCA approximation of the single layer G: q Gauss points per
    face axis of d omega_t, ACA tolerance eps (relative to the first pivot),
    ranks capped at kmax."""

    def __init__(self, mesh, q: int = 4, eta: float = 2.0, leaf: int = 32, eps: float = 1e-6, kmax: int = 64,
                 q_ss: int = 5):
        self.mesh = mesh
        v = _f64(mesh.vertices)
        t = np.ascontiguousarray(mesh.triangles, dtype=np.int32)
        self._keep = (v, t)
        h = lib().or_gca_create(_p(v), v.shape[0], _p(t), t.shape[0], q, float(eta), leaf, float(eps), kmax, q_ss)
        if not h:
            raise ValueError("or_gca_create failed")
        self.h = ctypes.c_void_p(h)
        sz = np.zeros(5, dtype=np.int64)
        lib().or_gca_sizes(self.h, _p(sz))
        self.nclusters, self.nfar, self.nnear, self.maxrank, self.k = (int(a) for a in sz)
        self.n = mesh.nt

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            lib().or_gca_destroy(h)
            self.h = None

    def ranks(self) -> np.ndarray:
        r = np.zeros(self.nclusters, np.int32)
        lib().or_gca_ranks(self.h, _p(r))
        return r

    def pivots(self, c: int) -> np.ndarray:
        p = np.zeros(int(self.ranks()[c]), np.int64)
        lib().or_gca_pivots(self.h, c, _p(p))
        return p

    def leaf_basis(self, c: int, size: int) -> np.ndarray:
        V = np.zeros((size, int(self.ranks()[c])))
        if lib().or_gca_basis(self.h, c, _p(V)):
            raise ValueError("not a leaf")
        return V

    def transfer(self, c: int, parent: int) -> np.ndarray:
        r = self.ranks()
        E = np.zeros((int(r[c]), int(r[parent])))
        if lib().or_gca_transfer(self.h, c, _p(E)):
            raise ValueError("bad cluster")
        return E

    def L(self, c: int):
        nr = int(lib().or_gca_rowcount(self.h, c))
        rows = np.zeros(nr, np.int64)
        L = np.zeros((nr, 2 * self.k))
        lib().or_gca_L(self.h, c, _p(rows), _p(L))
        return rows, L

    def matvec(self, x: np.ndarray, parts: int = PART_ALL) -> np.ndarray:
        """x: (nrhs, n) -> (nrhs, n)."""
        x = _f64(x)
        if x.ndim == 1:
            x = x[None, :]
        y = np.zeros_like(x)
        lib().or_gca_matvec(self.h, _p(x), x.shape[0], _p(y), int(parts))
        return y


class HCA:
    """The oracle's hybrid cross approximation of the single layer G (section 3)
    and its compression into an H^2-matrix: interpolation order m for the
    coupling matrix S of each block, cross approximation of S to eps_aca (at
    most kaca steps), compression with relative truncation eps_c, cluster
    ranks capped at kmax."""

    def __init__(self, mesh, m: int = 4, eta: float = 2.0, leaf: int = 32, eps_aca: float = 1e-6, kaca: int = 64,
                 eps_c: float = 1e-6, kmax: int = 64, q_ss: int = 5):
        self.mesh = mesh
        v = _f64(mesh.vertices)
        t = np.ascontiguousarray(mesh.triangles, dtype=np.int32)
        self._keep = (v, t)
        h = lib().or_hca_create(_p(v), v.shape[0], _p(t), t.shape[0], m, float(eta), leaf, float(eps_aca), kaca,
                                float(eps_c), kmax, q_ss)
        if not h:
            raise ValueError("or_hca_create failed")
        self.h = ctypes.c_void_p(h)
        sz = np.zeros(6, dtype=np.int64)
        lib().or_hca_sizes(self.h, _p(sz))
        self.nclusters, self.nfar, self.nnear, self.maxrank, self.k, self.maxblockrank = (int(a) for a in sz)
        self.n = mesh.nt

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            lib().or_hca_destroy(h)
            self.h = None

    def ranks(self) -> np.ndarray:
        r = np.zeros(self.nclusters, np.int32)
        lib().or_hca_ranks(self.h, _p(r), None)
        return r

    def block_ranks(self) -> np.ndarray:
        r = np.zeros(self.nfar, np.int32)
        lib().or_hca_ranks(self.h, None, _p(r))
        return r

    def blocks(self):
        ft = np.zeros(self.nfar, np.int64)
        fs = np.zeros(self.nfar, np.int64)
        lib().or_hca_blocks(self.h, _p(ft), _p(fs))
        return ft, fs

    def cluster(self, c: int) -> np.ndarray:
        idx = np.zeros(self.n, np.int64)
        cnt = int(lib().or_hca_cluster(self.h, c, _p(idx)))
        return idx[:cnt].copy()

    def block(self, b: int):
        """(tau, sigma, C) of farfield block b."""
        tau = np.zeros(self.k, np.int32)
        sig = np.zeros(self.k, np.int32)
        C = np.zeros(self.k * self.k)
        r = int(lib().or_hca_block(self.h, b, _p(tau), _p(sig), _p(C)))
        return tau[:r].copy(), sig[:r].copy(), C[:r * r].reshape(r, r).copy()

    def node(self, c: int, nu: int) -> np.ndarray:
        x = np.zeros(3)
        lib().or_hca_node(self.h, c, nu, _p(x))
        return x

    def kernel(self, b: int, x, y) -> float:
        return float(lib().or_hca_kernel(self.h, b, _p(_f64(x)), _p(_f64(y))))

    def block_matrix(self, b: int) -> np.ndarray:
        ft, fs = self.blocks()
        nt_, ns = len(self.cluster(int(ft[b]))), len(self.cluster(int(fs[b])))
        out = np.zeros((nt_, ns))
        lib().or_hca_block_matrix(self.h, b, _p(out))
        return out

    def basis(self, c: int) -> np.ndarray:
        Q = np.zeros((len(self.cluster(c)), int(self.ranks()[c])))
        lib().or_hca_basis(self.h, c, _p(Q))
        return Q

    def transfer(self, c: int, parent: int) -> np.ndarray:
        r = self.ranks()
        E = np.zeros((int(r[c]), int(r[parent])))
        if lib().or_hca_transfer(self.h, c, _p(E)):
            raise ValueError("bad cluster")
        return E

    def coupling(self, b: int) -> np.ndarray:
        ft, fs = self.blocks()
        r = self.ranks()
        S = np.zeros((int(r[ft[b]]), int(r[fs[b]])))
        lib().or_hca_coupling(self.h, b, _p(S))
        return S

    def matvec(self, x: np.ndarray, parts: int = PART_ALL, hmatrix: bool = False) -> np.ndarray:
        """x: (nrhs, n) -> (nrhs, n); hmatrix: the uncompressed HCA blocks."""
        x = _f64(x)
        if x.ndim == 1:
            x = x[None, :]
        y = np.zeros_like(x)
        lib().or_hca_matvec(self.h, _p(x), x.shape[0], _p(y), int(parts), int(hmatrix))
        return y


# ---------------------------------------------------------------------------
# Hypersingular operator W on continuous piecewise-linear functions (section 1,
# eq. (slp) ff.: w_ij = -int phi_i d/dn_x int dg/dn_y phi_j).  Section 1 sets
# it up through its representation by the single-layer operator (the
# integration-by-parts identity it cites from Sauter and Schwab): for the
# Laplace kernel on a closed surface
#     w_ij = int int g(x, y) curl phi_i(x) . curl phi_j(y) dy dx,
# with the surface curl curl phi = n x grad phi.  A hat function is linear on
# each triangle, so its curl is a constant vector there, and
#     W = sum_{d=1..3} C_d^T G C_d,   (C_d)_{tau j} = (curl phi_j |_tau)_d,
# G the piecewise-constant single-layer matrix of eq. (slp).  Plain numpy;
# the Galerkin matrix G (or its H^2 product) comes from the functions above.
# ---------------------------------------------------------------------------
def curl_p1(mesh):
    """Surface curls of the hat functions, constant per triangle.

    For tau = (a, b, c) with n = (b - a) x (c - a) / (2 |tau|):
        grad phi_a = n x (c - b) / (2 |tau|),  curl phi_a = n x grad phi_a = (b - c) / (2 |tau|),
    and cyclically curl phi_b = (c - a) / (2 |tau|), curl phi_c = (a - b) / (2 |tau|).
    Returns (rows, cols, vals): vals[d] are the entries of C_d at (tau, j)."""
    v = np.asarray(mesh.vertices, float)
    t = np.asarray(mesh.triangles, np.int64)
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    two_area = np.linalg.norm(np.cross(b - a, c - a), axis=1)[:, None]
    curls = [(b - c) / two_area, (c - a) / two_area, (a - b) / two_area]  # corner k of each triangle
    rows = np.repeat(np.arange(len(t)), 3)
    cols = t.reshape(-1)
    vals = np.stack([np.stack([curls[k][:, d] for k in range(3)], axis=1).reshape(-1) for d in range(3)])
    return rows, cols, vals


def curl_matrices(mesh):
    """C_d as scipy.sparse matrices (nt x nv), d = 0, 1, 2."""
    import scipy.sparse as sp

    rows, cols, vals = curl_p1(mesh)
    shape = (mesh.nt, mesh.vertices.shape[0])
    return [sp.csr_matrix((vals[d], (rows, cols)), shape=shape) for d in range(3)]


def hypersingular_matvec(mesh, x: np.ndarray, slp_matvec=None, q_ss: int = 5) -> np.ndarray:
    """W x = sum_d C_d^T G (C_d x); x: (nrhs, nv) -> (nrhs, nv).  slp_matvec
    applies G to (k, nt) arrays (default: the dense Galerkin product)."""
    x = _f64(x)
    if slp_matvec is None:
        slp_matvec = lambda z: dense_matvec(SLP, mesh, z, q_ss)  # noqa: E731
    C = curl_matrices(mesh)
    z = np.concatenate([(C[d] @ x.T).T for d in range(3)])  # (3 nrhs, nt)
    w = slp_matvec(z)
    nr = x.shape[0]
    return sum((C[d].T @ w[d * nr:(d + 1) * nr].T).T for d in range(3))


def hypersingular_dense(mesh, q_ss: int = 5) -> np.ndarray:
    """The matrix W (nv x nv) from the dense Galerkin matrix G."""
    G = dense_matrix(SLP, mesh, q_ss)
    C = curl_matrices(mesh)
    return sum((C[d].T @ (C[d].T @ G.T).T) for d in range(3))
