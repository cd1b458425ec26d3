"""Thin Python binding of libh2bem (the C ABI in include/h2bem.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  There is no CPU fallback; if the compiled library is missing the
import of a function raises.  Functions keep the C names; torch tensors (CUDA
or CPU) and numpy arrays are accepted for vectors.  A vector block of nrhs
right-hand sides is a (nrhs, n) row-major array, i.e. the column-major n x nrhs
layout with leading dimension n.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libh2bem.so")

H2BEM_OK, H2BEM_ERR_ARG, H2BEM_ERR_MESH, H2BEM_ERR_OOM, H2BEM_ERR_CUDA, H2BEM_ERR_TIMEOUT, H2BEM_ERR_STATE = range(7)
H2BEM_SLP, H2BEM_DLP = 0, 1
H2BEM_BASIS_CHEBYSHEV, H2BEM_BASIS_GCA, H2BEM_BASIS_HCA = 0, 1, 2
H2BEM_FP64, H2BEM_MIXED_FP32, H2BEM_MIXED_TF32, H2BEM_MIXED_BF16 = 0, 1, 2, 3
PRECISIONS = {"fp64": H2BEM_FP64, "mixed_fp32": H2BEM_MIXED_FP32, "mixed_tf32": H2BEM_MIXED_TF32,
              "mixed_bf16": H2BEM_MIXED_BF16}

EXPORTED = [
    "h2bem_last_error", "h2bem_mesh_create", "h2bem_mesh_destroy", "h2bem_tree_build", "h2bem_tree_upload",
    "h2bem_tree_info", "h2bem_tree_export", "h2bem_tree_destroy", "h2bem_blocks", "h2bem_opts_default",
    "h2bem_operator_create", "h2bem_operator_destroy", "h2bem_stats_get", "h2bem_apply", "h2bem_apply_transpose",
    "h2bem_apply_timed", "h2bem_apply_noalloc", "h2bem_batch_create", "h2bem_grad", "h2bem_apply_mass", "h2bem_apply_hypersingular",
    "h2bem_cg", "h2bem_gca_bases", "h2bem_apply_dlp_p1", "h2bem_cg_hypersingular", "h2bem_hca_ranks",
]


class H2bemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"h2bem error {code}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("q_ss", ctypes.c_int), ("precision", ctypes.c_int), ("cache_singular", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("autotune", ctypes.c_int),
                ("singular_fp64", ctypes.c_int), ("recompute_basis", ctypes.c_int), ("store_near", ctypes.c_int),
                ("basis", ctypes.c_int), ("gca_q", ctypes.c_int), ("gca_kmax", ctypes.c_int),
                ("tc_wait_test", ctypes.c_int), ("gca_eps", ctypes.c_double),
                ("hca_kaca", ctypes.c_int), ("hca_kmax", ctypes.c_int), ("hca_eps_aca", ctypes.c_double),
                ("hca_eps", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nclusters", ctypes.c_int64), ("nleaves", ctypes.c_int64),
                ("depth", ctypes.c_int64), ("nfar", ctypes.c_int64), ("nnear", ctypes.c_int64),
                ("near_pairs", ctypes.c_int64), ("regular_pairs", ctypes.c_int64),
                ("singular_pairs", ctypes.c_int64 * 3), ("k", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("last_apply_ms", ctypes.c_double),
                ("stage_ms", ctypes.c_double * 8), ("launch_variant", ctypes.c_int64 * 5),
                ("regular_evals", ctypes.c_int64), ("near_stored_bytes", ctypes.c_int64),
                ("far_stored_bytes", ctypes.c_int64), ("mean_rank", ctypes.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["singular_pairs"] = list(self.singular_pairs)
        d["stage_ms"] = list(self.stage_ms)
        d["launch_variant"] = list(self.launch_variant)
        return d


_lib = None


def lib():
    """Load libh2bem.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libh2bem.so not built ({LIB_PATH}); run paper_2001_05523_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
        pp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "h2bem_last_error": [ctypes.c_char_p, sz],
            "h2bem_mesh_create": [vp, i64, vp, i64, pp],
            "h2bem_mesh_destroy": [vp],
            "h2bem_tree_build": [vp, i32, pp],
            "h2bem_tree_upload": [vp, i64, vp, vp, vp, vp, vp, pp],
            "h2bem_tree_info": [vp, vp, vp, vp],
            "h2bem_tree_export": [vp] * 8,
            "h2bem_tree_destroy": [vp],
            "h2bem_blocks": [vp, d, vp, vp, vp, vp, vp, vp],
            "h2bem_gca_bases": [vp, vp, vp, vp, vp, vp],
            "h2bem_hca_ranks": [vp, vp, i32, d, vp, vp, vp, vp],
            "h2bem_apply_dlp_p1": [vp, d, vp, i64, i32, vp, i64, i32, vp],
            "h2bem_cg_hypersingular": [vp, vp, vp, i64, i32, vp, i64, d, i32, vp, vp, vp],
            "h2bem_opts_default": [vp],
            "h2bem_operator_create": [vp, vp, i32, i32, d, vp, pp],
            "h2bem_operator_destroy": [vp],
            "h2bem_stats_get": [vp, vp],
            "h2bem_apply": [vp, vp, i64, i32, vp, i64, vp],
            "h2bem_apply_transpose": [vp, vp, i64, i32, vp, i64, vp],
            "h2bem_apply_timed": [vp, vp, i64, i32, vp, i64, vp],
            "h2bem_apply_noalloc": [vp, vp, i64, i32, vp, i64, vp],
            "h2bem_batch_create": [i32, vp, i32, i32, i32, d, vp, pp],
            "h2bem_grad": [vp, vp, vp, i64, i32, vp, vp, vp],
            "h2bem_apply_mass": [vp, d, vp, i64, i32, vp, i64, vp],
            "h2bem_apply_hypersingular": [vp, vp, i64, i32, vp, i64, vp],
            "h2bem_cg": [vp, vp, i64, i32, vp, i64, d, i32, vp, vp, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = i32
        _lib = L
    return _lib


def _check(rc: int):
    if rc != H2BEM_OK:
        buf = ctypes.create_string_buffer(512)
        lib().h2bem_last_error(buf, 512)
        raise H2bemError(rc, buf.value.decode())


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- C names
def h2bem_mesh_create(vertices, triangles):
    v = np.ascontiguousarray(vertices, dtype=np.float64)
    t = np.ascontiguousarray(triangles, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(lib().h2bem_mesh_create(_np_ptr(v), v.shape[0], _np_ptr(t), t.shape[0], ctypes.byref(h)))
    return h


def h2bem_mesh_destroy(h):
    _check(lib().h2bem_mesh_destroy(h))


def h2bem_tree_build(mesh, leaf_size: int = 32):
    h = ctypes.c_void_p()
    _check(lib().h2bem_tree_build(mesh, int(leaf_size), ctypes.byref(h)))
    return h


def h2bem_tree_upload(mesh, perm, begin, end, child0, child1):
    arrs = [np.ascontiguousarray(a, dtype=np.int64) for a in (perm, begin, end, child0, child1)]
    h = ctypes.c_void_p()
    _check(lib().h2bem_tree_upload(mesh, arrs[1].size, *(_np_ptr(a) for a in arrs), ctypes.byref(h)))
    return h


def h2bem_tree_info(tree):
    nc, nl, dp = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().h2bem_tree_info(tree, ctypes.byref(nc), ctypes.byref(nl), ctypes.byref(dp)))
    return nc.value, nl.value, dp.value


def h2bem_tree_export(tree, n: int):
    nc, _, _ = h2bem_tree_info(tree)
    out = dict(perm=np.zeros(n, np.int64), begin=np.zeros(nc, np.int64), end=np.zeros(nc, np.int64),
               child0=np.zeros(nc, np.int64), child1=np.zeros(nc, np.int64), bmin=np.zeros((nc, 3)),
               bmax=np.zeros((nc, 3)))
    _check(lib().h2bem_tree_export(tree, *(_np_ptr(out[k]) for k in ("perm", "begin", "end", "child0", "child1",
                                                                      "bmin", "bmax"))))
    return out


def h2bem_tree_destroy(h):
    _check(lib().h2bem_tree_destroy(h))


def h2bem_blocks(tree, eta: float):
    nf, nn = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().h2bem_blocks(tree, float(eta), ctypes.byref(nf), ctypes.byref(nn), None, None, None, None))
    ft, fs = np.zeros(nf.value, np.int64), np.zeros(nf.value, np.int64)
    nt, ns = np.zeros(nn.value, np.int64), np.zeros(nn.value, np.int64)
    _check(lib().h2bem_blocks(tree, float(eta), None, None, _np_ptr(ft), _np_ptr(fs), _np_ptr(nt), _np_ptr(ns)))
    return (ft, fs), (nt, ns)


def h2bem_gca_bases(mesh, tree, nclusters: int, q: int = 4, kmax: int = 64, eps: float = 1e-6):
    """Ranks (per cluster) and pivot tree positions (cluster by cluster) of the
    GCA cluster bases, computed on the host."""
    o = h2bem_opts_default()
    o.basis, o.gca_q, o.gca_kmax, o.gca_eps = H2BEM_BASIS_GCA, int(q), int(kmax), float(eps)
    rank = np.zeros(nclusters, np.int64)
    npiv = ctypes.c_int64()
    _check(lib().h2bem_gca_bases(mesh, tree, ctypes.byref(o), _np_ptr(rank), ctypes.byref(npiv), None))
    piv = np.zeros(npiv.value, np.int64)
    _check(lib().h2bem_gca_bases(mesh, tree, ctypes.byref(o), None, None, _np_ptr(piv)))
    return rank, piv


def h2bem_hca_ranks(mesh, tree, nclusters: int, m: int = 4, eta: float = 2.0, kaca: int = 64, kmax: int = 64,
                    eps_aca: float = 1e-6, eps: float = 1e-6):
    """Ranks of the HCA construction on the host: per cluster (compressed bases)
    and per farfield block in the order of h2bem_blocks (cross approximation)."""
    o = h2bem_opts_default()
    o.basis, o.hca_kaca, o.hca_kmax, o.hca_eps_aca, o.hca_eps = H2BEM_BASIS_HCA, int(kaca), int(kmax), float(eps_aca), float(eps)
    rank = np.zeros(nclusters, np.int64)
    nfar = ctypes.c_int64()
    _check(lib().h2bem_hca_ranks(mesh, tree, int(m), float(eta), ctypes.byref(o), None, ctypes.byref(nfar), None))
    brank = np.zeros(nfar.value, np.int64)
    _check(lib().h2bem_hca_ranks(mesh, tree, int(m), float(eta), ctypes.byref(o), _np_ptr(rank), None,
                                 _np_ptr(brank)))
    return rank, brank


def h2bem_opts_default() -> Opts:
    o = Opts()
    _check(lib().h2bem_opts_default(ctypes.byref(o)))
    return o


def h2bem_operator_create(mesh, tree, kernel: int, m: int, eta: float, opts: Opts | None = None):
    h = ctypes.c_void_p()
    _check(lib().h2bem_operator_create(mesh, tree, int(kernel), int(m), float(eta),
                                       ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)))
    return h


def h2bem_batch_create(meshes, leaf_size: int, kernel: int, m: int, eta: float, opts: Opts | None = None):
    arr = (ctypes.c_void_p * len(meshes))(*[mh.value for mh in meshes])
    h = ctypes.c_void_p()
    _check(lib().h2bem_batch_create(len(meshes), ctypes.cast(arr, ctypes.c_void_p), int(leaf_size), int(kernel),
                                    int(m), float(eta), ctypes.byref(opts) if opts is not None else None,
                                    ctypes.byref(h)))
    return h


def h2bem_operator_destroy(h):
    _check(lib().h2bem_operator_destroy(h))


def h2bem_stats_get(op) -> dict:
    s = Stats()
    _check(lib().h2bem_stats_get(op, ctypes.byref(s)))
    return s.as_dict()


def _vec_args(x, y):
    """(pointer, ld, nrhs) for (nrhs, n) row-major torch tensors or numpy arrays."""
    def one(a):
        if isinstance(a, np.ndarray):
            if a.dtype != np.float64 or not a.flags.c_contiguous or a.ndim != 2:
                raise ValueError("vectors must be C-contiguous float64 arrays of shape (nrhs, n)")
            return ctypes.c_void_p(a.ctypes.data), a.shape[1], a.shape[0]
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous() or a.dim() != 2:
            raise ValueError("vectors must be contiguous float64 tensors of shape (nrhs, n)")
        return ctypes.c_void_p(a.data_ptr()), a.shape[1], a.shape[0]
    px, lx, rx = one(x)
    py, ly, ry = one(y)
    if rx != ry:
        raise ValueError("x and y must have the same number of right-hand sides")
    return px, lx, rx, py, ly


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def h2bem_apply(op, x, y, stream=None):
    px, lx, nr, py, ly = _vec_args(x, y)
    _check(lib().h2bem_apply(op, px, lx, nr, py, ly, _stream(stream)))


def h2bem_apply_transpose(op, x, y, stream=None):
    px, lx, nr, py, ly = _vec_args(x, y)
    _check(lib().h2bem_apply_transpose(op, px, lx, nr, py, ly, _stream(stream)))


def h2bem_grad(op, w, x, dxyz, dx=None, stream=None):
    """dxyz (nv, 3) = d/dX sum_r <w_r, G x_r>; optional dx = G^T w.  Device tensors."""
    pw, lw, nw, px, lx = _vec_args(w, x)
    if lw != lx:
        raise ValueError("w and x must have the same shape")
    pd = ctypes.c_void_p(dxyz.data_ptr())
    pdx = ctypes.c_void_p(dx.data_ptr()) if dx is not None else None
    _check(lib().h2bem_grad(op, pw, px, lx, nw, pd, pdx, _stream(stream)))


def h2bem_apply_noalloc(op, x, y, stream=None):
    """y = A x without any allocation by the library (device buffers only)."""
    px, lx, nr, py, ly = _vec_args(x, y)
    _check(lib().h2bem_apply_noalloc(op, px, lx, nr, py, ly, _stream(stream)))


def h2bem_apply_timed(op, x, y, stream=None):
    px, lx, nr, py, ly = _vec_args(x, y)
    _check(lib().h2bem_apply_timed(op, px, lx, nr, py, ly, _stream(stream)))


def h2bem_apply_mass(op, alpha, x, y, stream=None):
    """y = A x + alpha M x, M = diag(|tau_i|) (device buffers)."""
    px, lx, nr, py, ly = _vec_args(x, y)
    _check(lib().h2bem_apply_mass(op, ctypes.c_double(alpha), px, lx, nr, py, ly, _stream(stream)))


def h2bem_apply_hypersingular(op, x, y, stream=None):
    """y = W x, the hypersingular operator on piecewise-linear functions through
    the single layer `op` (device buffers, (nrhs, nv))."""
    px, lx, nr, py, ly = _vec_args(x, y)
    _check(lib().h2bem_apply_hypersingular(op, px, lx, nr, py, ly, _stream(stream)))


def h2bem_apply_dlp_p1(op, x, y, transpose: bool = False, alpha: float = 0.0, stream=None):
    """y = K1 x + alpha M1 x (x: (nrhs, nv), y: (nrhs, n)) or K1^T x + alpha M1^T x (x: (nrhs, n),
    y: (nrhs, nv)); device tensors."""
    px, lx, nr, py, ly = _vec_args(x, y)
    _check(lib().h2bem_apply_dlp_p1(op, ctypes.c_double(alpha), px, lx, nr, py, ly, int(transpose), _stream(stream)))


def h2bem_cg_hypersingular(op, m, b, x, rtol=1e-8, maxit=1000, stream=None):
    """CG for (W + m m^T) x = b on the vertices (device tensors (nrhs, nv); m: (nv,) or None);
    returns (iterations, relres per column)."""
    pb, lb, nr, px, lx = _vec_args(b, x)
    pm = ctypes.c_void_p(m.data_ptr()) if m is not None else None
    it = ctypes.c_int(0)
    rel = (ctypes.c_double * nr)()
    _check(lib().h2bem_cg_hypersingular(op, pm, pb, lb, nr, px, lx, ctypes.c_double(rtol), int(maxit),
                                        ctypes.byref(it), rel, _stream(stream)))
    return it.value, list(rel)


def h2bem_cg(op, b, x, rtol=1e-8, maxit=1000, stream=None):
    """Conjugate gradients for G x = b (device buffers, (nrhs, n)); returns (iterations, relres per column)."""
    pb, lb, nr, px, lx = _vec_args(b, x)
    it = ctypes.c_int(0)
    rel = (ctypes.c_double * nr)()
    _check(lib().h2bem_cg(op, pb, lb, nr, px, lx, ctypes.c_double(rtol), int(maxit), ctypes.byref(it), rel,
                          _stream(stream)))
    return it.value, list(rel)


# ---------------------------------------------------------------- convenience
class BatchOperator:
    """Block-diagonal operator over many meshes (vectors concatenated in mesh order)."""

    def __init__(self, meshes, kernel: str | int = "slp", m: int = 4, eta: float = 2.0, leaf_size: int = 32,
                 precision: str | int = "fp64", q_ss: int = 5, cache_singular: bool = False,
                 use_graph: bool = False, autotune: int = 0, singular_fp64: bool = False,
                 recompute_basis: bool = False, store_near: bool = False, gca: bool = False, gca_q: int = 4,
                 gca_kmax: int = 64, gca_eps: float = 1e-6, tc_wait_test: bool = False, hca: bool = False,
                 hca_kaca: int = 64, hca_kmax: int = 64, hca_eps_aca: float = 1e-6, hca_eps: float = 1e-6):
        kernel = {"slp": H2BEM_SLP, "dlp": H2BEM_DLP}.get(kernel, kernel) if isinstance(kernel, str) else kernel
        self.meshes = [h2bem_mesh_create(mh.vertices, mh.triangles) for mh in meshes]
        self.sizes = [int(mh.nt) for mh in meshes]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.n = int(self.offsets[-1])
        o = h2bem_opts_default()
        o.q_ss = q_ss
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.cache_singular = int(cache_singular)
        o.use_graph = int(use_graph)
        o.autotune = int(autotune)
        o.singular_fp64 = int(singular_fp64)
        o.recompute_basis = int(recompute_basis)
        o.store_near = int(store_near)
        if gca:
            o.basis = H2BEM_BASIS_GCA
            o.gca_q, o.gca_kmax, o.gca_eps = int(gca_q), int(gca_kmax), float(gca_eps)
        if hca:
            o.basis = H2BEM_BASIS_HCA
            o.hca_kaca, o.hca_kmax = int(hca_kaca), int(hca_kmax)
            o.hca_eps_aca, o.hca_eps = float(hca_eps_aca), float(hca_eps)
        o.tc_wait_test = int(tc_wait_test)
        self.op = h2bem_batch_create(self.meshes, leaf_size, kernel, m, eta, o)

    def close(self):
        if getattr(self, "op", None) is not None and self.op.value:
            h2bem_operator_destroy(self.op)
            self.op = None
        for mh in getattr(self, "meshes", []):
            if mh.value:
                h2bem_mesh_destroy(mh)
        self.meshes = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, x, y=None, stream=None, transpose: bool = False):
        if y is None:
            y = x.new_empty(x.shape) if not isinstance(x, np.ndarray) else np.empty_like(x)
        (h2bem_apply_transpose if transpose else h2bem_apply)(self.op, x, y, stream)
        return y

    def stats(self) -> dict:
        return h2bem_stats_get(self.op)


class Operator:
    """Owns mesh, tree and operator handles for one surface mesh."""

    def __init__(self, vertices, triangles, kernel: str | int = "slp", m: int = 4, eta: float = 2.0,
                 leaf_size: int = 32, precision: str | int = "fp64", q_ss: int = 5, cache_singular: bool = False,
                 use_graph: bool = False, autotune: int = 0, singular_fp64: bool = False,
                 recompute_basis: bool = False, store_near: bool = False, gca: bool = False, gca_q: int = 4,
                 gca_kmax: int = 64, gca_eps: float = 1e-6, tc_wait_test: bool = False, hca: bool = False,
                 hca_kaca: int = 64, hca_kmax: int = 64, hca_eps_aca: float = 1e-6, hca_eps: float = 1e-6):
        self.kernel = {"slp": H2BEM_SLP, "dlp": H2BEM_DLP}.get(kernel, kernel) if isinstance(kernel, str) else kernel
        self.n = int(np.asarray(triangles).shape[0])
        self.nv = int(np.asarray(vertices).shape[0])
        self.mesh = h2bem_mesh_create(vertices, triangles)
        self.tree = h2bem_tree_build(self.mesh, leaf_size)
        o = h2bem_opts_default()
        o.q_ss = q_ss
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.cache_singular = int(cache_singular)
        o.use_graph = int(use_graph)
        o.autotune = int(autotune)
        o.singular_fp64 = int(singular_fp64)
        o.recompute_basis = int(recompute_basis)
        o.store_near = int(store_near)
        if gca:
            o.basis = H2BEM_BASIS_GCA
            o.gca_q, o.gca_kmax, o.gca_eps = int(gca_q), int(gca_kmax), float(gca_eps)
        if hca:
            o.basis = H2BEM_BASIS_HCA
            o.hca_kaca, o.hca_kmax = int(hca_kaca), int(hca_kmax)
            o.hca_eps_aca, o.hca_eps = float(hca_eps_aca), float(hca_eps)
        o.tc_wait_test = int(tc_wait_test)
        self.op = h2bem_operator_create(self.mesh, self.tree, self.kernel, m, eta, o)

    def close(self):
        for name, fn in (("op", h2bem_operator_destroy), ("tree", h2bem_tree_destroy), ("mesh", h2bem_mesh_destroy)):
            h = getattr(self, name, None)
            if h is not None and h.value:
                fn(h)
                setattr(self, name, None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, x, y=None, stream=None, transpose: bool = False):
        if y is None:
            y = x.new_empty(x.shape) if not isinstance(x, np.ndarray) else np.empty_like(x)
        (h2bem_apply_transpose if transpose else h2bem_apply)(self.op, x, y, stream)
        return y

    def stats(self) -> dict:
        return h2bem_stats_get(self.op)
