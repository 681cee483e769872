"""ctypes wrapper of the Flowtree CPU oracle (test infrastructure only).

Every call forwards to oracle.cpp, the plain FP64 restatement of the paper's
definitions; see that file's header for the readings of the paper it takes.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

__all__ = [
    "OracleTree",
    "Supports",
    "exact_w1",
    "mean_distance",
    "min_cost_flow",
    "topk_ids",
    "MASS_ONE",
    "QUANT_BITS",
    "load",
]

MASS_ONE = 1 << 24
QUANT_BITS = 40

_lib = None

_f32p = C.POINTER(C.c_float)
_f64p = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)
_u64p = C.POINTER(C.c_uint64)


def _sig(fn, res, *args):
    fn.restype = res
    fn.argtypes = list(args)


def load():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is not None:
        return _lib
    # FT_ORACLE_SO lets the mutation test load a deliberately broken copy.
    path = os.environ.get("FT_ORACLE_SO") or _build.build()
    lib = C.CDLL(path)
    vp = C.c_void_p
    _sig(lib.oracle_tree_build, vp, _f32p, C.c_int64, C.c_int32, C.c_int32, _u64p)
    _sig(lib.oracle_tree_free, None, vp)
    _sig(lib.oracle_tree_params, None, vp, _f32p, _i32p, _i64p)
    _sig(lib.oracle_tree_z, None, vp, _u64p)
    _sig(lib.oracle_tree_ranks, None, vp, _i64p, _i64p)
    _sig(lib.oracle_tree_lcp, None, vp, _i32p)
    _sig(lib.oracle_lca_depth, C.c_int32, vp, C.c_int64, C.c_int64)
    _sig(lib.oracle_node_of, C.c_int32, vp, C.c_int64, C.c_int32)
    _sig(lib.oracle_embed_docs, C.c_int64, vp, _i64p, _i32p, _f32p, C.c_int64, _i64p, _i64p, _i64p)
    _sig(lib.oracle_quadtree_l1, C.c_int64, vp, _i64p, _i64p, C.c_int64, _i64p, _i64p, C.c_int64)
    _sig(lib.oracle_tree_distance, C.c_int64, vp, C.c_int64, C.c_int64)
    _sig(lib.oracle_flow, C.c_int64, vp, _i64p, _i64p, C.c_int64, _i64p, _i64p, C.c_int64,
         _i64p, _i64p, _i64p, _i32p, C.c_int64)
    _sig(lib.oracle_flowtree, C.c_double, vp, _f32p, _i64p, _i64p, C.c_int64, _i64p, _i64p, C.c_int64)
    _sig(lib.oracle_flowtree_batch, None, vp, _f32p, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p,
         _i64p, _i64p, C.c_int64, C.c_int32, _f64p)
    _sig(lib.oracle_quadtree_l1_batch, None, vp, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p,
         _i64p, _i64p, C.c_int64, C.c_int32, _i64p)
    _sig(lib.oracle_flowtree_grad_batch, None, vp, _f32p, _i64p, _i64p, _i64p, _i64p, _i64p, _i64p,
         _i64p, _i64p, _f64p, C.c_int64, _f64p)
    _sig(lib.oracle_exact_w1, C.c_double, _f32p, C.c_int32, _i64p, _i64p, C.c_int64, _i64p, _i64p, C.c_int64)
    _sig(lib.oracle_mean_distance, C.c_double, _f32p, C.c_int32, _i64p, _i64p, C.c_int64, _i64p, _i64p, C.c_int64)
    _sig(lib.oracle_tree_w1_mcf, C.c_double, vp, _i64p, _i64p, C.c_int64, _i64p, _i64p, C.c_int64)
    _sig(lib.oracle_min_cost_flow, C.c_double, _i64p, C.c_int64, _i64p, C.c_int64, _f64p)
    _lib = lib
    return lib


def _p(a: np.ndarray, ptype):
    return a.ctypes.data_as(ptype)


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int64)


@dataclass
class Supports:
    """Documents as rank-sorted supports with integer masses (sum 2^24 each)."""

    ptr: np.ndarray    # int64 [n_docs + 1]
    point: np.ndarray  # int64 [nnz] ground-point ids
    mass: np.ndarray   # int64 [nnz]

    @property
    def n_docs(self) -> int:
        return len(self.ptr) - 1

    def doc(self, i: int):
        s, e = int(self.ptr[i]), int(self.ptr[i + 1])
        return self.point[s:e], self.mass[s:e]


class OracleTree:
    """The oracle's explicit quadtree over the ground points (Sec. 2)."""

    def __init__(self, points: np.ndarray, levels: int, shift: np.ndarray):
        lib = load()
        self.points = np.ascontiguousarray(points, dtype=np.float32)
        if self.points.ndim != 2:
            raise ValueError("points must be [n, d]")
        self.n, self.d = self.points.shape
        self.levels = int(levels)
        self.shift = np.ascontiguousarray(shift, dtype=np.uint64)
        h = lib.oracle_tree_build(_p(self.points, _f32p), self.n, self.d, self.levels, _p(self.shift, _u64p))
        if not h:
            raise ValueError("oracle_tree_build rejected its arguments")
        self._h = C.c_void_p(h)
        lo = np.zeros(self.d, np.float32)
        pl = C.c_int32(0)
        nn = C.c_int64(0)
        lib.oracle_tree_params(self._h, _p(lo, _f32p), C.byref(pl), C.byref(nn))
        self.lo, self.phi_log2, self.n_nodes = lo, int(pl.value), int(nn.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.oracle_tree_free(h)
            self._h = None

    # -- tree structure ----------------------------------------------------
    def z(self) -> np.ndarray:
        out = np.zeros((self.n, self.d), np.uint64)
        _lib.oracle_tree_z(self._h, _p(out, _u64p))
        return out

    def ranks(self):
        rop = np.zeros(self.n, np.int64)
        por = np.zeros(self.n, np.int64)
        _lib.oracle_tree_ranks(self._h, _p(rop, _i64p), _p(por, _i64p))
        return rop, por

    def lcp(self) -> np.ndarray:
        out = np.zeros(max(self.n - 1, 0), np.int32)
        if self.n > 1:
            _lib.oracle_tree_lcp(self._h, _p(out, _i32p))
        return out

    def lca_depth(self, p: int, q: int) -> int:
        return int(_lib.oracle_lca_depth(self._h, int(p), int(q)))

    def node_of(self, p: int, k: int) -> int:
        return int(_lib.oracle_node_of(self._h, int(p), int(k)))

    def tree_distance(self, p: int, q: int) -> int:
        """Tree distance in units of u = 2*Phi / 2^(L+1)."""
        return int(_lib.oracle_tree_distance(self._h, int(p), int(q)))

    # -- distributions -----------------------------------------------------
    def embed_docs(self, row_ptr, word, weight) -> Supports:
        row_ptr = _i64(row_ptr)
        word = np.ascontiguousarray(word, dtype=np.int32)
        weight = np.ascontiguousarray(weight, dtype=np.float32)
        n_docs = len(row_ptr) - 1
        nnz = int(row_ptr[-1])
        ptr = np.zeros(n_docs + 1, np.int64)
        pt = np.zeros(max(nnz, 1), np.int64)
        ms = np.zeros(max(nnz, 1), np.int64)
        rc = _lib.oracle_embed_docs(self._h, _p(row_ptr, _i64p), _p(word, _i32p), _p(weight, _f32p), n_docs,
                                    _p(ptr, _i64p), _p(pt, _i64p), _p(ms, _i64p))
        if rc != 0:
            raise ValueError("invalid document %d" % (-1 - rc))
        tot = int(ptr[-1])
        return Supports(ptr, pt[:tot].copy(), ms[:tot].copy())

    # -- per-pair quantities -----------------------------------------------
    def quadtree_l1(self, pa, ma, pb, mb) -> int:
        pa, ma, pb, mb = map(_i64, (pa, ma, pb, mb))
        return int(_lib.oracle_quadtree_l1(self._h, _p(pa, _i64p), _p(ma, _i64p), len(pa),
                                           _p(pb, _i64p), _p(mb, _i64p), len(pb)))

    def flow(self, pa, ma, pb, mb):
        """Greedy tree flow: arrays (ia, ib, f, depth) in emission order."""
        pa, ma, pb, mb = map(_i64, (pa, ma, pb, mb))
        cap = len(pa) + len(pb) + 1
        ia, ib, f = (np.zeros(cap, np.int64) for _ in range(3))
        dep = np.zeros(cap, np.int32)
        n = _lib.oracle_flow(self._h, _p(pa, _i64p), _p(ma, _i64p), len(pa), _p(pb, _i64p), _p(mb, _i64p),
                             len(pb), _p(ia, _i64p), _p(ib, _i64p), _p(f, _i64p), _p(dep, _i32p), cap)
        if n < 0:
            raise RuntimeError("oracle_flow: more pairs than s_a + s_b")
        return ia[:n].copy(), ib[:n].copy(), f[:n].copy(), dep[:n].copy()

    def flowtree(self, vocab, pa, ma, pb, mb) -> float:
        vocab = np.ascontiguousarray(vocab, dtype=np.float32)
        pa, ma, pb, mb = map(_i64, (pa, ma, pb, mb))
        return float(_lib.oracle_flowtree(self._h, _p(vocab, _f32p), _p(pa, _i64p), _p(ma, _i64p), len(pa),
                                          _p(pb, _i64p), _p(mb, _i64p), len(pb)))

    def tree_w1_mcf(self, pa, ma, pb, mb) -> float:
        pa, ma, pb, mb = map(_i64, (pa, ma, pb, mb))
        return float(_lib.oracle_tree_w1_mcf(self._h, _p(pa, _i64p), _p(ma, _i64p), len(pa),
                                             _p(pb, _i64p), _p(mb, _i64p), len(pb)))

    # -- batched -----------------------------------------------------------
    def flowtree_batch(self, vocab, A: Supports, B: Supports, pair_a, pair_b, n_threads: int = 1) -> np.ndarray:
        vocab = np.ascontiguousarray(vocab, dtype=np.float32)
        pair_a, pair_b = _i64(pair_a), _i64(pair_b)
        out = np.zeros(len(pair_a), np.float64)
        _lib.oracle_flowtree_batch(self._h, _p(vocab, _f32p), _p(A.ptr, _i64p), _p(A.point, _i64p),
                                   _p(A.mass, _i64p), _p(B.ptr, _i64p), _p(B.point, _i64p), _p(B.mass, _i64p),
                                   _p(pair_a, _i64p), _p(pair_b, _i64p), len(pair_a), int(n_threads),
                                   _p(out, _f64p))
        return out

    def quadtree_l1_batch(self, A: Supports, B: Supports, pair_a, pair_b, n_threads: int = 1) -> np.ndarray:
        pair_a, pair_b = _i64(pair_a), _i64(pair_b)
        out = np.zeros(len(pair_a), np.int64)
        _lib.oracle_quadtree_l1_batch(self._h, _p(A.ptr, _i64p), _p(A.point, _i64p), _p(A.mass, _i64p),
                                      _p(B.ptr, _i64p), _p(B.point, _i64p), _p(B.mass, _i64p),
                                      _p(pair_a, _i64p), _p(pair_b, _i64p), len(pair_a), int(n_threads),
                                      _p(out, _i64p))
        return out

    def grad_batch(self, vocab, A: Supports, B: Supports, pair_a, pair_b, grad_cost) -> np.ndarray:
        vocab = np.ascontiguousarray(vocab, dtype=np.float32)
        pair_a, pair_b = _i64(pair_a), _i64(pair_b)
        g = np.ascontiguousarray(grad_cost, dtype=np.float64)
        out = np.zeros(vocab.shape, np.float64)
        _lib.oracle_flowtree_grad_batch(self._h, _p(vocab, _f32p), _p(A.ptr, _i64p), _p(A.point, _i64p),
                                        _p(A.mass, _i64p), _p(B.ptr, _i64p), _p(B.point, _i64p),
                                        _p(B.mass, _i64p), _p(pair_a, _i64p), _p(pair_b, _i64p), _p(g, _f64p),
                                        len(pair_a), _p(out, _f64p))
        return out


def exact_w1(vocab, pa, ma, pb, mb) -> float:
    """Exact W1 (Eq. 1) by min-cost flow, Euclidean ground metric."""
    lib = load()
    vocab = np.ascontiguousarray(vocab, dtype=np.float32)
    pa, ma, pb, mb = map(_i64, (pa, ma, pb, mb))
    return float(lib.oracle_exact_w1(_p(vocab, _f32p), vocab.shape[1], _p(pa, _i64p), _p(ma, _i64p), len(pa),
                                     _p(pb, _i64p), _p(mb, _i64p), len(pb)))


def mean_distance(vocab, pa, ma, pb, mb) -> float:
    """The Mean method (Sec. 5): distance between the mass-weighted centroids."""
    lib = load()
    vocab = np.ascontiguousarray(vocab, dtype=np.float32)
    pa, ma, pb, mb = map(_i64, (pa, ma, pb, mb))
    return float(lib.oracle_mean_distance(_p(vocab, _f32p), vocab.shape[1], _p(pa, _i64p), _p(ma, _i64p), len(pa),
                                          _p(pb, _i64p), _p(mb, _i64p), len(pb)))


def min_cost_flow(supply, demand, cost) -> float:
    """Min-cost transportation value for integer supply/demand (equal totals)."""
    lib = load()
    s, t = _i64(supply), _i64(demand)
    c = np.ascontiguousarray(cost, dtype=np.float64)
    return float(lib.oracle_min_cost_flow(_p(s, _i64p), len(s), _p(t, _i64p), len(t), _p(c, _f64p)))


def topk_ids(values, k: int, ids=None) -> np.ndarray:
    """k smallest values, ties broken by the smaller id (full sort)."""
    values = np.asarray(values)
    ids = np.arange(len(values)) if ids is None else np.asarray(ids)
    order = np.lexsort((ids, values))
    return ids[order[:k]]
