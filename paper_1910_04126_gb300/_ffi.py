"""ctypes declarations of libflowtree.so (C ABI in include/flowtree.h).

Loading fails loudly when the library has not been built: there is no CPU
fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

FT_OK = 0
STATUS = {0: "FT_OK", -1: "FT_EINVAL", -2: "FT_ENOMEM", -3: "FT_ECUDA", -4: "FT_ETIMEOUT",
          -5: "FT_EOVERFLOW", -6: "FT_EUNSUPPORTED", -7: "FT_EWORKSPACE", -8: "FT_ETOOBIG"}


class FlowtreeError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (where, STATUS.get(code, "unknown"), code))


class TreeInfo(C.Structure):
    _fields_ = [("n_points", C.c_int64), ("dim", C.c_int32), ("levels", C.c_int32),
                ("phi_log2", C.c_int32), ("rmq_levels", C.c_int32)]


class DocsInfo(C.Structure):
    _fields_ = [("n_docs", C.c_int64), ("n_items", C.c_int64), ("max_support", C.c_int32),
                ("n_embed", C.c_int64)]


ALGO_AUTO, ALGO_WARP, ALGO_THREAD, ALGO_BLOCKED = 0, 1, 2, 3
BLOCKED_MAX_ITEMS = 7936  # longest merged pair of the blocked form (a CTA of 256 threads, 31 items each)
BLOCKED_WARP_ITEMS = 416  # the warp's default staging; longer pairs take a CTA each


class FlowtreeConfig(C.Structure):
    _fields_ = [("warps_per_cta", C.c_int32), ("stage_items", C.c_int32), ("algo", C.c_int32),
                ("stage_tables", C.c_int32), ("deep_loads", C.c_int32)]


vp = C.c_void_p
i64 = C.c_int64
i32 = C.c_int32
sz = C.c_size_t

# name -> (restype, argtypes); every entry point of include/flowtree.h
SIGNATURES = {
    "ft_status_string": (C.c_char_p, [i32]),
    "ft_build_quadtree": (i32, [vp, i64, i32, i32, vp, C.c_uint64, vp, C.POINTER(vp)]),
    "ft_tree_free": (None, [vp]),
    "ft_tree_get_info": (i32, [vp, C.POINTER(TreeInfo)]),
    "ft_tree_export": (i32, [vp, vp, vp, vp, vp]),
    "ft_tree_status": (i32, [vp, vp]),
    "ft_embed_docs": (i32, [vp, vp, vp, vp, i64, vp, C.POINTER(vp)]),
    "ft_docs_free": (None, [vp]),
    "ft_docs_get_info": (i32, [vp, C.POINTER(DocsInfo)]),
    "ft_docs_export": (i32, [vp, vp, vp, vp]),
    "ft_flowtree_batch_workspace_size": (sz, [vp, vp, vp, i64]),
    "ft_flowtree_batch": (i32, [vp, vp, vp, vp, vp, vp, i64, vp, vp, vp, sz, vp]),
    "ft_flowtree_plain": (i32, [vp, vp, vp, vp, vp, vp, i64, vp, vp, sz, vp]),
    "ft_flowtree_set_config": (i32, [vp, C.POINTER(FlowtreeConfig)]),
    "ft_flowtree_get_config": (i32, [vp, C.POINTER(FlowtreeConfig)]),
    "ft_flowtree_autotune": (i32, [vp, vp, vp, vp, vp, vp, i64, vp, vp, sz, vp, C.POINTER(FlowtreeConfig)]),
    "ft_flows_create": (i32, [vp, vp, vp, vp, vp, i64, vp, C.POINTER(vp)]),
    "ft_flows_free": (None, [vp]),
    "ft_flows_capacity": (i32, [vp, C.POINTER(i64), C.POINTER(i64)]),
    "ft_flows_export": (i32, [vp, vp, vp, vp, vp, vp, vp]),
    "ft_flows_create_capacity": (i32, [vp, vp, vp, i64, C.POINTER(vp)]),
    "ft_flows_bind": (i32, [vp, vp, vp, i64, vp]),
    "ft_flowtree_backward_workspace_size": (sz, [vp, vp]),
    "ft_flowtree_backward": (i32, [vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]),
    "ft_quadtree_scan_workspace_size": (sz, [vp, vp, vp, i32]),
    "ft_quadtree_scan": (i32, [vp, vp, vp, i32, vp, sz, vp, vp, vp]),
    "ft_quadtree_l1_dense": (i32, [vp, vp, vp, vp, vp]),
    "ft_quadtree_scan_matches": (i32, [vp, vp, vp, C.POINTER(i64)]),
    "ft_knn_workspace_size": (sz, [vp, vp, vp, i32, i32]),
    "ft_knn": (i32, [vp, vp, vp, vp, i32, i32, vp, sz, vp, vp, vp]),
    "ft_mean_scan_workspace_size": (sz, [vp, vp, i32]),
    "ft_mean_scan": (i32, [vp, vp, vp, i32, vp, sz, vp, vp, vp]),
    "ft_exact_w1_workspace_size": (sz, [vp, vp, i64]),
    "ft_exact_w1_batch": (i32, [vp, vp, vp, vp, vp, i64, vp, vp, sz, vp]),
    "ft_knn_exact_workspace_size": (sz, [vp, vp, vp, i32, i32, i32]),
    "ft_knn_exact": (i32, [vp, vp, vp, vp, i32, i32, i32, vp, sz, vp, vp, vp]),
    "ft_topk_f32_workspace_size": (sz, [i64, i64]),
    "ft_topk_f32": (i32, [vp, i64, i64, i32, vp, sz, vp, vp, vp]),
    "ft_read_probe": (i32, [vp, sz, i32, vp, vp]),
    "ft_flowtree_batch_static": (i32, [vp, vp, vp, vp, vp, vp, i64, vp, vp]),
}

_lib = None


def load() -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError("libflowtree.so is not built (%s); run `python -m paper_1910_04126_gb300.build` "
                           "or __graft_entry__.build() on a machine with nvcc" % LIB)
    lib = C.CDLL(LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code: int, where: str) -> None:
    if code != FT_OK:
        raise FlowtreeError(code, where)
