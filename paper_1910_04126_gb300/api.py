"""PyTorch-facing binding of libflowtree (argument marshalling only).

Every computation runs in the library's CUDA kernels; PyTorch provides device
memory (tensors, workspaces) and streams.  Names follow the C ABI
(include/flowtree.h): ft_build_quadtree -> Tree, ft_embed_docs -> Docs,
ft_flowtree_batch -> flowtree_batch, and so on.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np
import torch

from . import _ffi
from ._ffi import check

MASS_ONE = 1 << 24


def _stream(stream: Optional[torch.cuda.Stream]) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[C.c_void_p]:
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev(x, dtype, device) -> torch.Tensor:
    if isinstance(x, torch.Tensor):
        t = x.to(device=device, dtype=dtype)
    else:
        t = torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=device)
    return t.contiguous()


def _workspace(nbytes: int, device, workspace: Optional[torch.Tensor]) -> torch.Tensor:
    if workspace is not None:
        if workspace.numel() * workspace.element_size() < nbytes:
            raise ValueError("workspace too small: %d < %d bytes" % (workspace.numel(), nbytes))
        return workspace
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


class Tree:
    """Randomly shifted quadtree over the ground points (ft_build_quadtree)."""

    def __init__(self, points: torch.Tensor, levels: int, shift=None, seed: int = 0,
                 stream: Optional[torch.cuda.Stream] = None):
        lib = _ffi.load()
        if not (isinstance(points, torch.Tensor) and points.is_cuda):
            raise TypeError("points must be a CUDA tensor")
        self.points = points.to(torch.float32).contiguous()
        self.device = self.points.device
        n, d = self.points.shape
        self.levels = int(levels)
        sh = None if shift is None else np.ascontiguousarray(shift, dtype=np.uint64)
        if sh is not None and sh.shape != (d,):
            raise ValueError("shift must have one entry per dimension")
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            code = lib.ft_build_quadtree(_ptr(self.points), n, d, self.levels,
                                         None if sh is None else sh.ctypes.data_as(C.c_void_p),
                                         C.c_uint64(seed), _stream(stream), C.byref(h))
        check(code, "ft_build_quadtree")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _ffi.load().ft_tree_free(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    @property
    def info(self) -> _ffi.TreeInfo:
        info = _ffi.TreeInfo()
        check(_ffi.load().ft_tree_get_info(self._h, C.byref(info)), "ft_tree_get_info")
        return info

    def export(self):
        n, d = self.points.shape
        rop = np.zeros(n, np.uint32)
        por = np.zeros(n, np.uint32)
        lcp = np.zeros(max(n - 1, 1), np.uint8)
        sh = np.zeros(d, np.uint64)
        check(_ffi.load().ft_tree_export(self._h, rop.ctypes.data, por.ctypes.data, lcp.ctypes.data,
                                         sh.ctypes.data), "ft_tree_export")
        return rop, por, lcp[: max(n - 1, 0)], sh

    def status(self, stream=None) -> int:
        return int(_ffi.load().ft_tree_status(self._h, _stream(stream)))

    def get_config(self):
        """(warps_per_cta, stage_items, algo, stage_tables, deep_loads); 0 = default."""
        cfg = _ffi.FlowtreeConfig()
        check(_ffi.load().ft_flowtree_get_config(self._h, C.byref(cfg)), "ft_flowtree_get_config")
        return (int(cfg.warps_per_cta), int(cfg.stage_items), int(cfg.algo), int(cfg.stage_tables),
                int(cfg.deep_loads))

    def set_config(self, warps_per_cta: int = 0, stage_items: int = 0, algo: int = 0, stage_tables: int = 0,
                   deep_loads: int = 0):
        cfg = _ffi.FlowtreeConfig(warps_per_cta, stage_items, algo, stage_tables, deep_loads)
        check(_ffi.load().ft_flowtree_set_config(self._h, C.byref(cfg)), "ft_flowtree_set_config")

    # -- checkpoint / resume ---------------------------------------------------
    # The build is deterministic in (points, levels, shift), so a saved index
    # is those inputs plus the launch configuration; loading rebuilds the same
    # tree bit for bit (the shift is the realised one, also when it was drawn
    # from a seed).
    def save(self, path) -> None:
        np.savez(path, points=self.points.cpu().numpy(), levels=np.int64(self.levels), shift=self.export()[3],
                 config=np.asarray(self.get_config(), np.int64))

    @classmethod
    def load(cls, path, device="cuda", stream=None) -> "Tree":
        z = np.load(path)
        t = cls(torch.as_tensor(z["points"], device=device), int(z["levels"]), z["shift"], stream=stream)
        t.set_config(*(int(x) for x in z["config"]))
        return t


class Docs:
    """Distributions on the tree (ft_embed_docs): rank-sorted supports, 2^24 masses."""

    def __init__(self, tree: Tree, row_ptr, word, weight, stream=None):
        lib = _ffi.load()
        self.tree = tree
        dev = tree.device
        self.row_ptr = _dev(row_ptr, torch.int64, dev)
        self.word = _dev(word, torch.int32, dev)
        self.weight = _dev(weight, torch.float32, dev)
        h = C.c_void_p()
        with torch.cuda.device(dev):
            code = lib.ft_embed_docs(tree.handle, _ptr(self.row_ptr), _ptr(self.word), _ptr(self.weight),
                                     self.row_ptr.numel() - 1, _stream(stream), C.byref(h))
        check(code, "ft_embed_docs")
        self._h = h

    @classmethod
    def from_csr(cls, tree: Tree, docs, stream=None) -> "Docs":
        return cls(tree, docs.row_ptr, docs.word, docs.weight, stream)

    def save(self, path) -> None:
        """The CSR input (the embedding is rebuilt from it deterministically on load)."""
        np.savez(path, row_ptr=self.row_ptr.cpu().numpy(), word=self.word.cpu().numpy(),
                 weight=self.weight.cpu().numpy())

    @classmethod
    def load(cls, tree: Tree, path, stream=None) -> "Docs":
        z = np.load(path)
        return cls(tree, z["row_ptr"], z["word"], z["weight"], stream)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _ffi.load().ft_docs_free(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    @property
    def info(self) -> _ffi.DocsInfo:
        info = _ffi.DocsInfo()
        check(_ffi.load().ft_docs_get_info(self._h, C.byref(info)), "ft_docs_get_info")
        return info

    @property
    def n_docs(self) -> int:
        return int(self.info.n_docs)

    def export(self):
        info = self.info
        ptr = np.zeros(info.n_docs + 1, np.int64)
        pt = np.zeros(max(info.n_items, 1), np.uint32)
        ms = np.zeros(max(info.n_items, 1), np.uint32)
        check(_ffi.load().ft_docs_export(self._h, ptr.ctypes.data, pt.ctypes.data, ms.ctypes.data),
              "ft_docs_export")
        return ptr, pt[: info.n_items], ms[: info.n_items]


class Flows:
    """Saved tree flows of a batch of pairs (ft_flows_create), or rebindable
    flows sized for up to max_pairs pairs (Flows.with_capacity + bind)."""

    def __init__(self, tree: Tree, a: Docs, b: Docs, pair_a=None, pair_b=None, stream=None):
        lib = _ffi.load()
        self.tree, self.a, self.b = tree, a, b
        self.pair_a, self.pair_b, n_pairs = _pairs(a, b, pair_a, pair_b, tree.device)
        h = C.c_void_p()
        code = lib.ft_flows_create(tree.handle, a.handle, b.handle, _ptr(self.pair_a), _ptr(self.pair_b),
                                   n_pairs, _stream(stream), C.byref(h))
        check(code, "ft_flows_create")
        self._h = h
        self.n_pairs = n_pairs
        self.max_pairs = 0

    @classmethod
    def with_capacity(cls, tree: Tree, a: Docs, b: Docs, max_pairs: int) -> "Flows":
        """Flows with room for any max_pairs pairs of (a, b), allocated once (ft_flows_create_capacity)."""
        self = cls.__new__(cls)
        self.tree, self.a, self.b = tree, a, b
        h = C.c_void_p()
        check(_ffi.load().ft_flows_create_capacity(tree.handle, a.handle, b.handle, int(max_pairs), C.byref(h)),
              "ft_flows_create_capacity")
        self._h = h
        self.max_pairs = int(max_pairs)
        self.pair_a = self.pair_b = None
        self.n_pairs = 0
        return self

    def bind(self, pair_a=None, pair_b=None, stream=None) -> "Flows":
        """Point the flows at a pair list (None, None = the cross product): no allocation, no host sync."""
        pa, pb, n_pairs = _pairs(self.a, self.b, pair_a, pair_b, self.tree.device)
        check(_ffi.load().ft_flows_bind(self._h, _ptr(pa), _ptr(pb), n_pairs, _stream(stream)), "ft_flows_bind")
        self.pair_a, self.pair_b, self.n_pairs = pa, pb, n_pairs
        return self

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _ffi.load().ft_flows_free(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def export(self):
        lib = _ffi.load()
        npairs, cap = C.c_int64(), C.c_int64()
        check(lib.ft_flows_capacity(self._h, C.byref(npairs), C.byref(cap)), "ft_flows_capacity")
        sp = np.zeros(npairs.value + 1, np.int64)
        cnt = np.zeros(max(npairs.value, 1), np.int32)
        ia, ib, f = (np.zeros(max(cap.value, 1), np.uint32) for _ in range(3))
        dep = np.zeros(max(cap.value, 1), np.uint8)
        check(lib.ft_flows_export(self._h, sp.ctypes.data, cnt.ctypes.data, ia.ctypes.data, ib.ctypes.data,
                                  f.ctypes.data, dep.ctypes.data), "ft_flows_export")
        out = []
        for i in range(npairs.value):
            s, c = int(sp[i]), int(cnt[i])
            out.append((ia[s:s + c].copy(), ib[s:s + c].copy(), f[s:s + c].copy(), dep[s:s + c].copy()))
        return out


def _pairs(a: Docs, b: Docs, pair_a, pair_b, device):
    if pair_a is None and pair_b is None:
        return None, None, a.n_docs * b.n_docs
    pa = _dev(pair_a, torch.int32, device)
    pb = _dev(pair_b, torch.int32, device)
    if pa.numel() != pb.numel():
        raise ValueError("pair_a and pair_b differ in length")
    return pa, pb, pa.numel()


def flowtree_workspace_size(tree: Tree, a: Docs, b: Docs, n_pairs: int) -> int:
    return int(_ffi.load().ft_flowtree_batch_workspace_size(tree.handle, a.handle, b.handle, n_pairs))


def flowtree_batch(tree: Tree, vocab: torch.Tensor, a: Docs, b: Docs, pair_a=None, pair_b=None,
                   flows: Optional[Flows] = None, out: Optional[torch.Tensor] = None,
                   workspace: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Flowtree value of every pair (ft_flowtree_batch); cross product if no pairs."""
    lib = _ffi.load()
    pa, pb, n_pairs = _pairs(a, b, pair_a, pair_b, tree.device)
    if out is None:
        out = torch.empty(n_pairs, dtype=torch.float32, device=tree.device)
    ws_n = lib.ft_flowtree_batch_workspace_size(tree.handle, a.handle, b.handle, n_pairs)
    ws = _workspace(ws_n, tree.device, workspace)
    code = lib.ft_flowtree_batch(tree.handle, _ptr(vocab), a.handle, b.handle, _ptr(pa), _ptr(pb), n_pairs,
                                 _ptr(out), None if flows is None else flows.handle, _ptr(ws),
                                 ws.numel(), _stream(stream))
    check(code, "ft_flowtree_batch")
    return out


def flowtree_plain(tree: Tree, vocab: torch.Tensor, a: Docs, b: Docs, pair_a=None, pair_b=None,
                   out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
                   stream=None) -> torch.Tensor:
    """The one-launch-per-pair form (ft_flowtree_plain)."""
    lib = _ffi.load()
    pa, pb, n_pairs = _pairs(a, b, pair_a, pair_b, tree.device)
    if out is None:
        out = torch.empty(n_pairs, dtype=torch.float32, device=tree.device)
    ws_n = lib.ft_flowtree_batch_workspace_size(tree.handle, a.handle, b.handle, 1)
    ws = _workspace(ws_n, tree.device, workspace)
    code = lib.ft_flowtree_plain(tree.handle, _ptr(vocab), a.handle, b.handle, _ptr(pa), _ptr(pb), n_pairs,
                                 _ptr(out), _ptr(ws), ws.numel(), _stream(stream))
    check(code, "ft_flowtree_plain")
    return out


def flowtree_autotune(tree: Tree, vocab: torch.Tensor, a: Docs, b: Docs, pair_a=None, pair_b=None,
                      stream=None):
    """Time a few launch configurations on these pairs and keep the fastest."""
    lib = _ffi.load()
    pa, pb, n_pairs = _pairs(a, b, pair_a, pair_b, tree.device)
    scratch = torch.empty(max(n_pairs, 1), dtype=torch.float32, device=tree.device)
    # the largest candidate staging needs the most workspace: size for it
    saved = tree.get_config()
    best_ws = 0
    shapes = [(w, cap, _ffi.ALGO_WARP) for w in (2, 3, 4, 5, 6, 7, 8) for cap in (32, 256, 384, 512, 768, 1024)]
    shapes += [(w, 0, _ffi.ALGO_THREAD) for w in (2, 4, 8)]
    for w, cap, algo in shapes:
        try:
            tree.set_config(w, cap, algo)
            best_ws = max(best_ws, lib.ft_flowtree_batch_workspace_size(tree.handle, a.handle, b.handle, n_pairs))
        except _ffi.FlowtreeError:
            pass
    tree.set_config(*saved)
    ws = _workspace(best_ws, tree.device, None)
    cfg = _ffi.FlowtreeConfig()
    code = lib.ft_flowtree_autotune(tree.handle, _ptr(vocab), a.handle, b.handle, _ptr(pa), _ptr(pb), n_pairs,
                                    _ptr(scratch), _ptr(ws), ws.numel(), _stream(stream), C.byref(cfg))
    check(code, "ft_flowtree_autotune")
    return (int(cfg.warps_per_cta), int(cfg.stage_items), int(cfg.algo), int(cfg.stage_tables),
            int(cfg.deep_loads))


def flowtree_backward(tree: Tree, a: Docs, b: Docs, flows: Flows, vocab: torch.Tensor, grad_cost: torch.Tensor,
                      grad_vocab: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
                      stream=None) -> torch.Tensor:
    """Adjoint for the frozen flow (ft_flowtree_backward); accumulates into grad_vocab."""
    lib = _ffi.load()
    if grad_vocab is None:
        grad_vocab = torch.zeros_like(vocab, dtype=torch.float32)
    ws_n = lib.ft_flowtree_backward_workspace_size(tree.handle, flows.handle)
    ws = _workspace(ws_n, tree.device, workspace)
    gc = grad_cost.to(torch.float32).contiguous()
    code = lib.ft_flowtree_backward(tree.handle, a.handle, b.handle, flows.handle, _ptr(vocab), _ptr(gc),
                                    _ptr(grad_vocab), _ptr(ws), ws.numel(), _stream(stream))
    check(code, "ft_flowtree_backward")
    return grad_vocab


def quadtree_scan(tree: Tree, queries: Docs, db: Docs, k1: int, with_l1: bool = False,
                  workspace: Optional[torch.Tensor] = None, stream=None):
    """k1 smallest quadtree-W1 candidates per query (ft_quadtree_scan)."""
    lib = _ffi.load()
    nq = queries.n_docs
    ids = torch.empty((nq, k1), dtype=torch.int32, device=tree.device)
    l1 = torch.empty((nq, k1), dtype=torch.int64, device=tree.device) if with_l1 else None
    ws_n = lib.ft_quadtree_scan_workspace_size(tree.handle, queries.handle, db.handle, k1)
    ws = _workspace(ws_n, tree.device, workspace)
    code = lib.ft_quadtree_scan(tree.handle, queries.handle, db.handle, k1, _ptr(ws), ws.numel(), _ptr(ids),
                                _ptr(l1), _stream(stream))
    check(code, "ft_quadtree_scan")
    return (ids, l1) if with_l1 else ids


def quadtree_l1_dense(tree: Tree, queries: Docs, db: Docs, stream=None) -> torch.Tensor:
    lib = _ffi.load()
    out = torch.empty((queries.n_docs, db.n_docs), dtype=torch.int64, device=tree.device)
    check(lib.ft_quadtree_l1_dense(tree.handle, queries.handle, db.handle, _ptr(out), _stream(stream)),
          "ft_quadtree_l1_dense")
    return out


def quadtree_scan_matches(tree: Tree, queries: Docs, db: Docs) -> int:
    """(query node, database document) matches the scan visits (ft_quadtree_scan_matches)."""
    n = C.c_int64(0)
    check(_ffi.load().ft_quadtree_scan_matches(tree.handle, queries.handle, db.handle, C.byref(n)),
          "ft_quadtree_scan_matches")
    return int(n.value)


def knn_workspace_size(tree: Tree, db: Docs, queries: Docs, k1: int, k: int) -> int:
    return int(_ffi.load().ft_knn_workspace_size(tree.handle, db.handle, queries.handle, k1, k))


def knn(tree: Tree, vocab: torch.Tensor, db: Docs, queries: Docs, k1: int, k: int,
        workspace: Optional[torch.Tensor] = None, ids: Optional[torch.Tensor] = None,
        dist: Optional[torch.Tensor] = None, stream=None):
    """Quadtree scan -> top-k1 -> Flowtree -> top-k per query (ft_knn)."""
    lib = _ffi.load()
    nq = queries.n_docs
    if ids is None:
        ids = torch.empty((nq, k), dtype=torch.int32, device=tree.device)
    if dist is None:
        dist = torch.empty((nq, k), dtype=torch.float32, device=tree.device)
    ws = _workspace(knn_workspace_size(tree, db, queries, k1, k), tree.device, workspace)
    code = lib.ft_knn(tree.handle, _ptr(vocab), db.handle, queries.handle, k1, k, _ptr(ws), ws.numel(),
                      _ptr(ids), _ptr(dist), _stream(stream))
    check(code, "ft_knn")
    return ids, dist


def mean_scan(tree: Tree, vocab: torch.Tensor, queries: Docs, db: Docs, k1: int,
              workspace: Optional[torch.Tensor] = None, stream=None):
    """k1 nearest database documents per query by centroid distance (ft_mean_scan): (ids, distances)."""
    lib = _ffi.load()
    nq = queries.n_docs
    ids = torch.empty((nq, k1), dtype=torch.int32, device=tree.device)
    dist = torch.empty((nq, k1), dtype=torch.float32, device=tree.device)
    ws = _workspace(lib.ft_mean_scan_workspace_size(queries.handle, db.handle, k1), tree.device, workspace)
    code = lib.ft_mean_scan(_ptr(vocab), queries.handle, db.handle, k1, _ptr(ws), ws.numel(), _ptr(ids), _ptr(dist),
                            _stream(stream))
    check(code, "ft_mean_scan")
    return ids, dist


def exact_w1_workspace_size(a: Docs, b: Docs, n_pairs: int) -> int:
    return int(_ffi.load().ft_exact_w1_workspace_size(a.handle, b.handle, n_pairs))


def exact_w1(tree: Tree, vocab: torch.Tensor, a: Docs, b: Docs, pair_a, pair_b,
             out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None, stream=None):
    """Exact W1 of the pairs (a[pair_a[i]], b[pair_b[i]]) by min-cost flow (ft_exact_w1_batch)."""
    lib = _ffi.load()
    pa = _dev(pair_a, torch.int32, tree.device)
    pb = _dev(pair_b, torch.int32, tree.device)
    n = int(pa.numel())
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=tree.device)
    ws = _workspace(exact_w1_workspace_size(a, b, n), tree.device, workspace)
    code = lib.ft_exact_w1_batch(_ptr(vocab), a.handle, b.handle, _ptr(pa), _ptr(pb), n, _ptr(out), _ptr(ws),
                                 ws.numel(), _stream(stream))
    check(code, "ft_exact_w1_batch")
    return out


def knn_exact_workspace_size(tree: Tree, db: Docs, queries: Docs, k1: int, k2: int, k: int) -> int:
    return int(_ffi.load().ft_knn_exact_workspace_size(tree.handle, db.handle, queries.handle, k1, k2, k))


def knn_exact(tree: Tree, vocab: torch.Tensor, db: Docs, queries: Docs, k1: int, k2: int, k: int,
              workspace: Optional[torch.Tensor] = None, ids: Optional[torch.Tensor] = None,
              dist: Optional[torch.Tensor] = None, stream=None):
    """Quadtree scan -> top-k1 -> Flowtree -> top-k2 -> exact W1 -> top-k per query (ft_knn_exact)."""
    lib = _ffi.load()
    nq = queries.n_docs
    if ids is None:
        ids = torch.empty((nq, k), dtype=torch.int32, device=tree.device)
    if dist is None:
        dist = torch.empty((nq, k), dtype=torch.float32, device=tree.device)
    ws = _workspace(knn_exact_workspace_size(tree, db, queries, k1, k2, k), tree.device, workspace)
    code = lib.ft_knn_exact(tree.handle, _ptr(vocab), db.handle, queries.handle, k1, k2, k, _ptr(ws), ws.numel(),
                            _ptr(ids), _ptr(dist), _stream(stream))
    check(code, "ft_knn_exact")
    return ids, dist


def topk_f32(values: torch.Tensor, k: int, ids: Optional[torch.Tensor] = None,
             vals: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None, stream=None):
    """Per-row k smallest of a [rows, cols] FP32 tensor, ties by column (ft_topk_f32)."""
    lib = _ffi.load()
    v = values.contiguous()
    rows, cols = v.shape
    if ids is None:
        ids = torch.empty((rows, k), dtype=torch.int32, device=v.device)
    if vals is None:
        vals = torch.empty((rows, k), dtype=torch.float32, device=v.device)
    ws = _workspace(lib.ft_topk_f32_workspace_size(rows, cols), v.device, workspace)
    check(lib.ft_topk_f32(_ptr(v), rows, cols, k, _ptr(ws), ws.numel(), _ptr(ids), _ptr(vals), _stream(stream)),
          "ft_topk_f32")
    return ids, vals


def read_probe(buf: torch.Tensor, passes: int, sink: torch.Tensor, stream=None) -> None:
    """Read buf `passes` times from every SM, bypassing L1 (ft_read_probe): the measured read-bandwidth peak
    of the L2 roofline.  buf: contiguous device tensor (16-byte aligned, size a multiple of 16 bytes);
    sink: one int32/uint32 device word."""
    check(_ffi.load().ft_read_probe(_ptr(buf), buf.numel() * buf.element_size(), passes, _ptr(sink),
                                    _stream(stream)), "ft_read_probe")


class FlowtreeFunction(torch.autograd.Function):
    """Flowtree values of a batch of pairs, differentiable in the vocabulary rows.

    The tree flow is piecewise constant in the coordinates (it depends on the
    quadtree cells only), so the gradient is that of the pricing sum for the
    frozen flow, computed by the library's adjoint kernels.
    """

    @staticmethod
    def forward(ctx, vocab, tree, a, b, pair_a, pair_b, flows=None):
        if flows is None:
            flows = Flows(tree, a, b, pair_a, pair_b)
        elif flows.max_pairs:  # caller-held rebindable flows: bound to this call's pairs (no allocation, no sync)
            flows.bind(pair_a, pair_b)
        # else: caller-held flows created for exactly these pairs, reused as they are
        cost = flowtree_batch(tree, vocab.detach(), a, b, flows.pair_a, flows.pair_b, flows=flows)
        ctx.tree, ctx.a, ctx.b, ctx.flows = tree, a, b, flows
        ctx.save_for_backward(vocab)
        return cost

    @staticmethod
    def backward(ctx, grad_cost):
        (vocab,) = ctx.saved_tensors
        g = flowtree_backward(ctx.tree, ctx.a, ctx.b, ctx.flows, vocab.detach().contiguous(),
                              grad_cost.contiguous())
        return g, None, None, None, None, None, None


def flowtree(vocab: torch.Tensor, tree: Tree, a: Docs, b: Docs, pair_a=None, pair_b=None,
             flows: Optional[Flows] = None) -> torch.Tensor:
    """Differentiable Flowtree values (FlowtreeFunction).  flows: optional caller-held Flows reused across
    calls, so a training step allocates and synchronises nothing: either created for exactly these pairs
    (used as they are) or rebindable (Flows.with_capacity; bound to the pairs of each call)."""
    return FlowtreeFunction.apply(vocab, tree, a, b, pair_a, pair_b, flows)
