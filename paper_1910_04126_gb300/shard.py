"""Data parallelism over documents (host logic; no data-path kernel).

Flowtree pairs are independent, so the batch shards without any exchange
inside the hot path.  Two layouts are used:

* weak scaling (the benchmark): every rank scores its own query batch
  against the full database; nothing is exchanged.
* database sharding (kNN serving): the database is split into contiguous
  shards and every rank holds one.  Per query batch:
    1. every shard takes its k1 smallest quadtree-W1 documents per query
       (ft_quadtree_scan), ids made global;
    2. the lists are gathered and the k1 smallest (W1, global id) per query
       kept: the global top-k1, exact because it is contained in the union
       of the local lists;
    3. every shard runs Flowtree on the (query, candidate) pairs whose
       candidate it owns (ft_flowtree_batch on explicit pairs) and keeps its
       k best per query by (Flowtree value, global id);
    4. those lists are gathered and merged by (value, global id).
  The result equals the unsharded pipeline (ft_knn) on the whole database:
  the same candidates, the same per-pair values, the same tie rule.

The gathers use torch.distributed (NCCL between GPUs, gloo on CPU), or, for
shards held in one process, plain lists.
"""
from __future__ import annotations

from typing import Callable, List, Tuple

import numpy as np


def shard_range(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous block [lo, hi) of n items owned by `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def merge_topk(ids: np.ndarray, dists: np.ndarray, k: int) -> Tuple[np.ndarray, np.ndarray]:
    """Merge per-rank top-k lists.

    ids, dists: [world, n_queries, k_local] with ids already global.  Returns
    the k best per query by (distance, id), ascending.
    """
    world, nq, kl = ids.shape
    out_i = np.empty((nq, k), dtype=ids.dtype)
    out_d = np.empty((nq, k), dtype=dists.dtype)
    for q in range(nq):
        i = ids[:, q, :].reshape(-1)
        d = dists[:, q, :].reshape(-1)
        order = np.lexsort((i, d))[:k]
        out_i[q] = i[order]
        out_d[q] = d[order]
    return out_i, out_d


def gather_topk(local_ids, local_dists, k: int):
    """All-gather per-rank (global ids, distances) [nq, k_local] and merge them.

    local_ids / local_dists are torch tensors on the rank's device (CPU for
    gloo).  Returns numpy arrays (ids, dists) [nq, k] on every rank.
    """
    import torch
    import torch.distributed as dist

    world = dist.get_world_size()
    gi = [torch.empty_like(local_ids) for _ in range(world)]
    gd = [torch.empty_like(local_dists) for _ in range(world)]
    dist.all_gather(gi, local_ids)
    dist.all_gather(gd, local_dists)
    ids = np.stack([t.cpu().numpy() for t in gi])
    dists = np.stack([t.cpu().numpy() for t in gd])
    return merge_topk(ids, dists, k)


def merge_candidates(ids: List[np.ndarray], l1: List[np.ndarray], k1: int) -> np.ndarray:
    """Step 2: the global top-k1 per query from the shards' lists.

    ids, l1: per shard, [n_queries, k1_shard] global document ids and their
    quadtree-W1 values (int64).  Returns [n_queries, k1] global ids, the k1
    smallest by (W1, id) ascending.
    """
    i = np.concatenate(ids, axis=1)
    v = np.concatenate(l1, axis=1)
    nq = i.shape[0]
    k = min(k1, i.shape[1])
    out = np.empty((nq, k), dtype=np.int64)
    for q in range(nq):
        out[q] = i[q][np.lexsort((i[q], v[q]))[:k]]
    return out


def scan_local(tree, db_shard, id_base: int, queries, k1: int) -> Tuple[np.ndarray, np.ndarray]:
    """Step 1 on one shard (documents id_base .. id_base + n - 1 of the whole
    database): its k1 smallest quadtree-W1 documents per query, as global ids
    with their W1 values (int64 [n_queries, min(k1, n)])."""
    from . import api
    k = min(k1, db_shard.n_docs)
    ids, l1 = api.quadtree_scan(tree, queries, db_shard, k, with_l1=True)
    return ids.cpu().numpy().astype(np.int64) + id_base, l1.cpu().numpy().astype(np.int64)


def flowtree_local(tree, vocab, db_shard, id_base: int, queries, cand: np.ndarray,
                   k: int) -> Tuple[np.ndarray, np.ndarray]:
    """Step 3 on one shard: Flowtree of every (query, candidate) pair of the
    global candidate lists `cand` [n_queries, k1] whose candidate the shard
    owns, and its k best per query by (value, global id).  Returns global ids
    (int64) and values (float32) [n_queries, k], padded with (-1, +inf)."""
    from . import api
    nq = cand.shape[0]
    lo, hi = id_base, id_base + db_shard.n_docs
    qi, ci = np.nonzero((cand >= lo) & (cand < hi))
    gid = cand[qi, ci]
    cost = np.empty(0, dtype=np.float32)
    if len(qi):
        cost = api.flowtree_batch(tree, vocab, queries, db_shard, qi.astype(np.int32),
                                  (gid - lo).astype(np.int32)).cpu().numpy()
    ids = np.full((nq, k), -1, dtype=np.int64)
    vals = np.full((nq, k), np.inf, dtype=np.float32)
    for q in range(nq):
        sel = np.nonzero(qi == q)[0]
        order = sel[np.lexsort((gid[sel], cost[sel]))][:k]
        ids[q, :len(order)] = gid[order]
        vals[q, :len(order)] = cost[order]
    return ids, vals


def merge_local_topk(ids: List[np.ndarray], vals: List[np.ndarray], k: int) -> Tuple[np.ndarray, np.ndarray]:
    """Step 4: merge the shards' [n_queries, k] lists by (value, global id)."""
    return merge_topk(np.stack(ids), np.stack(vals), k)


def knn_sharded(tree, vocab, db_shard, id_base: int, queries, k1: int, k: int,
                gather: Callable[[np.ndarray], List[np.ndarray]] = None) -> Tuple[np.ndarray, np.ndarray]:
    """Steps 1-4 for the rank holding `db_shard`; `gather(x)` returns every
    rank's x in rank order (default: torch.distributed all_gather)."""
    if gather is None:
        gather = _allgather_np
    ids1, l11 = scan_local(tree, db_shard, id_base, queries, k1)
    cand = merge_candidates(gather(ids1), gather(l11), k1)
    ids2, vals2 = flowtree_local(tree, vocab, db_shard, id_base, queries, cand, k)
    return merge_local_topk(gather(ids2), gather(vals2), k)


def _allgather_np(x: np.ndarray) -> List[np.ndarray]:
    import torch
    import torch.distributed as dist

    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.as_tensor(np.ascontiguousarray(x)).to(dev)
    out = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(out, t)
    return [o.cpu().numpy() for o in out]
