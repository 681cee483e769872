"""Data parallelism over documents (host logic; no data-path kernel).

Flowtree pairs are independent, so the batch shards without any exchange
inside the hot path.  Two layouts are used:

* weak scaling (the benchmark): every rank scores its own query batch
  against the full database; nothing is exchanged.
* database sharding (kNN serving): the database is split into contiguous
  shards, every rank runs the whole pipeline (quadtree scan -> top-k1 ->
  Flowtree -> top-k) on its shard for the same queries, and the per-rank
  top-k lists are gathered once per batch and merged by (distance, global
  document id).  The global top-k is contained in the union of the local
  ones, so the merge is exact.

The gather uses torch.distributed (NCCL between GPUs, gloo on CPU).
"""
from __future__ import annotations

from typing import Tuple

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
