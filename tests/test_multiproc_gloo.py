"""The N > 1 host path on CPU: two gloo ranks shard the database, score their
shard with the oracle, all-gather their local top-k lists and merge them; the
result must equal the unsharded top-k.  (The GPU ranks run ft_knn on their
shard instead of the oracle; the sharding and the merge are the same code.)
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1910_04126_gb300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, k, out_dir):
    import torch
    import torch.distributed as dist

    import oracle as O

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.tiny(n_points=600, n_db=257, n_queries=5)
    ot = O.OracleTree(w.points, w.levels, w.shift)
    lo, hi = shard.shard_range(w.db.n, rank, world)
    local = w.db.subset(np.arange(lo, hi))
    Sd = ot.embed_docs(local.row_ptr, local.word, local.weight)
    Sq = ot.embed_docs(w.queries.row_ptr, w.queries.word, w.queries.weight)
    nq, nd = w.queries.n, local.n
    cost = ot.flowtree_batch(w.points, Sq, Sd, np.repeat(np.arange(nq), nd), np.tile(np.arange(nd), nq)).reshape(nq, nd)
    ids = np.stack([O.topk_ids(cost[q], k) for q in range(nq)])
    d = np.take_along_axis(cost, ids, axis=1)
    gi, gd = shard.gather_topk(torch.as_tensor(ids + lo), torch.as_tensor(d), k)
    if rank == 0:
        np.save(os.path.join(out_dir, "ids.npy"), gi)
        np.save(os.path.join(out_dir, "d.npy"), gd)
    dist.barrier()
    dist.destroy_process_group()


def test_shard_range_partitions():
    for n in (0, 1, 7, 100, 101):
        for world in (1, 2, 3, 8):
            spans = [shard.shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.slow
def test_two_gloo_ranks_sharded_topk_equals_unsharded(tmp_path):
    import oracle as O

    k, world = 7, 2
    mp.start_processes(_worker, args=(world, _free_port(), k, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    gi, gd = np.load(tmp_path / "ids.npy"), np.load(tmp_path / "d.npy")
    w = synth.tiny(n_points=600, n_db=257, n_queries=5)
    ot = O.OracleTree(w.points, w.levels, w.shift)
    Sd = ot.embed_docs(w.db.row_ptr, w.db.word, w.db.weight)
    Sq = ot.embed_docs(w.queries.row_ptr, w.queries.word, w.queries.weight)
    nq, nd = w.queries.n, w.db.n
    cost = ot.flowtree_batch(w.points, Sq, Sd, np.repeat(np.arange(nq), nd), np.tile(np.arange(nd), nq)).reshape(nq, nd)
    for q in range(nq):
        want = O.topk_ids(cost[q], k)
        assert np.array_equal(gi[q], want)
        assert np.array_equal(gd[q], cost[q][want])
