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


def _oracle_scan_local(ot, Sq, db, lo, k1):
    import oracle as O
    Sd = ot.embed_docs(db.row_ptr, db.word, db.weight)
    nq, nd = Sq.n_docs, db.n
    l1 = ot.quadtree_l1_batch(Sq, Sd, np.repeat(np.arange(nq), nd), np.tile(np.arange(nd), nq)).reshape(nq, nd)
    k = min(k1, nd)
    ids = np.stack([O.topk_ids(l1[q], k) for q in range(nq)])
    return ids.astype(np.int64) + lo, np.take_along_axis(l1, ids, axis=1).astype(np.int64)


def _oracle_flowtree_local(ot, pts, Sq, db, lo, cand, k):
    Sd = ot.embed_docs(db.row_ptr, db.word, db.weight)
    nq = cand.shape[0]
    ids = np.full((nq, k), -1, dtype=np.int64)
    vals = np.full((nq, k), np.inf, dtype=np.float32)
    for q in range(nq):
        mine = cand[q][(cand[q] >= lo) & (cand[q] < lo + db.n)]
        if len(mine) == 0:
            continue
        c = ot.flowtree_batch(pts, Sq, Sd, np.full(len(mine), q), mine - lo).astype(np.float32)
        order = np.lexsort((mine, c))[:k]
        ids[q, :len(order)] = mine[order]
        vals[q, :len(order)] = c[order]
    return ids, vals


def _worker_two_stage(rank, world, port, k1, k, out_dir):
    import torch.distributed as dist

    import oracle as O

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.tiny(n_points=600, n_db=257, n_queries=5)
    ot = O.OracleTree(w.points, w.levels, w.shift)
    Sq = ot.embed_docs(w.queries.row_ptr, w.queries.word, w.queries.weight)
    lo, hi = shard.shard_range(w.db.n, rank, world)
    local = w.db.subset(np.arange(lo, hi))
    # the GPU steps of the sharded pipeline, computed by the oracle; the
    # gathers are the pipeline's own (torch.distributed over gloo)
    shard.scan_local = lambda tree, db_shard, id_base, queries, k1_: _oracle_scan_local(ot, Sq, local, lo, k1_)
    shard.flowtree_local = lambda tree, vocab, db_shard, id_base, queries, cand, k_: _oracle_flowtree_local(
        ot, w.points, Sq, local, lo, cand, k_)
    ids, d = shard.knn_sharded(None, None, local, lo, Sq, k1, k)
    if rank == 0:
        np.save(os.path.join(out_dir, "ids2.npy"), ids)
        np.save(os.path.join(out_dir, "d2.npy"), d)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.slow
def test_two_gloo_ranks_two_stage_pipeline_equals_unsharded(tmp_path):
    """Scan -> global top-k1 -> Flowtree -> top-k, sharded over two ranks, equals the unsharded pipeline."""
    import oracle as O

    k1, k, world = 30, 6, 2
    mp.start_processes(_worker_two_stage, args=(world, _free_port(), k1, k, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    gi, gd = np.load(tmp_path / "ids2.npy"), np.load(tmp_path / "d2.npy")
    w = synth.tiny(n_points=600, n_db=257, n_queries=5)
    ot = O.OracleTree(w.points, w.levels, w.shift)
    Sd = ot.embed_docs(w.db.row_ptr, w.db.word, w.db.weight)
    Sq = ot.embed_docs(w.queries.row_ptr, w.queries.word, w.queries.weight)
    nq, nd = w.queries.n, w.db.n
    pa, pb = np.repeat(np.arange(nq), nd), np.tile(np.arange(nd), nq)
    l1 = ot.quadtree_l1_batch(Sq, Sd, pa, pb).reshape(nq, nd)
    for q in range(nq):
        cand = O.topk_ids(l1[q], k1)
        c = ot.flowtree_batch(w.points, Sq, Sd, np.full(k1, q), cand).astype(np.float32)
        order = np.lexsort((cand, c))[:k]
        assert np.array_equal(gi[q], cand[order])
        assert np.array_equal(gd[q], c[order])


def test_merge_candidates_is_global_topk():
    rng = np.random.default_rng(3)
    nq, n, k1 = 4, 90, 12
    l1 = rng.integers(0, 6, (nq, n)).astype(np.int64)  # many ties
    spans = [shard.shard_range(n, r, 3) for r in range(3)]
    ids_l, l1_l = [], []
    for lo, hi in spans:
        part = l1[:, lo:hi]
        loc = np.stack([np.lexsort((np.arange(hi - lo), part[q]))[:k1] for q in range(nq)])
        ids_l.append(loc + lo)
        l1_l.append(np.take_along_axis(part, loc, axis=1))
    got = shard.merge_candidates(ids_l, l1_l, k1)
    for q in range(nq):
        assert np.array_equal(got[q], np.lexsort((np.arange(n), l1[q]))[:k1])
