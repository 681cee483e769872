"""Database sharding on one GPU: two shards in one process, the exact
sharded pipeline (scan per shard -> global top-k1 -> Flowtree per shard on
its candidates -> merge) against the unsharded ft_knn (bit-identical ids and
values) and, for two queries, against the oracle's Flowtree of the global
candidates.  The gathers are plain lists here; the multi-process path uses
the same functions with torch.distributed (tests/test_multiproc_gloo.py
covers that path on CPU ranks)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1910_04126_gb300 import api, shard, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("algo", [1, 3])
def test_two_shards_equal_unsharded_knn(algo):
    vocab = synth.mixture_vocab(3000, 30, 50, 0.3, 40)
    shift = synth.random_shift(30, 41)
    db = synth.zipf_docs(3000, 700, 42, median=30, s_lo=5, s_hi=120)
    q = synth.zipf_docs(3000, 9, 43, median=30, s_lo=5, s_hi=120)
    tree = api.Tree(torch.as_tensor(vocab, device="cuda"), 12, shift)
    tree.set_config(0, 0, algo)
    D, Q = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    k1, k = 60, 10
    ref_ids, ref_d = api.knn(tree, tree.points, D, Q, k1, k)
    ref_ids, ref_d = ref_ids.cpu().numpy(), ref_d.cpu().numpy()

    spans = [shard.shard_range(db.n, r, 2) for r in range(2)]
    shards = [api.Docs.from_csr(tree, db.subset(np.arange(lo, hi))) for lo, hi in spans]
    s1 = [shard.scan_local(tree, S, lo, Q, k1) for S, (lo, _) in zip(shards, spans)]
    cand = shard.merge_candidates([a for a, _ in s1], [b for _, b in s1], k1)
    s2 = [shard.flowtree_local(tree, tree.points, S, lo, Q, cand, k) for S, (lo, _) in zip(shards, spans)]
    ids, d = shard.merge_local_topk([a for a, _ in s2], [b for _, b in s2], k)
    assert np.array_equal(ids, ref_ids.astype(np.int64))
    assert np.array_equal(d, ref_d)
    assert tree.status() == 0

    # the candidates equal the unsharded scan's, and two queries' values the oracle's
    ref_cand = api.quadtree_scan(tree, Q, D, k1).cpu().numpy()
    assert np.array_equal(cand, ref_cand.astype(np.int64))
    ot = O.OracleTree(vocab, 12, shift)
    Sd, Sq = ot.embed_docs(db.row_ptr, db.word, db.weight), ot.embed_docs(q.row_ptr, q.word, q.weight)
    for qi in (0, 5):
        c = ot.flowtree_batch(vocab, Sq, Sd, np.full(k1, qi), cand[qi], n_threads=4)
        oi = O.topk_ids(c, k)
        np.testing.assert_allclose(d[qi], c[oi], rtol=1e-5)
