"""GPU parity of the quadtree-W1 prefilter, the top-k select and the kNN pipeline.

L1 values and top-k1 ids are bit-exact against the oracle (ties broken by
the smaller document id).  The final Flowtree top-k equals the oracle's
except for swaps between candidates whose FP64 values differ by at most
2e-5 relative (FP32 versus FP64 ranking of near-ties).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1910_04126_gb300 import api, synth

pytestmark = pytest.mark.gpu


def workloads():
    w = synth.tiny(n_points=1000, n_db=400, n_queries=9)
    yield "tiny2d", w.points, w.levels, w.shift, w.db, w.queries
    yield "grid", synth.grid_points(), 12, synth.random_shift(2, 21), synth.stroke_images(300, 22), \
        synth.stroke_images(6, 23)
    V = synth.mixture_vocab(5000, 300, 100, 0.3, 24)
    yield "d300", V, 12, synth.random_shift(300, 25), synth.zipf_docs(5000, 600, 26, median=60), \
        synth.zipf_docs(5000, 5, 27, median=60)
    V1 = np.random.default_rng(28).random((800, 1)).astype(np.float32)
    yield "line", V1, 14, synth.random_shift(1, 29), synth.uniform_docs(800, 350, 1, 50, 30), \
        synth.uniform_docs(800, 4, 1, 50, 31)


WL = {w[0]: w[1:] for w in workloads()}


def both(name):
    pts, L, shift, db, q = WL[name]
    tree = api.Tree(torch.as_tensor(pts, device="cuda"), L, shift)
    ot = O.OracleTree(pts, L, shift)
    return pts, tree, ot, db, q, api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q), \
        ot.embed_docs(db.row_ptr, db.word, db.weight), ot.embed_docs(q.row_ptr, q.word, q.weight)


@pytest.mark.parametrize("name", sorted(WL))
def test_l1_dense_bit_exact(name):
    pts, tree, ot, db, q, Dd, Dq, Sd, Sq = both(name)
    got = api.quadtree_l1_dense(tree, Dq, Dd).cpu().numpy()
    qa = np.repeat(np.arange(q.n), db.n)
    qb = np.tile(np.arange(db.n), q.n)
    ref = ot.quadtree_l1_batch(Sq, Sd, qa, qb, n_threads=4).reshape(q.n, db.n)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("name", sorted(WL))
@pytest.mark.parametrize("k1", [1, 37, 256])
def test_scan_topk_ids_bit_exact(name, k1):
    pts, tree, ot, db, q, Dd, Dq, Sd, Sq = both(name)
    ids, l1 = api.quadtree_scan(tree, Dq, Dd, k1, with_l1=True)
    ids, l1 = ids.cpu().numpy(), l1.cpu().numpy()
    qa = np.repeat(np.arange(q.n), db.n)
    qb = np.tile(np.arange(db.n), q.n)
    ref = ot.quadtree_l1_batch(Sq, Sd, qa, qb, n_threads=4).reshape(q.n, db.n)
    for i in range(q.n):
        want = O.topk_ids(ref[i], k1)
        assert np.array_equal(ids[i], want)
        assert np.array_equal(l1[i], ref[i][want])


@pytest.mark.parametrize("name", sorted(WL))
def test_knn_pipeline_vs_oracle(name):
    pts, tree, ot, db, q, Dd, Dq, Sd, Sq = both(name)
    k1, k = 64, 10
    ids, dist = api.knn(tree, tree.points, Dd, Dq, k1, k)
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy().astype(np.float64)
    qa = np.repeat(np.arange(q.n), db.n)
    qb = np.tile(np.arange(db.n), q.n)
    l1 = ot.quadtree_l1_batch(Sq, Sd, qa, qb, n_threads=4).reshape(q.n, db.n)
    for i in range(q.n):
        cand = O.topk_ids(l1[i], k1)
        cost = ot.flowtree_batch(pts, Sq, Sd, np.full(k1, i), cand, n_threads=2)
        order = np.lexsort((cand, cost))
        want_ids, want_cost = cand[order[:k]], cost[order[:k]]
        np.testing.assert_allclose(dist[i], want_cost, rtol=1e-5, atol=1e-30)
        costmap = dict(zip(cand.tolist(), cost.tolist()))
        for a, b in zip(ids[i], want_ids):
            if a != b:  # allowed only between near-ties
                assert abs(costmap[int(a)] - costmap[int(b)]) <= 2e-5 * max(costmap[int(b)], 1e-30)


def test_knn_graph_capture_replay():
    pts, tree, ot, db, q, Dd, Dq, Sd, Sq = both("d300")
    k1, k = 32, 5
    ws = torch.empty(api.knn_workspace_size(tree, Dd, Dq, k1, k), dtype=torch.uint8, device="cuda")
    ids = torch.empty((q.n, k), dtype=torch.int32, device="cuda")
    dist = torch.empty((q.n, k), dtype=torch.float32, device="cuda")
    ref_ids, ref_dist = api.knn(tree, tree.points, Dd, Dq, k1, k)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        api.knn(tree, tree.points, Dd, Dq, k1, k, workspace=ws, ids=ids, dist=dist, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        api.knn(tree, tree.points, Dd, Dq, k1, k, workspace=ws, ids=ids, dist=dist)
    ids.zero_()
    dist.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(ids, ref_ids) and torch.equal(dist, ref_dist)


def test_l1_dense_many_tiles_and_ranges():
    """Documents spanning several 4,096-document tiles with a ragged tail, and
    enough queries that each block covers a range of more than one tile: the
    posting cursors carry over tile and range boundaries.  Exact against the
    oracle on every pair of three queries and on 20,000 sampled pairs."""
    V = synth.mixture_vocab(5000, 300, 100, 0.3, 40)
    shift = synth.random_shift(300, 41)
    db = synth.zipf_docs(5000, 3 * 4096 + 123, 42, median=30)
    q = synth.zipf_docs(5000, 1000, 43, median=30)
    tree = api.Tree(torch.as_tensor(V, device="cuda"), 12, shift)
    ot = O.OracleTree(V, 12, shift)
    Dd, Dq = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    Sd, Sq = ot.embed_docs(db.row_ptr, db.word, db.weight), ot.embed_docs(q.row_ptr, q.word, q.weight)
    got = api.quadtree_l1_dense(tree, Dq, Dd).cpu().numpy()
    rng = np.random.default_rng(44)
    full_q = np.array([0, 517, q.n - 1])
    qa = np.concatenate([np.repeat(full_q, db.n), rng.integers(0, q.n, 20000)])
    qb = np.concatenate([np.tile(np.arange(db.n), len(full_q)), rng.integers(0, db.n, 20000)])
    ref = ot.quadtree_l1_batch(Sq, Sd, qa, qb, n_threads=4)
    assert np.array_equal(got[qa, qb], ref)
    ids, l1 = api.quadtree_scan(tree, Dq, Dd, 100, with_l1=True)
    for j, i in enumerate(full_q):
        row = ref[j * db.n:(j + 1) * db.n]
        want = O.topk_ids(row, 100)
        assert np.array_equal(ids[i].cpu().numpy(), want)
        assert np.array_equal(l1[i].cpu().numpy(), row[want])


def test_scan_matches_count():
    """The scan's work count: a document against itself matches each of its
    embedding entries once, and counts add over a split of the database."""
    pts, L, shift, db, q = WL["d300"]
    tree = api.Tree(torch.as_tensor(pts, device="cuda"), L, shift)
    Dq = api.Docs.from_csr(tree, q)
    for i in range(q.n):
        one = api.Docs.from_csr(tree, q.subset([i]))
        assert api.quadtree_scan_matches(tree, one, one) == one.info.n_embed
    half = db.n // 2
    D = api.Docs.from_csr(tree, db)
    D1 = api.Docs.from_csr(tree, db.subset(np.arange(half)))
    D2 = api.Docs.from_csr(tree, db.subset(np.arange(half, db.n)))
    m = api.quadtree_scan_matches(tree, Dq, D)
    assert m == api.quadtree_scan_matches(tree, Dq, D1) + api.quadtree_scan_matches(tree, Dq, D2)
    assert m > 0


@pytest.mark.parametrize("n,k,kind", [(1, 1, "rand"), (100, 37, "ties3"), (4095, 4095, "ties3"), (4096, 4096, "rand"),
                                      (4097, 4096, "ties3"), (100000, 4096, "equal"), (300003, 1000, "ties3"),
                                      (300003, 4096, "rand"), (200000, 10, "inf")])
def test_topk_f32_select_edge_cases(n, k, kind):
    """The radix select (11-bit digits, early exit once the prefix's keys fit its 4,096-entry buffer) against a
    plain stable sort: ascending values, ties to the smaller column; ragged row lengths around the buffer size,
    k at the buffer size, all-equal rows (the digits run out on the values and decide on the columns), three
    distinct values, and +inf entries."""
    rng = np.random.default_rng(n + k)
    rows = 3
    if kind == "rand":
        v = rng.random((rows, n)).astype(np.float32)
    elif kind == "ties3":
        v = rng.integers(0, 3, (rows, n)).astype(np.float32)
    elif kind == "equal":
        v = np.full((rows, n), 0.5, np.float32)
    else:
        v = rng.random((rows, n)).astype(np.float32)
        v[:, rng.integers(0, n, n // 2)] = np.inf
    ids, vals = api.topk_f32(torch.as_tensor(v, device="cuda"), k)
    ids, vals = ids.cpu().numpy(), vals.cpu().numpy()
    for r in range(rows):
        want = np.lexsort((np.arange(n), v[r]))[:k]  # by value, then by column
        assert np.array_equal(ids[r], want), r
        assert np.array_equal(vals[r], v[r][want])
