"""GPU parity of the exact-W1 re-ranking stage (Eq. 1 by min-cost flow) and of
the three-stage pipeline quadtree -> Flowtree -> exact W1 (Sec. 5.2)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1910_04126_gb300 import api, synth

pytestmark = pytest.mark.gpu
REL = 1e-5


def setup(pts, L, shift, db, q):
    tree = api.Tree(torch.as_tensor(pts, device="cuda"), L, shift)
    ot = O.OracleTree(pts, L, shift)
    Dd, Dq = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    Sd, Sq = ot.embed_docs(db.row_ptr, db.word, db.weight), ot.embed_docs(q.row_ptr, q.word, q.weight)
    return tree, ot, Dd, Dq, Sd, Sq


def cases():
    w = synth.tiny(n_points=1000, n_db=200, n_queries=5)
    yield "tiny2d", w.points, w.levels, w.shift, w.db, w.queries, 60
    V = synth.mixture_vocab(3000, 300, 60, 0.3, 70)
    yield "d300", V, 12, synth.random_shift(300, 71), synth.zipf_docs(3000, 200, 72, median=40, s_lo=5, s_hi=150), \
        synth.zipf_docs(3000, 5, 73, median=40, s_lo=5, s_hi=150), 40
    yield "grid", synth.grid_points(), 12, synth.random_shift(2, 74), synth.stroke_images(40, 75), \
        synth.stroke_images(3, 76), 12


CASES = {c[0]: c[1:] for c in cases()}


@pytest.mark.parametrize("name", sorted(CASES))
def test_exact_w1_vs_oracle(name):
    pts, L, shift, db, q, n_pairs = CASES[name]
    tree, ot, Dd, Dq, Sd, Sq = setup(pts, L, shift, db, q)
    rng = np.random.default_rng(1)
    pa = rng.integers(0, q.n, n_pairs)
    pb = rng.integers(0, db.n, n_pairs)
    got = api.exact_w1(tree, tree.points, Dq, Dd, pa, pb).cpu().numpy().astype(np.float64)
    ref = np.array([O.exact_w1(pts, *Sq.doc(a), *Sd.doc(b)) for a, b in zip(pa, pb)])
    np.testing.assert_allclose(got, ref, rtol=REL, atol=1e-6)
    # Flowtree prices a feasible flow, so it is never below W1
    ft = api.flowtree_batch(tree, tree.points, Dq, Dd, torch.as_tensor(pa, dtype=torch.int32, device="cuda"),
                            torch.as_tensor(pb, dtype=torch.int32, device="cuda")).cpu().numpy()
    assert np.all(ft >= got * (1 - 2 * REL) - 1e-6)
    assert tree.status() == 0


def test_exact_w1_edge_cases():
    rng = np.random.default_rng(5)
    pts = rng.random((50, 3)).astype(np.float32)
    tree = api.Tree(torch.as_tensor(pts, device="cuda"), 8, synth.random_shift(3, 6))
    words = [np.array([3]), np.array([7]), np.array([3, 7, 11, 20]), np.array([3, 7, 11, 20]), np.array([9, 30])]
    weights = [np.ones(1, np.float32), np.ones(1, np.float32), np.array([1, 2, 3, 4], np.float32),
               np.array([1, 2, 3, 4], np.float32), np.array([5, 1], np.float32)]
    docs = synth.csr_from_lists(words, weights)
    D = api.Docs.from_csr(tree, docs)
    pa = np.array([0, 2, 0, 4, 2, 1])
    pb = np.array([1, 3, 2, 0, 4, 1])
    got = api.exact_w1(tree, tree.points, D, D, pa, pb).cpu().numpy().astype(np.float64)
    ot = O.OracleTree(pts, 8, synth.random_shift(3, 6))
    S = ot.embed_docs(docs.row_ptr, docs.word, docs.weight)
    ref = np.array([O.exact_w1(pts, *S.doc(a), *S.doc(b)) for a, b in zip(pa, pb)])
    np.testing.assert_allclose(got, ref, rtol=REL, atol=1e-6)
    assert got[5] == 0.0 and got[1] == 0.0                      # identical distributions
    assert abs(got[0] - np.linalg.norm(pts[3] - pts[7])) < 1e-6  # Dirac vs Dirac
    # Dirac vs any distribution: the unique coupling, sum_j nu_j ||x - y_j||
    p3, m3 = S.doc(2)
    dirac = float(np.sum(m3 / 2.0**24 * np.linalg.norm(pts[p3].astype(np.float64) - pts[3], axis=1)))
    assert abs(got[2] - dirac) <= 1e-5 * dirac


def test_knn_exact_pipeline_vs_oracle():
    pts, L, shift, db, q, _ = CASES["d300"]
    tree, ot, Dd, Dq, Sd, Sq = setup(pts, L, shift, db, q)
    k1, k2, k = 60, 20, 5
    ids, dist = api.knn_exact(tree, tree.points, Dd, Dq, k1, k2, k)
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy().astype(np.float64)
    qa = np.repeat(np.arange(q.n), db.n)
    qb = np.tile(np.arange(db.n), q.n)
    l1 = ot.quadtree_l1_batch(Sq, Sd, qa, qb, n_threads=4).reshape(q.n, db.n)
    for i in range(q.n):
        cand = O.topk_ids(l1[i], k1)
        fcost = ot.flowtree_batch(pts, Sq, Sd, np.full(k1, i), cand, n_threads=2)
        order = np.lexsort((cand, fcost))
        surv = cand[order[:k2]]
        w = np.array([O.exact_w1(pts, *Sq.doc(i), *Sd.doc(int(j))) for j in surv])
        o2 = np.lexsort((surv, w))
        np.testing.assert_allclose(dist[i], w[o2[:k]], rtol=REL, atol=1e-6)
        wmap = dict(zip(surv.tolist(), w.tolist()))
        for a, b in zip(ids[i], surv[o2[:k]]):
            if a != b:  # only between near-ties (FP32 against FP64)
                assert abs(wmap[int(a)] - wmap[int(b)]) <= 2e-5 * max(wmap[int(b)], 1e-30)


def test_knn_exact_graph_capture_replay():
    pts, L, shift, db, q, _ = CASES["d300"]
    tree = api.Tree(torch.as_tensor(pts, device="cuda"), L, shift)
    Dd, Dq = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    k1, k2, k = 32, 10, 4
    ws = torch.empty(api.knn_exact_workspace_size(tree, Dd, Dq, k1, k2, k), dtype=torch.uint8, device="cuda")
    ids = torch.empty((q.n, k), dtype=torch.int32, device="cuda")
    dist = torch.empty((q.n, k), dtype=torch.float32, device="cuda")
    ref_ids, ref_dist = api.knn_exact(tree, tree.points, Dd, Dq, k1, k2, k)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        api.knn_exact(tree, tree.points, Dd, Dq, k1, k2, k, workspace=ws, ids=ids, dist=dist, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        api.knn_exact(tree, tree.points, Dd, Dq, k1, k2, k, workspace=ws, ids=ids, dist=dist)
    ids.zero_()
    dist.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(ids, ref_ids) and torch.equal(dist, ref_dist)


def test_exact_and_pipeline_reject_bad_inputs():
    pts, L, shift, db, q, _ = CASES["tiny2d"]
    tree = api.Tree(torch.as_tensor(pts, device="cuda"), L, shift)
    Dd, Dq = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    # a pair index out of range: NaN for that pair, FT_EINVAL in the status word, the others exact
    pa = np.array([0, 1, q.n + 5])
    pb = np.array([3, 4, 0])
    got = api.exact_w1(tree, tree.points, Dq, Dd, pa, pb).cpu().numpy()
    assert np.isnan(got[2]) and np.all(np.isfinite(got[:2]))
    assert tree.status() == -1
    assert tree.status() == 0  # read and cleared
    # stage sizes out of order, and documents of another tree
    with pytest.raises(api._ffi.FlowtreeError):
        api.knn_exact(tree, tree.points, Dd, Dq, 20, 30, 5)
    with pytest.raises(api._ffi.FlowtreeError):
        api.knn_exact(tree, tree.points, Dd, Dq, 20, 10, 11)
    other = api.Tree(torch.as_tensor(pts, device="cuda"), L, shift)
    Do = api.Docs.from_csr(other, db)
    with pytest.raises(api._ffi.FlowtreeError):
        api.exact_w1(tree, tree.points, Dq, Do, [0], [0])
    with pytest.raises(api._ffi.FlowtreeError):
        api.mean_scan(tree, tree.points, Dq, Dd, db.n + 1)
