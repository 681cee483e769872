"""GPU parity of the mean-distance prefilter (the Mean method of Sec. 5)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1910_04126_gb300 import api, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["tiny2d", "d300"])
def test_mean_scan_vs_oracle(name):
    if name == "tiny2d":
        w = synth.tiny(n_points=1000, n_db=500, n_queries=6)
        pts, L, shift, db, q = w.points, w.levels, w.shift, w.db, w.queries
    else:
        pts = synth.mixture_vocab(4000, 300, 80, 0.3, 90)
        L, shift = 12, synth.random_shift(300, 91)
        db = synth.zipf_docs(4000, 700, 92, median=40, s_lo=5, s_hi=150)
        q = synth.zipf_docs(4000, 6, 93, median=40, s_lo=5, s_hi=150)
    tree = api.Tree(torch.as_tensor(pts, device="cuda"), L, shift)
    ot = O.OracleTree(pts, L, shift)
    Dd, Dq = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    Sd, Sq = ot.embed_docs(db.row_ptr, db.word, db.weight), ot.embed_docs(q.row_ptr, q.word, q.weight)
    k1 = 50
    ids, dist = api.mean_scan(tree, tree.points, Dq, Dd, k1)
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy().astype(np.float64)
    for i in range(q.n):
        ref = np.array([O.mean_distance(pts, *Sq.doc(i), *Sd.doc(j)) for j in range(db.n)])
        # FP32 centroids and the expansion |c_q|^2 + |c_d|^2 - 2 c_q.c_d: the
        # error sits in the squared distance, a few FP32 ulps of the norms
        tol2 = 1e-5 * max(1.0, float(ref.max()) ** 2)
        assert np.all(np.abs(dist[i] ** 2 - ref[ids[i]] ** 2) <= tol2)
        want = O.topk_ids(ref, k1)
        # the same set up to near-ties with the k1-th value
        kth = np.sort(ref)[k1 - 1]
        for a in set(ids[i].tolist()) ^ set(want.tolist()):
            assert abs(ref[a] ** 2 - kth ** 2) <= 2 * tol2
        assert np.all(np.diff(dist[i]) >= -1e-6)


@pytest.mark.parametrize("dim,n_db,n_q", [(300, 3001, 130), (30, 2500, 257), (2, 1300, 129)])
def test_mean_scan_many_tiles_ragged(dim, n_db, n_q):
    """Distances over several 128 x 128 tiles with ragged edges (and a dimension that is not a multiple of 4),
    against FP64 centroid distances; the selected ids are the k1 smallest up to near-ties, in order."""
    pts = synth.mixture_vocab(2000, dim, 40, 0.3, 95) if dim > 2 else np.random.default_rng(95).random((2000, 2)).astype(np.float32)
    db = synth.zipf_docs(2000, n_db, 96, median=30, s_lo=5, s_hi=100)
    q = synth.zipf_docs(2000, n_q, 97, median=30, s_lo=5, s_hi=100)
    tree = api.Tree(torch.as_tensor(pts, device="cuda"), 12, synth.random_shift(dim, 98))
    Dd, Dq = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    k1 = 100
    ids, dist = api.mean_scan(tree, tree.points, Dq, Dd, k1)
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy().astype(np.float64)

    def centroids(D):
        c = np.zeros((D.n, dim))
        for i in range(D.n):
            w = D.weight[D.row_ptr[i]:D.row_ptr[i + 1]].astype(np.float64)
            c[i] = (w / w.sum()) @ pts[D.word[D.row_ptr[i]:D.row_ptr[i + 1]]].astype(np.float64)
        return c

    cd, cq = centroids(db), centroids(q)
    for i in range(0, n_q, 16):
        ref = np.sqrt(((cd - cq[i]) ** 2).sum(1))
        tol2 = 1e-5 * max(1.0, float(ref.max()) ** 2)
        assert np.all(np.abs(dist[i] ** 2 - ref[ids[i]] ** 2) <= tol2)
        kth = np.sort(ref)[k1 - 1]
        want = O.topk_ids(ref, k1)
        for a in set(ids[i].tolist()) ^ set(want.tolist()):
            assert abs(ref[a] ** 2 - kth ** 2) <= 2 * tol2
        assert np.all(np.diff(dist[i]) >= 0)


def test_mean_scan_ties_go_to_the_smaller_id():
    """Identical documents have identical distances: the select keeps the smaller ids, including when the
    tied documents at the threshold outnumber the candidate buffer (4,096)."""
    pts = synth.mixture_vocab(500, 30, 20, 0.3, 99)
    base = synth.zipf_docs(500, 3, 100, median=20, s_lo=5, s_hi=40)
    db = base.subset(np.array([0] * 5000 + [1] * 20 + [2] * 3000))  # 5,000 copies of doc 0 first
    q = base.subset(np.array([1, 0, 2]))
    tree = api.Tree(torch.as_tensor(pts, device="cuda"), 12, synth.random_shift(30, 101))
    Dd, Dq = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    k1 = 50
    ids, dist = api.mean_scan(tree, tree.points, Dq, Dd, k1)
    ids = ids.cpu().numpy()
    # query 0 (= doc 1): its 20 copies (ids 5000..5019) are at distance 0, then the smallest ids of the
    # nearer of the other two groups
    assert np.array_equal(ids[0][:20], np.arange(5000, 5020))
    # query 1 (= doc 0): 5,000 tied copies at distance 0, more than the buffer: the 50 smallest ids
    assert np.array_equal(ids[1], np.arange(50))
    # query 2 (= doc 2): copies at ids 5020..8019
    assert np.array_equal(ids[2], np.arange(5020, 5070))
    assert np.all(dist.cpu().numpy()[1] == 0.0)
