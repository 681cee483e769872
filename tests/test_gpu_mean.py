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
