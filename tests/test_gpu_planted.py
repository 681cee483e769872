"""GPU parity of the random-model experiment (Sec. 4.2 model): the scores the
experiment ranks come from the library and agree with the oracle, and the
success decisions follow from them."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1910_04126_gb300 import api, planted, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rep", range(3))
def test_planted_scores_match_oracle(rep):
    n, d, s, eps = 60, 6, 4, 0.25
    pts, support, query = synth.planted_instance(n, d, s, eps, 50 + rep)
    shift = synth.random_shift(d, 60 + rep)
    cand = synth.single_swap_docs(support, n)
    qdoc = synth.csr_from_lists([query])
    tree = api.Tree(torch.as_tensor(pts, device="cuda"), 12, shift)
    D, Q = api.Docs.from_csr(tree, cand), api.Docs.from_csr(tree, qdoc)
    l1 = api.quadtree_l1_dense(tree, Q, D)[0].cpu().numpy()
    cost = api.flowtree_batch(tree, tree.points, Q, D).cpu().numpy().astype(np.float64)
    ot = O.OracleTree(pts, 12, shift)
    Sd, Sq = ot.embed_docs(cand.row_ptr, cand.word, cand.weight), ot.embed_docs(qdoc.row_ptr, qdoc.word, qdoc.weight)
    qa, qb = np.zeros(cand.n, np.int64), np.arange(cand.n)
    l1_ref = ot.quadtree_l1_batch(Sq, Sd, qa, qb)
    assert np.array_equal(l1, l1_ref)
    ref = ot.flowtree_batch(pts, Sq, Sd, qa, qb)
    np.testing.assert_allclose(cost, ref, rtol=1e-5, atol=1e-30)
    # the decisions the experiment takes, wherever the FP64 margin is clear
    if abs(ref[0] - ref[1:].min()) > 1e-4 * ref[0]:
        assert (cost[0] < cost[1:].min()) == (ref[0] < ref[1:].min())
    assert (l1[0] < l1[1:].min()) == (l1_ref[0] < l1_ref[1:].min())
    assert tree.status() == 0


def test_planted_run_small():
    out = planted.run([40, 80], dim=6, s=4, eps=0.25, reps=5, seed=1)
    assert [r["n_points"] for r in out["results"]] == [40, 80]
    for r in out["results"]:
        assert 0.0 <= r["quadtree_success"] <= 1.0 and 0.0 <= r["flowtree_success"] <= 1.0
        assert r["pairs_scored"] == 5 * r["candidates_per_query"]
