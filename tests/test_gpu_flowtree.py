"""GPU parity of the quadtree, the supports and the batched Flowtree against the oracle.

Bit-exact: ranks, lcp, supports (points and integer masses), saved flows
(as sets of (item_a, item_b, flow, depth)).  Costs: FP32 within 1e-5 relative
of the FP64 oracle.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1910_04126_gb300 import api, synth

pytestmark = pytest.mark.gpu

REL = 1e-5


def build_both(points, levels, shift):
    tree = api.Tree(torch.as_tensor(points, device="cuda"), levels, shift)
    otree = O.OracleTree(points, levels, shift)
    return tree, otree


def oracle_supports(otree, docs):
    return otree.embed_docs(docs.row_ptr, docs.word, docs.weight)


def cases():
    out = {}
    w = synth.tiny(n_points=1000, n_db=300, n_queries=7)
    out["tiny2d"] = (w.points, w.levels, w.shift, w.db, w.queries)
    img_db = synth.stroke_images(150, 1)
    img_q = synth.stroke_images(5, 2)
    out["grid"] = (synth.grid_points(), 12, synth.random_shift(2, 3), img_db, img_q)
    rng = np.random.default_rng(4)
    p1 = rng.random((500, 1)).astype(np.float32)
    out["line"] = (p1, 14, synth.random_shift(1, 5), synth.uniform_docs(500, 80, 1, 40, 6),
                   synth.uniform_docs(500, 3, 1, 40, 7))
    v30 = synth.mixture_vocab(3000, 30, 50, 0.3, 8)
    out["d30"] = (v30, 12, synth.random_shift(30, 9), synth.zipf_docs(3000, 120, 10, median=40, s_lo=5, s_hi=200),
                  synth.zipf_docs(3000, 4, 11, median=40, s_lo=5, s_hi=200))
    # more than 65,536 ground points: the blocked form's per-support point ids
    wide = np.random.default_rng(16).random((70000, 2)).astype(np.float32)
    out["wide2d"] = (wide, 12, synth.random_shift(2, 17), synth.uniform_docs(70000, 120, 10, 60, 18),
                     synth.uniform_docs(70000, 4, 10, 60, 19))
    v300 = synth.mixture_vocab(4000, 300, 100, 0.3, 12)
    out["d300"] = (v300, 12, synth.random_shift(300, 13),
                   synth.zipf_docs(4000, 100, 14, median=80, s_lo=20, s_hi=400),
                   synth.zipf_docs(4000, 3, 15, median=80, s_lo=20, s_hi=400))
    return out


CASES = cases()


@pytest.mark.parametrize("name", sorted(CASES))
def test_tree_bit_exact(name):
    pts, L, shift, _, _ = CASES[name]
    tree, otree = build_both(pts, L, shift)
    rop, por, lcp, sh = tree.export()
    orop, opor = otree.ranks()
    assert np.array_equal(rop.astype(np.int64), orop)
    assert np.array_equal(por.astype(np.int64), opor)
    assert np.array_equal(lcp.astype(np.int32), otree.lcp())
    assert np.array_equal(sh, shift)
    assert tree.info.phi_log2 == otree.phi_log2


@pytest.mark.parametrize("name", sorted(CASES))
def test_supports_bit_exact(name):
    pts, L, shift, db, _ = CASES[name]
    tree, otree = build_both(pts, L, shift)
    D = api.Docs.from_csr(tree, db)
    ptr, pt, ms = D.export()
    S = oracle_supports(otree, db)
    assert np.array_equal(ptr, S.ptr)
    assert np.array_equal(pt.astype(np.int64), S.point)
    assert np.array_equal(ms.astype(np.int64), S.mass)


def _oracle_costs(otree, pts, SA, SB, pa, pb):
    return otree.flowtree_batch(pts, SA, SB, pa, pb, n_threads=4)


def algo_cases(names):
    """(case, algorithm): every case with the default (the blocked form where the pairs fit it) and the
    compacting warp form, plus the thread form where dim <= 8."""
    out = []
    for n in names:
        out += [(n, 0), (n, 1)]
        if CASES[n][0].shape[1] <= 8:
            out.append((n, 2))
    return out


@pytest.mark.parametrize("name,algo", algo_cases(sorted(CASES)))
def test_flowtree_cross_and_pairs_vs_oracle(name, algo):
    pts, L, shift, db, q = CASES[name]
    tree, otree = build_both(pts, L, shift)
    tree.set_config(0, 0, algo)
    Dd, Dq = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    Sd, Sq = oracle_supports(otree, db), oracle_supports(otree, q)
    vocab = tree.points
    # cross product queries x db
    got = api.flowtree_batch(tree, vocab, Dq, Dd).cpu().numpy().astype(np.float64)
    qa = np.repeat(np.arange(q.n), db.n)
    qb = np.tile(np.arange(db.n), q.n)
    ref = _oracle_costs(otree, pts, Sq, Sd, qa, qb)
    np.testing.assert_allclose(got, ref, rtol=REL, atol=1e-30)
    # explicit random pairs (db x db), including repeated and self pairs
    rng = np.random.default_rng(0)
    pa = rng.integers(0, db.n, 700)
    pb = rng.integers(0, db.n, 700)
    pb[:20] = pa[:20]
    got2 = api.flowtree_batch(tree, vocab, Dd, Dd, pa, pb).cpu().numpy().astype(np.float64)
    ref2 = _oracle_costs(otree, pts, Sd, Sd, pa, pb)
    np.testing.assert_allclose(got2, ref2, rtol=REL, atol=1e-30)
    assert np.all(got2[:20] == 0.0)
    assert tree.status() == 0


@pytest.mark.parametrize("name,algo", algo_cases(["tiny2d", "d300", "line", "grid", "wide2d"]))
def test_saved_flows_bit_exact(name, algo):
    pts, L, shift, db, _ = CASES[name]
    tree, otree = build_both(pts, L, shift)
    tree.set_config(0, 0, algo)
    Dd = api.Docs.from_csr(tree, db)
    Sd = oracle_supports(otree, db)
    rng = np.random.default_rng(1)
    pa = rng.integers(0, db.n, 200)
    pb = rng.integers(0, db.n, 200)
    flows = api.Flows(tree, Dd, Dd, pa, pb)
    api.flowtree_batch(tree, tree.points, Dd, Dd, flows.pair_a, flows.pair_b, flows=flows)
    got = flows.export()
    for i in range(200):
        ia, ib, f, dep = otree.flow(*Sd.doc(pa[i]), *Sd.doc(pb[i]))
        ref = sorted(zip(ia.tolist(), ib.tolist(), f.tolist(), dep.tolist()))
        g = got[i]
        mine = sorted(zip(g[0].tolist(), g[1].tolist(), g[2].tolist(), g[3].tolist()))
        assert mine == ref, i


@pytest.mark.parametrize("name", ["tiny2d", "d300"])
def test_plain_form_equals_batched(name):
    pts, L, shift, db, q = CASES[name]
    tree, _ = build_both(pts, L, shift)
    Dd, Dq = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    b = api.flowtree_plain(tree, tree.points, Dq, Dd)
    # the plain form runs the warp-per-pair code: bitwise equal to the batched warp path
    tree.set_config(0, 0, 1)
    a = api.flowtree_batch(tree, tree.points, Dq, Dd)
    assert torch.equal(a, b)
    # the default algorithm agrees within the FP32 tolerance
    tree.set_config(0, 0, 0)
    c = api.flowtree_batch(tree, tree.points, Dq, Dd)
    torch.testing.assert_close(c, b, rtol=2 * REL, atol=0)


@pytest.mark.parametrize("cap", [32, 64, 96])
def test_long_pairs_use_workspace_staging(cap):
    # The compacting warp form: pairs longer than its on-chip staging take the workspace path, bitwise equal
    # to the same form with enough staging.
    pts, L, shift, db, q = CASES["d300"]
    tree, otree = build_both(pts, L, shift)
    Dd, Dq = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    tree.set_config(0, 0, 1)
    ref = api.flowtree_batch(tree, tree.points, Dq, Dd).cpu().numpy()
    tree.set_config(2, cap, 1)
    got = api.flowtree_batch(tree, tree.points, Dq, Dd).cpu().numpy()
    assert np.array_equal(got, ref)
    Sd, Sq = oracle_supports(otree, db), oracle_supports(otree, q)
    qa = np.repeat(np.arange(q.n), db.n)
    qb = np.tile(np.arange(db.n), q.n)
    np.testing.assert_allclose(got, _oracle_costs(otree, pts, Sq, Sd, qa, qb), rtol=REL)


def test_edge_cases_dirac_single_and_identical():
    rng = np.random.default_rng(3)
    pts = rng.random((257, 3)).astype(np.float32)
    pts[5] = pts[6]  # duplicate coordinates, distinct points
    shift = synth.random_shift(3, 4)
    words = [np.array([5]), np.array([6]), np.array([0, 1, 2]), np.array([2, 1, 0]),
             np.arange(0, 257), np.array([256]), np.array([3, 3, 3])]
    weights = [np.ones(len(w), np.float32) for w in words]
    weights[3] = np.array([3.0, 2.0, 1.0], np.float32)
    docs = synth.csr_from_lists(words, weights)
    tree, otree = build_both(pts, 10, shift)
    D = api.Docs.from_csr(tree, docs)
    S = oracle_supports(otree, docs)
    n = docs.n
    pa = np.repeat(np.arange(n), n)
    pb = np.tile(np.arange(n), n)
    got = api.flowtree_batch(tree, tree.points, D, D, pa, pb).cpu().numpy().astype(np.float64)
    ref = otree.flowtree_batch(pts, S, S, pa, pb)
    np.testing.assert_allclose(got, ref, rtol=REL, atol=1e-30)
    assert got[0 * n + 1] == 0.0  # same coordinates, different points
    for i in range(n):
        assert got[i * n + i] == 0.0


def test_rejects_bad_inputs():
    pts = np.random.default_rng(0).random((10, 2)).astype(np.float32)
    tree = api.Tree(torch.as_tensor(pts, device="cuda"), 6, synth.random_shift(2, 0))
    bad = [synth.csr_from_lists([np.array([0, 1])], [np.array([1.0, -1.0], np.float32)]),
           synth.csr_from_lists([np.array([0])], [np.array([0.0], np.float32)]),
           synth.csr_from_lists([np.array([10])]),
           synth.csr_from_lists([np.array([0])], [np.array([np.nan], np.float32)])]
    for d in bad:
        with pytest.raises(api._ffi.FlowtreeError):
            api.Docs.from_csr(tree, d)
    with pytest.raises(api._ffi.FlowtreeError):
        api.Tree(torch.as_tensor(pts, device="cuda"), 0)
    with pytest.raises(api._ffi.FlowtreeError):
        api.Tree(torch.as_tensor(pts, device="cuda"), 6, np.array([2 ** 40 + 1, 0], np.uint64))
    # a pair index out of range is caught by the kernel's bounds check and
    # reported through the device status word; its cost is NaN
    good = api.Docs.from_csr(tree, synth.csr_from_lists([np.array([1, 2])]))
    out = api.flowtree_batch(tree, tree.points, good, good, np.array([0, 0]), np.array([3, 0]))
    assert tree.status() == -1
    o = out.cpu().numpy()
    assert np.isnan(o[0]) and o[1] == 0.0
    assert tree.status() == 0


@pytest.mark.parametrize("name", ["grid", "tiny2d"])
@pytest.mark.parametrize("warps", [1, 8])
def test_thread_form_block_shapes(name, warps):
    """Thread-per-pair form with one and eight warps per CTA (every lane takes
    pairs from the shared queue): costs and saved flows exact."""
    pts, L, shift, db, q = CASES[name]
    tree, otree = build_both(pts, L, shift)
    tree.set_config(warps, 0, 2)
    Dd, Dq = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    Sd, Sq = oracle_supports(otree, db), oracle_supports(otree, q)
    got = api.flowtree_batch(tree, tree.points, Dq, Dd).cpu().numpy().astype(np.float64)
    qa = np.repeat(np.arange(q.n), db.n)
    qb = np.tile(np.arange(db.n), q.n)
    np.testing.assert_allclose(got, _oracle_costs(otree, pts, Sq, Sd, qa, qb), rtol=REL, atol=1e-30)
    rng = np.random.default_rng(7)
    pa = rng.integers(0, db.n, 100)
    pb = rng.integers(0, db.n, 100)
    flows = api.Flows(tree, Dd, Dd, pa, pb)
    api.flowtree_batch(tree, tree.points, Dd, Dd, flows.pair_a, flows.pair_b, flows=flows)
    got_f = flows.export()
    for i in range(100):
        ia, ib, f, dep = otree.flow(*Sd.doc(pa[i]), *Sd.doc(pb[i]))
        ref = sorted(zip(ia.tolist(), ib.tolist(), f.tolist(), dep.tolist()))
        g = got_f[i]
        assert sorted(zip(g[0].tolist(), g[1].tolist(), g[2].tolist(), g[3].tolist())) == ref, i
    assert tree.status() == 0


@pytest.mark.parametrize("algo,stage", [(0, 0), (3, 224)])
def test_long_pairs_cta_form_bit_exact(algo, stage):
    """Supports of 2,000 points on both sides (the scale workload's longest documents) mixed with short ones: the
    pairs beyond the warp's staging go to a CTA each (the default staging, or one forced down to 224 items), and
    their saved flows are bit-exact against the oracle, their values within 1e-5."""
    rng = np.random.default_rng(30)
    pts = rng.random((6000, 2)).astype(np.float32)
    shift = synth.random_shift(2, 31)
    lens = np.array([2000, 2000, 1500, 40, 900, 20, 300, 2000, 64, 1200])
    docs = synth.csr_from_lists([rng.choice(6000, s, replace=False) for s in lens],
                                [rng.random(s).astype(np.float32) + 0.1 for s in lens])
    tree, otree = build_both(pts, 12, shift)
    tree.set_config(0, stage, algo)
    D = api.Docs.from_csr(tree, docs)
    S = oracle_supports(otree, docs)
    n = docs.n
    pa = np.repeat(np.arange(n), n)
    pb = np.tile(np.arange(n), n)
    flows = api.Flows(tree, D, D, pa, pb)
    got = api.flowtree_batch(tree, tree.points, D, D, flows.pair_a, flows.pair_b, flows=flows).cpu().numpy()
    ref = _oracle_costs(otree, pts, S, S, pa, pb)
    np.testing.assert_allclose(got.astype(np.float64), ref, rtol=REL, atol=1e-30)
    ex = flows.export()
    for i in range(len(pa)):
        ia, ib, f, dep = otree.flow(*S.doc(pa[i]), *S.doc(pb[i]))
        want = sorted(zip(ia.tolist(), ib.tolist(), f.tolist(), dep.tolist()))
        g = ex[i]
        assert sorted(zip(g[0].tolist(), g[1].tolist(), g[2].tolist(), g[3].tolist())) == want, i
    # the cross-product form of the same documents (no saved flows), and a second run gives the same bits
    c1 = api.flowtree_batch(tree, tree.points, D, D).cpu().numpy()
    c2 = api.flowtree_batch(tree, tree.points, D, D).cpu().numpy()
    np.testing.assert_allclose(c1.astype(np.float64), ref, rtol=REL, atol=1e-30)
    assert np.array_equal(c1, c2)
    assert tree.status() == 0


@pytest.mark.parametrize("name", ["d300", "d30"])
def test_deep_loads_build_same_values(name):
    """The warp form's deep-loads build (more registers per thread, the pricing rounds' row loads in flight
    together) computes the same costs and saved flows (pairs, flows, depths, distances) bit for bit as the
    occupancy build, over long pairs in the global staging too; the costs stay within 1e-5 of the oracle."""
    pts, L, shift, db, q = CASES[name]
    tree, otree = build_both(pts, L, shift)
    Dd = api.Docs.from_csr(tree, db)
    rng = np.random.default_rng(21)
    n = 300
    pa = rng.integers(0, db.n, n)
    pb = rng.integers(0, db.n, n)
    res = []
    for deep in (0, 1):
        for cap in (0, 64):  # 64: most pairs exceed the staging and run from the workspace
            tree.set_config(4, cap, 1, 0, deep)
            assert tree.get_config() == (4, cap, 1, 0, deep)
            flows = api.Flows(tree, Dd, Dd, pa, pb)
            cost = api.flowtree_batch(tree, tree.points, Dd, Dd, flows.pair_a, flows.pair_b, flows=flows)
            plain = api.flowtree_batch(tree, tree.points, Dd, Dd, flows.pair_a, flows.pair_b)
            assert tree.status() == 0
            assert torch.equal(cost, plain)
            # the saved distances through the adjoint
            g = api.flowtree_backward(tree, Dd, Dd, flows, tree.points, torch.ones(n, device="cuda"))
            res.append((cost.cpu().numpy(), flows.export(), g.cpu().numpy()))
    for cost, ex, g in res[1:]:
        assert np.array_equal(cost, res[0][0])
        assert np.array_equal(g, res[0][2])
        for i in range(n):
            assert all(np.array_equal(x, y) for x, y in zip(ex[i], res[0][1][i])), i
    Sd = oracle_supports(otree, db)
    sel = np.arange(0, n, 15)
    ref = _oracle_costs(otree, pts, Sd, Sd, pa[sel], pb[sel])
    np.testing.assert_allclose(res[-1][0][sel].astype(np.float64), ref, rtol=REL, atol=1e-30)
