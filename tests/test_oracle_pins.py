"""Pins of the CPU oracle to facts other than itself (CPU only).

Each test checks the oracle against what the paper and the mathematics fix:
hand-worked cases (tests/golden), the geometric definition of the shifted
grid (Sec. 2), closed forms of W1 (1-D, Dirac), brute force over couplings,
the tree-optimality of the greedy flow (App. A.1) via an independent
min-cost flow, and the planted-model exactness of Sec. 4.2.
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1910_04126_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")
ONE = 1 << 24


def _supports(tree, words, weights):
    docs = synth.csr_from_lists([np.asarray(words)], [np.asarray(weights, np.float32)])
    S = tree.embed_docs(docs.row_ptr, docs.word, docs.weight)
    return S.doc(0)


def tree_dist_units(L, m):
    return 0 if m >= L + 1 else 2 * ((1 << (L + 1 - m)) - 1)


# ---------------------------------------------------------------------------
# golden hand-worked cases
# ---------------------------------------------------------------------------

with open(GOLDEN) as fh:
    _CASES = json.load(fh)["cases"]


@pytest.mark.parametrize("case", _CASES, ids=[c["name"] for c in _CASES])
def test_golden_hand_examples(case):
    pts = np.array(case["points"], np.float32)
    T = O.OracleTree(pts, case["levels"], np.array(case["shift"], np.uint64))
    rop, _ = T.ranks()
    assert rop.tolist() == case["expect_rank_of_point"]
    assert T.lcp().tolist() == case["expect_lcp"]
    pa, ma = _supports(T, case["mu"]["word"], case["mu"]["weight"])
    pb, mb = _supports(T, case["nu"]["word"], case["nu"]["weight"])
    assert ma.tolist() == case["expect_mu_mass"]
    assert mb.tolist() == case["expect_nu_mass"]
    ia, ib, f, dep = T.flow(pa, ma, pb, mb)
    got = [[int(a), int(b), int(c), int(d)] for a, b, c, d in zip(ia, ib, f, dep)]
    assert got == case["expect_flow"]
    assert T.quadtree_l1(pa, ma, pb, mb) == case["expect_l1"]
    assert T.flowtree(pts, pa, ma, pb, mb) == pytest.approx(case["expect_cost"], rel=1e-15)
    assert O.exact_w1(pts, pa, ma, pb, mb) == pytest.approx(case["expect_exact_w1"], rel=1e-12)


# ---------------------------------------------------------------------------
# tree (Sec. 2 "Generic Quadtree")
# ---------------------------------------------------------------------------

def _exact_cells(pts, shift, phi_log2, k):
    """Cell index of every point at depth k from the geometric definition.

    Root cube [sigma - Phi, sigma + Phi) per dimension after translating by the
    per-dimension minimum, sigma = s * Phi / 2^40; depth-k cells are half-open
    cubes of side 2 Phi / 2^k.  Exact rational arithmetic.
    """
    phi = Fraction(2) ** phi_log2
    lo = pts.min(axis=0)
    side = 2 * phi / (2 ** k)
    out = []
    for p in range(pts.shape[0]):
        cell = []
        for c in range(pts.shape[1]):
            sigma = Fraction(int(shift[c])) * phi / (2 ** 40)
            x = Fraction(float(pts[p, c])) - Fraction(float(lo[c]))
            x = min(x, phi)
            pos = x - (sigma - phi)
            idx = int(pos // side)
            idx = min(idx, 2 ** k - 1)
            cell.append(idx)
        out.append(tuple(cell))
    return out


@pytest.mark.parametrize("d,n,seed", [(1, 40, 1), (2, 60, 2), (3, 50, 3), (5, 30, 4)])
def test_tree_matches_geometric_cells(d, n, seed):
    rng = np.random.default_rng(seed)
    pts = (rng.random((n, d)) * 7.3 - 2.0).astype(np.float32)
    shift = synth.random_shift(d, seed + 10)
    L = 6
    T = O.OracleTree(pts, L, shift)
    rng_range = float((pts.max(axis=0).astype(np.float64) - pts.min(axis=0)).max())
    assert 2 ** T.phi_log2 >= rng_range > 2 ** (T.phi_log2 - 1)
    for k in range(0, L + 1):
        cells = _exact_cells(pts, shift, T.phi_log2, k)
        for p in range(n):
            for q in range(p + 1, n):
                same_geo = cells[p] == cells[q]
                same_tree = T.node_of(p, k) == T.node_of(q, k)
                assert same_geo == same_tree, (k, p, q)


def test_tree_nodes_are_contiguous_rank_intervals():
    w = synth.tiny(n_points=300, n_db=1)
    T = O.OracleTree(w.points, w.levels, w.shift)
    rop, por = T.ranks()
    assert sorted(rop.tolist()) == list(range(300))
    assert np.array_equal(rop[por], np.arange(300))
    for k in range(0, w.levels + 2):
        node_by_rank = [T.node_of(int(por[r]), k) for r in range(300)]
        seen = set()
        prev = None
        for v in node_by_rank:
            if v != prev:
                assert v not in seen, "node split into two rank runs"
                seen.add(v)
                prev = v


def test_tree_one_dimension_rank_is_coordinate_order():
    # In one dimension the halving order is the order of the coordinate.
    rng = np.random.default_rng(7)
    x = rng.random(200).astype(np.float32)
    T = O.OracleTree(x[:, None], 20, synth.random_shift(1, 8))
    _, por = T.ranks()
    assert np.all(np.diff(x[por].astype(np.float64)) >= 0)


def test_tree_lcp_is_adjacent_lca():
    w = synth.tiny(n_points=200, n_db=1)
    T = O.OracleTree(w.points, w.levels, w.shift)
    _, por = T.ranks()
    lcp = T.lcp()
    for r in range(199):
        p, q = int(por[r]), int(por[r + 1])
        k = max(k for k in range(w.levels + 1) if T.node_of(p, k) == T.node_of(q, k))
        assert lcp[r] == k


def test_grid_cells_at_unit_side_hold_one_pixel():
    # 28x28 grid: range 27 -> Phi = 32, depth 6 cells have side 64/64 = 1, so
    # no two grid points share a depth-6 cell whatever the shift.
    pts = synth.grid_points()
    for seed in range(3):
        T = O.OracleTree(pts, 12, synth.random_shift(2, seed))
        assert T.phi_log2 == 5
        assert T.lcp().max() <= 5


# ---------------------------------------------------------------------------
# masses (Sec. 5: distributions normalised to total mass one)
# ---------------------------------------------------------------------------

def test_masses_uniform_closed_form():
    w = synth.tiny(n_points=500, n_db=50)
    T = O.OracleTree(w.points, w.levels, w.shift)
    S = T.embed_docs(w.db.row_ptr, w.db.word, w.db.weight)
    rop, _ = T.ranks()
    for i in range(S.n_docs):
        pts, m = S.doc(i)
        s = len(pts)
        assert s == w.db.lengths()[i]
        assert np.all(np.diff(rop[pts]) > 0), "support sorted by rank"
        base, rem = divmod(ONE, s)
        expect = np.full(s, base)
        expect[:rem] += 1
        assert m.tolist() == expect.tolist()


def test_masses_proportional_and_exact_sum():
    rng = np.random.default_rng(3)
    pts = rng.random((100, 2)).astype(np.float32)
    T = O.OracleTree(pts, 8, synth.random_shift(2, 4))
    words = [rng.choice(100, size=s, replace=False) for s in (1, 2, 7, 50, 100)]
    weights = [rng.random(len(x)).astype(np.float32) + 0.01 for x in words]
    docs = synth.csr_from_lists(words, weights)
    S = T.embed_docs(docs.row_ptr, docs.word, docs.weight)
    for i in range(S.n_docs):
        p, m = S.doc(i)
        assert m.sum() == ONE
        wmap = dict(zip(words[i].tolist(), weights[i].astype(np.float64).tolist()))
        tot = sum(weights[i].astype(np.float64))
        ideal = np.array([wmap[int(x)] / tot * ONE for x in p])
        assert np.all(np.abs(m - ideal) < 1.0)


def test_masses_largest_remainder_by_fraction():
    # weights (1, 2): exact shares 5592405.33, 11184810.67 -> floors sum to
    # 2^24 - 1, and the unit goes to the larger fractional part.
    pts = np.array([[0.0], [1.0]], np.float32)
    T = O.OracleTree(pts, 3, np.zeros(1, np.uint64))
    _, m = _supports(T, [0, 1], [1.0, 2.0])
    assert m.tolist() == [5592405, 11184811]


def test_masses_merge_duplicates_drop_zeros():
    pts = np.array([[0.0], [1.0], [2.0]], np.float32)
    T = O.OracleTree(pts, 3, np.zeros(1, np.uint64))
    p, m = _supports(T, [2, 0, 2, 1], [1.0, 2.0, 1.0, 0.0])
    assert p.tolist() == [0, 2] and m.tolist() == [ONE // 2, ONE // 2]


@pytest.mark.parametrize("words,weights", [([0, 1], [1.0, -1.0]), ([0], [0.0]), ([5], [1.0]),
                                           ([0], [float("nan")]), ([0], [float("inf")])])
def test_masses_reject_bad_documents(words, weights):
    pts = np.array([[0.0], [1.0]], np.float32)
    T = O.OracleTree(pts, 3, np.zeros(1, np.uint64))
    docs = synth.csr_from_lists([np.asarray(words)], [np.asarray(weights, np.float32)])
    with pytest.raises(ValueError):
        T.embed_docs(docs.row_ptr, docs.word, docs.weight)


# ---------------------------------------------------------------------------
# exact W1 (Eq. 1) against brute force and closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("s,d,seed", [(1, 2, 0), (2, 3, 1), (4, 2, 2), (8, 5, 3)])
def test_exact_w1_brute_force_permutations(s, d, seed):
    # Uniform equal-size supports with equal masses: an optimal coupling is a
    # permutation (Birkhoff), so W1 = min over permutations of the mean distance.
    rng = np.random.default_rng(seed)
    X = rng.random((2 * s, d)).astype(np.float32)
    Dm = np.linalg.norm(X[:s, None, :].astype(np.float64) - X[None, s:, :].astype(np.float64), axis=2)
    best = min(sum(Dm[i, perm[i]] for i in range(s)) for perm in itertools.permutations(range(s))) / s
    m = np.full(s, ONE // s)
    got = O.exact_w1(X, np.arange(s), m, np.arange(s, 2 * s), m)
    assert got == pytest.approx(best, rel=1e-12)


def test_exact_w1_linear_sum_assignment():
    opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(11)
    s, d = 16, 7
    X = rng.standard_normal((2 * s, d)).astype(np.float32)
    Dm = np.linalg.norm(X[:s, None, :].astype(np.float64) - X[None, s:, :].astype(np.float64), axis=2)
    r, c = opt.linear_sum_assignment(Dm)
    m = np.full(s, ONE // s)
    assert O.exact_w1(X, np.arange(s), m, np.arange(s, 2 * s), m) == pytest.approx(Dm[r, c].sum() / s, rel=1e-12)


@pytest.mark.parametrize("seed", range(5))
def test_exact_w1_one_dimension_closed_form(seed):
    # W1 on the line = integral of |F_mu - F_nu|, with arbitrary integer masses.
    rng = np.random.default_rng(seed)
    n = 12
    x = np.sort(rng.random(n)).astype(np.float32)
    ma = rng.integers(0, 5, n) * (rng.random(n) < 0.6)
    mb = rng.integers(0, 5, n) * (rng.random(n) < 0.6)
    ma[0] += 1
    mb[-1] += 1
    tot = ma.sum() * mb.sum()
    ma, mb = ma * mb.sum(), mb * ma.sum()
    F = np.cumsum(ma - mb)[:-1].astype(np.float64)
    gaps = np.diff(x.astype(np.float64))
    expect = float(np.sum(np.abs(F) * gaps))
    ia, ib = np.nonzero(ma)[0], np.nonzero(mb)[0]
    cost = np.abs(x[ia, None].astype(np.float64) - x[None, ib].astype(np.float64))
    got = O.min_cost_flow(ma[ia], mb[ib], cost)
    assert got == pytest.approx(expect, rel=1e-12, abs=1e-12 * tot)


# ---------------------------------------------------------------------------
# greedy flow (App. A.1) and the tree closed form (Sec. 2)
# ---------------------------------------------------------------------------

def _tiny_tree_and_docs(n_points=400, n_docs=60, levels=12):
    w = synth.tiny(n_points=n_points, n_db=n_docs, levels=levels)
    T = O.OracleTree(w.points, w.levels, w.shift)
    S = T.embed_docs(w.db.row_ptr, w.db.word, w.db.weight)
    return w, T, S


def test_flow_marginals_pair_bound_and_lca_depth():
    w, T, S = _tiny_tree_and_docs()
    for i in range(0, S.n_docs - 1, 2):
        pa, ma = S.doc(i)
        pb, mb = S.doc(i + 1)
        ia, ib, f, dep = T.flow(pa, ma, pb, mb)
        assert np.all(f > 0)
        assert np.array_equal(np.bincount(ia, weights=f, minlength=len(pa)).astype(np.int64), ma)
        assert np.array_equal(np.bincount(ib, weights=f, minlength=len(pb)).astype(np.int64), mb)
        assert len(f) <= len(pa) + len(pb) - 1
        for a, b, k in zip(ia, ib, dep):
            assert k == T.lca_depth(pa[a], pb[b])
        assert len(set(zip(ia.tolist(), ib.tolist()))) == len(ia)


def test_flow_tree_cost_equals_closed_form_and_min_cost_flow():
    # The greedy flow is optimal for the tree metric (App. A.1, citing
    # Kalantari), so its tree cost equals the closed form of Sec. 2 and the
    # optimum of an independent min-cost-flow solve under the tree metric.
    w, T, S = _tiny_tree_and_docs()
    for i in range(0, 40, 2):
        pa, ma = S.doc(i)
        pb, mb = S.doc(i + 1)
        ia, ib, f, dep = T.flow(pa, ma, pb, mb)
        tree_cost = sum(int(x) * tree_dist_units(w.levels, int(k)) for x, k in zip(f, dep))
        l1 = T.quadtree_l1(pa, ma, pb, mb)
        assert tree_cost == l1
        assert T.tree_w1_mcf(pa, ma, pb, mb) == float(l1)


def test_quadtree_l1_dense_embedding_brute_force():
    # Sec. 2: L1 distance between the per-node embeddings 2^l(v) mu(v).
    w, T, S = _tiny_tree_and_docs(n_points=150, n_docs=10)
    L = w.levels
    for i in range(0, 10, 2):
        pa, ma = S.doc(i)
        pb, mb = S.doc(i + 1)
        emb = {}
        for pts, ms, sign in ((pa, ma, 1), (pb, mb, -1)):
            for p, m in zip(pts, ms):
                for k in range(1, L + 2):
                    key = (k, T.node_of(p, k))
                    emb[key] = emb.get(key, 0) + sign * (1 << (L + 1 - k)) * int(m)
        assert T.quadtree_l1(pa, ma, pb, mb) == sum(abs(v) for v in emb.values())


def test_flow_swap_symmetry_and_identity():
    w, T, S = _tiny_tree_and_docs()
    for i in range(0, 20, 2):
        pa, ma = S.doc(i)
        pb, mb = S.doc(i + 1)
        f1 = T.flow(pa, ma, pb, mb)
        f2 = T.flow(pb, mb, pa, ma)
        s1 = sorted(zip(f1[0].tolist(), f1[1].tolist(), f1[2].tolist(), f1[3].tolist()))
        s2 = sorted(zip(f2[1].tolist(), f2[0].tolist(), f2[2].tolist(), f2[3].tolist()))
        assert s1 == s2
        assert T.flowtree(w.points, pa, ma, pb, mb) == pytest.approx(T.flowtree(w.points, pb, mb, pa, ma), rel=1e-14)
        ia, ib, f, dep = T.flow(pa, ma, pa, ma)
        assert np.all(ia == ib) and np.all(dep == w.levels + 1)
        assert T.flowtree(w.points, pa, ma, pa, ma) == 0.0


def test_flowtree_bounds_exact_w1_and_dirac_case():
    # The tree flow is a feasible coupling, so its Euclidean cost is >= W1
    # (Eq. 1); against a Dirac the coupling is unique and the two coincide.
    w, T, S = _tiny_tree_and_docs()
    X = w.points.astype(np.float64)
    for i in range(0, 60, 2):
        pa, ma = S.doc(i)
        pb, mb = S.doc(i + 1)
        ft = T.flowtree(w.points, pa, ma, pb, mb)
        w1 = O.exact_w1(w.points, pa, ma, pb, mb)
        assert ft >= w1 * (1 - 1e-12)
        # also bounded by sqrt(d) * tree W1 in length units
        u = 2.0 * 2.0 ** T.phi_log2 / 2 ** (w.levels + 1)
        assert ft <= np.sqrt(2) * T.quadtree_l1(pa, ma, pb, mb) * u / ONE * (1 + 1e-12)
    pa, ma = S.doc(0)
    q = np.array([int(S.doc(1)[0][0])])
    dirac = np.array([ONE])
    expect = sum(int(m) * np.linalg.norm(X[p] - X[q[0]]) for p, m in zip(pa, ma)) / ONE
    assert T.flowtree(w.points, pa, ma, q, dirac) == pytest.approx(expect, rel=1e-13)
    assert O.exact_w1(w.points, pa, ma, q, dirac) == pytest.approx(expect, rel=1e-12)


def test_flow_pairs_lie_in_their_match_cell():
    # A pair matched in a depth-k node lies in one cell of side 2 Phi / 2^k.
    w, T, S = _tiny_tree_and_docs()
    X = w.points.astype(np.float64)
    side0 = 2.0 * 2.0 ** T.phi_log2
    for i in range(0, 30, 2):
        pa, ma = S.doc(i)
        pb, mb = S.doc(i + 1)
        ia, ib, f, dep = T.flow(pa, ma, pb, mb)
        for a, b, k in zip(ia, ib, dep):
            gap = np.abs(X[pa[a]] - X[pb[b]]).max()
            assert gap <= side0 / 2 ** min(k, w.levels) * (1 + 1e-9)


def test_planted_model_flowtree_equals_w1():
    # Sec. 4.2 / proof of the random-model theorem: when the smallest cell
    # holding x_k and y_k contains no other support point, the tree flow is
    # the planted matching and Flowtree equals W1 exactly.
    hits = 0
    for seed in range(12):
        pts, sup, qry = synth.planted(200, 6, 6, 0.02, seed)
        T = O.OracleTree(pts, 14, synth.random_shift(6, 1000 + seed))
        m = np.full(6, 0)
        docs = synth.csr_from_lists([sup, qry])
        S = T.embed_docs(docs.row_ptr, docs.word, docs.weight)
        pa, ma = S.doc(0)
        pb, mb = S.doc(1)
        allpts = set(pa.tolist()) | set(pb.tolist())
        partner = {int(s): int(q) for s, q in zip(sup, qry)}
        separated = True
        for x in pa.tolist():
            y = partner[x]
            k = T.lca_depth(x, y)
            others = [z for z in allpts if z not in (x, y) and T.node_of(z, k) == T.node_of(x, k)]
            separated &= not others
        if not separated:
            continue
        hits += 1
        ft = T.flowtree(pts, pa, ma, pb, mb)
        assert ft == pytest.approx(O.exact_w1(pts, pa, ma, pb, mb), rel=1e-12)
        del m
    assert hits >= 3


def test_gradient_dirac_closed_form_and_finite_differences():
    # Dirac-Dirac: d|x - y|/dx = (x - y)/|x - y|.
    rng = np.random.default_rng(5)
    pts = rng.standard_normal((30, 4)).astype(np.float32)
    T = O.OracleTree(pts, 10, synth.random_shift(4, 6))
    A = O.Supports(np.array([0, 1]), np.array([3]), np.array([ONE]))
    B = O.Supports(np.array([0, 1]), np.array([17]), np.array([ONE]))
    g = T.grad_batch(pts, A, B, [0], [0], [1.0])
    u = (pts[3].astype(np.float64) - pts[17]) / np.linalg.norm(pts[3].astype(np.float64) - pts[17])
    assert np.allclose(g[3], u, rtol=1e-12) and np.allclose(g[17], -u, rtol=1e-12)
    assert np.abs(np.delete(g, [3, 17], axis=0)).max() == 0.0
    # Frozen-flow central differences on a batch of random pairs.
    w, T2, S = _tiny_tree_and_docs(n_points=200, n_docs=20)
    pa_idx, pb_idx = np.arange(0, 20, 2), np.arange(1, 20, 2)
    gc = rng.random(10) + 0.5
    G = T2.grad_batch(w.points, S, S, pa_idx, pb_idx, gc)
    for p, c in [(int(S.point[0]), 0), (int(S.point[5]), 1), (int(S.point[40]), 0)]:
        h = 1e-3
        vp, vm = w.points.copy(), w.points.copy()
        vp[p, c] += h
        vm[p, c] -= h
        fp = (T2.flowtree_batch(vp, S, S, pa_idx, pb_idx) * gc).sum()
        fm = (T2.flowtree_batch(vm, S, S, pa_idx, pb_idx) * gc).sum()
        fd = (fp - fm) / (float(vp[p, c]) - float(vm[p, c]))
        assert fd == pytest.approx(G[p, c], rel=1e-4, abs=1e-6)


def test_batch_entry_points_agree_with_single_calls():
    w, T, S = _tiny_tree_and_docs(n_points=300, n_docs=30)
    pa_idx = np.arange(0, 30)
    pb_idx = (np.arange(0, 30) * 7) % 30
    c1 = T.flowtree_batch(w.points, S, S, pa_idx, pb_idx, n_threads=1)
    c4 = T.flowtree_batch(w.points, S, S, pa_idx, pb_idx, n_threads=4)
    l1 = T.quadtree_l1_batch(S, S, pa_idx, pb_idx, n_threads=3)
    assert np.array_equal(c1, c4)
    for i in range(30):
        pa, ma = S.doc(pa_idx[i])
        pb, mb = S.doc(pb_idx[i])
        assert c1[i] == T.flowtree(w.points, pa, ma, pb, mb)
        assert l1[i] == T.quadtree_l1(pa, ma, pb, mb)


def test_topk_ties_by_smaller_id():
    v = np.array([3.0, 1.0, 2.0, 1.0, 0.5])
    assert O.topk_ids(v, 3).tolist() == [4, 1, 3]


# ---------------------------------------------------------------------------
# the Mean method (Sec. 5): centroid distance, a lower bound on W1
# ---------------------------------------------------------------------------

def test_mean_distance_pins():
    rng = np.random.default_rng(31)
    X = rng.random((40, 3)).astype(np.float32)
    # Dirac against Dirac: the distance of the two points
    d = O.mean_distance(X, [3], [ONE], [17], [ONE])
    assert d == pytest.approx(np.linalg.norm(X[3].astype(np.float64) - X[17]), rel=1e-12)
    # a distribution against itself: 0
    m = np.array([ONE // 4, ONE // 4, ONE // 2])
    assert O.mean_distance(X, [1, 2, 5], m, [1, 2, 5], m) == 0.0
    # the centroid of two equal masses is the midpoint: distance to the midpoint's Dirac-like pair
    half = [ONE // 2, ONE // 2]
    mid = (X[4].astype(np.float64) + X[9]) / 2
    assert O.mean_distance(X, [4, 9], half, [11], [ONE]) == pytest.approx(np.linalg.norm(mid - X[11]), rel=1e-12)
    # Jensen: never above exact W1, on random distributions
    for t in range(20):
        na, nb = rng.integers(1, 7), rng.integers(1, 7)
        pa = rng.choice(40, na, replace=False)
        pb = rng.choice(40, nb, replace=False)
        ma = rng.integers(1, 100, na)
        mb = rng.integers(1, 100, nb)
        ma = ma * ONE // ma.sum()
        ma[0] += ONE - ma.sum()
        mb = mb * ONE // mb.sum()
        mb[0] += ONE - mb.sum()
        assert O.mean_distance(X, pa, ma, pb, mb) <= O.exact_w1(X, pa, ma, pb, mb) * (1 + 1e-12) + 1e-15
