"""GPU parity of the Flowtree adjoint (ft_flowtree_backward, FlowtreeFunction).

Checks: against the oracle's FP64 gradient of sum_i g_i W~_i for the frozen
flow; against FP64 central finite differences (frozen tree, and rebuilt tree
for coordinates whose cells do not move); bitwise determinism; autograd.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1910_04126_gb300 import api, synth

pytestmark = pytest.mark.gpu


def setup(n_words=3000, dim=300, n_pairs=256, seed=0, levels=12):
    V = synth.mixture_vocab(n_words, dim, 60, 0.3, 500 + seed)
    shift = synth.random_shift(dim, 501 + seed)
    rng = np.random.default_rng(502 + seed)
    A = synth.zipf_docs(n_words, n_pairs, 503 + seed, lengths=rng.integers(20, 301, n_pairs))
    B = synth.zipf_docs(n_words, n_pairs, 504 + seed, lengths=rng.integers(20, 301, n_pairs))
    tree = api.Tree(torch.as_tensor(V, device="cuda"), levels, shift)
    ot = O.OracleTree(V, levels, shift)
    return V, shift, A, B, tree, ot


def test_backward_matches_oracle_gradient():
    V, shift, A, B, tree, ot = setup()
    DA, DB = api.Docs.from_csr(tree, A), api.Docs.from_csr(tree, B)
    n = A.n
    pa = np.arange(n)
    pb = np.arange(n)
    g = np.random.default_rng(1).standard_normal(n).astype(np.float32)
    flows = api.Flows(tree, DA, DB, pa, pb)
    api.flowtree_batch(tree, tree.points, DA, DB, flows.pair_a, flows.pair_b, flows=flows)
    grad = api.flowtree_backward(tree, DA, DB, flows, tree.points, torch.as_tensor(g, device="cuda"))
    got = grad.cpu().numpy().astype(np.float64)
    SA = ot.embed_docs(A.row_ptr, A.word, A.weight)
    SB = ot.embed_docs(B.row_ptr, B.word, B.weight)
    ref = ot.grad_batch(V, SA, SB, pa, pb, g.astype(np.float64))
    scale = max(1.0, float(np.abs(ref).max()))
    assert np.abs(got - ref).max() <= 1e-4 * scale
    # rows untouched by any pair stay exactly zero
    touched = np.zeros(len(V), bool)
    touched[A.word] = True
    touched[B.word] = True
    assert np.all(got[~touched] == 0.0)


def test_backward_is_deterministic_and_accumulates():
    V, shift, A, B, tree, _ = setup(n_pairs=128, seed=3)
    DA, DB = api.Docs.from_csr(tree, A), api.Docs.from_csr(tree, B)
    flows = api.Flows(tree, DA, DB, np.arange(A.n), np.arange(A.n))
    api.flowtree_batch(tree, tree.points, DA, DB, flows.pair_a, flows.pair_b, flows=flows)
    gc = torch.ones(A.n, device="cuda")
    g1 = api.flowtree_backward(tree, DA, DB, flows, tree.points, gc)
    g2 = api.flowtree_backward(tree, DA, DB, flows, tree.points, gc)
    assert torch.equal(g1, g2)
    g3 = api.flowtree_backward(tree, DA, DB, flows, tree.points, gc, grad_vocab=g1.clone())
    assert torch.allclose(g3, 2 * g1, rtol=1e-6, atol=1e-7)


def test_autograd_function_and_finite_differences_frozen_tree():
    V, shift, A, B, tree, ot = setup(n_words=2000, n_pairs=96, seed=5)
    DA, DB = api.Docs.from_csr(tree, A), api.Docs.from_csr(tree, B)
    n = A.n
    pa = torch.arange(n, dtype=torch.int32, device="cuda")
    vocab = tree.points.clone().requires_grad_(True)
    cost = api.flowtree(vocab, tree, DA, DB, pa, pa)
    w = torch.linspace(0.5, 1.5, n, device="cuda")
    (cost * w).sum().backward()
    grad = vocab.grad.cpu().numpy().astype(np.float64)
    SA = ot.embed_docs(A.row_ptr, A.word, A.weight)
    SB = ot.embed_docs(B.row_ptr, B.word, B.weight)
    wn = w.cpu().numpy().astype(np.float64)
    idx = np.arange(n)
    rng = np.random.default_rng(7)
    used = np.unique(np.concatenate([A.word, B.word]))
    coords = [(int(rng.choice(used)), int(rng.integers(0, V.shape[1]))) for _ in range(64)]
    for p, c in coords:
        h = 1e-3
        vp, vm = V.copy(), V.copy()
        vp[p, c] += h
        vm[p, c] -= h
        fp = float((ot.flowtree_batch(vp, SA, SB, idx, idx, n_threads=4) * wn).sum())
        fm = float((ot.flowtree_batch(vm, SA, SB, idx, idx, n_threads=4) * wn).sum())
        fd = (fp - fm) / (float(vp[p, c]) - float(vm[p, c]))
        assert abs(fd - grad[p, c]) <= 1e-4 * max(1.0, abs(fd)), (p, c, fd, grad[p, c])


def test_finite_differences_with_rebuilt_tree_away_from_cell_edges():
    # Full FD: the tree is rebuilt from the perturbed points.  Coordinates are
    # used only if the perturbation leaves the rank order and every lcp
    # unchanged (the flow is then the same), i.e. away from cell boundaries.
    V, shift, A, B, tree, _ = setup(n_words=1500, n_pairs=64, seed=9)
    DA, DB = api.Docs.from_csr(tree, A), api.Docs.from_csr(tree, B)
    n = A.n
    pa = torch.arange(n, dtype=torch.int32, device="cuda")
    vocab = tree.points.clone().requires_grad_(True)
    api.flowtree(vocab, tree, DA, DB, pa, pa).sum().backward()
    grad = vocab.grad.cpu().numpy().astype(np.float64)
    rop0, por0, lcp0, _ = tree.export()
    idx = np.arange(n)
    rng = np.random.default_rng(11)
    used = np.unique(np.concatenate([A.word, B.word]))
    checked = 0
    for _ in range(40):
        p, c = int(rng.choice(used)), int(rng.integers(0, V.shape[1]))
        h = 2e-3
        vals = []
        ok = True
        for sgn in (1, -1):
            Vp = V.copy()
            Vp[p, c] += sgn * h
            ot = O.OracleTree(Vp, 12, shift)
            rop, _ = ot.ranks()
            if not (np.array_equal(rop, rop0) and np.array_equal(ot.lcp(), lcp0.astype(np.int32))):
                ok = False
                break
            SA = ot.embed_docs(A.row_ptr, A.word, A.weight)
            SB = ot.embed_docs(B.row_ptr, B.word, B.weight)
            vals.append((float(ot.flowtree_batch(Vp, SA, SB, idx, idx, n_threads=4).sum()), float(Vp[p, c])))
        if not ok:
            continue
        fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
        assert abs(fd - grad[p, c]) <= 1e-4 * max(1.0, abs(fd)), (p, c, fd, grad[p, c])
        checked += 1
        if checked >= 12:
            break
    assert checked >= 4


@pytest.mark.parametrize("dim,n_words,n_pairs", [(2, 400, 160), (7, 500, 120), (300, 800, 96), (520, 600, 48)])
def test_backward_any_dimension_and_long_runs(dim, n_words, n_pairs):
    # Dimensions that are not a multiple of 4 (scalar row loads), above one
    # column block (520 > 384), and small vocabularies, so that the frequent
    # words' contributions span many chunks of the sorted list.
    V = synth.mixture_vocab(n_words, dim, 12, 0.3, 610 + dim)
    shift = synth.random_shift(dim, 611 + dim)
    rng = np.random.default_rng(612 + dim)
    A = synth.zipf_docs(n_words, n_pairs, 613 + dim, lengths=rng.integers(20, 301, n_pairs))
    B = synth.zipf_docs(n_words, n_pairs, 614 + dim, lengths=rng.integers(20, 301, n_pairs))
    tree = api.Tree(torch.as_tensor(V, device="cuda"), 12, shift)
    ot = O.OracleTree(V, 12, shift)
    DA, DB = api.Docs.from_csr(tree, A), api.Docs.from_csr(tree, B)
    pa = np.arange(n_pairs)
    g = np.random.default_rng(615).standard_normal(n_pairs).astype(np.float32)
    flows = api.Flows(tree, DA, DB, pa, pa)
    api.flowtree_batch(tree, tree.points, DA, DB, flows.pair_a, flows.pair_b, flows=flows)
    gc = torch.as_tensor(g, device="cuda")
    grad = api.flowtree_backward(tree, DA, DB, flows, tree.points, gc)
    got = grad.cpu().numpy().astype(np.float64)
    SA = ot.embed_docs(A.row_ptr, A.word, A.weight)
    SB = ot.embed_docs(B.row_ptr, B.word, B.weight)
    ref = ot.grad_batch(V, SA, SB, pa, pa, g.astype(np.float64))
    scale = max(1.0, float(np.abs(ref).max()))
    assert np.abs(got - ref).max() <= 1e-4 * scale
    assert torch.equal(grad, api.flowtree_backward(tree, DA, DB, flows, tree.points, gc))
    touched = np.zeros(n_words, bool)
    touched[A.word] = True
    touched[B.word] = True
    assert np.all(got[~touched] == 0.0)


def test_backward_single_point_runs_over_many_chunks():
    # Every pair moves all of its mass from point 0 to point 1: the sorted
    # contributions are n_pairs entries of point 0 then n_pairs of point 1,
    # each run crossing many chunk boundaries.  Closed form:
    #   grad[0] = sum_i g_i (x0 - x1)/||x0 - x1||,  grad[1] = -grad[0].
    n_pairs = 5000
    V = np.array([[0.1, 0.2, 0.3, 0.4], [0.9, -0.5, 0.25, 0.0], [0.5, 0.5, 0.5, 0.5]], np.float32)
    tree = api.Tree(torch.as_tensor(V, device="cuda"), 12, synth.random_shift(4, 620))
    DA = api.Docs.from_csr(tree, synth.csr_from_lists([[0]] * n_pairs))
    DB = api.Docs.from_csr(tree, synth.csr_from_lists([[1]] * n_pairs))
    g = np.random.default_rng(621).standard_normal(n_pairs)
    pa = np.arange(n_pairs)
    flows = api.Flows(tree, DA, DB, pa, pa)
    api.flowtree_batch(tree, tree.points, DA, DB, flows.pair_a, flows.pair_b, flows=flows)
    grad = api.flowtree_backward(tree, DA, DB, flows, tree.points, torch.as_tensor(g, dtype=torch.float32,
                                                                                    device="cuda"))
    got = grad.cpu().numpy().astype(np.float64)
    d = V[0].astype(np.float64) - V[1].astype(np.float64)
    u = d / np.linalg.norm(d)
    gs = float(g.astype(np.float32).astype(np.float64).sum())
    assert np.allclose(got[0], gs * u, rtol=1e-5, atol=1e-4)
    assert np.allclose(got[1], -gs * u, rtol=1e-5, atol=1e-4)
    assert np.all(got[2] == 0.0)


def test_rebindable_flows_match_created_flows():
    """Flows.with_capacity + bind (no allocation, no host sync per step) give the same values and bitwise the
    same gradients as flows created for each pair list, over two binds in a row with different pair lists,
    a cross-product bind, and through autograd."""
    V, shift, A, B, tree, ot = setup(n_pairs=160, seed=7)
    DA, DB = api.Docs.from_csr(tree, A), api.Docs.from_csr(tree, B)
    rng = np.random.default_rng(8)
    F = api.Flows.with_capacity(tree, DA, DB, 600)
    for n in (600, 237):
        pa = torch.as_tensor(rng.integers(0, A.n, n), dtype=torch.int32, device="cuda")
        pb = torch.as_tensor(rng.integers(0, B.n, n), dtype=torch.int32, device="cuda")
        gc = torch.as_tensor(rng.standard_normal(n).astype(np.float32), device="cuda")
        F.bind(pa, pb)
        c1 = api.flowtree_batch(tree, tree.points, DA, DB, pa, pb, flows=F)
        g1 = api.flowtree_backward(tree, DA, DB, F, tree.points, gc)
        ref = api.Flows(tree, DA, DB, pa, pb)
        c2 = api.flowtree_batch(tree, tree.points, DA, DB, ref.pair_a, ref.pair_b, flows=ref)
        g2 = api.flowtree_backward(tree, DA, DB, ref, tree.points, gc)
        assert torch.equal(c1, c2)
        assert torch.equal(g1, g2)
        # the saved records themselves
        got, want = F.export(), ref.export()
        for i in range(n):
            assert all(np.array_equal(x, y) for x, y in zip(got[i], want[i])), i
    # a cross product bound to the same capacity
    DAs, DBs = api.Docs.from_csr(tree, A.subset(np.arange(12))), api.Docs.from_csr(tree, B.subset(np.arange(40)))
    Fx = api.Flows.with_capacity(tree, DAs, DBs, 12 * 40).bind()
    gc = torch.ones(12 * 40, device="cuda")
    c1 = api.flowtree_batch(tree, tree.points, DAs, DBs, flows=Fx)
    g1 = api.flowtree_backward(tree, DAs, DBs, Fx, tree.points, gc)
    ref = api.Flows(tree, DAs, DBs)
    c2 = api.flowtree_batch(tree, tree.points, DAs, DBs, flows=ref)
    g2 = api.flowtree_backward(tree, DAs, DBs, ref, tree.points, gc)
    assert torch.equal(c1, c2) and torch.equal(g1, g2)
    # autograd with the caller-held flows, two steps
    vocab = tree.points.clone().requires_grad_(True)
    for n in (300, 300):
        pa = torch.as_tensor(rng.integers(0, A.n, n), dtype=torch.int32, device="cuda")
        pb = torch.as_tensor(rng.integers(0, B.n, n), dtype=torch.int32, device="cuda")
        vocab.grad = None
        api.flowtree(vocab, tree, DA, DB, pa, pb, flows=F).sum().backward()
        ref = api.Flows(tree, DA, DB, pa, pb)
        api.flowtree_batch(tree, tree.points, DA, DB, ref.pair_a, ref.pair_b, flows=ref)
        want = api.flowtree_backward(tree, DA, DB, ref, tree.points, torch.ones(n, device="cuda"))
        assert torch.equal(vocab.grad, want)
    assert tree.status() == 0
