"""Checkpoint / resume of an index: a saved tree and saved documents load back
into the same device structures, bit for bit, with the same launch
configuration, and give the same Flowtree values."""
import numpy as np
import pytest
import torch

from paper_1910_04126_gb300 import api, synth

pytestmark = pytest.mark.gpu


def test_tree_and_docs_save_load_roundtrip(tmp_path):
    V = synth.mixture_vocab(3000, 300, 40, 0.3, 700)
    db = synth.zipf_docs(3000, 200, 701, median=60)
    q = synth.zipf_docs(3000, 4, 702, median=60)
    tree = api.Tree(torch.as_tensor(V, device="cuda"), 12, None, seed=703)  # shift drawn from the seed
    tree.set_config(6, 256, 1, 0)
    D, Q = api.Docs.from_csr(tree, db), api.Docs.from_csr(tree, q)
    c1 = api.flowtree_batch(tree, tree.points, Q, D)
    tree.save(tmp_path / "tree.npz")
    D.save(tmp_path / "db.npz")
    Q.save(tmp_path / "q.npz")

    t2 = api.Tree.load(tmp_path / "tree.npz")
    D2, Q2 = api.Docs.load(t2, tmp_path / "db.npz"), api.Docs.load(t2, tmp_path / "q.npz")
    assert t2.get_config() == tree.get_config()
    for a, b in zip(tree.export(), t2.export()):
        assert np.array_equal(a, b)
    for a, b in zip(D.export(), D2.export()):
        assert np.array_equal(a, b)
    c2 = api.flowtree_batch(t2, t2.points, Q2, D2)
    assert torch.equal(c1, c2)
    assert tree.status() == 0 and t2.status() == 0
