"""The allocation-free entry point ft_flowtree_batch_static, called through the C ABI.

It serves callers that cannot allocate device memory (and so cannot hand
ft_flowtree_batch a workspace): its scratch is a fixed device array compiled
into the library.  Checked against the workspace entry point on the same
pairs, twice in a row (the shared array keeps the previous call's contents),
plus the rejection of a batch that needs more scratch than the array holds.
This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1910_04126_gb300 import _ffi, api, synth

pytestmark = pytest.mark.gpu

REL = 1e-5


def _call_static(tree, vocab, a, b, pa, pb, n_pairs, out):
    lib = _ffi.load()
    return lib.ft_flowtree_batch_static(tree.handle, C.c_void_p(vocab.data_ptr()), a.handle, b.handle,
                                        None if pa is None else C.c_void_p(pa.data_ptr()),
                                        None if pb is None else C.c_void_p(pb.data_ptr()), n_pairs,
                                        C.c_void_p(out.data_ptr()),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("shape", ["tiny2d_pairs", "grid_cross", "d300_pairs"])
def test_static_scratch_matches_workspace_entry_point(shape):
    dev = torch.device("cuda")
    if shape == "tiny2d_pairs":
        w = synth.tiny(n_points=1000, n_db=400, n_queries=1)
        pts, L, shift, A, B = w.points, w.levels, w.shift, w.db, w.db
    elif shape == "grid_cross":
        pts, L, shift = synth.grid_points(), 12, synth.random_shift(2, 7)
        A, B = synth.stroke_images(16, 8), synth.stroke_images(500, 9)
    else:
        pts = synth.mixture_vocab(5000, 300, 100, 0.3, 10)
        L, shift = 12, synth.random_shift(300, 11)
        A = B = synth.zipf_docs(5000, 300, 12, median=60, s_lo=20, s_hi=200)
    tree = api.Tree(torch.as_tensor(pts, device=dev), L, shift)
    Da, Db = api.Docs.from_csr(tree, A), api.Docs.from_csr(tree, B)
    if shape.endswith("_pairs"):
        rng = np.random.default_rng(13)
        n = 20000
        pa = torch.as_tensor(rng.integers(0, A.n, n), dtype=torch.int32, device=dev)
        pb = torch.as_tensor(rng.integers(0, B.n, n), dtype=torch.int32, device=dev)
    else:
        pa = pb = None
        n = A.n * B.n
    ref = api.flowtree_batch(tree, tree.points, Da, Db, pa, pb)
    for _ in range(2):
        out = torch.full((n,), float("nan"), dtype=torch.float32, device=dev)
        code = _call_static(tree, tree.points, Da, Db, pa, pb, n, out)
        assert code == _ffi.FT_OK, _ffi.STATUS.get(code)
        torch.cuda.synchronize()
        torch.testing.assert_close(out, ref, rtol=REL, atol=0)
    assert tree.status() == 0


def test_static_scratch_rejects_batches_beyond_its_size():
    dev = torch.device("cuda")
    w = synth.tiny(n_points=500, n_db=50, n_queries=1)
    tree = api.Tree(torch.as_tensor(w.points, device=dev), w.levels, w.shift)
    D = api.Docs.from_csr(tree, w.db)
    n = 4_000_000  # explicit pairs: order and sort buffers exceed the fixed scratch
    pa = torch.zeros(n, dtype=torch.int32, device=dev)
    out = torch.empty(n, dtype=torch.float32, device=dev)
    code = _call_static(tree, tree.points, D, D, pa, pa, n, out)
    assert code == -8  # FT_ETOOBIG, refused before any launch


def test_static_scratch_large_cross_product():
    """A cross product far beyond the explicit-pair limit (2.5 million pairs):
    it needs no pair order, so it fits the fixed scratch and must match the
    workspace entry point."""
    dev = torch.device("cuda")
    pts = np.random.default_rng(0).random((1000, 2)).astype(np.float32)
    tree = api.Tree(torch.as_tensor(pts, device=dev), 12, synth.random_shift(2, 21))
    Da = api.Docs.from_csr(tree, synth.uniform_docs(1000, 50, 10, 30, 22))
    Db = api.Docs.from_csr(tree, synth.uniform_docs(1000, 50000, 10, 30, 23))
    n = 50 * 50000
    ref = api.flowtree_batch(tree, tree.points, Da, Db)
    for _ in range(2):
        out = torch.full((n,), float("nan"), dtype=torch.float32, device=dev)
        code = _call_static(tree, tree.points, Da, Db, None, None, n, out)
        assert code == _ffi.FT_OK, _ffi.STATUS.get(code)
        torch.cuda.synchronize()
        torch.testing.assert_close(out, ref, rtol=REL, atol=0)
    assert tree.status() == 0
