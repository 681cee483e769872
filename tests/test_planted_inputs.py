"""Inputs of the random-model experiment (Sec. 4.2): the spherical-cap sampler
and the single-swap candidate set."""
import pytest
import numpy as np
from scipy import integrate, stats

from paper_1910_04126_gb300 import synth


def test_sphere_cap_point_is_uniform_on_the_cap():
    d, eps = 10, 0.25
    rng = np.random.default_rng(0)
    x = rng.standard_normal(d)
    x /= np.linalg.norm(x)
    ys = np.array([synth.sphere_cap_point(x, eps, rng) for _ in range(3000)])
    assert np.allclose(np.linalg.norm(ys, axis=1), 1.0, atol=1e-12)
    assert np.all(np.linalg.norm(ys - x, axis=1) <= eps + 1e-12)
    # the angle to x has density proportional to sin(t)^(d-2) on [0, t_max]
    t = np.arccos(np.clip(ys @ x, -1.0, 1.0))
    t_max = 2 * np.arcsin(eps / 2)
    z = integrate.quad(lambda u: np.sin(u) ** (d - 2), 0, t_max)[0]
    cdf = lambda v: np.array([integrate.quad(lambda u: np.sin(u) ** (d - 2), 0, min(a, t_max))[0] / z
                              for a in np.atleast_1d(v)])
    assert stats.kstest(t, cdf).pvalue > 1e-3
    # the direction orthogonal to x is uniform: its mean is near 0
    v = ys - np.outer(ys @ x, x)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    assert np.linalg.norm(v.mean(axis=0)) < 0.1


def test_planted_instance_layout():
    pts, support, query = synth.planted_instance(500, 8, 6, 0.3, 3)
    assert pts.shape == (506, 8) and pts.dtype == np.float32
    assert len(set(support.tolist())) == 6 and support.max() < 500
    assert np.array_equal(query, np.arange(500, 506))
    assert np.all(np.linalg.norm(pts[query] - pts[support], axis=1) <= 0.3 + 1e-6)


def test_single_swap_docs():
    support = np.array([5, 2, 9])
    D = synth.single_swap_docs(support, 12)
    assert D.n == 1 + 3 * 9
    docs = [tuple(D.word[D.row_ptr[i]:D.row_ptr[i + 1]].tolist()) for i in range(D.n)]
    assert docs[0] == (5, 2, 9)
    assert len(set(frozenset(d) for d in docs)) == D.n  # all distinct supports
    for d in docs[1:]:
        assert len(set(d)) == 3 and len(set(d) & {5, 2, 9}) == 2
    assert np.all(D.weight == 1.0)


def test_random_subset_competitors():
    support = np.array([3, 17, 5, 40])
    d = synth.random_subset_docs(support, 50, 300, seed=1)
    assert d.n == 301
    assert np.array_equal(d.word[:4], support)
    planted = np.sort(support)
    for i in range(1, d.n):
        w = d.word[d.row_ptr[i]:d.row_ptr[i + 1]]
        assert len(w) == 4 and len(set(w.tolist())) == 4 and w.min() >= 0 and w.max() < 50
        assert not np.array_equal(np.sort(w), planted)


@pytest.mark.parametrize("n_points,s", [(200, 100), (20, 10), (5000, 100)])
def test_random_subset_competitors_dense_supports(n_points, s):
    """Supports of half the ground set (s = 100 of N = 200, the model's smallest N at s = 100): every row holds s
    distinct points of the ground set and differs from the planted support; the draw finishes (s independent
    draws per row would almost never be distinct here)."""
    support = np.arange(s) * (n_points // s)
    d = synth.random_subset_docs(support, n_points, 2000, seed=3)
    assert d.n == 2001
    rows = d.word.reshape(d.n, s)
    assert np.array_equal(rows[0], support)
    planted = np.sort(support)
    srt = np.sort(rows[1:], axis=1)
    assert np.all(np.diff(srt, axis=1) > 0) and srt.min() >= 0 and srt.max() < n_points
    assert not np.any(np.all(srt == planted, axis=1))
    # every point of the ground set is drawn about equally often (uniform s-subsets)
    counts = np.bincount(rows[1:].reshape(-1), minlength=n_points)
    expect = 2000 * s / n_points
    tol = 6.0 * np.sqrt(expect)  # six standard deviations of a count
    assert counts.min() > expect - tol and counts.max() < expect + tol
