"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only: ground points, the random shift of
the quadtree (passed explicitly to both the library and the oracle), and
documents in CSR form (row_ptr int64, word int32, weight float32).  It holds
none of the Flowtree arithmetic (no quantisation, no masses, no flow).

Workloads (the paper's datasets, Sec. 5 Table "Dataset properties", are not
available; these stand in for them with the same shapes):

* tiny   -- 1,000 points uniform in [0,1]^2, documents uniform over 10..30
            distinct points.
* image  -- the 28x28 integer grid {(i, j)}, i, j = 1..28, as in the paper's
            image setting; each image is 1..3 cubic Bezier strokes rendered with
            a Gaussian brush, keeping the s ~ U{100..200} brightest pixels with
            mass proportional to intensity (mean s about 150, like MNIST's
            150.07).
* text   -- a vocabulary of unit vectors from a Gaussian-mixture of 1,000
            clusters; documents are uniform over distinct words drawn
            Zipf-distributed over word ids, with log-normal lengths.
* planted -- the random model of Sec. 4.2: points uniform on the sphere, a
            query made of points within distance eps of a planted document's
            support.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

QUANT_BITS = 40  # width of the integer shift range [0, 2^40]


@dataclass
class Docs:
    row_ptr: np.ndarray  # int64 [n + 1]
    word: np.ndarray     # int32 [nnz]
    weight: np.ndarray   # float32 [nnz]

    @property
    def n(self) -> int:
        return len(self.row_ptr) - 1

    def lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def subset(self, idx) -> "Docs":
        idx = np.asarray(idx, dtype=np.int64)
        lens = self.lengths()[idx]
        rp = np.zeros(len(idx) + 1, np.int64)
        np.cumsum(lens, out=rp[1:])
        words = [self.word[self.row_ptr[i]:self.row_ptr[i + 1]] for i in idx]
        weights = [self.weight[self.row_ptr[i]:self.row_ptr[i + 1]] for i in idx]
        w = np.concatenate(words) if words else np.zeros(0, np.int32)
        g = np.concatenate(weights) if weights else np.zeros(0, np.float32)
        return Docs(rp, w.astype(np.int32), g.astype(np.float32))


def csr_from_lists(words, weights=None) -> Docs:
    lens = np.array([len(w) for w in words], dtype=np.int64)
    rp = np.zeros(len(words) + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    w = np.concatenate([np.asarray(x, np.int32) for x in words]) if len(words) else np.zeros(0, np.int32)
    if weights is None:
        g = np.ones(len(w), np.float32)
    else:
        g = np.concatenate([np.asarray(x, np.float32) for x in weights]) if len(words) else np.zeros(0, np.float32)
    return Docs(rp, w, g)


def random_shift(d: int, seed: int) -> np.ndarray:
    """Integer shift s_c uniform in [0, 2^40] per dimension (Sec. 2 random shift)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, (1 << QUANT_BITS) + 1, size=d, dtype=np.uint64)


# ---------------------------------------------------------------------------
# tiny
# ---------------------------------------------------------------------------

def uniform_docs(n_points: int, n_docs: int, s_lo: int, s_hi: int, seed: int) -> Docs:
    rng = np.random.default_rng(seed)
    words = []
    for _ in range(n_docs):
        s = int(rng.integers(s_lo, s_hi + 1))
        words.append(rng.choice(n_points, size=s, replace=False))
    return csr_from_lists(words)


@dataclass
class Workload:
    points: np.ndarray   # float32 [n, d] ground points (the vocabulary)
    shift: np.ndarray    # uint64 [d]
    levels: int
    db: Docs
    queries: Docs


def tiny(n_points: int = 1000, n_db: int = 1000, n_queries: int = 1, levels: int = 12) -> Workload:
    pts = np.random.default_rng(0).random((n_points, 2)).astype(np.float32)
    return Workload(pts, random_shift(2, 101), levels,
                    uniform_docs(n_points, n_db, 10, 30, 102), uniform_docs(n_points, n_queries, 10, 30, 103))


# ---------------------------------------------------------------------------
# image
# ---------------------------------------------------------------------------

def grid_points(side: int = 28) -> np.ndarray:
    """Pixel (i, j), i, j = 1..side, as point id (i-1)*side + (j-1)."""
    i, j = np.meshgrid(np.arange(1, side + 1), np.arange(1, side + 1), indexing="ij")
    return np.stack([i.ravel(), j.ravel()], axis=1).astype(np.float32)


def stroke_images(n: int, seed: int, side: int = 28, samples: int = 200, sigma: float = 0.8,
                  s_lo: int = 100, s_hi: int = 200, chunk: int = 2048) -> Docs:
    """Images of 1..3 cubic Bezier strokes; keep the s brightest pixels.

    Intensity at pixel (i, j) is sum over stroke samples c of
    exp(-|(i, j) - c|^2 / (2 sigma^2)), which factorises as gx(i) * gy(j) per
    sample, so an image is a [side, S] x [S, side] product.
    """
    rng = np.random.default_rng(seed)
    n_strokes = rng.integers(1, 4, size=n)
    ctrl = rng.uniform(5.0, 24.0, size=(n, 3, 4, 2))
    keep = rng.integers(s_lo, s_hi + 1, size=n)
    t = np.linspace(0.0, 1.0, samples)
    bern = np.stack([(1 - t) ** 3, 3 * t * (1 - t) ** 2, 3 * t ** 2 * (1 - t), t ** 3], axis=1)  # [S, 4]
    import torch  # CPU tensor ops only: fast multi-threaded rendering of the strokes

    coords = torch.arange(1, side + 1, dtype=torch.float32)
    inv = -1.0 / (2 * sigma * sigma)
    words, weights = [], []
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        c = torch.from_numpy(np.einsum("sk,nmkd->nmsd", bern, ctrl[lo:hi]).astype(np.float32))  # [m, 3, S, 2]
        mask = torch.from_numpy((np.arange(3)[None, :] < n_strokes[lo:hi, None]).astype(np.float32))
        gx = torch.exp((coords - c[..., 0:1]).square() * inv) * mask[:, :, None, None]
        gy = torch.exp((coords - c[..., 1:2]).square() * inv)
        gx = gx.reshape(hi - lo, 3 * samples, side)
        gy = gy.reshape(hi - lo, 3 * samples, side)
        img = torch.bmm(gx.transpose(1, 2), gy).reshape(hi - lo, side * side).numpy()
        order = np.argsort(-img, axis=1, kind="stable")
        for r in range(hi - lo):
            idx = np.sort(order[r, : int(keep[lo + r])])
            words.append(idx.astype(np.int32))
            weights.append(img[r, idx].astype(np.float32))
    return csr_from_lists(words, weights)


def image(n_db: int = 60000, n_queries: int = 1000, levels: int = 12) -> Workload:
    return Workload(grid_points(), random_shift(2, 201), levels,
                    stroke_images(n_db, 202), stroke_images(n_queries, 203))


# ---------------------------------------------------------------------------
# text
# ---------------------------------------------------------------------------

def mixture_vocab(n_words: int, dim: int, n_clusters: int, sigma: float, seed: int) -> np.ndarray:
    """Unit vectors: normalise(centre + sigma/sqrt(dim) * N(0, I)), centres unit."""
    rng = np.random.default_rng(seed)
    centres = rng.standard_normal((n_clusters, dim))
    centres /= np.linalg.norm(centres, axis=1, keepdims=True)
    which = rng.integers(0, n_clusters, size=n_words)
    out = np.empty((n_words, dim), np.float32)
    step = 65536
    for lo in range(0, n_words, step):
        hi = min(n_words, lo + step)
        x = centres[which[lo:hi]] + (sigma / np.sqrt(dim)) * rng.standard_normal((hi - lo, dim))
        x /= np.linalg.norm(x, axis=1, keepdims=True)
        out[lo:hi] = x
    return out


def zipf_docs(n_words: int, n_docs: int, seed: int, exponent: float = 1.1, median: float = 100.0,
              log_sigma: float = 0.6, s_lo: int = 20, s_hi: int = 500, lengths=None) -> Docs:
    """Uniform documents over distinct words, word id w drawn with p ~ (w+1)^-exponent."""
    rng = np.random.default_rng(seed)
    p = np.arange(1, n_words + 1, dtype=np.float64) ** (-exponent)
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    if lengths is None:
        lengths = np.clip(np.rint(rng.lognormal(np.log(median), log_sigma, size=n_docs)), s_lo, s_hi).astype(np.int64)
    lengths = np.minimum(np.asarray(lengths, np.int64), n_words)
    words = []
    for s in lengths:
        s = int(s)
        got = np.zeros(0, np.int64)
        draw = 2 * s
        while len(got) < s:
            cand = np.searchsorted(cdf, rng.random(draw), side="right")
            cand = np.minimum(cand, n_words - 1)
            got = np.concatenate([got, cand])
            _, first = np.unique(got, return_index=True)
            got = got[np.sort(first)]
            draw *= 2
        words.append(got[:s])
    return csr_from_lists(words)


def zipf_docs_bulk(n_words: int, n_docs: int, seed: int, exponent: float = 1.05, median: float = 150.0,
                   log_sigma: float = 0.8, s_lo: int = 10, s_hi: int = 2000, device: str = "cpu",
                   chunk: int = 100000) -> Docs:
    """Vectorised variant of zipf_docs for millions of documents (torch, any device).

    Per document: s = clip(round(LogNormal(ln median, log_sigma)), s_lo, s_hi)
    target distinct words; 2 s + 64 Zipf draws are made, duplicates removed,
    and the distinct words kept in random order up to s.  A document whose
    draws hold fewer than s distinct words keeps all of them (documents near
    s_hi come out slightly shorter).
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    p = torch.arange(1, n_words + 1, dtype=torch.float64, device=device).pow(-exponent)
    cdf = torch.cumsum(p, 0)
    cdf /= cdf[-1].clone()
    lens = torch.exp(torch.randn(n_docs, generator=g, device=device, dtype=torch.float64) * log_sigma
                     + np.log(median)).round().clamp(s_lo, min(s_hi, n_words)).to(torch.int64)
    words_out, lens_out = [], []
    for lo in range(0, n_docs, chunk):
        hi = min(n_docs, lo + chunk)
        s = lens[lo:hi]
        m = 2 * s + 64
        doc = torch.repeat_interleave(torch.arange(hi - lo, device=device), m)
        u = torch.rand(doc.numel(), generator=g, device=device, dtype=torch.float64)
        w = torch.searchsorted(cdf, u, right=True).clamp(max=n_words - 1)
        key = torch.unique(doc * n_words + w)                     # distinct (doc, word), sorted
        kdoc = key // n_words
        pri = torch.rand(key.numel(), generator=g, device=device)
        order = torch.argsort(kdoc.to(torch.float64) * 2.0 + pri.to(torch.float64))  # by doc, random within
        key, kdoc = key[order], kdoc[order]
        start = torch.zeros(hi - lo + 1, dtype=torch.int64, device=device)
        start[1:] = torch.cumsum(torch.bincount(kdoc, minlength=hi - lo), 0)
        pos = torch.arange(key.numel(), device=device) - start[kdoc]
        keep = pos < s[kdoc]
        key, kdoc = key[keep], kdoc[keep]
        words_out.append((key % n_words).to(torch.int32).cpu().numpy())
        lens_out.append(torch.bincount(kdoc, minlength=hi - lo).cpu().numpy())
    ln = np.concatenate(lens_out).astype(np.int64)
    rp = np.zeros(n_docs + 1, np.int64)
    np.cumsum(ln, out=rp[1:])
    w = np.concatenate(words_out)
    return Docs(rp, w, np.ones(len(w), np.float32))


def scale(n_words: int = 400000, dim: int = 300, n_db: int = 1000000, n_queries: int = 256,
          levels: int = 12, device: str = "cpu") -> Workload:
    """The scale configuration: 400,000 x 300 vocabulary, 1,000,000 documents (log-normal
    lengths, median 150, 10..2,000 words, Zipf(1.05)), one 256-query batch."""
    vocab = mixture_vocab(n_words, dim, 1000, 0.3, 500)
    return Workload(vocab, random_shift(dim, 501), levels,
                    zipf_docs_bulk(n_words, n_db, 502, device=device),
                    zipf_docs_bulk(n_words, n_queries, 503, device=device))


def text(n_words: int = 100000, dim: int = 300, n_db: int = 100000, n_queries: int = 1000,
         levels: int = 12) -> Workload:
    vocab = mixture_vocab(n_words, dim, 1000, 0.3, 300)
    return Workload(vocab, random_shift(dim, 301), levels,
                    zipf_docs(n_words, n_db, 302), zipf_docs(n_words, n_queries, 303))


def diff_pairs(n_words: int = 30000, dim: int = 300, n_pairs: int = 4096, levels: int = 12):
    """Vocabulary + two document sets A, B of n_pairs docs each; pair i = (A_i, B_i)."""
    vocab = mixture_vocab(n_words, dim, 1000, 0.3, 400)
    rng = np.random.default_rng(402)
    la = rng.integers(20, 301, size=n_pairs)
    lb = rng.integers(20, 301, size=n_pairs)
    A = zipf_docs(n_words, n_pairs, 403, lengths=la)
    B = zipf_docs(n_words, n_pairs, 404, lengths=lb)
    return Workload(vocab, random_shift(dim, 401), levels, A, B)


# ---------------------------------------------------------------------------
# planted random model (Sec. 4.2)
# ---------------------------------------------------------------------------

def sphere_points(n: int, dim: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, dim))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x


def planted(n_points: int, dim: int, s: int, eps: float, seed: int):
    """Ground set = n_points random unit vectors plus s planted near-copies.

    Returns (points float32, planted support ids, query support ids).
    """
    rng = np.random.default_rng(seed)
    X = sphere_points(n_points, dim, seed + 1)
    support = rng.choice(n_points, size=s, replace=False)
    ys = []
    for k in support:
        v = rng.standard_normal(dim)
        v -= v.dot(X[k]) * X[k]
        v /= np.linalg.norm(v)
        r = eps * rng.random()
        y = X[k] * np.sqrt(max(0.0, 1 - r * r)) + v * r
        y /= np.linalg.norm(y)
        ys.append(y)
    pts = np.concatenate([X, np.array(ys)], axis=0).astype(np.float32)
    query = np.arange(n_points, n_points + s)
    return pts, support.astype(np.int64), query.astype(np.int64)


def sphere_cap_point(x: np.ndarray, eps: float, rng: np.random.Generator) -> np.ndarray:
    """A point uniform on {y in S^(d-1) : ||y - x|| <= eps} (x a unit vector).

    The angle t between y and x has density proportional to sin(t)^(d-2) on
    [0, t_max], t_max = 2 asin(eps / 2) (drawn by rejection against the
    uniform density); the direction orthogonal to x is uniform.
    """
    d = x.shape[0]
    t_max = 2.0 * np.arcsin(min(eps, 2.0) / 2.0)
    s_max = np.sin(min(t_max, np.pi / 2))
    while True:
        t = rng.random() * t_max
        if d <= 2 or rng.random() <= (np.sin(t) / s_max) ** (d - 2):
            break
    v = rng.standard_normal(d)
    v -= v.dot(x) * x
    v /= np.linalg.norm(v)
    y = x * np.cos(t) + v * np.sin(t)
    return y / np.linalg.norm(y)


def planted_instance(n_points: int, dim: int, s: int, eps: float, seed: int):
    """One repetition of the random model of Sec. 4.2.

    Ground set X: n_points i.i.d. uniform on S^(dim-1); a planted support of s
    distinct points of X; the query support y_1..y_s, y_k uniform among the
    points of the sphere within distance eps of x_k.  Returns (points float32
    [n_points + s][dim] = X then the y's, planted support ids, query ids).
    """
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n_points, dim))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    support = rng.choice(n_points, size=s, replace=False)
    Y = np.array([sphere_cap_point(X[k], eps, rng) for k in support])
    pts = np.concatenate([X, Y], axis=0).astype(np.float32)
    return pts, support.astype(np.int64), np.arange(n_points, n_points + s, dtype=np.int64)


def random_subset_docs(support: np.ndarray, n_points: int, n_docs: int, seed: int) -> Docs:
    """The planted support (document 0) and n_docs uniformly random s-subsets of
    the ground set (documents 1 .. n_docs), drawn from the model's dataset of all
    s-subsets; a draw equal to the planted support is redrawn.  Uniform
    weights."""
    support = np.asarray(support, dtype=np.int64)
    s = len(support)
    rng = np.random.default_rng(seed)
    planted = np.sort(support)
    out = np.empty((n_docs, s), dtype=np.int64)
    todo = np.arange(n_docs)
    while len(todo):  # redraw the rows equal to the planted support
        if n_points <= 4096:
            # small ground sets: the first s of a random permutation per row (a row of s independent draws
            # would repeat a point too often: for s = 100 of 200 points, all but about 1e-11 of the rows)
            d = np.argsort(rng.random((len(todo), n_points)), axis=1)[:, :s]
        else:
            # large ground sets: s independent draws, rows with a repeated point redrawn (at s <= 100 and
            # more than 4,096 points, at least 30% of the rows have none)
            d = rng.integers(0, n_points, (len(todo), s))
        srt = np.sort(d, axis=1)
        bad = (np.diff(srt, axis=1) == 0).any(axis=1) | (srt == planted).all(axis=1)
        out[todo[~bad]] = d[~bad]
        todo = todo[bad]
    words = np.concatenate([support[None, :], out]).astype(np.int32)
    rp = np.arange(n_docs + 2, dtype=np.int64) * s
    return Docs(rp, words.reshape(-1), np.ones(words.size, np.float32))


def single_swap_docs(support: np.ndarray, n_points: int) -> Docs:
    """The planted support (document 0) and every support that differs from it
    in one point: x_k replaced by any x' of the ground set outside the support
    (documents 1 .. s (n_points - s), in order of k, then x').  Uniform
    weights."""
    support = np.asarray(support, dtype=np.int64)
    s = len(support)
    others = np.setdiff1d(np.arange(n_points, dtype=np.int64), support)
    m = len(others)
    words = np.empty((1 + s * m, s), dtype=np.int32)
    words[0] = support
    base = np.broadcast_to(support, (m, s))
    for k in range(s):
        block = base.copy()
        block[:, k] = others
        words[1 + k * m: 1 + (k + 1) * m] = block
    n = words.shape[0]
    return Docs(np.arange(0, n * s + 1, s, dtype=np.int64), words.reshape(-1).astype(np.int32),
                np.ones(n * s, dtype=np.float32))
