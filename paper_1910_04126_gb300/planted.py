"""The random-model experiment (model of Sec. 4.2, experiment of Sec. 5.1,
figure "Results on random data") on the GPU path.

Model: a ground set X of N points i.i.d. uniform on the unit sphere
S^(d-1); documents are uniform distributions over s-subsets of X; a query is
planted on a document's support x_1..x_s by drawing y_k uniformly among the
points of the sphere within distance eps of x_k.  The theorem of Sec. 4.2:
Quadtree recovers the planted document with a probability that decays as N
grows, Flowtree with a probability independent of N.

The dataset of the model holds all C(N, s) subsets.  The competitors that
decide the theorem's events are the subsets one point away from the planted
support (x_k replaced by another point of X): Quadtree fails exactly when a
cell holding x_k and y_k holds another point, i.e. when such a swap ties or
beats the planted document.  The experiment therefore ranks the planted
document against all s (N - s) single swaps; "success" = the planted
document's score is strictly the smallest (a tie is a failure: the method
cannot tell the documents apart); the rate at which it is among the
minimisers is reported too.  For Flowtree this is a necessary condition for
success over the whole dataset.  A second reading ranks the planted document
against a uniform sample of the dataset (random s-subsets of X) instead.

Every repetition draws a new instance and a new random shift of the tree;
both scores come from the library (ft_quadtree_l1_dense, ft_flowtree_batch).
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import api, synth


def run(n_points_list, dim: int = 10, s: int = 10, eps: float = 0.25, reps: int = 100, seed: int = 0,
        levels: int = 12, device: str = "cuda", competitors: str = "swaps", n_random: int = 2000) -> dict:
    """Success fractions of Quadtree and Flowtree for every N in n_points_list.

    competitors: "swaps" -- every single swap of the planted support (the
    documents that decide the theorem's events); "random" -- n_random
    uniformly random s-subsets, a sample of the model's dataset."""
    dev = torch.device(device)
    out = []
    for n in n_points_list:
        ok_qt = ok_ft = tie_qt = tie_ft = 0
        pairs = 0
        gpu_s = 0.0
        for r in range(reps):
            inst_seed = 1_000_003 * (seed + 1) + 7919 * int(n) + r
            pts, support, query = synth.planted_instance(int(n), dim, s, eps, inst_seed)
            shift = synth.random_shift(dim, inst_seed + 17)
            if competitors == "swaps":
                cand = synth.single_swap_docs(support, int(n))
            else:
                cand = synth.random_subset_docs(support, int(n), n_random, inst_seed + 29)
            qdoc = synth.csr_from_lists([query])
            tree = api.Tree(torch.as_tensor(pts, device=dev), levels, shift)
            D, Q = api.Docs.from_csr(tree, cand), api.Docs.from_csr(tree, qdoc)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            l1 = api.quadtree_l1_dense(tree, Q, D)[0]
            cost = api.flowtree_batch(tree, tree.points, Q, D)
            torch.cuda.synchronize(dev)
            gpu_s += time.perf_counter() - t0
            l1, cost = l1.cpu().numpy(), cost.cpu().numpy()
            ok_qt += int(l1[0] < l1[1:].min())
            ok_ft += int(cost[0] < cost[1:].min())
            tie_qt += int(l1[0] <= l1[1:].min())
            tie_ft += int(cost[0] <= cost[1:].min())
            pairs += cand.n
            status = tree.status()
            if status != 0:
                raise RuntimeError("device status %d in the planted experiment (N=%d, rep %d)" % (status, n, r))
        out.append({"n_points": int(n), "candidates_per_query": cand.n,
                    "quadtree_success": ok_qt / reps, "flowtree_success": ok_ft / reps,
                    "quadtree_among_minimizers": tie_qt / reps, "flowtree_among_minimizers": tie_ft / reps,
                    "pairs_scored": pairs, "gpu_seconds": gpu_s})
    return {"dim": dim, "s": s, "eps": eps, "reps": reps, "levels": levels, "competitors": competitors,
            "results": out}


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, nargs="+", default=[100, 1000, 10000])
    ap.add_argument("--dim", type=int, default=10)
    ap.add_argument("--s", type=int, default=10)
    ap.add_argument("--eps", type=float, default=0.25)
    ap.add_argument("--reps", type=int, default=100)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--competitors", choices=["swaps", "random"], default="swaps")
    a = ap.parse_args()
    print(json.dumps(run(a.n, a.dim, a.s, a.eps, a.reps, a.seed, competitors=a.competitors)))
