"""Plant plausible mistakes in a copy of the oracle and check the pins catch them.

Each mutation edits one line of oracle/oracle.cpp in a temporary copy, builds
it, and runs tests/test_oracle_pins.py against it; the pins must fail.  This is
the evidence that the pins constrain the oracle rather than restate it.
"""
import os
import subprocess
import sys

import pytest

from oracle import build as obuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    # children visited in reverse bit-vector order (Sec. 2 child order)
    "child_order_reversed": ("for (auto& g : groups) {", "for (auto it = groups.rbegin(); it != groups.rend(); ++it) { auto& g = *it;"),
    # shift added instead of subtracted (Sec. 2 random shift)
    "shift_sign": ("uint64_t zz = q + one_b - T->shift[c];", "uint64_t zz = q + T->shift[c];"),
    # halving bit off by one level
    "halving_bit": ("const int bit = kQuantBits - k;", "const int bit = kQuantBits - k - 1;"),
    # edge weight 2^(L-k) instead of 2^(L+1-k) (Sec. 2 closed form)
    "edge_weight": ("total += (int64_t(1) << (T.levels + 1 - k)) * level_sum;", "total += (int64_t(1) << (T.levels - k)) * level_sum;"),
    # remainder units to the smallest fractional parts
    "remainder_order": ("return items[a].frac > items[b].frac;", "return items[a].frac < items[b].frac;"),
    # pricing with the squared distance (Sec. 3)
    "squared_distance": ("    return std::sqrt(s);", "    return s;"),
    # no matching at the point level (a point carried by both sides)
    "skip_point_level": ("for (int k = leaf_depth; k >= 0; --k) {", "for (int k = leaf_depth; k >= 0; --k) { if (k == leaf_depth) { for (auto& kv : level) { int v = kv.second.first; int p = T.nodes[v].parent; auto& pe = parents_hold[T.nodes[p].rank_lo]; pe.first = p; for (auto& x : kv.second.second.mu) pe.second.mu.push_back(x); for (auto& x : kv.second.second.nu) pe.second.nu.push_back(x);} level.swap(parents_hold); continue; }"),
    # leftovers not passed for the nu side
    "drop_nu_leftover": ("for (; j < nl.nu.size(); ++j) pe.second.nu.push_back(nl.nu[j]);", ";"),
    # total weight taken as the number of entries (uniform assumption)
    "uniform_total": ("total += double(w);", "total += 1.0;"),
    # adjoint: the nu endpoint moved with the same sign as the mu endpoint
    "grad_sign_nu": ("grad[size_t(q) * d + c] -= coef * diff;", "grad[size_t(q) * d + c] += coef * diff;"),
    # adjoint: the unit direction not normalised by the distance
    "grad_no_normalise": ("double coef = grad_cost[i] * (double(e.f) / double(kMassOne)) / dist;",
                          "double coef = grad_cost[i] * (double(e.f) / double(kMassOne));"),
    # exact W1: successive shortest paths without the potential update
    "mcf_no_potentials": ("if (dist[v] < INF) pot[v] += dist[v];", "if (dist[v] < INF) pot[v] += 0.0;"),
    # Mean: unweighted centroid of the support instead of the mass-weighted one
    "mean_unweighted": ("for (int64_t i = 0; i < na; ++i) ca += double(ma[i]) / double(kMassOne) * double(vocab[size_t(pa[i]) * d + t]);",
                        "for (int64_t i = 0; i < na; ++i) ca += 1.0 / double(na) * double(vocab[size_t(pa[i]) * d + t]);"),
}

EXTRA = {
    "skip_point_level": ("    std::map<int64_t, std::pair<int, NodeLists>> level;  // rank_lo -> (node, lists)",
                         "    std::map<int64_t, std::pair<int, NodeLists>> level, parents_hold;  // rank_lo -> (node, lists)"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, tmp_path):
    src = open(os.path.join(ROOT, "oracle", "oracle.cpp")).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, name
    src = src.replace(old, new)
    if name in EXTRA:
        o2, n2 = EXTRA[name]
        assert src.count(o2) == 1
        src = src.replace(o2, n2)
    cpp = tmp_path / "mut.cpp"
    cpp.write_text(src)
    so = obuild.compile_source(str(cpp), str(tmp_path / "mut.so"))
    env = dict(os.environ, FT_ORACLE_SO=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "mutation %s survived the pins:\n%s" % (name, r.stdout[-2000:])
