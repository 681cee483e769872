// Flowtree CPU oracle.  TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, obviously-correct FP64 restatement of what the Flowtree
// estimate (Backurs, Dong, Indyk, Razenshteyn, Wagner, arXiv 1910.04126)
// computes.  It is written from the paper's text, shares no code, header,
// table or constant generator with the CUDA library, and is only ever loaded
// by the test-suite, by the smoke check and by the benchmark's CPU-baseline
// leg.  Nothing in the product path may call it.
//
// Every function cites the passage it follows:
//   Sec. 2 "Generic Quadtree"              random shift, recursive halving, levels
//   Sec. 2 "Wasserstein-1 on Quadtree"     closed form sum_v 2^l(v) |mu(v)-nu(v)|
//   Sec. 3 "Flowtree"                      tree-optimal flow, priced in the ground metric
//   App. A.1 "Flowtree Computation"        bottom-up greedy matching per node
//   Eq. (1)                                 the W1 definition (exact W1 for small cases)
//   Sec. 5 "Datasets"                      documents as uniform distributions, images
//                                           as intensity-proportional distributions
//
// Readings of the paper where it is silent or ambiguous (all are restated in
// the project's design notes):
//   * fixed depth: L subdivided levels (depths 1..L) below the root (depth 0),
//     plus an implicit point level L+1 (the paper's singleton leaves);
//   * the ground metric for pricing is Euclidean (l2);
//   * inside a node, leftover demands are matched in north-west-corner order:
//     mu-items in rank order against nu-items in rank order (the paper says
//     "arbitrarily"); equal heads advance both pointers;
//   * a point carried by both distributions is matched at the point level;
//   * masses are 24-bit fixed point: integers summing to exactly 2^24;
//   * coordinates are quantised once to B = 40 bits; cells are half-open.
//
// Parity pins: every function here is checked by tests/test_oracle_pins.py
// against closed forms, brute force and invariants; none is "parity unpinned".

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <map>
#include <thread>
#include <vector>

namespace {

constexpr int kQuantBits = 40;                 // B: coordinate quantisation bits
constexpr int64_t kMassOne = int64_t(1) << 24; // total mass of every distribution

struct Node {
    int depth = 0;
    int parent = -1;
    std::vector<int> children;
    int64_t rank_lo = 0, rank_hi = 0;  // the node's points are ranks [lo, hi)
};

struct Tree {
    int64_t n = 0;
    int d = 0;
    int levels = 0;                // L
    std::vector<float> lo;         // per-dimension minimum
    int phi_log2 = 0;              // Phi = 2^phi_log2
    std::vector<uint64_t> shift;   // integer shift s_c in [0, 2^B]
    std::vector<uint64_t> z;       // [n][d] shifted integer coordinates
    std::vector<Node> nodes;       // nodes[0] = root (depth 0)
    std::vector<int64_t> rank_of_point, point_of_rank;
    std::vector<int> anc;          // [n][L+2]: node containing the point at depth k
    int anc_at(int64_t p, int k) const { return anc[size_t(p) * (levels + 2) + k]; }
};

// ---------------------------------------------------------------------------
// Sec. 2 "Generic Quadtree": quantise the points, shift the enclosing cube,
// halve it recursively.  Only non-empty cells are created.
// ---------------------------------------------------------------------------

// Phi = smallest power of two >= the largest coordinate range (Phi = 1 when
// all points coincide).  The paper assumes coordinates in [0, Phi]; we
// translate by the per-dimension minimum, which changes no distance.
int phi_log2_for(double range) {
    if (!(range > 0.0)) return 0;
    int ex = 0;
    double m = std::frexp(range, &ex);  // range = m * 2^ex, m in [0.5, 1)
    return (m == 0.5) ? ex - 1 : ex;
}

void build_rec(Tree& T, int node, const std::vector<int64_t>& pts, int k, int64_t& next_rank) {
    T.nodes[node].rank_lo = next_rank;
    if (k == T.levels) {
        // Below the deepest cell every point is its own leaf (point level L+1),
        // ordered by point id.
        for (int64_t p : pts) {
            Node leaf;
            leaf.depth = T.levels + 1;
            leaf.parent = node;
            leaf.rank_lo = next_rank;
            leaf.rank_hi = next_rank + 1;
            T.nodes.push_back(leaf);
            int leaf_id = int(T.nodes.size()) - 1;
            T.nodes[node].children.push_back(leaf_id);
            T.rank_of_point[p] = next_rank;
            T.point_of_rank[next_rank] = p;
            ++next_rank;
        }
    } else {
        // Halve the cell along every dimension: the child cell at depth k+1
        // is z >> (B - k); relative to the parent it is selected by bit
        // (B - k) of each coordinate.  Children are ordered by that d-bit
        // vector compared dimension 0 first.
        const int bit = kQuantBits - k;
        std::map<std::vector<uint8_t>, std::vector<int64_t>> groups;
        std::vector<uint8_t> key(T.d);
        for (int64_t p : pts) {
            for (int c = 0; c < T.d; ++c) key[c] = uint8_t((T.z[size_t(p) * T.d + c] >> bit) & 1u);
            groups[key].push_back(p);
        }
        for (auto& g : groups) {
            Node child;
            child.depth = k + 1;
            child.parent = node;
            T.nodes.push_back(child);
            int child_id = int(T.nodes.size()) - 1;
            T.nodes[node].children.push_back(child_id);
            build_rec(T, child_id, g.second, k + 1, next_rank);
        }
    }
    T.nodes[node].rank_hi = next_rank;
}

Tree* build_tree(const float* pts, int64_t n, int d, int levels, const uint64_t* shift) {
    Tree* T = new Tree;
    T->n = n;
    T->d = d;
    T->levels = levels;
    T->lo.assign(d, 0.0f);
    double range = 0.0;
    for (int c = 0; c < d; ++c) {
        float mn = pts[c], mx = pts[c];
        for (int64_t p = 1; p < n; ++p) {
            mn = std::min(mn, pts[size_t(p) * d + c]);
            mx = std::max(mx, pts[size_t(p) * d + c]);
        }
        T->lo[c] = mn;
        range = std::max(range, double(mx) - double(mn));
    }
    T->phi_log2 = phi_log2_for(range);
    T->shift.assign(shift, shift + d);
    // q = floor((x - lo) * 2^B / Phi), capped at 2^B; z = q + 2^B - s, capped at
    // 2^(B+1) - 1.  The root cube [sigma - Phi, sigma + Phi) maps to z in
    // [0, 2^(B+1)), with sigma = s * Phi / 2^B uniform in [0, Phi].
    const double scale = std::ldexp(1.0, kQuantBits - T->phi_log2);
    const uint64_t one_b = uint64_t(1) << kQuantBits;
    T->z.resize(size_t(n) * d);
    for (int64_t p = 0; p < n; ++p)
        for (int c = 0; c < d; ++c) {
            double diff = double(pts[size_t(p) * d + c]) - double(T->lo[c]);
            double scaled = diff * scale;
            uint64_t q = uint64_t(std::floor(scaled));
            if (q > one_b) q = one_b;
            uint64_t zz = q + one_b - T->shift[c];
            if (zz > 2 * one_b - 1) zz = 2 * one_b - 1;
            T->z[size_t(p) * d + c] = zz;
        }
    T->rank_of_point.assign(n, -1);
    T->point_of_rank.assign(n, -1);
    T->nodes.clear();
    T->nodes.push_back(Node{});  // root, depth 0
    std::vector<int64_t> all(n);
    for (int64_t p = 0; p < n; ++p) all[p] = p;
    int64_t next_rank = 0;
    build_rec(*T, 0, all, 0, next_rank);
    // Ancestor table: walk up from each point's leaf.
    T->anc.assign(size_t(n) * (levels + 2), -1);
    for (size_t v = 0; v < T->nodes.size(); ++v) {
        if (T->nodes[v].depth != levels + 1) continue;
        int64_t p = T->point_of_rank[T->nodes[v].rank_lo];
        int u = int(v);
        while (u >= 0) {
            T->anc[size_t(p) * (levels + 2) + T->nodes[u].depth] = u;
            u = T->nodes[u].parent;
        }
    }
    return T;
}

// Depth of the lowest common ancestor of two points (L+1 when p == q).
int lca_depth(const Tree& T, int64_t p, int64_t q) {
    int k = T.levels + 1;
    while (T.anc_at(p, k) != T.anc_at(q, k)) --k;
    return k;
}

// ---------------------------------------------------------------------------
// Sec. 5 "Datasets": a document is a distribution over its terms (uniform
// weights for text, intensities for images), normalised to total mass one.
// Reading: masses are integers summing to exactly 2^24 (largest remainder).
// ---------------------------------------------------------------------------

struct Support {
    std::vector<int64_t> point;  // ground-point ids, sorted by quadtree rank
    std::vector<int64_t> mass;   // integer masses, sum 2^24
};

// Returns 0 on success, -1 on invalid input (negative / non-finite weight,
// word out of range, or no positive weight).
int make_support(const Tree& T, const int32_t* word, const float* weight, int64_t len, Support* out) {
    double total = 0.0;
    std::map<int64_t, double> merged;  // point -> summed weight (CSR order)
    for (int64_t i = 0; i < len; ++i) {
        float w = weight[i];
        int64_t p = word[i];
        if (p < 0 || p >= T.n) return -1;
        if (!std::isfinite(w) || w < 0.0f) return -1;
        if (w == 0.0f) continue;
        total += double(w);
        merged[p] += double(w);
    }
    if (merged.empty()) return -1;
    struct Item { int64_t rank, point; double x; int64_t m; double frac; };
    std::vector<Item> items;
    for (auto& kv : merged) {
        Item it;
        it.point = kv.first;
        it.rank = T.rank_of_point[kv.first];
        it.x = (kv.second / total) * double(kMassOne);
        it.m = int64_t(std::floor(it.x));
        it.frac = it.x - double(it.m);
        items.push_back(it);
    }
    std::sort(items.begin(), items.end(), [](const Item& a, const Item& b) { return a.rank < b.rank; });
    int64_t assigned = 0;
    for (auto& it : items) assigned += it.m;
    int64_t remainder = kMassOne - assigned;
    // The remaining units go one each to the largest fractional parts; ties
    // go to the smaller rank.
    std::vector<size_t> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return items[a].frac > items[b].frac; });
    for (int64_t r = 0; r < remainder; ++r) items[order[size_t(r)]].m += 1;
    out->point.clear();
    out->mass.clear();
    for (auto& it : items)
        if (it.m > 0) {
            out->point.push_back(it.point);
            out->mass.push_back(it.m);
        }
    return 0;
}

// ---------------------------------------------------------------------------
// Sec. 2 "Wasserstein-1 on Quadtree": tree W1 = sum over nodes of
// (edge weight above the node) * |mu(v) - nu(v)|.  Length unit
// u = 2 Phi / 2^(L+1); the edge above a depth-k node weighs 2^(L+1-k) u.
// Result in units of u * 2^-24 (exact integer).
// ---------------------------------------------------------------------------

int64_t quadtree_l1(const Tree& T, const Support& a, const Support& b) {
    int64_t total = 0;
    for (int k = 1; k <= T.levels + 1; ++k) {
        std::map<int, int64_t> diff;
        for (size_t i = 0; i < a.point.size(); ++i) diff[T.anc_at(a.point[i], k)] += a.mass[i];
        for (size_t j = 0; j < b.point.size(); ++j) diff[T.anc_at(b.point[j], k)] -= b.mass[j];
        int64_t level_sum = 0;
        for (auto& kv : diff) level_sum += std::llabs(kv.second);
        total += (int64_t(1) << (T.levels + 1 - k)) * level_sum;
    }
    return total;
}

// Tree distance between points matched inside a depth-m node, in units of u:
// twice the sum of the edge weights from depth m+1 down to the point level.
int64_t tree_distance_units(int levels, int m) {
    if (m >= levels + 1) return 0;
    return 2 * ((int64_t(1) << (levels + 1 - m)) - 1);
}

// ---------------------------------------------------------------------------
// App. A.1 "Flowtree Computation": bottom-up greedy flow.  Nodes are visited
// from the point level up to the root; each node matches the unmatched mu- and
// nu-demands collected from its children and hands the rest to its parent.
// ---------------------------------------------------------------------------

struct FlowPair { int64_t ia, ib, f; int depth; };

struct Demand { int64_t item; int64_t res; };
struct NodeLists { std::vector<Demand> mu, nu; };

void greedy_flow(const Tree& T, const Support& a, const Support& b, std::vector<FlowPair>* out) {
    out->clear();
    // Start at the point level: one node per support point, keyed by rank so
    // that iterating the map visits nodes left to right.
    std::map<int64_t, std::pair<int, NodeLists>> level;  // rank_lo -> (node, lists)
    const int leaf_depth = T.levels + 1;
    for (size_t i = 0; i < a.point.size(); ++i) {
        int v = T.anc_at(a.point[i], leaf_depth);
        auto& e = level[T.nodes[v].rank_lo];
        e.first = v;
        e.second.mu.push_back({int64_t(i), a.mass[i]});
    }
    for (size_t j = 0; j < b.point.size(); ++j) {
        int v = T.anc_at(b.point[j], leaf_depth);
        auto& e = level[T.nodes[v].rank_lo];
        e.first = v;
        e.second.nu.push_back({int64_t(j), b.mass[j]});
    }
    for (int k = leaf_depth; k >= 0; --k) {
        std::map<int64_t, std::pair<int, NodeLists>> parents;
        for (auto& kv : level) {
            int v = kv.second.first;
            NodeLists& nl = kv.second.second;
            // Match: while both sides have demand, move eta = min of the two
            // heads (north-west-corner order).
            size_t i = 0, j = 0;
            while (i < nl.mu.size() && j < nl.nu.size()) {
                int64_t eta = std::min(nl.mu[i].res, nl.nu[j].res);
                out->push_back({nl.mu[i].item, nl.nu[j].item, eta, k});
                nl.mu[i].res -= eta;
                nl.nu[j].res -= eta;
                if (nl.mu[i].res == 0) ++i;
                if (nl.nu[j].res == 0) ++j;
            }
            // At most one side is left; pass it to the parent.
            if (k == 0) continue;
            int p = T.nodes[v].parent;
            auto& pe = parents[T.nodes[p].rank_lo];
            pe.first = p;
            for (; i < nl.mu.size(); ++i) pe.second.mu.push_back(nl.mu[i]);
            for (; j < nl.nu.size(); ++j) pe.second.nu.push_back(nl.nu[j]);
        }
        level.swap(parents);
    }
}

// Sec. 3: the Flowtree estimate prices the tree flow in the ground metric.
double euclid(const float* vocab, int d, int64_t p, int64_t q) {
    double s = 0.0;
    for (int c = 0; c < d; ++c) {
        double t = double(vocab[size_t(p) * d + c]) - double(vocab[size_t(q) * d + c]);
        s += t * t;
    }
    return std::sqrt(s);
}

double price_flow(const float* vocab, int d, const Support& a, const Support& b, const std::vector<FlowPair>& fl) {
    double cost = 0.0;
    for (const FlowPair& e : fl)
        cost += (double(e.f) / double(kMassOne)) * euclid(vocab, d, a.point[size_t(e.ia)], b.point[size_t(e.ib)]);
    return cost;
}

// ---------------------------------------------------------------------------
// Eq. (1): exact W1 by successive shortest paths (Dijkstra with potentials)
// on the complete bipartite graph between the two supports.  Integer
// supplies, FP64 costs.  Small inputs only.
// ---------------------------------------------------------------------------

double min_cost_flow(const std::vector<int64_t>& supply, const std::vector<int64_t>& demand,
                     const std::vector<double>& cost /* [na][nb] */) {
    const int na = int(supply.size()), nb = int(demand.size());
    const int V = na + nb + 2, S = na + nb, Tn = na + nb + 1;
    struct Edge { int to; int64_t cap; double cost; int rev; };
    std::vector<std::vector<Edge>> g(V);
    auto add = [&](int u, int v, int64_t cap, double c) {
        g[u].push_back({v, cap, c, int(g[v].size())});
        g[v].push_back({u, 0, -c, int(g[u].size()) - 1});
    };
    const int64_t inf_cap = std::numeric_limits<int64_t>::max() / 4;
    for (int i = 0; i < na; ++i) add(S, i, supply[i], 0.0);
    for (int j = 0; j < nb; ++j) add(na + j, Tn, demand[j], 0.0);
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j) add(i, na + j, inf_cap, cost[size_t(i) * nb + j]);
    int64_t need = 0;
    for (int64_t s : supply) need += s;
    std::vector<double> pot(V, 0.0), dist(V);
    std::vector<int> prev_node(V), prev_edge(V);
    std::vector<char> done(V);
    double total = 0.0;
    const double INF = std::numeric_limits<double>::infinity();
    while (need > 0) {
        std::fill(dist.begin(), dist.end(), INF);
        std::fill(done.begin(), done.end(), 0);
        dist[S] = 0.0;
        for (int it = 0; it < V; ++it) {  // dense Dijkstra
            int u = -1;
            for (int v = 0; v < V; ++v)
                if (!done[v] && dist[v] < INF && (u < 0 || dist[v] < dist[u])) u = v;
            if (u < 0) break;
            done[u] = 1;
            for (size_t e = 0; e < g[u].size(); ++e) {
                const Edge& ed = g[u][e];
                if (ed.cap <= 0) continue;
                double rc = ed.cost + pot[u] - pot[ed.to];
                if (rc < 0.0) rc = 0.0;  // rounding only; reduced costs are >= 0
                if (dist[u] + rc < dist[ed.to]) {
                    dist[ed.to] = dist[u] + rc;
                    prev_node[ed.to] = u;
                    prev_edge[ed.to] = int(e);
                }
            }
        }
        if (!(dist[Tn] < INF)) return std::numeric_limits<double>::quiet_NaN();
        for (int v = 0; v < V; ++v)
            if (dist[v] < INF) pot[v] += dist[v];
        int64_t push = need;
        for (int v = Tn; v != S; v = prev_node[v]) push = std::min(push, g[prev_node[v]][prev_edge[v]].cap);
        for (int v = Tn; v != S; v = prev_node[v]) {
            Edge& ed = g[prev_node[v]][prev_edge[v]];
            ed.cap -= push;
            g[v][ed.rev].cap += push;
            total += double(push) * ed.cost;
        }
        need -= push;
    }
    return total;
}

Tree* as_tree(void* h) { return static_cast<Tree*>(h); }

Support support_from(const int64_t* point, const int64_t* mass, int64_t len) {
    Support s;
    s.point.assign(point, point + len);
    s.mass.assign(mass, mass + len);
    return s;
}

}  // namespace

extern "C" {

// Build the oracle's explicit quadtree (Sec. 2).  `shift` holds d integers
// in [0, 2^40].  Returns an opaque handle, or NULL on bad arguments.
void* oracle_tree_build(const float* pts, int64_t n, int32_t d, int32_t levels, const uint64_t* shift) {
    if (n <= 0 || d <= 0 || levels < 1 || levels > kQuantBits) return nullptr;
    for (int c = 0; c < d; ++c)
        if (shift[c] > (uint64_t(1) << kQuantBits)) return nullptr;
    return build_tree(pts, n, d, levels, shift);
}

void oracle_tree_free(void* h) { delete as_tree(h); }

// lo[d] (float), phi_log2, number of nodes (all depths, including point leaves).
void oracle_tree_params(void* h, float* lo, int32_t* phi_log2, int64_t* n_nodes) {
    Tree* T = as_tree(h);
    for (int c = 0; c < T->d; ++c) lo[c] = T->lo[c];
    *phi_log2 = T->phi_log2;
    *n_nodes = int64_t(T->nodes.size());
}

void oracle_tree_z(void* h, uint64_t* z) {
    Tree* T = as_tree(h);
    std::memcpy(z, T->z.data(), T->z.size() * sizeof(uint64_t));
}

void oracle_tree_ranks(void* h, int64_t* rank_of_point, int64_t* point_of_rank) {
    Tree* T = as_tree(h);
    for (int64_t p = 0; p < T->n; ++p) {
        rank_of_point[p] = T->rank_of_point[p];
        point_of_rank[p] = T->point_of_rank[p];
    }
}

// lcp[r] = depth of the lowest common ancestor of the points at ranks r, r+1.
void oracle_tree_lcp(void* h, int32_t* lcp) {
    Tree* T = as_tree(h);
    for (int64_t r = 0; r + 1 < T->n; ++r) lcp[r] = lca_depth(*T, T->point_of_rank[r], T->point_of_rank[r + 1]);
}

int32_t oracle_lca_depth(void* h, int64_t p, int64_t q) { return lca_depth(*as_tree(h), p, q); }

// Node (global id) containing point p at depth k in 0..L+1.
int32_t oracle_node_of(void* h, int64_t p, int32_t k) { return as_tree(h)->anc_at(p, k); }

// Document masses (Sec. 5): per doc, the support sorted by rank with integer
// masses summing to 2^24.  Output arrays must hold nnz entries; sup_ptr has
// n_docs+1 entries.  Returns 0, or -1 - (index of the first bad document).
int64_t oracle_embed_docs(void* h, const int64_t* row_ptr, const int32_t* word, const float* weight, int64_t n_docs,
                          int64_t* sup_ptr, int64_t* sup_point, int64_t* sup_mass) {
    Tree* T = as_tree(h);
    sup_ptr[0] = 0;
    for (int64_t i = 0; i < n_docs; ++i) {
        Support s;
        int64_t len = row_ptr[i + 1] - row_ptr[i];
        if (make_support(*T, word + row_ptr[i], weight + row_ptr[i], len, &s) != 0) return -1 - i;
        int64_t base = sup_ptr[i];
        for (size_t j = 0; j < s.point.size(); ++j) {
            sup_point[base + int64_t(j)] = s.point[j];
            sup_mass[base + int64_t(j)] = s.mass[j];
        }
        sup_ptr[i + 1] = base + int64_t(s.point.size());
    }
    return 0;
}

// Quadtree W1 (Sec. 2 closed form), units of u * 2^-24.
int64_t oracle_quadtree_l1(void* h, const int64_t* pa, const int64_t* ma, int64_t na,
                           const int64_t* pb, const int64_t* mb, int64_t nb) {
    return quadtree_l1(*as_tree(h), support_from(pa, ma, na), support_from(pb, mb, nb));
}

// Tree distance in units of u between two points.
int64_t oracle_tree_distance(void* h, int64_t p, int64_t q) {
    Tree* T = as_tree(h);
    return tree_distance_units(T->levels, lca_depth(*T, p, q));
}

// Greedy tree flow (App. A.1).  Writes up to `cap` pairs (index into a,
// index into b, flow, depth) and returns the number of pairs (or -1 if cap
// is too small).
int64_t oracle_flow(void* h, const int64_t* pa, const int64_t* ma, int64_t na, const int64_t* pb,
                    const int64_t* mb, int64_t nb, int64_t* out_ia, int64_t* out_ib, int64_t* out_f,
                    int32_t* out_depth, int64_t cap) {
    std::vector<FlowPair> fl;
    greedy_flow(*as_tree(h), support_from(pa, ma, na), support_from(pb, mb, nb), &fl);
    if (int64_t(fl.size()) > cap) return -1;
    for (size_t i = 0; i < fl.size(); ++i) {
        out_ia[i] = fl[i].ia;
        out_ib[i] = fl[i].ib;
        out_f[i] = fl[i].f;
        out_depth[i] = fl[i].depth;
    }
    return int64_t(fl.size());
}

// Flowtree estimate (Sec. 3) for one pair, FP64.
double oracle_flowtree(void* h, const float* vocab, const int64_t* pa, const int64_t* ma, int64_t na,
                       const int64_t* pb, const int64_t* mb, int64_t nb) {
    Support a = support_from(pa, ma, na), b = support_from(pb, mb, nb);
    std::vector<FlowPair> fl;
    greedy_flow(*as_tree(h), a, b, &fl);
    return price_flow(vocab, as_tree(h)->d, a, b, fl);
}

// Flowtree estimate for many pairs of documents given as supports in CSR
// form (sup_ptr / sup_point / sup_mass, as written by oracle_embed_docs).
// Pair i is (doc pair_a[i] of set A, doc pair_b[i] of set B).  Runs on
// `n_threads` host threads (plain partition of the pairs).
void oracle_flowtree_batch(void* h, const float* vocab, const int64_t* a_ptr, const int64_t* a_point,
                           const int64_t* a_mass, const int64_t* b_ptr, const int64_t* b_point,
                           const int64_t* b_mass, const int64_t* pair_a, const int64_t* pair_b, int64_t n_pairs,
                           int32_t n_threads, double* out_cost) {
    Tree* T = as_tree(h);
    auto work = [&](int64_t lo, int64_t hi) {
        std::vector<FlowPair> fl;
        for (int64_t i = lo; i < hi; ++i) {
            int64_t da = pair_a[i], db = pair_b[i];
            Support a = support_from(a_point + a_ptr[da], a_mass + a_ptr[da], a_ptr[da + 1] - a_ptr[da]);
            Support b = support_from(b_point + b_ptr[db], b_mass + b_ptr[db], b_ptr[db + 1] - b_ptr[db]);
            greedy_flow(*T, a, b, &fl);
            out_cost[i] = price_flow(vocab, T->d, a, b, fl);
        }
    };
    if (n_threads <= 1) {
        work(0, n_pairs);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < n_threads; ++t) {
        int64_t lo = n_pairs * t / n_threads, hi = n_pairs * (t + 1) / n_threads;
        th.emplace_back(work, lo, hi);
    }
    for (auto& x : th) x.join();
}

// Quadtree W1 for many pairs (same layout as oracle_flowtree_batch).
void oracle_quadtree_l1_batch(void* h, const int64_t* a_ptr, const int64_t* a_point, const int64_t* a_mass,
                              const int64_t* b_ptr, const int64_t* b_point, const int64_t* b_mass,
                              const int64_t* pair_a, const int64_t* pair_b, int64_t n_pairs, int32_t n_threads,
                              int64_t* out_l1) {
    Tree* T = as_tree(h);
    auto work = [&](int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) {
            int64_t da = pair_a[i], db = pair_b[i];
            Support a = support_from(a_point + a_ptr[da], a_mass + a_ptr[da], a_ptr[da + 1] - a_ptr[da]);
            Support b = support_from(b_point + b_ptr[db], b_mass + b_ptr[db], b_ptr[db + 1] - b_ptr[db]);
            out_l1[i] = quadtree_l1(*T, a, b);
        }
    };
    if (n_threads <= 1) {
        work(0, n_pairs);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < n_threads; ++t) th.emplace_back(work, n_pairs * t / n_threads, n_pairs * (t + 1) / n_threads);
    for (auto& x : th) x.join();
}

// Gradient of sum_i g_i * Flowtree_i with respect to the vocabulary rows,
// for the frozen tree flow:  d/dx_a of f * |x_a - y_b| = f (x_a - y_b)/|x_a - y_b|,
// and the opposite sign for y_b; zero when the two points coincide.  FP64,
// accumulated into grad[n][d] (caller zeroes it).
void oracle_flowtree_grad_batch(void* h, const float* vocab, const int64_t* a_ptr, const int64_t* a_point,
                                const int64_t* a_mass, const int64_t* b_ptr, const int64_t* b_point,
                                const int64_t* b_mass, const int64_t* pair_a, const int64_t* pair_b,
                                const double* grad_cost, int64_t n_pairs, double* grad) {
    Tree* T = as_tree(h);
    const int d = T->d;
    std::vector<FlowPair> fl;
    for (int64_t i = 0; i < n_pairs; ++i) {
        int64_t da = pair_a[i], db = pair_b[i];
        Support a = support_from(a_point + a_ptr[da], a_mass + a_ptr[da], a_ptr[da + 1] - a_ptr[da]);
        Support b = support_from(b_point + b_ptr[db], b_mass + b_ptr[db], b_ptr[db + 1] - b_ptr[db]);
        greedy_flow(*T, a, b, &fl);
        for (const FlowPair& e : fl) {
            int64_t p = a.point[size_t(e.ia)], q = b.point[size_t(e.ib)];
            double dist = euclid(vocab, d, p, q);
            if (!(dist > 0.0)) continue;
            double coef = grad_cost[i] * (double(e.f) / double(kMassOne)) / dist;
            for (int c = 0; c < d; ++c) {
                double diff = double(vocab[size_t(p) * d + c]) - double(vocab[size_t(q) * d + c]);
                grad[size_t(p) * d + c] += coef * diff;
                grad[size_t(q) * d + c] -= coef * diff;
            }
        }
    }
}

// Exact W1 (Eq. 1) between two supports under the Euclidean ground metric,
// by min-cost flow.  Masses are the integer masses; the result is divided
// by 2^24.
double oracle_exact_w1(const float* vocab, int32_t d, const int64_t* pa, const int64_t* ma, int64_t na,
                       const int64_t* pb, const int64_t* mb, int64_t nb) {
    std::vector<int64_t> sup(ma, ma + na), dem(mb, mb + nb);
    std::vector<double> cost(size_t(na) * nb);
    for (int64_t i = 0; i < na; ++i)
        for (int64_t j = 0; j < nb; ++j) cost[size_t(i) * nb + j] = euclid(vocab, d, pa[i], pb[j]);
    return min_cost_flow(sup, dem, cost) / double(kMassOne);
}

// The "Mean" method of Sec. 5: the Euclidean distance between the two
// mass-weighted centroids sum_i (m_i / 2^24) x_i, in FP64.
double oracle_mean_distance(const float* vocab, int32_t d, const int64_t* pa, const int64_t* ma, int64_t na,
                            const int64_t* pb, const int64_t* mb, int64_t nb) {
    double sq = 0.0;
    for (int32_t t = 0; t < d; ++t) {
        double ca = 0.0, cb = 0.0;
        for (int64_t i = 0; i < na; ++i) ca += double(ma[i]) / double(kMassOne) * double(vocab[size_t(pa[i]) * d + t]);
        for (int64_t j = 0; j < nb; ++j) cb += double(mb[j]) / double(kMassOne) * double(vocab[size_t(pb[j]) * d + t]);
        sq += (ca - cb) * (ca - cb);
    }
    return std::sqrt(sq);
}

// Exact W1 under the quadtree metric t (units of u * 2^-24), by the same
// min-cost flow solver: an independent check of the closed form.
double oracle_tree_w1_mcf(void* h, const int64_t* pa, const int64_t* ma, int64_t na, const int64_t* pb,
                          const int64_t* mb, int64_t nb) {
    Tree* T = as_tree(h);
    std::vector<int64_t> sup(ma, ma + na), dem(mb, mb + nb);
    std::vector<double> cost(size_t(na) * nb);
    for (int64_t i = 0; i < na; ++i)
        for (int64_t j = 0; j < nb; ++j)
            cost[size_t(i) * nb + j] = double(tree_distance_units(T->levels, lca_depth(*T, pa[i], pb[j])));
    return min_cost_flow(sup, dem, cost);
}

// General min-cost flow entry (for pins against brute force): integer
// supplies/demands with equal totals and an FP64 cost matrix [na][nb].
double oracle_min_cost_flow(const int64_t* supply, int64_t na, const int64_t* demand, int64_t nb,
                            const double* cost) {
    std::vector<int64_t> s(supply, supply + na), t(demand, demand + nb);
    std::vector<double> c(cost, cost + size_t(na) * nb);
    return min_cost_flow(s, t, c);
}

}  // extern "C"
