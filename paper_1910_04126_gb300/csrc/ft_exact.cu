// Exact W1 (Eq. 1) of document pairs on the GPU: the re-ranking stage of the
// nearest-neighbour pipelines of Sec. 5.2 (the paper solves it with a
// network-simplex code on the CPU).
//
// Each pair is a transportation problem on the complete bipartite graph
// between the supports: supplies = the first document's masses, demands =
// the second's (2^24 fixed point, equal totals), arc costs = Euclidean
// distances between the ground points.  One warp solves it by successive
// shortest paths with node potentials (the primal-dual method for min-cost
// flow):
//   * potentials pi keep every residual arc's reduced cost
//     rc(u -> v) = c(u, v) + pi(u) - pi(v) non-negative (forward arcs
//     supply -> demand always exist; a backward arc demand -> supply exists
//     while the pair carries flow, with cost -c);
//   * Dijkstra on reduced costs from every supply node with supply left, over
//     the dense graph (the warp scans all nodes for the minimum and relaxes
//     one node's arcs per step), stopping at the first demand node with
//     demand left;
//   * pi(v) += min(dist(v), D) (D = the distance of that demand node) keeps
//     reduced costs non-negative and makes the path's arcs tight;
//   * the path is augmented by the smallest of: the source's supply, the
//     sink's demand, and the flow on its backward arcs.
// Flows are integers, so the flow is exact; costs, distances and potentials
// are FP32 (reduced costs that rounding pushes below zero are read as 0), so
// the value is optimal up to FP32 rounding of the costs.  The cost matrix and
// the flow of the pair live in the warp's workspace slice (L2-resident while
// the pair is solved); the node arrays live in shared memory.  Pairs are
// taken largest first (the work grows like the cube of the support sizes).
#include <algorithm>
#include <cfloat>

#include "ft_internal.cuh"

namespace {

constexpr int EX_WARPS = 4;  // warps per CTA

struct ExactCtx {
    const int64_t* a_ptr;
    const uint32_t* a_rank;
    const uint32_t* a_mass;
    const uint32_t* a_word;
    const int64_t* b_ptr;
    const uint32_t* b_rank;
    const uint32_t* b_mass;
    const uint32_t* b_word;
    const float* vocab;
    int dim;
    const int32_t* pair_a;
    const int32_t* pair_b;
    int64_t n_pairs;
    int64_t na_docs;
    int64_t nb_docs;
    float* cost_out;
    float* cmat;        // per warp [slice] cost matrix, row-major [na][nb]
    uint32_t* flow;     // per warp [slice] flow, row-major [na][nb]
    size_t slice;       // entries per warp slice (>= max_a * max_b)
    uint32_t* fbits;    // per warp [bslice] bitmap of arcs with flow, column-major: [nb][ceil(na/32)] words
    size_t bslice;
    int nmax;           // max_a + max_b: node arrays per warp
    const uint32_t* order;  // queue position -> pair, largest pairs first
    unsigned long long* queue;
    uint32_t* status;
};

__device__ __forceinline__ bool settled(float d) { return (__float_as_uint(d) >> 31) != 0u; }

__device__ __forceinline__ void warp_argmin(float& v, int& i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float v2 = __shfl_xor_sync(FULL_MASK, v, o);
        const int i2 = __shfl_xor_sync(FULL_MASK, i, o);
        if (v2 < v || (v2 == v && i2 < i)) {
            v = v2;
            i = i2;
        }
    }
}

// Solves one pair with the calling warp; returns W1 (all lanes), or NaN
// after flagging the status word when the phase limit is reached.
__device__ float exact_pair(const ExactCtx& c, int64_t da, int64_t db, float* cm, uint32_t* fl, uint32_t* fb,
                            float* dist, float* pi, int16_t* pred, uint32_t* resid) {
    const unsigned lane = lane_id();
    const int64_t ao = c.a_ptr[da], bo = c.b_ptr[db];
    const int na = int(c.a_ptr[da + 1] - ao), nb = int(c.b_ptr[db + 1] - bo);
    const int n = na + nb;
    const int W = (na + 31) >> 5;  // bitmap words per demand node
    for (int e = int(lane); e < nb * W; e += 32) fb[e] = 0u;
    // cost matrix (direct differences in FP32: no cancellation for near points)
    for (int i = 0; i < na; ++i) {
        const float* x = c.vocab + size_t(c.a_word[ao + i]) * c.dim;
        for (int j = int(lane); j < nb; j += 32) {
            const float* y = c.vocab + size_t(c.b_word[bo + j]) * c.dim;
            float s = 0.0f;
            for (int t = 0; t < c.dim; ++t) {
                const float df = __ldg(x + t) - __ldg(y + t);
                s = fmaf(df, df, s);
            }
            cm[size_t(i) * nb + j] = sqrtf(s);
            fl[size_t(i) * nb + j] = 0u;
        }
    }
    for (int v = int(lane); v < n; v += 32) {
        pi[v] = 0.0f;
        resid[v] = v < na ? c.a_mass[ao + v] : c.b_mass[bo + (v - na)];
    }
    __syncwarp();
    // A point carried by both sides ships min(a, b) to itself at cost 0: with
    // zero potentials every arc keeps a non-negative reduced cost and the flow
    // sits on zero-cost arcs, so this is a valid start for the shortest paths
    // (and some optimal flow keeps the shared mass in place, the cost being a
    // metric).  Supports are rank-sorted with distinct ranks.
    for (int i = int(lane); i < na; i += 32) {
        const uint32_t r = c.a_rank[ao + i];
        int lo = 0, hi = nb;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (c.b_rank[bo + mid] < r) lo = mid + 1; else hi = mid;
        }
        if (lo < nb && c.b_rank[bo + lo] == r) {
            const uint32_t f = min(resid[i], resid[na + lo]);
            fl[size_t(i) * nb + lo] = f;
            if (f) atomicOr(fb + size_t(lo) * W + (i >> 5), 1u << (i & 31));
            resid[i] -= f;
            resid[na + lo] -= f;
        }
    }
    __syncwarp();
    uint32_t remaining = 0;
    for (int v = int(lane); v < na; v += 32) remaining += resid[v];
    remaining = __reduce_add_sync(FULL_MASK, remaining);
    const int max_phases = 8 * n + 64;
    int phases = 0;
    bool failed = false;
    while (remaining > 0) {
        if (++phases > max_phases) {
            failed = true;
            break;
        }
        // Dijkstra on reduced costs from every supply node with supply left.
        // A settled node keeps its distance with the sign bit set (-0.0 for
        // 0), so one load tells both.
        for (int v = int(lane); v < n; v += 32) {
            dist[v] = (v < na && resid[v] > 0) ? 0.0f : FLT_MAX;
            pred[v] = -1;
        }
        __syncwarp();
        int t = -1;
        float D = 0.0f;
        for (int step = 0; step < n; ++step) {
            float best = FLT_MAX;
            int bi = 0x7fffffff;
            int v = int(lane);
            for (; v + 96 < n; v += 128) {  // four independent loads in flight
                const float d0 = dist[v], d1 = dist[v + 32], d2 = dist[v + 64], d3 = dist[v + 96];
                if (!settled(d0) && d0 < best) { best = d0; bi = v; }
                if (!settled(d1) && d1 < best) { best = d1; bi = v + 32; }
                if (!settled(d2) && d2 < best) { best = d2; bi = v + 64; }
                if (!settled(d3) && d3 < best) { best = d3; bi = v + 96; }
            }
            for (; v < n; v += 32) {
                const float dv = dist[v];
                if (!settled(dv) && dv < best) { best = dv; bi = v; }
            }
            warp_argmin(best, bi);
            if (best == FLT_MAX) break;  // nothing reachable (cannot happen: totals are equal)
            const int u = bi;
            __syncwarp();
            if (lane == 0) dist[u] = -best;
            if (u >= na && resid[u] > 0) {
                t = u;
                D = best;
                __syncwarp();
                break;
            }
            const float pu = pi[u];
            if (u < na) {  // forward arcs u -> every demand node
                const float* row = cm + size_t(u) * nb;
                // eight row entries per lane loaded before any store, so that
                // their (L2) latencies overlap
                for (int j0 = int(lane); j0 < nb; j0 += 32 * 8) {
                    float cv[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int j = j0 + 32 * k;
                        cv[k] = j < nb ? row[j] : 0.0f;
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int j = j0 + 32 * k;
                        if (j < nb) {
                            const float e0 = dist[na + j];
                            const float n0 = best + fmaxf(0.0f, cv[k] + pu - pi[na + j]);
                            if (!settled(e0) && n0 < e0) {
                                dist[na + j] = n0;
                                pred[na + j] = int16_t(u);
                            }
                        }
                    }
                }
            } else {  // backward arcs: demand node u -> supply nodes that ship to it (bitmap)
                const int j = u - na;
                for (int w = int(lane); w < W; w += 32) {
                    uint32_t m = fb[size_t(j) * W + w];
                    while (m) {
                        const int i = w * 32 + __ffs(m) - 1;
                        m &= m - 1;
                        const float di = dist[i];
                        if (settled(di)) continue;
                        const float nd = best + fmaxf(0.0f, pu - cm[size_t(i) * nb + j] - pi[i]);
                        if (nd < di) {
                            dist[i] = nd;
                            pred[i] = int16_t(u);
                        }
                    }
                }
            }
            __syncwarp();
        }
        if (t < 0) {
            failed = true;
            break;
        }
        for (int v = int(lane); v < n; v += 32) {
            const float dv = dist[v];
            pi[v] += settled(dv) ? -dv : fminf(dv, D);
        }
        __syncwarp();
        // augment along the path (one lane; the path has at most n arcs)
        uint32_t delta = 0;
        if (lane == 0) {
            delta = resid[t];
            int v = t, s = t, guard = 0;
            while (pred[v] >= 0 && guard++ < n) {
                const int u = pred[v];
                if (u >= na) delta = min(delta, fl[size_t(v) * nb + (u - na)]);  // backward arc u -> v
                s = u;
                v = u;
            }
            delta = min(delta, resid[s]);
            v = t;
            guard = 0;
            while (pred[v] >= 0 && guard++ < n) {
                const int u = pred[v];
                if (u < na) {  // forward arc u -> v
                    uint32_t& f = fl[size_t(u) * nb + (v - na)];
                    if (f == 0u) fb[size_t(v - na) * W + (u >> 5)] |= 1u << (u & 31);
                    f += delta;
                } else {       // backward arc u -> v
                    uint32_t& f = fl[size_t(v) * nb + (u - na)];
                    f -= delta;
                    if (f == 0u) fb[size_t(u - na) * W + (v >> 5)] &= ~(1u << (v & 31));
                }
                v = u;
            }
            resid[s] -= delta;
            resid[t] -= delta;
        }
        delta = __shfl_sync(FULL_MASK, delta, 0);
        __syncwarp();
        if (delta == 0u) {  // no progress would loop forever: report instead
            failed = true;
            break;
        }
        remaining -= delta;
    }
    if (failed) {
        if (lane == 0) ft_flag(c.status, FT_DEV_ETIMEOUT);
        return __int_as_float(0x7fc00000);
    }
    // value: sum f * c over the (sparse) flow, FP64 across the warp
    double acc = 0.0;
    const size_t m = size_t(na) * nb;
    for (size_t e = lane; e < m; e += 32) {
        const uint32_t f = fl[e];
        if (f) acc += double(f) * double(cm[e]);
    }
    acc = warp_sum_f64(acc);
    return float(acc / 16777216.0);
}

__global__ void __launch_bounds__(EX_WARPS * 32, 4) k_exact_w1(ExactCtx c) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = int(threadIdx.x >> 5);
    const unsigned lane = lane_id();
    const int nm = c.nmax;
    uint8_t* base = smem + size_t(warp) * (size_t(nm) * 16);
    float* dist = reinterpret_cast<float*>(base);
    float* pi = dist + nm;
    uint32_t* resid = reinterpret_cast<uint32_t*>(pi + nm);
    int16_t* pred = reinterpret_cast<int16_t*>(resid + nm);
    const int64_t gw = int64_t(blockIdx.x) * EX_WARPS + warp;
    float* cm = c.cmat + size_t(gw) * c.slice;
    uint32_t* fl = c.flow + size_t(gw) * c.slice;
    uint32_t* fb = c.fbits + size_t(gw) * c.bslice;
    for (;;) {
        unsigned long long q = 0;
        if (lane == 0) q = atomicAdd(c.queue, 1ull);
        q = __shfl_sync(FULL_MASK, q, 0);
        if (q >= (unsigned long long)c.n_pairs) break;
        const int64_t p = int64_t(c.order[q]);
        const int64_t da = c.pair_a[p], db = c.pair_b[p];
        if (da < 0 || da >= c.na_docs || db < 0 || db >= c.nb_docs) {
            if (lane == 0) {
                ft_flag(c.status, FT_DEV_EINVAL);
                c.cost_out[p] = __int_as_float(0x7fc00000);
            }
            continue;
        }
        const float w = exact_pair(c, da, db, cm, fl, fb, dist, pi, pred, resid);
        if (lane == 0) c.cost_out[p] = w;
    }
}

struct ExactPlan {
    int64_t n_pairs = 0;
    int blocks = 0;
    size_t smem = 0;
    size_t slice = 0;
    size_t bslice = 0;
    int nmax = 0;
};

ft_status plan_exact(const ft_docs* a, const ft_docs* b, int64_t n_pairs, ExactPlan* p) {
    p->n_pairs = n_pairs;
    const int max_a = std::max(a->max_support, 1), max_b = std::max(b->max_support, 1);
    p->nmax = (max_a + max_b + 31) & ~31;
    if (p->nmax > 32767) return FT_EUNSUPPORTED;  // node ids are int16 in the path records
    p->slice = (size_t(max_a) * max_b + 63) & ~size_t(63);
    p->bslice = (size_t(max_b) * ((max_a + 31) / 32) + 63) & ~size_t(63);
    p->smem = size_t(EX_WARPS) * size_t(p->nmax) * 16;  // dist, pi, resid (4 B), pred (2 B) per node
    int dev = 0, max_smem = 0, sms = 0;
    FT_CUDA(cudaGetDevice(&dev));
    FT_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    FT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (p->smem > size_t(max_smem)) return FT_EUNSUPPORTED;
    int bps = 0;
    FT_TRY(ft_prepare_kernel(reinterpret_cast<const void*>(&k_exact_w1), EX_WARPS * 32, p->smem, &bps));
    if (bps < 1) return FT_EUNSUPPORTED;
    // enough warps to cover the pairs, at most the resident ones
    const int64_t want = (std::max<int64_t>(n_pairs, 1) + EX_WARPS - 1) / EX_WARPS;
    p->blocks = int(std::min<int64_t>(want, int64_t(sms) * bps));
    return FT_OK;
}

struct ExactLayout {
    unsigned long long* queue;
    uint32_t* order;
    uint32_t* keys;
    void* sort_tmp;
    float* cmat;
    uint32_t* flow;
    uint32_t* fbits;
};

// sort key of a pair: larger supports first (the work grows like their
// cube, so the largest pairs go to the warps first)
__global__ void k_exact_key(const int64_t* __restrict__ a_ptr, const int64_t* __restrict__ b_ptr,
                            const int32_t* __restrict__ pa, const int32_t* __restrict__ pb, int64_t n,
                            int64_t na_docs, int64_t nb_docs, uint32_t* __restrict__ key) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t a = pa[i], b = pb[i];
        int64_t len = 0;
        if (a >= 0 && a < na_docs && b >= 0 && b < nb_docs) len = (a_ptr[a + 1] - a_ptr[a]) + (b_ptr[b + 1] - b_ptr[b]);
        key[i] = 0xFFFFu - uint32_t(min(len, int64_t(0xFFFF)));
    }
}

size_t exact_layout(const ExactPlan& p, void* base, ExactLayout* out) {
    WsCarver w(base);
    ExactLayout l{};
    l.queue = w.take<unsigned long long>(1);
    l.order = w.take<uint32_t>(size_t(p.n_pairs));
    l.keys = w.take<uint32_t>(size_t(p.n_pairs));
    l.sort_tmp = w.take<uint8_t>(ft_sort_tmp_bytes(p.n_pairs));
    const size_t per = size_t(p.blocks) * EX_WARPS * p.slice;
    l.cmat = w.take<float>(per);
    l.flow = w.take<uint32_t>(per);
    l.fbits = w.take<uint32_t>(size_t(p.blocks) * EX_WARPS * p.bslice);
    if (out) *out = l;
    return w.off + 256;
}

ft_status check_exact(const float* vocab, const ft_docs* a, const ft_docs* b, const int32_t* pa, const int32_t* pb,
                      int64_t n_pairs, const float* cost_out) {
    if (!vocab || !a || !b || !pa || !pb || !cost_out || n_pairs < 0) return FT_EINVAL;
    if (!a->tree || a->tree != b->tree) return FT_EINVAL;
    return FT_OK;
}

}  // namespace

extern "C" size_t ft_exact_w1_workspace_size(const ft_docs* a, const ft_docs* b, int64_t n_pairs) {
    if (!a || !b || n_pairs < 0 || !a->tree || a->tree != b->tree) return 0;
    ExactPlan p;
    if (plan_exact(a, b, n_pairs, &p) != FT_OK) return 0;
    return exact_layout(p, nullptr, nullptr);
}

extern "C" ft_status ft_exact_w1_batch(const float* vocab_dev, const ft_docs* a, const ft_docs* b,
                                       const int32_t* pair_a_dev, const int32_t* pair_b_dev, int64_t n_pairs,
                                       float* cost_out_dev, void* workspace, size_t ws_bytes, void* stream) {
    FtRange nvtx_range("ft_exact_w1_batch");
    FT_TRY(check_exact(vocab_dev, a, b, pair_a_dev, pair_b_dev, n_pairs, cost_out_dev));
    if (n_pairs == 0) return FT_OK;
    ExactPlan p;
    FT_TRY(plan_exact(a, b, n_pairs, &p));
    if (!workspace || ws_bytes < exact_layout(p, nullptr, nullptr)) return FT_EWORKSPACE;
    ExactLayout l;
    exact_layout(p, workspace, &l);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ExactCtx c{};
    c.a_ptr = a->d_ptr;
    c.a_rank = a->d_rank;
    c.a_mass = a->d_mass;
    c.a_word = a->d_word;
    c.b_ptr = b->d_ptr;
    c.b_rank = b->d_rank;
    c.b_mass = b->d_mass;
    c.b_word = b->d_word;
    c.vocab = vocab_dev;
    c.dim = a->tree->dim;
    c.pair_a = pair_a_dev;
    c.pair_b = pair_b_dev;
    c.n_pairs = n_pairs;
    c.na_docs = a->n_docs;
    c.nb_docs = b->n_docs;
    c.cost_out = cost_out_dev;
    c.cmat = l.cmat;
    c.flow = l.flow;
    c.slice = p.slice;
    c.fbits = l.fbits;
    c.bslice = p.bslice;
    c.nmax = p.nmax;
    c.queue = l.queue;
    c.order = l.order;
    c.status = a->tree->d_status;
    FT_CUDA(cudaMemsetAsync(l.queue, 0, 8, s));
    k_exact_key<<<int(std::min<int64_t>((n_pairs + 255) / 256, 65535 * 8)), 256, 0, s>>>(
        a->d_ptr, b->d_ptr, pair_a_dev, pair_b_dev, n_pairs, a->n_docs, b->n_docs, l.keys);
    FT_CUDA(cudaGetLastError());
    FT_TRY(ft_iota_u32(l.order, n_pairs, s));
    FT_TRY(ft_sort_perm_by_u32(l.keys, l.order, n_pairs, 16, l.sort_tmp, s));
    k_exact_w1<<<p.blocks, EX_WARPS * 32, p.smem, s>>>(c);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}
