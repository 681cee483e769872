// The per-pair Flowtree device code (Sec. 3; greedy flow of App. A.1),
// shared by the persistent batched kernel and the plain one-launch-per-pair
// kernel.
//
// One warp computes one (mu, nu) pair:
//   1. merge the two rank-sorted supports (rank order = depth-first order of
//      the quadtree, so every tree node is a contiguous run of the merged
//      list); equal ranks (a point carried by both) sit side by side;
//   2. D[i] = depth of the lowest common ancestor of merged items i, i+1
//      (L+1 for the same point), from the range-minimum table over lcp;
//   3. bottom-up matching, level-synchronously: at depth k the depth-k nodes
//      are the maximal runs with D >= k.  In every run, the mu-residuals and
//      nu-residuals are matched in north-west-corner order, which is the
//      intersection of their prefix-sum intervals clipped to
//      M = min(run mu-total, run nu-total); what lies beyond M stays for the
//      parent.  Only depths that occur among the D values change the runs,
//      so only those are visited; the smallest one clears everything.
//   4. every matched pair (x, y, f) is priced f * ||x - y|| (FP32 distance,
//      FP64 accumulation) and optionally saved.
// Masses are 24-bit fixed point, so the flow is exact integer arithmetic.
#pragma once

#include "ft_internal.cuh"

namespace ftk {

struct FlowCtx {
    // tree
    const uint8_t* rmq;   // [rmq_levels][n_points]
    int64_t n_points;
    int levels;
    // pricing
    const float* vocab;   // [n_points][dim]
    int dim;
    // supports
    const int64_t* a_ptr;
    const uint32_t* a_rank;
    const uint32_t* a_mass;
    const uint32_t* a_word;
    const int64_t* b_ptr;
    const uint32_t* b_rank;
    const uint32_t* b_mass;
    const uint32_t* b_word;
    // pairs
    const int32_t* pair_a;  // NULL -> cross product
    const int32_t* pair_b;
    int64_t nb_cross;
    int64_t n_pairs;
    int64_t na_docs;
    int64_t nb_docs;
    const uint32_t* order;  // NULL -> identity
    unsigned int* queue;
    float* cost_out;
    // saved flows (NULL = not saved)
    const int64_t* slot_ptr;
    int32_t* count;
    uint32_t* f_ia;
    uint32_t* f_ib;
    uint32_t* f_f;
    uint8_t* f_depth;
    float* f_dist;
    // long-pair scratch
    uint8_t* gscratch;
    size_t gscratch_warp_bytes;
    int gscratch_items;
    uint32_t* status;
};

// Per-warp working set for `cap` merged items (cap multiple of 32).
struct WarpBuf {
    uint32_t* G;      // own-side exclusive residual prefix (merge phase: ranks)
    uint32_t* res;    // residual mass
    uint32_t* word;   // ground-point id
    uint32_t* segS;   // [cap+32] mu prefix at run heads (and at n: totals)
    uint32_t* segSn;  // [cap+32] nu prefix at run heads
    uint32_t* sideG;  // live items compacted per side: prefix
    uint32_t* sideR;  // live items compacted per side: residual (merge phase: input ranks)
    uint16_t* meta;   // bit 15 side (0 mu, 1 nu), bits 0..14 index in its support
    uint16_t* segC;   // [cap+32] live mu count before the run head
    uint16_t* segCn;  // [cap+32] live nu count before the run head
    uint16_t* next;   // next run head of a run head
    uint16_t* headof; // run head of each item
    uint16_t* sideM;  // merged position of a compacted live item
    uint8_t* D;       // LCA depth to the next item
};

__host__ __device__ inline size_t warpbuf_bytes(int cap) {
    return size_t(cap) * (7 * 4 + 6 * 2 + 1) + 64 * 4 + 64 * 2 + 64;
}

__device__ __forceinline__ WarpBuf carve_warpbuf(uint8_t* base, int cap) {
    WarpBuf w;
    uint32_t* p32 = reinterpret_cast<uint32_t*>(base);
    w.G = p32;
    w.res = p32 + cap;
    w.word = p32 + 2 * cap;
    w.segS = p32 + 3 * cap;
    w.segSn = p32 + 4 * cap + 32;
    w.sideG = p32 + 5 * cap + 64;
    w.sideR = p32 + 6 * cap + 64;
    uint16_t* p16 = reinterpret_cast<uint16_t*>(p32 + 7 * cap + 64);
    w.meta = p16;
    w.segC = p16 + cap;
    w.segCn = p16 + 2 * cap + 32;
    w.next = p16 + 3 * cap + 64;
    w.headof = p16 + 4 * cap + 64;
    w.sideM = p16 + 5 * cap + 64;
    w.D = reinterpret_cast<uint8_t*>(p16 + 6 * cap + 64);
    return w;
}

// LCA depth of ranks lo < hi: min of lcp[lo .. hi-1] (range-minimum table).
__device__ __forceinline__ int lca_depth_ranks(const FlowCtx& c, uint32_t lo, uint32_t hi) {
    const uint32_t len = hi - lo;  // >= 1
    const int j = 31 - __clz(len);
    const uint8_t* row = c.rmq + size_t(j) * c.n_points;
    const uint32_t x = __ldg(row + lo);
    const uint32_t y = __ldg(row + hi - (1u << j));
    return int(min(x, y));
}

// Pricing: ||vocab[wa] - vocab[wb]||_2 in FP32.
// MODE 0: each lane prices its own pair (small dim, scalar loads).
// MODE 1: 8-lane groups per pair, float4 loads (dim % 4 == 0).
// MODE 2: 8-lane groups per pair, scalar loads.
__device__ __forceinline__ float dist_lane(const FlowCtx& c, uint32_t wa, uint32_t wb) {
    const float* x = c.vocab + size_t(wa) * c.dim;
    const float* y = c.vocab + size_t(wb) * c.dim;
    float s = 0.0f;
    for (int t = 0; t < c.dim; ++t) {
        const float df = __ldg(x + t) - __ldg(y + t);
        s = fmaf(df, df, s);
    }
    return sqrtf(s);
}

template <int MODE>
__device__ __forceinline__ float dist_group(const FlowCtx& c, uint32_t wa, uint32_t wb, unsigned sub) {
    float s = 0.0f;
    if (MODE == 1) {
        const float4* x = reinterpret_cast<const float4*>(c.vocab + size_t(wa) * c.dim);
        const float4* y = reinterpret_cast<const float4*>(c.vocab + size_t(wb) * c.dim);
        const int n4 = c.dim >> 2;
        for (int t = int(sub); t < n4; t += 8) {
            const float4 p = __ldg(x + t), q = __ldg(y + t);
            const float d0 = p.x - q.x, d1 = p.y - q.y, d2 = p.z - q.z, d3 = p.w - q.w;
            s = fmaf(d0, d0, s);
            s = fmaf(d1, d1, s);
            s = fmaf(d2, d2, s);
            s = fmaf(d3, d3, s);
        }
    } else {
        const float* x = c.vocab + size_t(wa) * c.dim;
        const float* y = c.vocab + size_t(wb) * c.dim;
        for (int t = int(sub); t < c.dim; t += 8) {
            const float df = __ldg(x + t) - __ldg(y + t);
            s = fmaf(df, df, s);
        }
    }
    s += __shfl_xor_sync(FULL_MASK, s, 1);
    s += __shfl_xor_sync(FULL_MASK, s, 2);
    s += __shfl_xor_sync(FULL_MASK, s, 4);
    return sqrtf(s);
}

// Documents of a pair, checked against the document counts; false (and the
// status word flagged) for an index out of range.
__device__ __forceinline__ bool pair_docs(const FlowCtx& c, int64_t pair, int64_t* da, int64_t* db) {
    if (c.pair_a) {
        *da = c.pair_a[pair];
        *db = c.pair_b[pair];
    } else {
        *da = pair / c.nb_cross;
        *db = pair - *da * c.nb_cross;
    }
    if (*da < 0 || *da >= c.na_docs || *db < 0 || *db >= c.nb_docs) {
        if (lane_id() == 0) ft_flag(c.status, FT_DEV_EINVAL);
        return false;
    }
    return true;
}

// Position of the n-th (0-based) set bit of mask; n < popc(mask).
__device__ __forceinline__ int nth_set_bit(unsigned mask, int n) {
    int pos = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const int c = __popc(mask & ((1u << s) - 1u));
        if (n >= c) {
            n -= c;
            mask >>= s;
            pos += s;
        }
    }
    return pos;
}

// Computes one pair with the warp; returns the Flowtree value on all lanes.
template <int MODE, bool SAVE>
__device__ float flowtree_pair(const FlowCtx& c, const WarpBuf& w, int64_t pair, int64_t da, int64_t db) {
    const unsigned lane = lane_id();
    const int64_t ao = c.a_ptr[da], bo = c.b_ptr[db];
    const int na = int(c.a_ptr[da + 1] - ao);
    const int nb = int(c.b_ptr[db + 1] - bo);
    const int n = na + nb;
    const int L = c.levels;

    // 1. stage the input ranks, then merge (equal ranks: mu first)
    uint32_t* stage = w.sideR;
    for (int i = lane; i < na; i += 32) stage[i] = __ldg(c.a_rank + ao + i);
    for (int j = lane; j < nb; j += 32) stage[na + j] = __ldg(c.b_rank + bo + j);
    __syncwarp();
    for (int i = lane; i < na; i += 32) {
        const uint32_t r = stage[i];
        const int pos = i + lower_bound_dev(stage + na, nb, r);
        w.G[pos] = r;
        w.res[pos] = __ldg(c.a_mass + ao + i);
        w.word[pos] = __ldg(c.a_word + ao + i);
        w.meta[pos] = uint16_t(i);
    }
    for (int j = lane; j < nb; j += 32) {
        const uint32_t r = stage[na + j];
        const int pos = j + upper_bound_dev(stage, na, r);
        w.G[pos] = r;
        w.res[pos] = __ldg(c.b_mass + bo + j);
        w.word[pos] = __ldg(c.b_word + bo + j);
        w.meta[pos] = uint16_t(0x8000u | unsigned(j));
    }
    __syncwarp();

    // 2. LCA depth between neighbours; the set of depths that occur
    uint32_t levelmask = 0;
    for (int i = lane; i < n - 1; i += 32) {
        const uint32_t r1 = w.G[i], r2 = w.G[i + 1];
        const int dd = (r1 == r2) ? L + 1 : lca_depth_ranks(c, r1, r2);
        w.D[i] = uint8_t(dd);
        levelmask |= 1u << dd;
    }
    levelmask = __reduce_or_sync(FULL_MASK, levelmask);
    __syncwarp();

    double acc = 0.0;
    int n_saved = 0;
    const int64_t slot0 = SAVE ? c.slot_ptr[pair] : 0;

    // 3. bottom-up matching over the depths present, deepest first
    for (int k = L + 1; k >= 0; --k) {
        if (!((levelmask >> k) & 1u)) continue;
        // pass A: prefixes, run heads, live items compacted per side
        uint32_t gm = 0, gn = 0, cm = 0, cn = 0;
        int lasthead = -1;
        for (int base = 0; base < n; base += 32) {
            const int i = base + int(lane);
            const bool valid = i < n;
            const uint32_t r = valid ? w.res[i] : 0u;
            const unsigned side = valid ? (unsigned(w.meta[i]) >> 15) : 0u;
            const bool live = r > 0;
            const bool head = valid && (i == 0 || int(w.D[i - 1]) < k);
            const uint64_t v = side ? (uint64_t(r) << 32) : uint64_t(r);
            const uint64_t inc = warp_incl_scan_u64(v);
            const uint64_t ex = inc - v;
            const uint32_t Gm = gm + uint32_t(ex);
            const uint32_t Gn = gn + uint32_t(ex >> 32);
            const unsigned bm = __ballot_sync(FULL_MASK, live && side == 0);
            const unsigned bn = __ballot_sync(FULL_MASK, live && side == 1);
            const uint32_t Cm = cm + __popc(bm & lanemask_lt());
            const uint32_t Cn = cn + __popc(bn & lanemask_lt());
            int hinc = warp_incl_max_i32(head ? i : -1);
            hinc = max(hinc, lasthead);
            int hprev = __shfl_up_sync(FULL_MASK, hinc, 1);
            if (lane == 0) hprev = lasthead;
            if (head) {
                w.segS[i] = Gm;
                w.segSn[i] = Gn;
                w.segC[i] = uint16_t(Cm);
                w.segCn[i] = uint16_t(Cn);
                if (hprev >= 0) w.next[hprev] = uint16_t(i);
            }
            if (valid) {
                w.headof[i] = uint16_t(hinc);
                w.G[i] = side ? Gn : Gm;
            }
            if (live) {
                const int idx = side ? na + int(Cn) : int(Cm);
                w.sideG[idx] = side ? Gn : Gm;
                w.sideR[idx] = r;
                w.sideM[idx] = uint16_t(i);
            }
            const uint64_t tot = __shfl_sync(FULL_MASK, inc, 31);
            gm += uint32_t(tot);
            gn += uint32_t(tot >> 32);
            cm += __popc(bm);
            cn += __popc(bn);
            lasthead = __shfl_sync(FULL_MASK, hinc, 31);
        }
        if (lane == 0) {
            w.segS[n] = gm;
            w.segSn[n] = gn;
            w.segC[n] = uint16_t(cm);
            w.segCn[n] = uint16_t(cn);
            w.next[lasthead] = uint16_t(n);
        }
        __syncwarp();
        if (cm == 0) break;  // all mass matched (the two totals are equal)

        // pass B: match inside every run, emit and price the pairs
        for (int base = 0; base < n; base += 32) {
            const int i = base + int(lane);
            bool emit = false;
            uint32_t f = 0, wa = 0, wb = 0;
            unsigned ia = 0, ib = 0;
            if (i < n) {
                const uint32_t r = w.res[i];
                if (r > 0) {
                    const unsigned side = unsigned(w.meta[i]) >> 15;
                    const int h = w.headof[i];
                    const int nx = w.next[h];
                    const uint32_t Sm = w.segS[h], Sn = w.segSn[h];
                    const uint32_t Tm = w.segS[nx] - Sm, Tn = w.segSn[nx] - Sn;
                    const uint32_t M = min(Tm, Tn);
                    const uint32_t S_own = side ? Sn : Sm;
                    const uint32_t S_oth = side ? Sm : Sn;
                    const uint32_t P = w.G[i] - S_own;
                    if (P < M) {
                        const uint32_t target = S_oth + P;
                        int lo = side ? int(w.segC[h]) : na + int(w.segCn[h]);
                        int hi = side ? int(w.segC[nx]) : na + int(w.segCn[nx]);
                        // last b in [lo, hi) with sideG[b] <= target
                        while (hi - lo > 1) {
                            const int mid = (lo + hi) >> 1;
                            if (w.sideG[mid] <= target) lo = mid; else hi = mid;
                        }
                        const uint32_t Gb = w.sideG[lo];
                        const uint32_t rb = w.sideR[lo];
                        if (!(side == 1 && Gb == target)) {
                            const uint32_t end_own = P + r;
                            const uint32_t end_oth = (Gb - S_oth) + rb;
                            f = min(min(end_own, end_oth), M) - P;
                            emit = f > 0;
                            const int pm = w.sideM[lo];
                            const unsigned mo = w.meta[pm];
                            if (side == 0) {
                                ia = unsigned(w.meta[i]) & 0x7FFFu;
                                ib = mo & 0x7FFFu;
                                wa = w.word[i];
                                wb = w.word[pm];
                            } else {
                                ia = mo & 0x7FFFu;
                                ib = unsigned(w.meta[i]) & 0x7FFFu;
                                wa = w.word[pm];
                                wb = w.word[i];
                            }
                        }
                        w.res[i] = r - min(r, M - P);
                    }
                }
            }
            const unsigned emask = __ballot_sync(FULL_MASK, emit);
            if (emask == 0) continue;
            float dist = 0.0f;
            if (k <= L) {
                if (MODE == 0) {
                    if (emit) dist = dist_lane(c, wa, wb);
                } else {
                    const int nemit = __popc(emask);
                    const unsigned grp = lane >> 3, sub = lane & 7u;
                    const int my_e = __popc(emask & lanemask_lt());
                    for (int r0 = 0; r0 < nemit; r0 += 4) {
                        const int e = r0 + int(grp);
                        const int src = e < nemit ? nth_set_bit(emask, e) : 0;
                        uint32_t ga = __shfl_sync(FULL_MASK, wa, src);
                        uint32_t gb = __shfl_sync(FULL_MASK, wb, src);
                        if (e >= nemit) ga = gb = 0;  // idle group: a zero-length pair (row 0 twice)
                        // every lane takes part: dist_group shuffles across the warp
                        const float dg = dist_group<MODE>(c, ga, gb, sub);
                        // hand each group's distance back to its emitting lane
                        const int from = ((my_e - r0) & 3) * 8;
                        const float got = __shfl_sync(FULL_MASK, dg, from);
                        if (emit && my_e >= r0 && my_e < r0 + 4) dist = got;
                    }
                }
            }
            if (emit) acc += double(f) * double(dist);
            if (SAVE) {
                const int o = n_saved + __popc(emask & lanemask_lt());
                if (emit) {
                    const int64_t slot = slot0 + o;
                    c.f_ia[slot] = ia;
                    c.f_ib[slot] = ib;
                    c.f_f[slot] = f;
                    c.f_depth[slot] = uint8_t(k);
                    c.f_dist[slot] = dist;
                }
                n_saved += __popc(emask);
            }
        }
        __syncwarp();
    }
    if (SAVE && lane == 0) c.count[pair] = n_saved;
    acc = warp_sum_f64(acc);
    return float(acc * (1.0 / 16777216.0));
}

}  // namespace ftk
