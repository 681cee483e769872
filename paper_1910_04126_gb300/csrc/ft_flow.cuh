// The per-pair Flowtree device code (Sec. 3; greedy flow of App. A.1),
// shared by the persistent batched kernel and the plain one-launch-per-pair
// kernel.
//
// One warp computes one (mu, nu) pair:
//   1. merge the two rank-sorted supports along the merge path (rank order =
//      depth-first order of the quadtree, so every tree node is a contiguous
//      run of the merged list; equal ranks -- a point carried by both -- sit
//      side by side, mu first);
//   2. D[i] = depth of the lowest common ancestor of merged items i, i+1
//      (L+1 for the same point), from the range-minimum table over lcp;
//   3. bottom-up matching, level-synchronously, deepest first.  After the
//      first depth, only the depths where a live mu item and a live nu item
//      are adjacent (D of an adjacency whose sides differ) get a pass: below
//      the deepest such depth every node holds one side only, so no other
//      depth can match anything.  At depth k the depth-k nodes are
//      the maximal runs with D >= k.  In every run the mu-residuals and the
//      nu-residuals are matched in north-west-corner order: with per-side
//      prefix sums, the unit at offset t of the run's mu stream meets the
//      unit at offset t of its nu stream, for t < M = min(run mu total, run
//      nu total); what lies beyond M stays for the parent.  Items left with
//      no residual are dropped before the next depth, and the LCA depths of
//      the survivors are recomputed (min over the dropped span = the LCA of
//      the two survivors), so each depth only touches live items.  The
//      shallowest depth present clears everything (the totals are equal).
//   4. every matched pair (x, y, f) is priced f * ||x - y|| (FP32 distance,
//      compensated FP32 sum) and optionally saved.  Pairs are queued and
//      priced 32 at a time, so every lane has a pair to price.
// Masses are 24-bit fixed point, so the flow itself is exact integer
// arithmetic.
#pragma once

#include "ft_internal.cuh"

namespace ftk {

struct FlowCtx {
    // tree
    const uint8_t* rmq;   // [rmq_levels][n_points]
    int64_t n_points;
    int levels;
    int rmq_levels;
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
    // blocked form: pairs beyond the warp's staging, left to the CTA-per-pair launch
    uint32_t* long_list;
    unsigned int* long_count;
    // long-pair scratch
    uint8_t* gscratch;
    size_t gscratch_warp_bytes;
    int gscratch_items;
    uint32_t* status;
};

// Vocabulary rows and the LCA range-minimum table, in shared memory when the
// tree is small enough, else in global memory.
struct Tables {
    const float* vocab;   // [n_points][dim]
    const uint8_t* rmq;   // [rmq_levels][n_points]
};

__host__ __device__ inline size_t tables_bytes(int64_t n_points, int dim, int rmq_levels) {
    return ((size_t(n_points) * dim * 4 + 15) & ~size_t(15)) + size_t(rmq_levels) * n_points;
}

// Copy the tables into shared memory (whole block); returns the shared copy.
__device__ __forceinline__ Tables stage_tables(const FlowCtx& c, uint8_t* smem) {
    float* sv = reinterpret_cast<float*>(smem);
    const int nv = int(c.n_points) * c.dim;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) sv[i] = c.vocab[i];
    uint8_t* sr = smem + ((size_t(nv) * 4 + 15) & ~size_t(15));
    const int nr = c.rmq_levels * int(c.n_points);
    for (int i = threadIdx.x; i < nr; i += blockDim.x) sr[i] = c.rmq[i];
    __syncthreads();
    return Tables{sv, sr};
}

// Neumaier-compensated FP32 sum
struct CompSum {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    __device__ __forceinline__ float value() const { return s + c; }
};

// hardware square-root approximation (relative error well below 1e-6)
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Per-warp working set for `cap` merged items (cap multiple of 32), 21 B/item
// plus a 64-entry queue of matched pairs waiting to be priced.
struct WarpBuf {
    uint32_t* rank;   // merged ranks (live items, compacted after every depth)
    uint32_t* res;    // residual mass
    uint32_t* Gm;     // [cap+32] exclusive mu-residual prefix at each position (+ total)
    uint32_t* Gn;     // [cap+32] exclusive nu-residual prefix
    uint32_t* qe;     // [64] queued pairs: mu index | nu index << 16
    uint32_t* qf;     // [64] their flow
    uint16_t* meta;   // bit 15 side (0 mu, 1 nu), bits 0..14 index in its support
    uint16_t* next;   // at run heads: position of the next run head
    uint8_t* D;       // LCA depth to the next item
};

__host__ __device__ inline size_t warpbuf_bytes(int cap) {
    return size_t(cap) * (4 * 4 + 2 * 2 + 1) + (64 + 128) * 4 + 64;
}

__device__ __forceinline__ WarpBuf carve_warpbuf(uint8_t* base, int cap) {
    WarpBuf w;
    uint32_t* p32 = reinterpret_cast<uint32_t*>(base);
    w.rank = p32;
    w.res = p32 + cap;
    w.Gm = p32 + 2 * cap;
    w.Gn = p32 + 3 * cap + 32;
    w.qe = p32 + 4 * cap + 64;
    w.qf = w.qe + 64;
    uint16_t* p16 = reinterpret_cast<uint16_t*>(p32 + 4 * cap + 64 + 128);
    w.meta = p16;
    w.next = p16 + cap;
    w.D = reinterpret_cast<uint8_t*>(p16 + 2 * cap);
    return w;
}

// LCA depth of ranks lo < hi: min of lcp[lo .. hi-1] (range-minimum table).
__device__ __forceinline__ int lca_ranks(const Tables& tb, int64_t n_points, uint32_t lo, uint32_t hi) {
    const uint32_t len = hi - lo;  // >= 1
    const int j = 31 - __clz(len);
    const uint8_t* row = tb.rmq + size_t(j) * n_points;
    return int(min(row[lo], row[hi - (1u << j)]));
}

// Pricing: ||vocab[wa] - vocab[wb]||_2 in FP32.
// MODE 0: each lane prices its own pair (small dim).
// MODE 1: 8-lane groups per pair, float4 loads (dim % 4 == 0).
// MODE 2: 8-lane groups per pair, scalar loads.
__device__ __forceinline__ float dist_lane(const Tables& tb, int dim, uint32_t wa, uint32_t wb) {
    const float* x = tb.vocab + size_t(wa) * dim;
    const float* y = tb.vocab + size_t(wb) * dim;
    float s = 0.0f;
    for (int t = 0; t < dim; ++t) {
        const float df = x[t] - y[t];
        s = fmaf(df, df, s);
    }
    return sqrt_approx(s);
}

template <int MODE>
__device__ __forceinline__ float dist_group(const FlowCtx& c, uint32_t wa, uint32_t wb, unsigned sub) {
    float s = 0.0f;
    if (MODE == 1) {
        const float4* x = reinterpret_cast<const float4*>(c.vocab + size_t(wa) * c.dim);
        const float4* y = reinterpret_cast<const float4*>(c.vocab + size_t(wb) * c.dim);
        const int n4 = c.dim >> 2;
#pragma unroll 4
        for (int t = int(sub); t < n4; t += 8) {  // several row loads in flight
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
#pragma unroll 4
        for (int t = int(sub); t < c.dim; t += 8) {
            const float df = __ldg(x + t) - __ldg(y + t);
            s = fmaf(df, df, s);
        }
    }
    s += __shfl_xor_sync(FULL_MASK, s, 1);
    s += __shfl_xor_sync(FULL_MASK, s, 2);
    s += __shfl_xor_sync(FULL_MASK, s, 4);
    return sqrt_approx(s);
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

// Prices the first cnt (<= 32) queued pairs: acc += f * ||x_a - y_b||, and
// with SAVE the distance goes to the pair's flow slot (queue entry j was
// saved in slot qslot + j).
template <int MODE, bool SAVE>
__device__ __forceinline__ void price_queue(const FlowCtx& c, const WarpBuf& w, const Tables& tb, int64_t ao,
                                            int64_t bo, int cnt, int64_t qslot, CompSum& acc) {
    const unsigned lane = lane_id();
    if (MODE == 0) {
        if (int(lane) < cnt) {
            const uint32_t e = w.qe[lane];
            const uint32_t wa = __ldg(c.a_word + ao + (e & 0xFFFFu));
            const uint32_t wb = __ldg(c.b_word + bo + (e >> 16));
            const float dist = dist_lane(tb, c.dim, wa, wb);
            acc.add(float(w.qf[lane]) * dist);
            if (SAVE) c.f_dist[qslot + lane] = dist;
        }
    } else {
        const unsigned grp = lane >> 3, sub = lane & 7u;
        // the words of all queued pairs at once, one pair per lane, so that the
        // rounds below wait on row loads only
        uint32_t my_wa = 0, my_wb = 0;
        if (int(lane) < cnt) {
            const uint32_t q = w.qe[lane];
            my_wa = __ldg(c.a_word + ao + (q & 0xFFFFu));
            my_wb = __ldg(c.b_word + bo + (q >> 16));
        }
        for (int r0 = 0; r0 < cnt; r0 += 4) {
            const int e = r0 + int(grp);
            uint32_t wa = __shfl_sync(FULL_MASK, my_wa, e & 31);
            uint32_t wb = __shfl_sync(FULL_MASK, my_wb, e & 31);
            if (e >= cnt) wa = wb = 0;  // idle group: a zero-length pair (row 0 twice)
            // every lane takes part: dist_group shuffles across the warp
            const float dist = dist_group<MODE>(c, wa, wb, sub);
            if (e < cnt && sub == 0) {
                acc.add(float(w.qf[e]) * dist);
                if (SAVE) c.f_dist[qslot + e] = dist;
            }
        }
    }
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
__device__ float flowtree_pair(const FlowCtx& c, const WarpBuf& w, const Tables& tb, int64_t pair, int64_t da,
                               int64_t db) {
    const unsigned lane = lane_id();
    const unsigned lmask_lt = lanemask_lt();
    const unsigned lmask_le = lmask_lt | (1u << lane);
    const int64_t ao = c.a_ptr[da], bo = c.b_ptr[db];
    const int na = int(c.a_ptr[da + 1] - ao);
    const int nb = int(c.b_ptr[db + 1] - bo);
    const int n = na + nb;
    const int L = c.levels;

    // 1. stage ranks (Gm) and masses (Gn) of both supports, then merge along
    //    the merge path: each lane writes a contiguous slice of the output
    for (int i = lane; i < na; i += 32) {
        w.Gm[i] = __ldg(c.a_rank + ao + i);
        w.Gn[i] = __ldg(c.a_mass + ao + i);
    }
    for (int j = lane; j < nb; j += 32) {
        w.Gm[na + j] = __ldg(c.b_rank + bo + j);
        w.Gn[na + j] = __ldg(c.b_mass + bo + j);
    }
    __syncwarp();
    {
        const uint32_t* A = w.Gm;
        const uint32_t* B = w.Gm + na;
        const int per = (n + 31) >> 5;
        const int d0 = min(n, int(lane) * per);
        const int d1 = min(n, d0 + per);
        int lo = max(0, d0 - nb), hi = min(d0, na);
        while (lo < hi) {  // split of the first d0 outputs: mu before nu on ties
            const int mid = (lo + hi) >> 1;
            if (A[mid] <= B[d0 - 1 - mid]) lo = mid + 1; else hi = mid;
        }
        int i = lo, j = d0 - lo;
        for (int d = d0; d < d1; ++d) {
            if (i < na && (j >= nb || A[i] <= B[j])) {
                w.rank[d] = A[i];
                w.res[d] = w.Gn[i];
                w.meta[d] = uint16_t(i);
                ++i;
            } else {
                w.rank[d] = B[j];
                w.res[d] = w.Gn[na + j];
                w.meta[d] = uint16_t(0x8000u | unsigned(j));
                ++j;
            }
        }
    }
    __syncwarp();

    CompSum acc;
    int n_saved = 0;
    const int64_t slot0 = SAVE ? c.slot_ptr[pair] : 0;

    // 2. LCA depth between neighbours; the set of depths that occur.  A point
    //    carried by both supports is a run of its own at the point level
    //    (depth L+1): its mu and nu items sit side by side and are matched
    //    here directly (distance 0), so the point level needs no pass.
    uint32_t levelmask = 0;
    for (int base = 0; base < n - 1; base += 32) {
        const int i = base + int(lane);
        const bool valid = i < n - 1;
        bool same = false;
        uint32_t f = 0;
        if (valid) {
            const uint32_t r1 = w.rank[i], r2 = w.rank[i + 1];
            same = r1 == r2;
            const int dd = same ? L + 1 : lca_ranks(tb, c.n_points, r1, r2);
            w.D[i] = uint8_t(dd);
            // every depth present: items emptied at the point level may still
            // separate a mu item from a nu item here, so the exact rule (a
            // depth where the sides meet) waits for the first compaction
            if (!same) levelmask |= 1u << dd;
            if (same) {  // i is the mu item, i + 1 the nu item of the same point
                const uint32_t ra = w.res[i], rb = w.res[i + 1];
                f = min(ra, rb);
                w.res[i] = ra - f;
                w.res[i + 1] = rb - f;
            }
        }
        if (SAVE) {
            const unsigned emask = __ballot_sync(FULL_MASK, same);
            if (same) {
                const int64_t slot = slot0 + n_saved + __popc(emask & lmask_lt);
                c.f_ia[slot] = unsigned(w.meta[i]) & 0x7FFFu;
                c.f_ib[slot] = unsigned(w.meta[i + 1]) & 0x7FFFu;
                c.f_f[slot] = f;
                c.f_depth[slot] = uint8_t(L + 1);
                c.f_dist[slot] = 0.0f;
            }
            n_saved += __popc(emask);
        }
    }
    levelmask = __reduce_or_sync(FULL_MASK, levelmask);
    __syncwarp();
    int qn = 0;                                   // pairs queued for pricing
    int64_t qslot = SAVE ? slot0 + n_saved : 0;   // flow slot of queue entry 0
    int nl = n;  // items in the working set (exhausted ones are dropped after the first depth)

    // 3. bottom-up matching over the depths present, deepest first
    while (nl > 0 && levelmask != 0) {
        const int k = 31 - __clz(levelmask);
        // pass A: per-side exclusive prefixes at every position; every run
        // head links to the next one, with bit 15 set when the run holds
        // residual on both sides (only such runs match anything)
        uint32_t gm = 0, gn = 0;
        int lasthead = -1;
        bool any_mixed = false;
        for (int base = 0; base < nl; base += 32) {
            const int i = base + int(lane);
            const bool valid = i < nl;
            const uint32_t r = valid ? w.res[i] : 0u;
            const unsigned side = valid ? (unsigned(w.meta[i]) >> 15) : 0u;
            const bool head = valid && (i == 0 || int(w.D[i - 1]) < k);
            const uint64_t v = side ? (uint64_t(r) << 32) : uint64_t(r);
            const uint64_t inc = warp_incl_scan_u64(v);
            const uint64_t ex = inc - v;
            const uint32_t Gmi = gm + uint32_t(ex), Gni = gn + uint32_t(ex >> 32);
            if (valid) {
                w.Gm[i] = Gmi;
                w.Gn[i] = Gni;
            }
            __syncwarp();
            const unsigned hb = __ballot_sync(FULL_MASK, head);
            const unsigned before = hb & lmask_lt;
            const int prev = before ? base + 31 - __clz(before) : lasthead;
            if (head && prev >= 0) {
                const bool mixed = (Gmi - w.Gm[prev]) > 0 && (Gni - w.Gn[prev]) > 0;
                any_mixed |= mixed;
                w.next[prev] = uint16_t(i | (mixed ? 0x8000 : 0));
            }
            if (hb) lasthead = base + 31 - __clz(hb);
            const uint64_t tot = __shfl_sync(FULL_MASK, inc, 31);
            gm += uint32_t(tot);
            gn += uint32_t(tot >> 32);
        }
        if (lane == 0) {
            w.Gm[nl] = gm;
            w.Gn[nl] = gn;
            const bool mixed = (gm - w.Gm[lasthead]) > 0 && (gn - w.Gn[lasthead]) > 0;
            any_mixed |= mixed;
            w.next[lasthead] = uint16_t(nl | (mixed ? 0x8000 : 0));
        }
        __syncwarp();
        // Every run one-sided (possible only before the first compaction,
        // while the depths are all those present): nothing to match, but
        // pass C still runs, to drop the items emptied at the point level and
        // find the depths where the sides meet.
        const int nl_b = __any_sync(FULL_MASK, any_mixed) ? nl : 0;

        // pass B: match inside every run, queue and save the pairs
        lasthead = -1;
        for (int base = 0; base < nl_b; base += 32) {
            const int i = base + int(lane);
            const bool valid = i < nl;
            const bool head = valid && (i == 0 || int(w.D[i - 1]) < k);
            const unsigned hb = __ballot_sync(FULL_MASK, head);
            const unsigned upto = hb & lmask_le;
            const int h = upto ? base + 31 - __clz(upto) : lasthead;
            if (hb) lasthead = base + 31 - __clz(hb);
            bool emit = false;
            uint32_t f = 0;
            unsigned ia = 0, ib = 0;
            const uint32_t r = valid ? w.res[i] : 0u;
            const unsigned link = valid ? unsigned(w.next[h]) : 0u;
            if (r > 0 && (link & 0x8000u)) {  // live item in a run with both sides
                const unsigned mi = w.meta[i];
                const unsigned side = mi >> 15;
                const int nx = int(link & 0x7FFFu);
                const uint32_t Sm = w.Gm[h], Sn = w.Gn[h];
                const uint32_t M = min(w.Gm[nx] - Sm, w.Gn[nx] - Sn);
                const uint32_t* Go = side ? w.Gm : w.Gn;
                const uint32_t S_own = side ? Sn : Sm;
                const uint32_t S_oth = side ? Sm : Sn;
                const uint32_t P = (side ? w.Gn[i] : w.Gm[i]) - S_own;
                if (P < M) {
                    const uint32_t target = S_oth + P;
                    // the other-side item holding offset P: last position in
                    // the run whose other-side prefix is <= target
                    int lo = h, hi = nx;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (Go[mid] <= target) lo = mid; else hi = mid;
                    }
                    const uint32_t Gp = Go[lo];
                    const uint32_t rp = Go[lo + 1] - Gp;
                    if (!(side == 1 && Gp == target)) {
                        f = min(min(P + r, (Gp - S_oth) + rp), M) - P;
                        emit = true;
                        const unsigned mp = w.meta[lo];
                        if (side == 0) {
                            ia = mi & 0x7FFFu;
                            ib = mp & 0x7FFFu;
                        } else {
                            ia = mp & 0x7FFFu;
                            ib = mi & 0x7FFFu;
                        }
                    }
                    w.res[i] = r - min(r, M - P);
                }
            }
            const unsigned emask = __ballot_sync(FULL_MASK, emit);
            if (emask == 0) continue;
            // queue the pairs (k <= L: distinct points); they are priced 32
            // at a time, one lane (MODE 0) or 8-lane group (MODE 1, 2) each
            const int pos = __popc(emask & lmask_lt);
            if (emit) {
                w.qe[qn + pos] = ia | (ib << 16);
                w.qf[qn + pos] = f;
            }
            if (SAVE) {
                if (emit) {
                    const int64_t slot = slot0 + n_saved + pos;
                    c.f_ia[slot] = ia;
                    c.f_ib[slot] = ib;
                    c.f_f[slot] = f;
                    c.f_depth[slot] = uint8_t(k);
                }
                n_saved += __popc(emask);
            }
            qn += __popc(emask);
            if (qn >= 32) {
                __syncwarp();
                price_queue<MODE, SAVE>(c, w, tb, ao, bo, 32, qslot, acc);
                __syncwarp();
                const int rest = qn - 32;
                uint32_t qe2 = 0, qf2 = 0;
                if (int(lane) < rest) {
                    qe2 = w.qe[32 + lane];
                    qf2 = w.qf[32 + lane];
                }
                __syncwarp();
                if (int(lane) < rest) {
                    w.qe[lane] = qe2;
                    w.qf[lane] = qf2;
                }
                __syncwarp();
                qn = rest;
                qslot += 32;
            }
        }
        __syncwarp();

        // pass C: drop exhausted items (stable, in place) and recompute the
        // LCA depth between consecutive survivors (the minimum over the
        // dropped span: a range-minimum lookup, unless the two were
        // neighbours already); only depths below k can remain.  Ranks are
        // below 2^24, so bit 31 carries the side.
        int cnt = 0;
        uint32_t nm = 0;
        uint32_t carry = 0;        // rank | side << 31 of the previous chunk's last survivor
        bool carry_adj = false;    // ... which was that chunk's last item
        unsigned carry_d = 0;      // ... and its D before this pass
        for (int base = 0; base < nl; base += 32) {
            const int i = base + int(lane);
            const bool valid = i < nl;
            const uint32_t r = valid ? w.res[i] : 0u;
            const uint32_t rk = valid ? w.rank[i] : 0u;
            const uint16_t mt = valid ? w.meta[i] : uint16_t(0);
            const unsigned d_old = valid ? unsigned(w.D[i]) : 0u;
            const bool keep = r > 0;
            const unsigned km = __ballot_sync(FULL_MASK, keep);
            const uint32_t rs = rk | ((unsigned(mt) >> 15) << 31);
            // the next survivor in this chunk (self if none)
            const unsigned above = km & ~lmask_le;
            const int nxt = above ? __ffs(above) - 1 : int(lane);
            const uint32_t rs_next = __shfl_sync(FULL_MASK, rs, nxt);
            const uint32_t rs_first = __shfl_sync(FULL_MASK, rs, km ? __ffs(km) - 1 : 0);
            const uint32_t rs_last = __shfl_sync(FULL_MASK, rs, km ? 31 - __clz(km) : 0);
            const unsigned d31 = __shfl_sync(FULL_MASK, d_old, 31);
            __syncwarp();
            const int o = cnt + __popc(km & lmask_lt);
            if (keep) {
                if (o != i) {
                    w.rank[o] = rk;
                    w.res[o] = r;
                    w.meta[o] = mt;
                }
                if (above) {
                    int dd = int(d_old);
                    if (nxt != int(lane) + 1) {
                        const uint32_t rn = rs_next & 0x7FFFFFFFu;
                        dd = (rk == rn) ? L + 1 : lca_ranks(tb, c.n_points, rk, rn);
                    }
                    if (o != i || dd != int(d_old)) w.D[o] = uint8_t(dd);
                    if ((rs ^ rs_next) >> 31) nm |= 1u << dd;
                }
            }
            if (lane == 0 && km && cnt > 0) {  // previous chunk's last survivor -> this chunk's first
                int dd;
                if (carry_adj && (km & 1u)) {
                    dd = int(carry_d);
                } else {
                    const uint32_t ra = carry & 0x7FFFFFFFu, rb = rs_first & 0x7FFFFFFFu;
                    dd = (ra == rb) ? L + 1 : lca_ranks(tb, c.n_points, ra, rb);
                }
                w.D[cnt - 1] = uint8_t(dd);
                if ((carry ^ rs_first) >> 31) nm |= 1u << dd;
            }
            if (km) carry = rs_last;
            carry_adj = (km >> 31) & 1u;
            carry_d = d31;
            cnt += __popc(km);
            __syncwarp();
        }
        nl = cnt;
        nm = __reduce_or_sync(FULL_MASK, nm);
        levelmask = nm & ((1u << k) - 1u);
        __syncwarp();
    }
    if (qn > 0) {
        __syncwarp();
        price_queue<MODE, SAVE>(c, w, tb, ao, bo, qn, qslot, acc);
    }
    if (nl > 0) {  // any mass left unmatched would be a bug: report it
        bool left = false;
        for (int i = lane; i < nl; i += 32) left |= w.res[i] > 0;
        if (__any_sync(FULL_MASK, left) && lane == 0) ft_flag(c.status, FT_DEV_EOVERFLOW);
    }
    if (SAVE && lane == 0) c.count[pair] = n_saved;
    float total = acc.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(FULL_MASK, total, o);
    return total * (1.0f / 16777216.0f);
}

}  // namespace ftk
