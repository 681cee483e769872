// Blocked warp-per-pair Flowtree (Sec. 3; greedy flow of App. A.1).
//
// The same flow as flowtree_pair (ft_flow.cuh), laid out for a lower
// instruction count per item:
//   * lane l owns the live merged items at positions [l*K, l*K + K) (K odd,
//     so that the strided shared-memory accesses below hit distinct banks);
//     an item is one 32-bit word: residual, LCA depth to the previous live
//     item, side;
//   * a depth costs two sequential walks over a lane's K items plus a few
//     warp-wide scans of per-lane totals;
//   * the items that match something at a depth are listed (by ballot, in
//     the second walk) and then processed 32 at a time, so the partner
//     searches run with every lane busy;
//   * the ground-point ids of the matched pairs come from shared memory: per
//     merged position (16-bit, moved with the items) for ground sets of at
//     most 65,536 points, else per support item;
//   * after the point level and after every depth the survivors are
//     compacted into a new blocked layout (the LCA depth between two
//     survivors is the minimum over the dropped span), which also yields the
//     exact next depth to visit: the deepest LCA depth of two neighbouring
//     survivors of different sides (below it every node holds one side
//     only, so nothing else can match).
// At depth k every run of positions with LCA depth >= k is a depth-k node.
// Its mu-residuals meet its nu-residuals in north-west-corner order: with G
// the exclusive prefix sums of the residuals over the whole pair (mu and nu
// packed in one 64-bit word), the item at position i whose own-side offset
// in its run [h, e) is P = G_own[i] - G_own[h] < M = min(G_m[e] - G_m[h],
// G_n[e] - G_n[h]) gives units [P, min(P + r, M)) of its residual r to the
// other-side items whose offsets cover them.  Every pair of the NW matching
// starts at a breakpoint of one of the two streams; the item starting there
// emits it (a nu item leaves it to a mu item that starts at the same
// offset), after a binary search for the other-side item that holds the
// breakpoint.
#pragma once

#include "ft_flow.cuh"

namespace ftk {

// Per-warp shared memory of the blocked form, for up to `cap` merged items.
struct BlockedBuf {
    uint64_t* G;      // [cap + 1] exclusive residual prefix (mu low word, nu high word); staging area
    uint32_t* it;     // [cap] items (it_make)
    uint32_t* list;   // [cap] items that match at the current depth: position | run head << 16
    uint32_t* M;      // [cap] at run heads: the run's matched mass min(mu total, nu total)
    uint32_t* qe;     // (queue) [64] queued pairs: (PT16) mu point | nu point << 16, else mu index | nu index << 16
    uint32_t* qf;     // (queue) [64] their flow
    uint32_t* wd;     // (not PT16) [cap] ground-point ids of the two supports (mu items, then nu items)
    uint16_t* meta;   // (with meta) [cap] bit 15 side (0 mu, 1 nu), bits 0..14 index in its support
    uint16_t* pt;     // (PT16) [cap] ground-point id of the item at each position
};

// PT16: ground sets of at most 65,536 points (16-bit point ids per position).
// The support indices (meta) are kept when flows are saved or the pricing
// resolves point ids through them (not PT16).
__host__ __device__ constexpr bool blocked_has_meta(bool pt16, bool save) { return save || !pt16; }

// The pricing queue (qe, qf) exists for the 8-lane-group pricing only (dim
// > 8); with small dims every lane prices its own pairs as they are found.
__host__ __device__ constexpr bool blocked_has_queue(int mode) { return mode != 0; }

__host__ __device__ inline size_t blockedbuf_bytes(int cap, bool pt16, bool meta, bool queue) {
    return (size_t(cap + 1) * 8 + size_t(cap) * (12 + (meta ? 2 : 0) + (pt16 ? 2 : 4)) + (queue ? 512 : 0) + 15) &
           ~size_t(15);
}

__device__ __forceinline__ BlockedBuf carve_blockedbuf(uint8_t* base, int cap, bool pt16, bool meta, bool queue) {
    BlockedBuf w;
    w.G = reinterpret_cast<uint64_t*>(base);
    w.it = reinterpret_cast<uint32_t*>(w.G + cap + 1);
    w.list = w.it + cap;
    w.M = w.list + cap;
    w.qe = queue ? w.M + cap : nullptr;
    w.qf = queue ? w.qe + 64 : nullptr;
    w.wd = queue ? w.qf + 64 : w.M + cap;
    w.meta = reinterpret_cast<uint16_t*>(w.wd + (pt16 ? 0 : cap));
    w.pt = w.meta + (meta ? cap : 0);
    return w;
}

// item word: residual (bits 0..24; at most 2^24) | LCA depth to the
// previous live item + 1 (bits 25..29; 0 = a run head at every depth) |
// side (bit 30: 0 mu, 1 nu)
constexpr uint32_t kItRes = 0x1FFFFFFu;
__device__ __forceinline__ uint32_t it_res(uint32_t x) { return x & kItRes; }
__device__ __forceinline__ uint32_t it_dp1(uint32_t x) { return (x >> 25) & 31u; }
__device__ __forceinline__ uint32_t it_side(uint32_t x) { return x >> 30; }
__device__ __forceinline__ uint32_t it_make(uint32_t r, uint32_t dp1, uint32_t side) {
    return r | (dp1 << 25) | (side << 30);
}

// smallest odd number of items per lane that holds n items
__device__ __forceinline__ int blocked_k(int n) { return ((max(n, 1) + 31) >> 5) | 1; }

__device__ __forceinline__ uint64_t side_word(uint32_t side, uint32_t r) {
    return side ? (uint64_t(r) << 32) : uint64_t(r);
}

// Per-lane carries for a depth from the lane's residual total `ls`, its last
// run head `nh` (position, -1 if none) and the local exclusive prefix `nl`
// at that head: g0 = exclusive prefix at the lane's first item, and the head
// h_in (with its prefix S_in) of the run holding the lane's first item.
__device__ __forceinline__ void blocked_carries(uint64_t ls, int nh, uint64_t nl, uint64_t* g0, int* h_in,
                                                uint64_t* S_in) {
    const unsigned lane = lane_id();
    const uint64_t incl = warp_incl_scan_u64(ls);
    *g0 = incl - ls;
    const uint64_t S_mine = *g0 + nl;
    // the last lane before this one that holds a head
    const int owner_incl = warp_incl_max_i32(nh >= 0 ? int(lane) : -1);
    int owner = __shfl_up_sync(FULL_MASK, owner_incl, 1);
    if (lane == 0) owner = -1;
    const int src = owner >= 0 ? owner : 0;
    const int hp = __shfl_sync(FULL_MASK, nh, src);
    const uint64_t sp = __shfl_sync(FULL_MASK, S_mine, src);
    *h_in = owner >= 0 ? hp : -1;
    *S_in = owner >= 0 ? sp : 0ull;
}

// Survivor bookkeeping of one lane during a walk, for the compaction:
// survivors kept, the running minimum of the LCA depths (+1) since the last
// survivor, and the depths where two neighbouring survivors of different
// sides meet (within the lane).
struct Survivors {
    int c = 0;
    uint32_t mn = 31;         // min (LCA depth + 1) since the last survivor (31: none yet)
    uint32_t lead = 31;       // ... up to the lane's first survivor
    uint32_t first_side = 0;
    uint32_t last_side = 0;
    uint32_t nm = 0;          // bit d: two neighbouring survivors of different sides with LCA depth d
};

// Item x seen in position order; returns it with a survivor's LCA depth
// (+1) replaced by the one to the previous survivor (the minimum over the
// span between them).
__device__ __forceinline__ uint32_t survivor_track(Survivors& s, uint32_t x) {
    s.mn = min(s.mn, it_dp1(x));
    if (it_res(x) > 0) {
        const uint32_t side = it_side(x);
        if (s.c == 0) {
            s.lead = s.mn;
            s.first_side = side;
        } else if (side != s.last_side) {
            s.nm |= 1u << (s.mn - 1u);
        }
        x = (x & ~(31u << 25)) | (s.mn << 25);
        s.last_side = side;
        ++s.c;
        s.mn = 31;
    }
    return x;
}

// Moves the survivors (residual > 0, LCA depths as left by survivor_track)
// of the lanes' blocks to a new blocked layout through the staging area (the
// prefix array, free at this point), items with their meta (and, PT16, their
// point ids), and returns the
// next depth to visit among the bits of `kmask` (-1: none).  On return Keff
// and n describe the new layout and (ls, nh, nl) are the carries' inputs for
// that depth.
template <bool PT16, bool META>
__device__ __forceinline__ int blocked_compact(const BlockedBuf& w, int& Keff, int& n, const Survivors& s,
                                               uint32_t kmask, uint64_t& ls, int& nh, uint64_t& nl) {
    const unsigned lane = lane_id();
    // segmented carry from the lanes before: has a survivor (bit 6), that
    // survivor's side (bit 5), min LCA depth (+1) over the span after it (bits 0..4)
    uint32_t v = (s.c > 0 ? 64u : 0u) | (s.last_side << 5) | s.mn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL_MASK, v, o);
        if (lane >= unsigned(o) && !(v & 64u)) v = (t & 0x60u) | min(t & 31u, v & 31u);
    }
    uint32_t cin = __shfl_up_sync(FULL_MASK, v, 1);
    if (lane == 0) cin = 0;
    uint32_t nm = s.nm;
    uint32_t first_dp1 = 0;  // the lane's first survivor: new position 0 if no survivor precedes it
    if (cin & 64u) {
        first_dp1 = min(cin & 31u, s.lead);
        if (s.c > 0 && ((cin >> 5) & 1u) != s.first_side) nm |= 1u << (first_dp1 - 1u);
    }
    const uint32_t incl = warp_incl_scan_u32(uint32_t(s.c));
    const int off = int(incl) - s.c;
    const int n_new = int(__shfl_sync(FULL_MASK, incl, 31));
    {
        const int base = int(lane) * Keff;
        int j = off;
        for (int t = 0; t < Keff; ++t) {
            uint32_t x = w.it[base + t];
            if (it_res(x) > 0) {
                if (j == off) x = (x & ~(31u << 25)) | (first_dp1 << 25);
                uint64_t e = uint64_t(x);
                if (META) e |= uint64_t(w.meta[base + t]) << 32;
                if (PT16) e |= uint64_t(w.pt[base + t]) << 48;
                w.G[j] = e;
                ++j;
            }
        }
    }
    nm = __reduce_or_sync(FULL_MASK, nm) & kmask;
    const int knext = nm ? 31 - __clz(nm) : -1;
    __syncwarp();
    n = n_new;
    Keff = blocked_k(n_new);
    const int base = int(lane) * Keff;
    ls = 0;
    nl = 0;
    nh = -1;
    for (int t = 0; t < Keff; ++t) {
        const int pos = base + t;
        const uint64_t e = pos < n_new ? w.G[pos] : 0ull;  // padding: no mass, a run head at every depth
        const uint32_t x = uint32_t(e);
        w.it[pos] = x;
        if (META) w.meta[pos] = uint16_t(e >> 32);
        if (PT16) w.pt[pos] = uint16_t(e >> 48);
        if (int(it_dp1(x)) <= knext) {
            nh = pos;
            nl = ls;
        }
        ls += side_word(it_side(x), it_res(x));
    }
    __syncwarp();  // staging reads done before the prefix array is rewritten
    return knext;
}


// Prices the first cnt (<= 32) queued pairs: acc += f * ||x_a - y_b||, and
// with SAVE the distance goes to the pair's flow slot (queue entry j was
// saved in slot qslot + j).  The queue holds the pairs' ground-point ids
// (PT16) or their support indices, resolved through the staged ids.  MODE as
// in price_queue.
template <int MODE, bool SAVE, bool PT16>
__device__ __forceinline__ void price_staged(const FlowCtx& c, const BlockedBuf& w, const Tables& tb, int na, int cnt,
                                             int64_t qslot, CompSum& acc) {
    const unsigned lane = lane_id();
    uint32_t my_wa = 0, my_wb = 0;
    if (int(lane) < cnt) {
        const uint32_t q = w.qe[lane];
        my_wa = PT16 ? (q & 0xFFFFu) : w.wd[q & 0xFFFFu];
        my_wb = PT16 ? (q >> 16) : w.wd[na + (q >> 16)];
    }
    if (MODE == 0) {
        if (int(lane) < cnt) {
            const float dist = dist_lane(tb, c.dim, my_wa, my_wb);
            acc.add(float(w.qf[lane]) * dist);
            if (SAVE) c.f_dist[qslot + lane] = dist;
        }
    } else {
        const unsigned grp = lane >> 3, sub = lane & 7u;
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

// Computes one pair with the warp, n = na + nb <= cap (the buffer's
// capacity, a multiple of 32 with cap / 32 odd); returns the Flowtree value
// on all lanes.
template <int MODE, bool SAVE, bool PT16>
__device__ float flowtree_pair_blocked(const FlowCtx& c, const BlockedBuf& w, const Tables& tb, int64_t pair,
                                       int64_t da, int64_t db) {
    constexpr bool META = SAVE || !PT16;  // blocked_has_meta
    const unsigned lane = lane_id();
    const unsigned lmask_lt = lanemask_lt();
    const int64_t ao = c.a_ptr[da], bo = c.b_ptr[db];
    const int na = int(c.a_ptr[da + 1] - ao);
    const int nb = int(c.b_ptr[db + 1] - bo);
    int n = na + nb;
    const int L = c.levels;
    int Keff = blocked_k(n);

    // 1. stage ranks (words [0, n)) and masses (words [n, 2n)) of both
    //    supports in the prefix array's space, and their ground-point ids
    //    (PT16: in the list's space until the merge moves them to their
    //    positions; else for the whole pair), 12 loads in flight per lane
    uint32_t* s32 = reinterpret_cast<uint32_t*>(w.G);
    uint32_t* swd = PT16 ? w.list : w.wd;
    for (int b0 = 0; b0 < max(na, nb); b0 += 64) {
        uint32_t v[12];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = b0 + 32 * u + int(lane);
            v[u] = i < na ? __ldg(c.a_rank + ao + i) : 0u;
            v[2 + u] = i < na ? __ldg(c.a_mass + ao + i) : 0u;
            v[4 + u] = i < na ? __ldg(c.a_word + ao + i) : 0u;
            v[6 + u] = i < nb ? __ldg(c.b_rank + bo + i) : 0u;
            v[8 + u] = i < nb ? __ldg(c.b_mass + bo + i) : 0u;
            v[10 + u] = i < nb ? __ldg(c.b_word + bo + i) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = b0 + 32 * u + int(lane);
            if (i < na) {
                s32[i] = v[u];
                s32[n + i] = v[2 + u];
                swd[i] = v[4 + u];
            }
            if (i < nb) {
                s32[na + i] = v[6 + u];
                s32[n + na + i] = v[8 + u];
                swd[na + i] = v[10 + u];
            }
        }
    }
    __syncwarp();

    // 2. merge along the merge path (lane l produces merged positions
    //    [l*Keff, (l+1)*Keff)); the LCA depth to the previous item (from the
    //    range-minimum table); a point carried by both supports (equal ranks,
    //    mu first) is matched with itself here (the point level, distance 0).
    uint32_t levelmask = 0;
    int n_pt = 0;
    uint32_t first_rank = 0xFFFFFFFFu, last_rank = 0xFFFFFFFFu, last_res = 0, first_res = 0;
    const int base0 = int(lane) * Keff;
    {
        const uint32_t* A = s32;
        const uint32_t* B = s32 + na;
        const int d0 = min(n, base0);
        int lo = max(0, d0 - nb), hi = min(d0, na);
        while (lo < hi) {  // split of the first d0 outputs: mu before nu on ties
            const int mid = (lo + hi) >> 1;
            if (A[mid] <= B[d0 - 1 - mid]) lo = mid + 1; else hi = mid;
        }
        int i = lo, j = d0 - lo;
        uint32_t ai = i < na ? A[i] : 0xFFFFFFFFu;  // ranks are < 2^24
        uint32_t bj = j < nb ? B[j] : 0xFFFFFFFFu;
        for (int t = 0; t < Keff; ++t) {
            const int pos = base0 + t;
            uint32_t rk = 0xFFFFFFFFu, r = 0, mi = 0, pid = 0;  // padding: no mass, a run head at every depth
            if (pos < n) {
                if (ai <= bj) {
                    rk = ai;
                    r = s32[n + i];
                    mi = uint32_t(i);
                    if (PT16) pid = swd[i];
                    ++i;
                    ai = i < na ? A[i] : 0xFFFFFFFFu;
                } else {
                    rk = bj;
                    r = s32[n + na + j];
                    mi = 0x8000u | uint32_t(j);
                    if (PT16) pid = swd[na + j];
                    ++j;
                    bj = j < nb ? B[j] : 0xFFFFFFFFu;
                }
            }
            uint32_t dp1 = 0;
            if (t > 0 && pos < n) {
                if (rk == last_rank) {  // mu item of the same point just before
                    dp1 = uint32_t(L + 2);
                    const uint32_t f = min(last_res, r);
                    r -= f;
                    w.it[pos - 1] -= f;
                    ++n_pt;
                } else {
                    const int dd = lca_ranks(tb, c.n_points, last_rank, rk);
                    dp1 = uint32_t(dd + 1);
                    levelmask |= 1u << dd;
                }
            }
            w.it[pos] = it_make(r, dp1, mi >> 15);
            if (META) w.meta[pos] = uint16_t(mi);
            if (PT16) w.pt[pos] = uint16_t(pid);
            if (t == 0) {
                first_rank = rk;
                first_res = r;
            }
            last_rank = rk;
            last_res = r;
        }
    }
    // the lane's first item against the previous lane's last one
    __syncwarp();
    {
        const uint32_t prev_rank = __shfl_up_sync(FULL_MASK, last_rank, 1);
        const uint32_t prev_res = __shfl_up_sync(FULL_MASK, last_res, 1);
        const uint32_t next_rank = __shfl_down_sync(FULL_MASK, first_rank, 1);
        const uint32_t next_res = __shfl_down_sync(FULL_MASK, first_res, 1);
        if (lane > 0 && base0 < n) {
            uint32_t x = w.it[base0];
            if (first_rank == prev_rank) {
                const uint32_t f = min(prev_res, first_res);
                x = it_make(it_res(x) - f, uint32_t(L + 2), it_side(x));
                ++n_pt;
            } else {
                const int dd = lca_ranks(tb, c.n_points, prev_rank, first_rank);
                x = it_make(it_res(x), uint32_t(dd + 1), it_side(x));
                levelmask |= 1u << dd;
            }
            w.it[base0] = x;
        }
        if (lane < 31 && base0 + Keff < n && next_rank == last_rank) {
            // this lane's last item is the mu item of a point whose nu item starts the next lane
            w.it[base0 + Keff - 1] -= min(last_res, next_res);
        }
    }
    levelmask = __reduce_or_sync(FULL_MASK, levelmask);
    CompSum acc;
    int n_saved = 0;
    const int64_t slot0 = SAVE ? c.slot_ptr[pair] : 0;
    if (SAVE) {
        // point-level pairs: the nu item of each (LCA depth L + 1 to the mu
        // item before it) writes the record; the flow is the smaller of the
        // two staged masses
        __syncwarp();
        const uint32_t incl = warp_incl_scan_u32(uint32_t(n_pt));
        int64_t slot = slot0 + int(incl) - n_pt;
        for (int t = 0; t < Keff; ++t) {
            const int pos = base0 + t;
            if (pos < n && it_dp1(w.it[pos]) == uint32_t(L + 2)) {
                const uint32_t ia = uint32_t(w.meta[pos - 1]) & 0x7FFFu, ib = uint32_t(w.meta[pos]) & 0x7FFFu;
                c.f_ia[slot] = ia;
                c.f_ib[slot] = ib;
                c.f_f[slot] = min(s32[n + ia], s32[n + na + ib]);
                c.f_depth[slot] = uint8_t(L + 1);
                c.f_dist[slot] = 0.0f;
                ++slot;
            }
        }
        n_saved = int(__shfl_sync(FULL_MASK, incl, 31));
    }
    __syncwarp();
    // 3. the survivors of the point level
    Survivors sv;
    for (int t = 0; t < Keff; ++t) {
        const uint32_t x = w.it[base0 + t];
        const uint32_t y = survivor_track(sv, x);
        if (y != x) w.it[base0 + t] = y;
    }
    uint32_t kmask = levelmask & ((2u << L) - 1u);

    int qn = 0;                                  // pairs queued for pricing
    int64_t qslot = SAVE ? slot0 + n_saved : 0;  // flow slot of queue entry 0
    const uint32_t* G32 = reinterpret_cast<const uint32_t*>(w.G);  // G32[2p] = mu prefix, G32[2p + 1] = nu prefix

    // 4. bottom-up matching over the depths where the sides meet, deepest
    //    first: every pass starts with the compaction of the survivors (one
    //    call site keeps the kernel small), which also names the next depth
    for (;;) {
        uint64_t ls, nl;
        int nh;
        const int k = blocked_compact<PT16, META>(w, Keff, n, sv, kmask, ls, nh, nl);
        if (k < 0) break;
        const int base = int(lane) * Keff;
        uint64_t g0, S_in;
        int h_in;
        blocked_carries(ls, nh, nl, &g0, &h_in, &S_in);
        // walk 1: prefixes of every position; at run heads the run's matched
        // mass M = min(mu total, nu total)
        {
            uint32_t glo = uint32_t(g0), ghi = uint32_t(g0 >> 32);
            uint32_t slo = uint32_t(S_in), shi = uint32_t(S_in >> 32);
            int cur = h_in;
            for (int t = 0; t < Keff; ++t) {
                const int pos = base + t;
                const uint32_t x = w.it[pos];
                if (int(it_dp1(x)) <= k) {
                    if (cur >= 0) {
                        w.M[cur] = min(glo - slo, ghi - shi);
                    }
                    slo = glo;
                    shi = ghi;
                    cur = pos;
                }
                w.G[pos] = uint64_t(glo) | (uint64_t(ghi) << 32);
                if (it_side(x)) ghi += it_res(x); else glo += it_res(x);
            }
            if (lane == 31) {
                const int end = 32 * Keff;
                w.M[cur] = min(glo - slo, ghi - shi);
                w.G[end] = uint64_t(glo) | (uint64_t(ghi) << 32);
            }
        }
        __syncwarp();
        // walk 2: residual updates, the list of matching items (by ballot),
        // and the survivor bookkeeping of the compaction
        int total = 0;
        sv = Survivors();
        {
            uint32_t rlo = uint32_t(g0) - uint32_t(S_in), rhi = uint32_t(g0 >> 32) - uint32_t(S_in >> 32);
            uint32_t M = h_in >= 0 ? w.M[h_in] : 0u;
            uint32_t hp = uint32_t(max(h_in, 0)) << 16;
            for (int t = 0; t < Keff; ++t) {
                const int pos = base + t;
                const uint32_t x = w.it[pos];
                const uint32_t side = it_side(x);
                if (int(it_dp1(x)) <= k) {
                    rlo = 0;
                    rhi = 0;
                    M = w.M[pos];
                    hp = uint32_t(pos) << 16;
                }
                const uint32_t P = side ? rhi : rlo;
                uint32_t r = it_res(x);
                if (side) rhi += r; else rlo += r;
                const bool emit = r > 0 && P < M;
                const unsigned em = __ballot_sync(FULL_MASK, emit);
                uint32_t y = x;
                if (emit) {
                    w.list[total + __popc(em & lmask_lt)] = uint32_t(pos) | (side << 15) | hp;
                    y = x - min(r, M - P);
                }
                total += __popc(em);
                y = survivor_track(sv, y);
                if (y != x) w.it[pos] = y;
            }
        }
        __syncwarp();
        // the matching items of this depth, 32 at a time
        for (int e0 = 0; e0 < total; e0 += 32) {
            const int e = e0 + int(lane);
            bool emit = false;
            uint32_t f = 0;
            unsigned ia = 0, ib = 0, qa = 0, qb = 0;
            if (e < total) {
                const uint32_t ent = w.list[e];
                const int pos = int(ent & 0x7FFFu), h = int(ent >> 16);
                const unsigned own = (ent >> 15) & 1u, oth = own ^ 1u;
                const int nx = 32 * Keff;  // the layout's end
                const uint32_t M = w.M[h];
                const uint32_t S_own = G32[2 * h + own], S_oth = G32[2 * h + oth];
                const uint32_t g_own = G32[2 * pos + own];
                const uint32_t r = G32[2 * pos + 2 + own] - g_own;
                const uint32_t P = g_own - S_own;
                const uint32_t t0 = S_oth + P;
                const uint32_t capv = S_oth + min(P + r, M);
                // the other-side item holding offset P: last position whose
                // other-side prefix is <= t0 (it lies in the run: the prefix
                // at the run's end exceeds t0)
                int lo = h, hi = nx;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (G32[2 * mid + oth] <= t0) lo = mid; else hi = mid;
                }
                const uint32_t gp = G32[2 * lo + oth];
                if (!(own == 1u && gp == t0)) {
                    f = min(capv, G32[2 * lo + 2 + oth]) - t0;
                    emit = true;
                    if (META) {
                        const unsigned mi = w.meta[pos], mp = w.meta[lo];
                        ia = (own ? mp : mi) & 0x7FFFu;
                        ib = (own ? mi : mp) & 0x7FFFu;
                    }
                    if (PT16) {
                        const uint32_t po = w.pt[pos], pp = w.pt[lo];
                        qa = own ? pp : po;
                        qb = own ? po : pp;
                    }
                }
            }
            const unsigned emask = __ballot_sync(FULL_MASK, emit);
            if (emask == 0) continue;
            const int qp = __popc(emask & lmask_lt);
            if (MODE == 0) {
                // small dim: each emitting lane prices its own pair at once (no queue)
                if (emit) {
                    const uint32_t wa = PT16 ? qa : w.wd[ia];
                    const uint32_t wb = PT16 ? qb : w.wd[na + ib];
                    const float dist = dist_lane(tb, c.dim, wa, wb);
                    acc.add(float(f) * dist);
                    if (SAVE) c.f_dist[slot0 + n_saved + qp] = dist;
                }
            } else if (emit) {
                w.qe[qn + qp] = PT16 ? (qa | (qb << 16)) : (ia | (ib << 16));
                w.qf[qn + qp] = f;
            }
            if (SAVE) {
                if (emit) {
                    const int64_t slot = slot0 + n_saved + qp;
                    c.f_ia[slot] = ia;
                    c.f_ib[slot] = ib;
                    c.f_f[slot] = f;
                    c.f_depth[slot] = uint8_t(k);
                }
                n_saved += __popc(emask);
            }
            if (MODE != 0) qn += __popc(emask);
            if (qn >= 32) {
                __syncwarp();
                price_staged<MODE, SAVE, PT16>(c, w, tb, na, 32, qslot, acc);
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
        __syncwarp();  // the list walk above read the prefix array the compaction reuses
        kmask = (1u << k) - 1u;
    }
    if (qn > 0) {
        __syncwarp();
        price_staged<MODE, SAVE, PT16>(c, w, tb, na, qn, qslot, acc);
    }
    {  // any mass left unmatched would be a bug: report it
        bool left = false;
        for (int t = 0; t < Keff; ++t) left |= it_res(w.it[int(lane) * Keff + t]) > 0;
        if (__any_sync(FULL_MASK, left) && lane == 0) ft_flag(c.status, FT_DEV_EOVERFLOW);
    }
    if (SAVE && lane == 0) c.count[pair] = n_saved;
    __syncwarp();  // the next pair's staging overwrites the prefix array
    float total = acc.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(FULL_MASK, total, o);
    return total * (1.0f / 16777216.0f);
}

}  // namespace ftk
