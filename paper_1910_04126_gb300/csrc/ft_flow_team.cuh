// A CTA per pair: the blocked Flowtree (ft_flow_blocked.cuh) for pairs whose
// merged supports exceed a warp's staging (Sec. 3; greedy flow of App. A.1).
//
// The whole CTA (W warps, T = 32W threads) is the team of one pair: thread t
// owns merged positions [t*K, t*K + K) (K odd), the warp scans of the warp
// form become team scans (warp scans, then a scan of the warp totals in
// shared memory), every warp lists the matching items of its own positions,
// and the lists are processed in team-wide rounds: in round r every warp
// takes its entries [32r, 32r + 32), and the flow records of the round are
// numbered in warp order, so saved flows land in the same slots on every
// run.  Each warp prices its own queue; the warps' compensated sums are
// added in warp order.
#pragma once

#include "ft_flow_blocked.cuh"

namespace ftk {

constexpr int kTeamWarps = 8;
constexpr int kTeamThreads = 32 * kTeamWarps;

// Team scratch in shared memory (besides the per-position arrays).
struct TeamScratch {
    uint64_t u64[kTeamThreads];   // per-thread 64-bit values (prefix at the last head, ...)
    uint32_t a[kTeamThreads];     // per-thread 32-bit values (first / last rank, ...)
    uint32_t b[kTeamThreads];
    uint32_t c[kTeamThreads];
    uint32_t d[kTeamThreads];
    uint64_t w64[kTeamWarps + 1]; // per-warp totals
    uint32_t w32[kTeamWarps + 1];
    uint32_t w32b[kTeamWarps + 1];
    unsigned long long pair;      // the pair the team works on
};

// team inclusive scan (sum) of a 64-bit value; all threads of the CTA call it
__device__ __forceinline__ uint64_t team_incl_scan_u64(uint64_t v, TeamScratch& ts) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    uint64_t x = warp_incl_scan_u64(v);
    if (lane == 31) ts.w64[warp] = x;
    __syncthreads();
    uint64_t off = 0;
    for (unsigned w = 0; w < warp; ++w) off += ts.w64[w];
    __syncthreads();
    return x + off;
}

__device__ __forceinline__ uint32_t team_incl_scan_u32(uint32_t v, TeamScratch& ts, uint32_t* total) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t x = warp_incl_scan_u32(v);
    if (lane == 31) ts.w32[warp] = x;
    __syncthreads();
    uint32_t off = 0, tot = 0;
    for (unsigned w = 0; w < kTeamWarps; ++w) {
        if (w < warp) off += ts.w32[w];
        tot += ts.w32[w];
    }
    __syncthreads();
    *total = tot;
    return x + off;
}

__device__ __forceinline__ int team_incl_max_i32(int v, TeamScratch& ts) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const int x = warp_incl_max_i32(v);
    if (lane == 31) ts.w32[warp] = uint32_t(x);
    __syncthreads();
    int off = -1;
    for (unsigned w = 0; w < warp; ++w) off = max(off, int(ts.w32[w]));
    __syncthreads();
    return max(x, off);
}

__device__ __forceinline__ uint32_t team_or(uint32_t v, TeamScratch& ts) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t x = __reduce_or_sync(FULL_MASK, v);
    if (lane == 0) ts.w32b[warp] = x;
    __syncthreads();
    uint32_t r = 0;
    for (unsigned w = 0; w < kTeamWarps; ++w) r |= ts.w32b[w];
    __syncthreads();
    return r;
}

__device__ __forceinline__ uint32_t team_max_u32(uint32_t v, TeamScratch& ts) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t x = __reduce_max_sync(FULL_MASK, v);
    if (lane == 0) ts.w32b[warp] = x;
    __syncthreads();
    uint32_t r = 0;
    for (unsigned w = 0; w < kTeamWarps; ++w) r = max(r, ts.w32b[w]);
    __syncthreads();
    return r;
}

// The survivors' segmented carry (see blocked_compact) over the team: the
// combination of a left value t and a right value v keeps v if v holds a
// survivor, else takes t's survivor and side and the smaller span minimum.
__device__ __forceinline__ uint32_t seg_combine(uint32_t t, uint32_t v) {
    return (v & 64u) ? v : ((t & 0x60u) | min(t & 31u, v & 31u));
}

__device__ __forceinline__ uint32_t team_excl_seg(uint32_t v, TeamScratch& ts) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= unsigned(o)) x = seg_combine(t, x);
    }
    if (lane == 31) ts.w32[warp] = x;
    uint32_t ex = __shfl_up_sync(FULL_MASK, x, 1);
    __syncthreads();
    uint32_t off = 31u;  // identity: no survivor, span minimum "none"
    for (unsigned w = 0; w < warp; ++w) off = seg_combine(off, ts.w32[w]);
    __syncthreads();
    return lane == 0 ? off : seg_combine(off, ex);
}

// Per-team shared memory for up to `cap` merged items (cap a multiple of
// 32 * kTeamWarps with cap / (32 * kTeamWarps) odd).
struct TeamBuf {
    uint64_t* G;      // [cap + 1] exclusive residual prefix (mu low word, nu high word); staging area
    uint32_t* it;     // [cap] items (it_make)
    uint32_t* list;   // [cap] matching items, warp w's at [w * 32K, ...): position | side << 15 | run head << 16
    uint32_t* M;      // [cap] at run heads: the run's matched mass
    uint32_t* wd;     // [cap] ground-point ids of the two supports (mu items, then nu items)
    uint32_t* qe;     // [kTeamWarps][64] queued pairs per warp: mu index | nu index << 16
    uint32_t* qf;     // [kTeamWarps][64] their flow
    uint32_t* qs;     // [kTeamWarps][64] their flow slot (relative to the pair's first slot)
    uint16_t* meta;   // [cap] bit 15 side, bits 0..14 index in its support
};

__host__ __device__ inline size_t teambuf_bytes(int cap) {
    return (size_t(cap + 1) * 8 + size_t(cap) * 18 + size_t(3) * kTeamWarps * 64 * 4 + 15) & ~size_t(15);
}

__device__ __forceinline__ TeamBuf carve_teambuf(uint8_t* base, int cap) {
    TeamBuf w;
    w.G = reinterpret_cast<uint64_t*>(base);
    w.it = reinterpret_cast<uint32_t*>(w.G + cap + 1);
    w.list = w.it + cap;
    w.M = w.list + cap;
    w.wd = w.M + cap;
    w.qe = w.wd + cap;
    w.qf = w.qe + kTeamWarps * 64;
    w.qs = w.qf + kTeamWarps * 64;
    w.meta = reinterpret_cast<uint16_t*>(w.qs + kTeamWarps * 64);
    return w;
}

// smallest odd number of items per thread that holds n items
__device__ __forceinline__ int team_k(int n) { return ((max(n, 1) + kTeamThreads - 1) / kTeamThreads) | 1; }

// Team version of blocked_compact: moves the survivors to a new blocked
// layout through the staging area, returns the next depth among kmask's
// bits (-1: none) and the carries' inputs (ls, nh, nl) for it.
__device__ int team_compact(const TeamBuf& w, TeamScratch& ts, int& Keff, const Survivors& s, uint32_t kmask,
                            uint64_t& ls, int& nh, uint64_t& nl) {
    const int tid = int(threadIdx.x);
    const uint32_t cin_raw = team_excl_seg((s.c > 0 ? 64u : 0u) | (s.last_side << 5) | s.mn, ts);
    const uint32_t cin = (cin_raw & 64u) ? cin_raw : 0u;
    uint32_t nm = s.nm;
    uint32_t first_dp1 = 0;
    if (cin & 64u) {
        first_dp1 = min(cin & 31u, s.lead);
        if (s.c > 0 && ((cin >> 5) & 1u) != s.first_side) nm |= 1u << (first_dp1 - 1u);
    }
    uint32_t n_new = 0;
    const uint32_t incl = team_incl_scan_u32(uint32_t(s.c), ts, &n_new);
    const int off = int(incl) - s.c;
    {
        const int base = tid * Keff;
        int j = off;
        for (int t = 0; t < Keff; ++t) {
            uint32_t x = w.it[base + t];
            if (it_res(x) > 0) {
                if (j == off) x = (x & ~(31u << 25)) | (first_dp1 << 25);
                w.G[j] = uint64_t(x) | (uint64_t(w.meta[base + t]) << 32);
                ++j;
            }
        }
    }
    nm = team_or(nm, ts) & kmask;  // (its barriers also order the staging writes before the reads below)
    const int knext = nm ? 31 - __clz(nm) : -1;
    Keff = team_k(int(n_new));
    const int base = tid * Keff;
    ls = 0;
    nl = 0;
    nh = -1;
    for (int t = 0; t < Keff; ++t) {
        const int pos = base + t;
        const uint64_t e = pos < int(n_new) ? w.G[pos] : 0ull;
        const uint32_t x = uint32_t(e);
        w.it[pos] = x;
        w.meta[pos] = uint16_t(e >> 32);
        if (int(it_dp1(x)) <= knext) {
            nh = pos;
            nl = ls;
        }
        ls += side_word(it_side(x), it_res(x));
    }
    __syncthreads();  // staging reads done before the prefix array is rewritten
    return knext;
}

// Team version of blocked_carries.
__device__ __forceinline__ void team_carries(uint64_t ls, int nh, uint64_t nl, TeamScratch& ts, uint64_t* g0,
                                             int* h_in, uint64_t* S_in) {
    const int tid = int(threadIdx.x);
    const uint64_t incl = team_incl_scan_u64(ls, ts);
    *g0 = incl - ls;
    const int owner_incl = team_incl_max_i32(nh >= 0 ? tid : -1, ts);
    ts.a[tid] = uint32_t(owner_incl);
    ts.b[tid] = uint32_t(nh);
    ts.u64[tid] = *g0 + nl;
    __syncthreads();
    const int owner = tid > 0 ? int(ts.a[tid - 1]) : -1;
    *h_in = owner >= 0 ? int(ts.b[owner]) : -1;
    *S_in = owner >= 0 ? ts.u64[owner] : 0ull;
    __syncthreads();
}

// Prices warp w's first cnt (<= 32) queued pairs; with SAVE the distance
// goes to the pair's flow slot slot0 + qs[j].  MODE as in price_queue.
template <int MODE, bool SAVE>
__device__ __forceinline__ void team_price(const FlowCtx& c, const TeamBuf& w, const Tables& tb, int na, int cnt,
                                           int64_t slot0, CompSum& acc) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t* qe = w.qe + warp * 64;
    const uint32_t* qf = w.qf + warp * 64;
    const uint32_t* qs = w.qs + warp * 64;
    uint32_t my_wa = 0, my_wb = 0;
    if (int(lane) < cnt) {
        const uint32_t q = qe[lane];
        my_wa = w.wd[q & 0xFFFFu];
        my_wb = w.wd[na + (q >> 16)];
    }
    if (MODE == 0) {
        if (int(lane) < cnt) {
            const float dist = dist_lane(tb, c.dim, my_wa, my_wb);
            acc.add(float(qf[lane]) * dist);
            if (SAVE) c.f_dist[slot0 + qs[lane]] = dist;
        }
    } else {
        const unsigned grp = lane >> 3, sub = lane & 7u;
        for (int r0 = 0; r0 < cnt; r0 += 4) {
            const int e = r0 + int(grp);
            uint32_t wa = __shfl_sync(FULL_MASK, my_wa, e & 31);
            uint32_t wb = __shfl_sync(FULL_MASK, my_wb, e & 31);
            if (e >= cnt) wa = wb = 0;
            const float dist = dist_group<MODE>(c, wa, wb, sub);
            if (e < cnt && sub == 0) {
                acc.add(float(qf[e]) * dist);
                if (SAVE) c.f_dist[slot0 + qs[e]] = dist;
            }
        }
    }
}

// Computes one pair with the whole CTA, n = na + nb <= cap; returns the
// Flowtree value on thread 0 (others: unspecified).
template <int MODE, bool SAVE>
__device__ float flowtree_pair_team(const FlowCtx& c, const TeamBuf& w, TeamScratch& ts, const Tables& tb,
                                    int64_t pair, int64_t da, int64_t db) {
    const int tid = int(threadIdx.x);
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const unsigned lmask_lt = lanemask_lt();
    const int64_t ao = c.a_ptr[da], bo = c.b_ptr[db];
    const int na = int(c.a_ptr[da + 1] - ao);
    const int nb = int(c.b_ptr[db + 1] - bo);
    const int n = na + nb;
    const int L = c.levels;
    int Keff = team_k(n);

    // 1. stage ranks (words [0, n)), masses (words [n, 2n)) and ground-point ids
    uint32_t* s32 = reinterpret_cast<uint32_t*>(w.G);
    for (int i = tid; i < na; i += kTeamThreads) {
        s32[i] = __ldg(c.a_rank + ao + i);
        s32[n + i] = __ldg(c.a_mass + ao + i);
        w.wd[i] = __ldg(c.a_word + ao + i);
    }
    for (int j = tid; j < nb; j += kTeamThreads) {
        s32[na + j] = __ldg(c.b_rank + bo + j);
        s32[n + na + j] = __ldg(c.b_mass + bo + j);
        w.wd[na + j] = __ldg(c.b_word + bo + j);
    }
    __syncthreads();

    // 2. merge (thread t produces positions [t*Keff, (t+1)*Keff)), LCA depth
    //    to the previous item, point-level matches (as in the warp form)
    uint32_t levelmask = 0;
    int n_pt = 0;
    uint32_t first_rank = 0xFFFFFFFFu, last_rank = 0xFFFFFFFFu, last_res = 0, first_res = 0;
    const int base0 = tid * Keff;
    {
        const uint32_t* A = s32;
        const uint32_t* B = s32 + na;
        const int d0 = min(n, base0);
        int lo = max(0, d0 - nb), hi = min(d0, na);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (A[mid] <= B[d0 - 1 - mid]) lo = mid + 1; else hi = mid;
        }
        int i = lo, j = d0 - lo;
        uint32_t ai = i < na ? A[i] : 0xFFFFFFFFu;
        uint32_t bj = j < nb ? B[j] : 0xFFFFFFFFu;
        for (int t = 0; t < Keff; ++t) {
            const int pos = base0 + t;
            uint32_t rk = 0xFFFFFFFFu, r = 0, mi = 0;
            if (pos < n) {
                if (ai <= bj) {
                    rk = ai;
                    r = s32[n + i];
                    mi = uint32_t(i);
                    ++i;
                    ai = i < na ? A[i] : 0xFFFFFFFFu;
                } else {
                    rk = bj;
                    r = s32[n + na + j];
                    mi = 0x8000u | uint32_t(j);
                    ++j;
                    bj = j < nb ? B[j] : 0xFFFFFFFFu;
                }
            }
            uint32_t dp1 = 0;
            if (t > 0 && pos < n) {
                if (rk == last_rank) {
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
            w.meta[pos] = uint16_t(mi);
            if (t == 0) {
                first_rank = rk;
                first_res = r;
            }
            last_rank = rk;
            last_res = r;
        }
    }
    ts.a[tid] = first_rank;
    ts.b[tid] = first_res;
    ts.c[tid] = last_rank;
    ts.d[tid] = last_res;
    __syncthreads();
    {
        if (tid > 0 && base0 < n) {
            const uint32_t prev_rank = ts.c[tid - 1], prev_res = ts.d[tid - 1];
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
        if (tid + 1 < kTeamThreads && base0 + Keff < n && ts.a[tid + 1] == last_rank)
            w.it[base0 + Keff - 1] -= min(last_res, ts.b[tid + 1]);
    }
    levelmask = team_or(levelmask, ts);  // (its barriers order the item writes above)
    CompSum acc;
    int n_saved = 0;
    const int64_t slot0 = SAVE ? c.slot_ptr[pair] : 0;
    if (SAVE) {
        uint32_t tot = 0;
        const uint32_t incl = team_incl_scan_u32(uint32_t(n_pt), ts, &tot);
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
        n_saved = int(tot);
    }
    __syncthreads();
    // 3. survivors of the point level
    Survivors sv;
    for (int t = 0; t < Keff; ++t) {
        const uint32_t x = w.it[base0 + t];
        const uint32_t y = survivor_track(sv, x);
        if (y != x) w.it[base0 + t] = y;
    }
    uint32_t kmask = levelmask & ((2u << L) - 1u);
    int qn = 0;  // this warp's queued pairs
    uint32_t* qe = w.qe + warp * 64;
    uint32_t* qf = w.qf + warp * 64;
    uint32_t* qs = w.qs + warp * 64;
    const uint32_t* G32 = reinterpret_cast<const uint32_t*>(w.G);

    // 4. bottom-up matching, deepest first; every pass starts with the compaction
    for (;;) {
        uint64_t ls, nl;
        int nh;
        const int k = team_compact(w, ts, Keff, sv, kmask, ls, nh, nl);
        if (k < 0) break;
        const int base = tid * Keff;
        const int end = kTeamThreads * Keff;
        uint64_t g0, S_in;
        int h_in;
        team_carries(ls, nh, nl, ts, &g0, &h_in, &S_in);
        // walk 1: prefixes of every position; at run heads the run's matched mass
        {
            uint32_t glo = uint32_t(g0), ghi = uint32_t(g0 >> 32);
            uint32_t slo = uint32_t(S_in), shi = uint32_t(S_in >> 32);
            int cur = h_in;
            for (int t = 0; t < Keff; ++t) {
                const int pos = base + t;
                const uint32_t x = w.it[pos];
                if (int(it_dp1(x)) <= k) {
                    if (cur >= 0) w.M[cur] = min(glo - slo, ghi - shi);
                    slo = glo;
                    shi = ghi;
                    cur = pos;
                }
                w.G[pos] = uint64_t(glo) | (uint64_t(ghi) << 32);
                if (it_side(x)) ghi += it_res(x); else glo += it_res(x);
            }
            if (tid == kTeamThreads - 1) {
                w.M[cur] = min(glo - slo, ghi - shi);
                w.G[end] = uint64_t(glo) | (uint64_t(ghi) << 32);
            }
        }
        __syncthreads();
        // walk 2: residual updates; every warp lists the matching items of its positions
        uint32_t* wl = w.list + warp * 32 * Keff;
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
                const uint32_t r = it_res(x);
                if (side) rhi += r; else rlo += r;
                const bool emit = r > 0 && P < M;
                const unsigned em = __ballot_sync(FULL_MASK, emit);
                uint32_t y = x;
                if (emit) {
                    wl[total + __popc(em & lmask_lt)] = uint32_t(pos) | (side << 15) | hp;
                    y = x - min(r, M - P);
                }
                total += __popc(em);
                y = survivor_track(sv, y);
                if (y != x) w.it[pos] = y;
            }
        }
        // the listed items in team-wide rounds (warp w takes its entries [32r, 32r + 32))
        const int rounds = int(team_max_u32(uint32_t((total + 31) >> 5), ts));  // (barriers: the lists are complete)
        for (int r = 0; r < rounds; ++r) {
            const int e = 32 * r + int(lane);
            bool emit = false;
            uint32_t f = 0;
            unsigned ia = 0, ib = 0;
            if (e < total) {
                const uint32_t ent = wl[e];
                const int pos = int(ent & 0x7FFFu), h = int(ent >> 16);
                const unsigned own = (ent >> 15) & 1u, oth = own ^ 1u;
                const uint32_t M = w.M[h];
                const uint32_t S_own = G32[2 * h + own], S_oth = G32[2 * h + oth];
                const uint32_t g_own = G32[2 * pos + own];
                const uint32_t rr = G32[2 * pos + 2 + own] - g_own;
                const uint32_t P = g_own - S_own;
                const uint32_t t0 = S_oth + P;
                const uint32_t capv = S_oth + min(P + rr, M);
                int lo = h, hi = end;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (G32[2 * mid + oth] <= t0) lo = mid; else hi = mid;
                }
                if (!(own == 1u && G32[2 * lo + oth] == t0)) {
                    f = min(capv, G32[2 * lo + 2 + oth]) - t0;
                    emit = true;
                    const unsigned mi = w.meta[pos], mp = w.meta[lo];
                    ia = (own ? mp : mi) & 0x7FFFu;
                    ib = (own ? mi : mp) & 0x7FFFu;
                }
            }
            const unsigned emask = __ballot_sync(FULL_MASK, emit);
            const int cw = __popc(emask);
            if (lane == 0) ts.w32[warp] = uint32_t(cw);
            __syncthreads();
            int woff = 0, rtot = 0;
            for (int v = 0; v < kTeamWarps; ++v) {
                if (v < int(warp)) woff += int(ts.w32[v]);
                rtot += int(ts.w32[v]);
            }
            __syncthreads();
            const int qp = __popc(emask & lmask_lt);
            if (emit) {
                const int rel = n_saved + woff + qp;  // flow slot, numbered in warp order
                qe[qn + qp] = ia | (ib << 16);
                qf[qn + qp] = f;
                qs[qn + qp] = uint32_t(rel);
                if (SAVE) {
                    c.f_ia[slot0 + rel] = ia;
                    c.f_ib[slot0 + rel] = ib;
                    c.f_f[slot0 + rel] = f;
                    c.f_depth[slot0 + rel] = uint8_t(k);
                }
            }
            n_saved += rtot;
            qn += cw;
            if (qn >= 32) {  // this warp's queue: priced 32 at a time
                __syncwarp();
                team_price<MODE, SAVE>(c, w, tb, na, 32, slot0, acc);
                __syncwarp();
                const int rest = qn - 32;
                uint32_t a2 = 0, b2 = 0, c2 = 0;
                if (int(lane) < rest) {
                    a2 = qe[32 + lane];
                    b2 = qf[32 + lane];
                    c2 = qs[32 + lane];
                }
                __syncwarp();
                if (int(lane) < rest) {
                    qe[lane] = a2;
                    qf[lane] = b2;
                    qs[lane] = c2;
                }
                __syncwarp();
                qn = rest;
            }
        }
        __syncthreads();  // list and prefix reads done before the compaction
        kmask = (1u << k) - 1u;
    }
    if (qn > 0) {
        __syncwarp();
        team_price<MODE, SAVE>(c, w, tb, na, qn, slot0, acc);
    }
    {  // any mass left unmatched would be a bug: report it
        bool left = false;
        for (int t = 0; t < Keff; ++t) left |= it_res(w.it[tid * Keff + t]) > 0;
        if (team_or(left ? 1u : 0u, ts) && tid == 0) ft_flag(c.status, FT_DEV_EOVERFLOW);
    }
    if (SAVE && tid == 0) c.count[pair] = n_saved;
    float v = acc.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    if (lane == 0) ts.u64[warp] = __float_as_uint(v);
    __syncthreads();
    float total = 0.0f;
    if (tid == 0)
        for (int v2 = 0; v2 < kTeamWarps; ++v2) total += __uint_as_float(uint32_t(ts.u64[v2]));
    __syncthreads();  // the next pair's staging overwrites the prefix array
    return total * (1.0f / 16777216.0f);
}

}  // namespace ftk
