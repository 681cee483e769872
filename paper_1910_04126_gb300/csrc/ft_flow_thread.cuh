// One thread per (mu, nu) pair: the bottom-up greedy of App. A.1 as a single
// left-to-right sweep over the merged rank-sorted supports.
//
// Quadtree nodes are contiguous runs of the rank order, and the depth of the
// lowest common ancestor of two neighbouring items (g, from the range-minimum
// table) says which nodes close between them.  The sweep keeps a stack of
// frames, one per child group of the nodes still open, with strictly
// increasing depths; a frame is a contiguous range of merged positions whose
// unmatched items all lie on one side once the frame is complete.  Before
// item x with left gap g is pushed, every top frame of depth >= g is merged
// into the frame below it, at the top frame's depth (the node they share).
// A merge of a left group into a right group matches their items first in
// first out, which for a node's children taken left to right is exactly the
// north-west-corner matching of the node's concatenated mu- and nu-lists
// (the k-th unit of mu mass meets the k-th unit of nu mass).  The sweep ends
// by merging everything down to the first frame (the root clears all mass,
// the two totals being equal).
//
// Positions are merged order and are never reused, so the per-thread state
// is small: a side bit, a matched bit and a partly-matched bit per position
// (a position's support index is the count of same-side positions before
// it) and the frame stack, in shared memory; the residuals of partly matched
// items (one may be left by every merge; an image pair has ~30 at once) in
// the thread's slice of the workspace.  Only the two items at the fronts of
// a merge change while it runs, and they are held in registers.
//
// The sweep is a flat state machine (fetch/merge-check, one match step per
// iteration), so the 32 threads of a warp, each on its own pair, go round the
// same loop and diverge only inside one iteration.  Per-thread arrays live in
// shared memory, interleaved over the lanes (word e of a lane at base[32 e]).
#pragma once

#include "ft_flow.cuh"

namespace ftk {

constexpr int kLaneFrames = FT_MAX_LEVELS + 3;

// shared-memory words per lane for positions up to nmax
__host__ __device__ inline int lane_words(int nmax) {
    const int W = (nmax + 31) / 32;
    return 4 * W + 1 + 2 * kLaneFrames;
}

template <bool SAVE>
struct LanePair {
    const FlowCtx& c;  // a __grid_constant__ kernel parameter: no local copy
    const Tables tb;
    uint32_t* sidew;  // [W] bit p: side of position p (1 = nu)
    uint32_t* usedw;  // [W] bit p: position p fully matched
    uint32_t* pcw;    // [W+1] nu positions before word w
    uint32_t* partw;  // [W] bit p: position p partly matched (residual in gres[p])
    uint32_t* fgb;    // [kLaneFrames] gap (biased by one) | first position << 5
    uint32_t* fhd;    // [kLaneFrames] first live position
    uint32_t* gres;   // this thread's residuals of partly matched positions (global)
    int W;
    // pair
    int64_t ao = 0, bo = 0, slot = 0;
    int na = 0, nb = 0, L = 0;
    int saved = 0;
    CompSum acc;

    __device__ __forceinline__ LanePair(const FlowCtx& c_, const Tables& tb_, uint32_t* lane_base, int W_,
                                        uint32_t* gres_)
        : c(c_), tb(tb_), gres(gres_), W(W_) {
        sidew = lane_base;
        usedw = lane_base + size_t(W_) * 32;
        pcw = lane_base + size_t(2 * W_) * 32;
        partw = lane_base + size_t(3 * W_ + 1) * 32;
        fgb = lane_base + size_t(4 * W_ + 1) * 32;
        fhd = fgb + size_t(kLaneFrames) * 32;
    }

    __device__ __forceinline__ uint32_t& S(uint32_t* a, int e) { return a[size_t(e) * 32]; }

    __device__ __forceinline__ unsigned side_of(int x) { return (S(sidew, x >> 5) >> (x & 31)) & 1u; }
    // support index of position x on its side s
    __device__ __forceinline__ int index_of(int x, unsigned s) {
        const int w = x >> 5;
        const int nu_before = int(S(pcw, w)) + __popc(S(sidew, w) & ((1u << (x & 31)) - 1u));
        return s ? nu_before : x - nu_before;
    }
    __device__ __forceinline__ void set_used(int x) { S(usedw, x >> 5) |= 1u << (x & 31); }
    // first position >= x that is not fully matched, or end
    __device__ __forceinline__ int next_live(int x, int end) {
        if (x >= end) return end;
        int w = x >> 5;
        uint32_t m = ~S(usedw, w) & (0xFFFFFFFFu << (x & 31));
        const int wl = (end - 1) >> 5;
        while (m == 0u && w < wl) m = ~S(usedw, ++w);
        if (m == 0u) return end;
        const int pos = w * 32 + __ffs(m) - 1;
        return pos < end ? pos : end;
    }
    // residual of a live position: its override (taken out of the table;
    // partial = true), else its full mass
    __device__ __forceinline__ uint32_t take_res(int x, unsigned s, int idx, bool& partial) {
        uint32_t& w = S(partw, x >> 5);
        const uint32_t bit = 1u << (x & 31);
        partial = (w & bit) != 0u;
        if (partial) {
            w &= ~bit;
            return gres[x];
        }
        return s ? c.b_mass[bo + idx] : c.a_mass[ao + idx];
    }
    __device__ __forceinline__ void keep_res(int x, uint32_t r) {
        S(partw, x >> 5) |= 1u << (x & 31);
        gres[x] = r;
    }
    __device__ __forceinline__ uint32_t word_of(unsigned s, int idx) {
        return SAVE ? uint32_t(idx) : (s ? c.b_word[bo + idx] : c.a_word[ao + idx]);
    }

    __device__ __forceinline__ void emit(int im, int in, uint32_t wm, uint32_t wn, uint32_t eta, int k) {
        float dist = 0.0f;
        if (k <= L) {
            const uint32_t wa = SAVE ? c.a_word[ao + im] : wm;
            const uint32_t wb = SAVE ? c.b_word[bo + in] : wn;
            dist = dist_lane(tb, c.dim, wa, wb);
        }
        acc.add(float(eta) * dist);
        if (SAVE) {
            const int64_t s = slot + saved;
            c.f_ia[s] = uint32_t(im);
            c.f_ib[s] = uint32_t(in);
            c.f_f[s] = eta;
            c.f_depth[s] = uint8_t(k);
            c.f_dist[s] = dist;
            ++saved;
        }
    }
};

// The sweep of one pair, driven by the caller one step at a time.
enum : int { LP_FETCH = 0, LP_CHECK = 1, LP_FINAL = 2, LP_MATCH = 3, LP_DONE = 4 };

template <bool SAVE>
struct LaneSweep {
    LanePair<SAVE> P;
    int phase = LP_DONE;
    int ret = LP_CHECK;   // phase to resume after a match
    // merging input
    int ia = 0, ib = 0;
    uint32_t ra = 0, rb = 0, prev = 0;
    int p = 0, nf = 0;
    // pending item
    unsigned ps = 0;  // its side
    int pg = 0;       // its gap: LCA depth with the previous item (-1 for the first)
    // current match: left front (pl, end le), right front (pr, end re)
    int mk = 0, pl = 0, le = 0, pr = 0, re = 0;
    unsigned sl = 0, sr = 0;
    int il = 0, ir = 0;
    uint32_t wl = 0, wr = 0, resl = 0, resr = 0;
    bool dl = false, dr = false;  // front residual below its full mass

    __device__ __forceinline__ LaneSweep(const FlowCtx& c, const Tables& tb, uint32_t* lane_base, int W,
                                         uint32_t* gres)
        : P(c, tb, lane_base, W, gres) {}

    __device__ __forceinline__ void start(int64_t pair, int64_t da, int64_t db) {
        const FlowCtx& c = P.c;
        P.ao = c.a_ptr[da];
        P.bo = c.b_ptr[db];
        P.na = int(c.a_ptr[da + 1] - P.ao);
        P.nb = int(c.b_ptr[db + 1] - P.bo);
        P.L = c.levels;
        P.saved = 0;
        P.acc = CompSum();
        if (SAVE) P.slot = c.slot_ptr[pair];
        ia = ib = 0;
        ra = P.na > 0 ? c.a_rank[P.ao] : 0xFFFFFFFFu;
        rb = P.nb > 0 ? c.b_rank[P.bo] : 0xFFFFFFFFu;
        p = 0;
        nf = 0;
        phase = LP_FETCH;
    }

    __device__ __forceinline__ int gap_top() { return int(P.S(P.fgb, nf - 1) & 31u) - 1; }

    // merge the top frame into the one below at depth gap_top(); O(1) unless
    // both fronts are live and on different sides, which starts a match
    __device__ __forceinline__ void merge_begin() {
        const int lf = nf - 2, rf = nf - 1;
        const int lh = int(P.S(P.fhd, lf)), rbeg = int(P.S(P.fgb, rf) >> 5), rh = int(P.S(P.fhd, rf));
        const int e = p;
        if (lh == rbeg) {  // left fully matched: the merged frame is the right one
            P.S(P.fhd, lf) = uint32_t(rh);
            --nf;
            return;
        }
        if (rh == e) {  // right fully matched
            --nf;
            return;
        }
        const unsigned s1 = P.side_of(lh), s2 = P.side_of(rh);
        if (s1 == s2) {  // one side: concatenation (the gap between them is fully matched)
            --nf;
            return;
        }
        mk = gap_top();
        pl = lh;
        le = rbeg;
        pr = rh;
        re = e;
        sl = s1;
        sr = s2;
        il = P.index_of(pl, sl);
        ir = P.index_of(pr, sr);
        resl = P.take_res(pl, sl, il, dl);
        resr = P.take_res(pr, sr, ir, dr);
        wl = P.word_of(sl, il);
        wr = P.word_of(sr, ir);
        ret = phase;
        phase = LP_MATCH;
    }

    // one step of the first-in first-out match between the two fronts
    __device__ __forceinline__ void match_step() {
        const uint32_t eta = min(resl, resr);
        if (sl == 0) P.emit(il, ir, wl, wr, eta, mk); else P.emit(ir, il, wr, wl, eta, mk);
        resl -= eta;
        resr -= eta;
        dl = true;
        dr = true;
        if (resl == 0u) {
            P.set_used(pl);
            pl = P.next_live(pl + 1, le);
            if (pl < le) {
                il = P.index_of(pl, sl);
                resl = P.take_res(pl, sl, il, dl);
                wl = P.word_of(sl, il);
            }
        }
        if (resr == 0u) {
            P.set_used(pr);
            pr = P.next_live(pr + 1, re);
            if (pr < re) {
                ir = P.index_of(pr, sr);
                resr = P.take_res(pr, sr, ir, dr);
                wr = P.word_of(sr, ir);
            }
        }
        if (pl >= le || pr >= re) {
            const int lf = nf - 2;
            if (pl >= le) {
                P.S(P.fhd, lf) = uint32_t(pr);  // the right remainder (or nothing: pr == re)
                if (pr < re && dr) P.keep_res(pr, resr);
            } else {
                P.S(P.fhd, lf) = uint32_t(pl);
                if (dl) P.keep_res(pl, resl);
            }
            --nf;
            phase = ret;
        }
    }

    // one iteration of the state machine
    __device__ __forceinline__ void step() {
        const FlowCtx& c = P.c;
        if (phase == LP_FETCH) {
            if (ia >= P.na && ib >= P.nb) {
                phase = LP_FINAL;
            } else {
                uint32_t r;
                if (ia < P.na && (ib >= P.nb || ra <= rb)) {
                    r = ra;
                    ps = 0;
                    ++ia;
                    ra = ia < P.na ? c.a_rank[P.ao + ia] : 0xFFFFFFFFu;
                } else {
                    r = rb;
                    ps = 1;
                    ++ib;
                    rb = ib < P.nb ? c.b_rank[P.bo + ib] : 0xFFFFFFFFu;
                }
                pg = p == 0 ? -1 : (r == prev ? P.L + 1 : lca_ranks(P.tb, c.n_points, prev, r));
                prev = r;
                phase = LP_CHECK;
            }
        }
        if (phase == LP_CHECK || phase == LP_FINAL) {
            const int g = phase == LP_FINAL ? -1 : pg;
            if (nf >= 2 && gap_top() >= g) {
                merge_begin();
            } else if (phase == LP_CHECK) {  // push the pending item as a frame of its own
                const int w = p >> 5, b = p & 31;
                if (b == 0) {
                    P.S(P.sidew, w) = 0u;
                    P.S(P.usedw, w) = 0u;
                    P.S(P.partw, w) = 0u;
                    P.S(P.pcw, w) = w == 0 ? 0u : P.S(P.pcw, w - 1) + uint32_t(__popc(P.S(P.sidew, w - 1)));
                }
                P.S(P.sidew, w) |= ps << b;
                P.S(P.fgb, nf) = uint32_t(pg + 1) | (uint32_t(p) << 5);
                P.S(P.fhd, nf) = uint32_t(p);
                ++nf;
                ++p;
                phase = LP_FETCH;
            } else {
                phase = LP_DONE;
            }
        } else if (phase == LP_MATCH) {
            match_step();
        }
    }
};

}  // namespace ftk
