// One thread per (mu, nu) pair: the bottom-up greedy of App. A.1 as a single
// left-to-right sweep over the merged rank-sorted supports.
//
// Quadtree nodes are contiguous runs of the rank order, and the depth of the
// lowest common ancestor of two neighbouring items (g, from the range-minimum
// table) says which nodes close between them.  The sweep keeps a stack of
// frames, one per child group of the nodes still open, with strictly
// increasing depths; each frame's leftover demands (all on one side once the
// frame is complete) are a contiguous run of a per-thread item buffer.
// Before item x with left gap g is pushed:
//   * every frame deeper than g is complete: the top frame is merged into the
//     frame below it, at the depth of the top frame (the node they share);
//   * a top frame at depth g is a complete earlier child of the node at depth
//     g that x joins: it is merged into the frame below as well.
// A merge of a left group into a right group matches their demands first in
// first out, which for a node's children taken left to right is exactly the
// north-west-corner matching of the node's concatenated mu- and nu-lists
// (the k-th unit of mu mass meets the k-th unit of nu mass).  The sweep ends
// by merging everything down to the first frame (the root clears all mass,
// the two totals being equal).
//
// Work per pair: one pass over the s_mu + s_nu items plus one step per matched
// pair, no warp-wide synchronisation.  Used for low-dimensional ground sets,
// where pricing a pair is a few instructions.  The item buffer lives in
// shared memory, interleaved over the 32 lanes of the warp (entry e of a lane
// at buf[32 e]); a pair whose buffer would outgrow `cap` entries stops and
// reports overflow (the caller hands it to the warp-per-pair kernel).
#pragma once

#include "ft_flow.cuh"

namespace ftk {

constexpr int kThreadFrames = FT_MAX_LEVELS + 3;

// buffer entry: residual (bits 0..24), side (bit 25), payload (bits 26..63):
// the support index when flows are saved, otherwise the ground-point id.
__device__ __forceinline__ uint64_t tentry(uint32_t res, uint32_t side, uint64_t payload) {
    return uint64_t(res) | (uint64_t(side) << 25) | (payload << 26);
}
__device__ __forceinline__ uint32_t tres(uint64_t e) { return uint32_t(e & 0x1FFFFFFu); }
__device__ __forceinline__ uint32_t tside(uint64_t e) { return uint32_t(e >> 25) & 1u; }
__device__ __forceinline__ uint64_t tpay(uint64_t e) { return e >> 26; }
__device__ __forceinline__ uint64_t tsetres(uint64_t e, uint32_t r) { return (e & ~uint64_t(0x1FFFFFFu)) | r; }

__device__ __forceinline__ float tdist(const Tables& tb, int dim, uint32_t wa, uint32_t wb) {
    return dist_lane(tb, dim, wa, wb);
}

template <bool SAVE>
struct ThreadPair {
    const FlowCtx& c;
    const Tables& tb;
    uint64_t* buf;  // this lane's entry 0; entry e at buf[32 e]
    int cap;
    bool overflow = false;
    uint8_t fgap[kThreadFrames];
    uint16_t fbeg[kThreadFrames];
    uint16_t fhead[kThreadFrames];
    int nf = 0;
    int bend = 0;
    int64_t ao = 0, bo = 0, slot = 0;
    int saved = 0;
    CompSum acc;

    __device__ ThreadPair(const FlowCtx& c_, const Tables& tb_, uint64_t* buf_, int cap_)
        : c(c_), tb(tb_), buf(buf_), cap(cap_) {}

    __device__ __forceinline__ uint64_t& B(int e) { return buf[size_t(e) * 32]; }

    __device__ __forceinline__ void emit(uint64_t em, uint64_t en, uint32_t eta, int k) {
        uint32_t wa, wb;
        if (SAVE) {
            wa = c.a_word[ao + int64_t(tpay(em))];
            wb = c.b_word[bo + int64_t(tpay(en))];
        } else {
            wa = uint32_t(tpay(em));
            wb = uint32_t(tpay(en));
        }
        const float dist = (k <= c.levels) ? tdist(tb, c.dim, wa, wb) : 0.0f;
        acc.add(float(eta) * dist);
        if (SAVE) {
            const int64_t s = slot + saved;
            c.f_ia[s] = uint32_t(tpay(em));
            c.f_ib[s] = uint32_t(tpay(en));
            c.f_f[s] = eta;
            c.f_depth[s] = uint8_t(k);
            c.f_dist[s] = dist;
            ++saved;
        }
    }

    // merge the top frame into the one below it, at node depth k
    __device__ __forceinline__ void merge_top(int k) {
        const int lf = nf - 2, rf = nf - 1;
        const int lh = fhead[lf], rb = fbeg[rf], rh = fhead[rf], e = bend;
        if (lh == rb) {
            fhead[lf] = uint16_t(rh);
        } else if (rh == e) {
            bend = rb;
        } else {
            uint64_t el = B(lh), er = B(rh);
            if (tside(el) == tside(er)) {
                if (rh != rb) {
                    for (int t = rh; t < e; ++t) B(rb + (t - rh)) = B(t);
                    bend = rb + (e - rh);
                }
            } else {
                int pl = lh, pr = rh;
                bool lx = false, rx = false;
                for (;;) {
                    const uint32_t rl = tres(el), rr = tres(er);
                    const uint32_t eta = min(rl, rr);
                    if (tside(el) == 0) emit(el, er, eta, k); else emit(er, el, eta, k);
                    if (rl == eta) {
                        if (++pl == rb) lx = true; else el = B(pl);
                    } else {
                        el = tsetres(el, rl - eta);
                    }
                    if (rr == eta) {
                        if (++pr == e) rx = true; else er = B(pr);
                    } else {
                        er = tsetres(er, rr - eta);
                    }
                    if (lx || rx) break;
                }
                if (lx && rx) {
                    fhead[lf] = uint16_t(rb);
                    bend = rb;
                } else if (lx) {
                    B(pr) = er;
                    fhead[lf] = uint16_t(pr);
                } else {
                    B(pl) = el;
                    fhead[lf] = uint16_t(pl);
                    bend = rb;
                }
            }
        }
        --nf;
    }

    // returns the Flowtree value of the pair (meaningless when overflow is set)
    __device__ float run(int64_t pair, int64_t da, int64_t db) {
        ao = c.a_ptr[da];
        bo = c.b_ptr[db];
        const int na = int(c.a_ptr[da + 1] - ao);
        const int nb = int(c.b_ptr[db + 1] - bo);
        if (SAVE) slot = c.slot_ptr[pair];
        const int L = c.levels;
        int i = 0, j = 0;
        uint32_t ra = na > 0 ? c.a_rank[ao] : 0xFFFFFFFFu;
        uint32_t rbk = nb > 0 ? c.b_rank[bo] : 0xFFFFFFFFu;
        uint32_t prev = 0;
        bool first = true;
        while (i < na || j < nb) {
            uint32_t r, m, side;
            uint64_t pay;
            if (i < na && (j >= nb || ra <= rbk)) {
                r = ra;
                m = c.a_mass[ao + i];
                side = 0;
                pay = SAVE ? uint64_t(i) : uint64_t(c.a_word[ao + i]);
                ++i;
                ra = i < na ? c.a_rank[ao + i] : 0xFFFFFFFFu;
            } else {
                r = rbk;
                m = c.b_mass[bo + j];
                side = 1;
                pay = SAVE ? uint64_t(j) : uint64_t(c.b_word[bo + j]);
                ++j;
                rbk = j < nb ? c.b_rank[bo + j] : 0xFFFFFFFFu;
            }
            int g = -1;
            if (!first) g = (r == prev) ? L + 1 : lca_ranks(tb, c.n_points, prev, r);
            first = false;
            prev = r;
            while (nf >= 2 && int(fgap[nf - 1]) - 1 > g) merge_top(int(fgap[nf - 1]) - 1);
            if (nf >= 2 && int(fgap[nf - 1]) - 1 == g) merge_top(g);
            if (bend >= cap) {  // the buffer is full: leave this pair to the warp kernel
                overflow = true;
                return 0.0f;
            }
            fgap[nf] = uint8_t(g + 1);  // stored biased by one (the first frame has gap -1)
            fbeg[nf] = uint16_t(bend);
            fhead[nf] = uint16_t(bend);
            ++nf;
            B(bend++) = tentry(m, side, pay);
        }
        while (nf >= 2) merge_top(int(fgap[nf - 1]) - 1);
        if (SAVE) c.count[pair] = saved;
        return acc.value() * (1.0f / 16777216.0f);
    }
};

}  // namespace ftk
