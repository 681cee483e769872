// Batched Flowtree forward: persistent launch, plain per-pair launch, saved
// flows, launch planning and autotuning.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ft_flow.cuh"
#include "ft_flow_blocked.cuh"
#include "ft_flow_team.cuh"
#include "ft_flow_thread.cuh"

using namespace ftk;

namespace {

constexpr int kDefaultWarps = 4;
constexpr int kMaxStage = 2048;
constexpr int kBlockedCap = 32 * 31;   // longest pair of a warp of the blocked form (31 items per lane)
constexpr int kWarpCapDefault = 32 * 13; // the warp's default staging when longer pairs go to the team launch

// A warp per pair, persistent: warps take `grab` consecutive queue entries at
// a time.  Dynamic shared memory: [tables (if staged)] [one WarpBuf per warp].
template <int MODE, bool SAVE>
__device__ __forceinline__ void persistent_body(const FlowCtx& c, int cap, int grab, int tables_bytes) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = int(threadIdx.x >> 5);
    const unsigned lane = lane_id();
    const Tables tb = tables_bytes > 0 ? stage_tables(c, smem) : Tables{c.vocab, c.rmq};
    uint8_t* wbase = smem + tables_bytes;
    const WarpBuf sbuf = carve_warpbuf(wbase + size_t(warp) * warpbuf_bytes(cap), cap);
    const int64_t gw = int64_t(blockIdx.x) * (blockDim.x >> 5) + warp;
    WarpBuf gbuf = sbuf;
    if (c.gscratch) gbuf = carve_warpbuf(c.gscratch + size_t(gw) * c.gscratch_warp_bytes, c.gscratch_items);
    const int64_t n_pairs = c.n_pairs;
    for (;;) {
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(reinterpret_cast<unsigned long long*>(c.queue), (unsigned long long)grab);
        first = __shfl_sync(FULL_MASK, first, 0);
        if (first >= (unsigned long long)n_pairs) break;
        const int64_t last = min(int64_t(first) + grab, n_pairs);
        for (int64_t q = int64_t(first); q < last; ++q) {
            const int64_t pair = c.order ? int64_t(c.order[q]) : q;
            int64_t da, db;
            if (!pair_docs(c, pair, &da, &db)) {
                if (lane == 0) c.cost_out[pair] = __int_as_float(0x7fc00000);
                continue;
            }
            const int n = int(c.a_ptr[da + 1] - c.a_ptr[da]) + int(c.b_ptr[db + 1] - c.b_ptr[db]);
            float cost;
            if (n <= cap) {
                cost = flowtree_pair<MODE, SAVE>(c, sbuf, tb, pair, da, db);
            } else if (c.gscratch && n <= c.gscratch_items) {
                cost = flowtree_pair<MODE, SAVE>(c, gbuf, tb, pair, da, db);
            } else {
                if (lane == 0) ft_flag(c.status, FT_DEV_EOVERFLOW);
                cost = __int_as_float(0x7fc00000);
            }
            if (lane == 0) c.cost_out[pair] = cost;
        }
    }
}

// The occupancy build: the compiler keeps registers low enough for many
// resident warps (throughput-bound batches: the row gathers of many pairs
// overlap across warps).
template <int MODE, bool SAVE>
__global__ void __launch_bounds__(256) k_flowtree_persistent(FlowCtx c, int cap, int grab, int tables_bytes) {
    persistent_body<MODE, SAVE>(c, cap, grab, tables_bytes);
}

// The deep-loads build (8-lane-group pricing only): one resident CTA is all
// the compiler must allow, so a warp keeps its pricing rounds' row loads in
// registers together; for batches too small to fill the GPU, whose time is
// the longest pairs' latency on their warps.
template <int MODE, bool SAVE>
__global__ void __launch_bounds__(256, 1) k_flowtree_persistent_deep(FlowCtx c, int cap, int grab, int tables_bytes) {
    persistent_body<MODE, SAVE>(c, cap, grab, tables_bytes);
}

// A warp per pair, register-blocked (ft_flow_blocked.cuh), persistent.
// Dynamic shared memory: [tables (if staged)] [one BlockedBuf per warp].
template <int MODE, bool SAVE, bool PT16>
__global__ void __launch_bounds__(256) k_flowtree_blocked(FlowCtx c, int grab, int cap, int tables_bytes) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = int(threadIdx.x >> 5);
    const unsigned lane = lane_id();
    const Tables tb = tables_bytes > 0 ? stage_tables(c, smem) : Tables{c.vocab, c.rmq};
    constexpr bool META = blocked_has_meta(PT16, SAVE), QUEUE = blocked_has_queue(MODE);
    const BlockedBuf w = carve_blockedbuf(smem + tables_bytes + size_t(warp) * blockedbuf_bytes(cap, PT16, META, QUEUE),
                                          cap, PT16, META, QUEUE);
    const int64_t n_pairs = c.n_pairs;
    for (;;) {
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(reinterpret_cast<unsigned long long*>(c.queue), (unsigned long long)grab);
        first = __shfl_sync(FULL_MASK, first, 0);
        if (first >= (unsigned long long)n_pairs) break;
        const int64_t last = min(int64_t(first) + grab, n_pairs);
        for (int64_t q = int64_t(first); q < last; ++q) {
            const int64_t pair = c.order ? int64_t(c.order[q]) : q;
            int64_t da, db;
            if (!pair_docs(c, pair, &da, &db)) {
                if (lane == 0) c.cost_out[pair] = __int_as_float(0x7fc00000);
                continue;
            }
            const int n = int(c.a_ptr[da + 1] - c.a_ptr[da]) + int(c.b_ptr[db + 1] - c.b_ptr[db]);
            float cost;
            if (n <= cap) {
                cost = flowtree_pair_blocked<MODE, SAVE, PT16>(c, w, tb, pair, da, db);
            } else if (c.long_list) {  // a CTA of the team launch takes it
                if (lane == 0) c.long_list[atomicAdd(c.long_count, 1u)] = uint32_t(pair);
                continue;
            } else {
                if (lane == 0) ft_flag(c.status, FT_DEV_EOVERFLOW);
                cost = __int_as_float(0x7fc00000);
            }
            if (lane == 0) c.cost_out[pair] = cost;
        }
    }
}

// A CTA per pair (ft_flow_team.cuh) for the pairs the blocked warp form
// listed as too long for its staging; persistent over that list.  Dynamic
// shared memory: [tables (if staged)] [TeamBuf].
template <int MODE, bool SAVE>
__global__ void __launch_bounds__(kTeamThreads) k_flowtree_team(FlowCtx c, unsigned int* team_queue, int cap,
                                                                int tables_bytes) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ TeamScratch ts;
    const Tables tb = tables_bytes > 0 ? stage_tables(c, smem) : Tables{c.vocab, c.rmq};
    const TeamBuf w = carve_teambuf(smem + tables_bytes, cap);
    const unsigned n_long = *c.long_count;
    for (;;) {
        if (threadIdx.x == 0) ts.pair = atomicAdd(team_queue, 1u);
        __syncthreads();
        const unsigned q = unsigned(ts.pair);
        __syncthreads();
        if (q >= n_long) break;
        const int64_t pair = int64_t(c.long_list[q]);
        int64_t da, db;
        if (!pair_docs(c, pair, &da, &db)) {  // cannot happen: the warp form checked the pair
            if (threadIdx.x == 0) c.cost_out[pair] = __int_as_float(0x7fc00000);
            continue;
        }
        const int n = int(c.a_ptr[da + 1] - c.a_ptr[da]) + int(c.b_ptr[db + 1] - c.b_ptr[db]);
        float cost;
        if (n <= cap) {
            cost = flowtree_pair_team<MODE, SAVE>(c, w, ts, tb, pair, da, db);
        } else {
            if (threadIdx.x == 0) ft_flag(c.status, FT_DEV_EOVERFLOW);
            cost = __int_as_float(0x7fc00000);
        }
        if (threadIdx.x == 0) c.cost_out[pair] = cost;
    }
}

// A thread per pair (low-dimensional ground sets).  The vocabulary and the
// LCA table are copied to shared memory when they fit.  Every lane runs the
// sweep of its own pair one state-machine step per iteration; a lane whose
// pair is done takes the next queue entry (one atomic per warp and
// iteration).  Dynamic shared memory: [tables (if staged)]
// [warps][lane_words(nmax)][32] uint32; gres: nmax residual words per thread.
template <bool SAVE>
__global__ void __launch_bounds__(256) k_flowtree_thread(const __grid_constant__ FlowCtx c, int W, int tables_bytes,
                                                         uint32_t* gres, int nmax) {
    extern __shared__ __align__(16) uint8_t smem[];
    const Tables tb = tables_bytes > 0 ? stage_tables(c, smem) : Tables{c.vocab, c.rmq};
    const unsigned lane = lane_id();
    const int words = 4 * W + 1 + 2 * kLaneFrames;
    uint32_t* base = reinterpret_cast<uint32_t*>(smem + tables_bytes) + size_t(threadIdx.x >> 5) * words * 32 + lane;
    const int64_t gt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    LaneSweep<SAVE> sw(c, tb, base, W, gres + size_t(gt) * nmax);
    int64_t pair = -1;
    bool active = false, drained = false;
    for (;;) {
        const unsigned need = __ballot_sync(FULL_MASK, !active);
        if (need && !drained) {
            const int leader = __ffs(need) - 1;
            unsigned long long first = 0;
            if (int(lane) == leader)
                first = atomicAdd(reinterpret_cast<unsigned long long*>(c.queue), (unsigned long long)__popc(need));
            first = __shfl_sync(FULL_MASK, first, leader);
            if (first + __popc(need) >= (unsigned long long)c.n_pairs) drained = true;
            if (!active) {
                const int64_t q = int64_t(first) + __popc(need & lanemask_lt());
                if (q < c.n_pairs) {
                    pair = c.order ? int64_t(c.order[q]) : q;
                    int64_t da, db;
                    if (c.pair_a) {
                        da = c.pair_a[pair];
                        db = c.pair_b[pair];
                    } else {
                        da = pair / c.nb_cross;
                        db = pair - da * c.nb_cross;
                    }
                    if (da < 0 || da >= c.na_docs || db < 0 || db >= c.nb_docs) {
                        ft_flag(c.status, FT_DEV_EINVAL);
                        c.cost_out[pair] = __int_as_float(0x7fc00000);
                    } else {
                        sw.start(pair, da, db);
                        active = true;
                    }
                }
            }
        }
        if (!__any_sync(FULL_MASK, active) && drained) break;
        if (active) {
            sw.step();
            if (sw.phase == LP_DONE) {
                c.cost_out[pair] = sw.P.acc.value() * (1.0f / 16777216.0f);
                if (SAVE) c.count[pair] = sw.P.saved;
                active = false;
            }
        }
    }
}

// The plain form: one warp, one pair per launch.
template <int MODE>
__global__ void __launch_bounds__(32) k_flowtree_one(FlowCtx c, int cap, int64_t pair) {
    extern __shared__ __align__(16) uint8_t smem[];
    const WarpBuf sbuf = carve_warpbuf(smem, cap);
    const Tables tb{c.vocab, c.rmq};
    int64_t da, db;
    if (!pair_docs(c, pair, &da, &db)) {
        if (lane_id() == 0) c.cost_out[pair] = __int_as_float(0x7fc00000);
        return;
    }
    const int n = int(c.a_ptr[da + 1] - c.a_ptr[da]) + int(c.b_ptr[db + 1] - c.b_ptr[db]);
    float cost;
    if (n <= cap) {
        cost = flowtree_pair<MODE, false>(c, sbuf, tb, pair, da, db);
    } else if (c.gscratch && n <= c.gscratch_items) {
        const WarpBuf gbuf = carve_warpbuf(c.gscratch, c.gscratch_items);
        cost = flowtree_pair<MODE, false>(c, gbuf, tb, pair, da, db);
    } else {
        if (lane_id() == 0) ft_flag(c.status, FT_DEV_EOVERFLOW);
        cost = __int_as_float(0x7fc00000);
    }
    if (lane_id() == 0) c.cost_out[pair] = cost;
}

// key = 0xFFFF - min(n, 0xFFFF): ascending key = longest pair first
__global__ void k_pair_len_key(const int64_t* __restrict__ a_ptr, const int64_t* __restrict__ b_ptr,
                               const int32_t* __restrict__ pa, const int32_t* __restrict__ pb, int64_t n_pairs,
                               int64_t na_docs, int64_t nb_docs, uint32_t* __restrict__ key, uint32_t* status) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_pairs; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t da = pa[i], db = pb[i];
        uint32_t n = 0;
        if (da < 0 || da >= na_docs || db < 0 || db >= nb_docs) {
            ft_flag(status, FT_DEV_EINVAL);
        } else {
            n = uint32_t((a_ptr[da + 1] - a_ptr[da]) + (b_ptr[db + 1] - b_ptr[db]));
        }
        key[i] = 0xFFFFu - min(n, 0xFFFFu);
    }
}

__global__ void k_slot_len(const int64_t* __restrict__ a_ptr, const int64_t* __restrict__ b_ptr,
                           const int32_t* __restrict__ pa, const int32_t* __restrict__ pb, int64_t n_pairs,
                           int64_t nb_cross, int64_t na_docs, int64_t nb_docs, int64_t* __restrict__ len,
                           uint32_t* status) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_pairs; i += int64_t(gridDim.x) * blockDim.x) {
        int64_t da, db;
        if (pa) {
            da = pa[i];
            db = pb[i];
        } else {
            da = i / nb_cross;
            db = i - da * nb_cross;
        }
        if (da < 0 || da >= na_docs || db < 0 || db >= nb_docs) {
            ft_flag(status, FT_DEV_EINVAL);
            len[i] = 0;
        } else {
            len[i] = (a_ptr[da + 1] - a_ptr[da]) + (b_ptr[db + 1] - b_ptr[db]);
        }
    }
}

int grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535 * 8) b = 65535 * 8;
    return int(b);
}

int round32(int x) { return (x + 31) & ~31; }

struct Plan {
    int algo = FT_ALGO_WARP;
    int mode = 0;
    int warps = kDefaultWarps;
    int cap = 0;
    int blocks = 0;
    size_t smem = 0;
    int gscratch_items = 0;
    size_t gscratch_warp_bytes = 0;
    bool need_order = false;
    int64_t n_pairs = 0;
    int tables_bytes = 0;  // vocabulary + LCA table staged in shared memory (0 = read from global)
    bool deep = false;     // warp form: the deep-loads build
    void* kernel = nullptr;  // blocked form: the instantiation to launch
    // blocked form, pairs longer than the warp's staging: a CTA per pair
    int team_cap = 0;        // 0: no team launch
    size_t team_smem = 0;
    int team_blocks = 0;
    void* team_kernel = nullptr;
    // thread algorithm: the lane-per-pair launch; cap, warps, blocks, smem
    // above then describe the warp-per-pair launch for its overflow pairs
    int tw = 0;            // words per bit array of a lane (positions up to the longest pair)
    int tmaxn = 0;         // positions per thread (the longest pair)
    int twarps = 0;
    int tblocks = 0;
    size_t tsmem = 0;
};

constexpr int kThreadMaxItems = 8192;
constexpr size_t kTablesMax = 32 * 1024;  // stage the tables when they are at most this big

int staged_tables_bytes(const ft_tree* t) {
    const size_t b = (tables_bytes(t->n, t->dim, t->rmq_levels) + 127) & ~size_t(127);
    return b <= kTablesMax ? int(b) : 0;
}

void* thread_kernel(bool save) {
    return save ? reinterpret_cast<void*>(&k_flowtree_thread<true>)
                : reinterpret_cast<void*>(&k_flowtree_thread<false>);
}

template <int MODE, bool SAVE>
void* persistent_fn() {
    return reinterpret_cast<void*>(&k_flowtree_persistent<MODE, SAVE>);
}

template <bool PT16>
void* blocked_fn(int mode, bool save) {
    switch (mode * 2 + (save ? 1 : 0)) {
        case 0: return reinterpret_cast<void*>(&k_flowtree_blocked<0, false, PT16>);
        case 1: return reinterpret_cast<void*>(&k_flowtree_blocked<0, true, PT16>);
        case 2: return reinterpret_cast<void*>(&k_flowtree_blocked<1, false, PT16>);
        case 3: return reinterpret_cast<void*>(&k_flowtree_blocked<1, true, PT16>);
        case 4: return reinterpret_cast<void*>(&k_flowtree_blocked<2, false, PT16>);
        default: return reinterpret_cast<void*>(&k_flowtree_blocked<2, true, PT16>);
    }
}

// 16-bit point ids per merged position when the ground set allows
bool blocked_pt16(const ft_tree* t) { return t->n <= 65536; }

void* blocked_kernel(const ft_tree* t, int mode, bool save) {
    return blocked_pt16(t) ? blocked_fn<true>(mode, save) : blocked_fn<false>(mode, save);
}

void* team_kernel(int mode, bool save) {
    switch (mode * 2 + (save ? 1 : 0)) {
        case 0: return reinterpret_cast<void*>(&k_flowtree_team<0, false>);
        case 1: return reinterpret_cast<void*>(&k_flowtree_team<0, true>);
        case 2: return reinterpret_cast<void*>(&k_flowtree_team<1, false>);
        case 3: return reinterpret_cast<void*>(&k_flowtree_team<1, true>);
        case 4: return reinterpret_cast<void*>(&k_flowtree_team<2, false>);
        default: return reinterpret_cast<void*>(&k_flowtree_team<2, true>);
    }
}

void* persistent_kernel(int mode, bool save, bool deep) {
    if (deep && mode >= 1) {
        switch ((mode - 1) * 2 + (save ? 1 : 0)) {
            case 0: return reinterpret_cast<void*>(&k_flowtree_persistent_deep<1, false>);
            case 1: return reinterpret_cast<void*>(&k_flowtree_persistent_deep<1, true>);
            case 2: return reinterpret_cast<void*>(&k_flowtree_persistent_deep<2, false>);
            default: return reinterpret_cast<void*>(&k_flowtree_persistent_deep<2, true>);
        }
    }
    switch (mode * 2 + (save ? 1 : 0)) {
        case 0: return persistent_fn<0, false>();
        case 1: return persistent_fn<0, true>();
        case 2: return persistent_fn<1, false>();
        case 3: return persistent_fn<1, true>();
        case 4: return persistent_fn<2, false>();
        default: return persistent_fn<2, true>();
    }
}

int pick_mode(const ft_tree* t, const float* vocab) {
    if (t->dim <= 8) return 0;
    if ((t->dim % 4) == 0 && (reinterpret_cast<uintptr_t>(vocab) % 16) == 0) return 1;
    return 2;
}

ft_status make_plan_algo(const ft_tree* t, const ft_docs* a, const ft_docs* b, int64_t n_pairs, int mode, bool save,
                         bool explicit_pairs, const ft_flowtree_config& cfg, Plan* p) {
    p->mode = mode;
    p->n_pairs = n_pairs;
    p->warps = cfg.warps_per_cta > 0 ? cfg.warps_per_cta : kDefaultWarps;
    const int maxn = round32(std::max(a->max_support + b->max_support, 32));
    p->need_order = explicit_pairs && n_pairs > 1;
    const bool thread_ok = t->dim <= 8 && maxn <= kThreadMaxItems;
    p->algo = cfg.algo;
    int dev = 0, max_smem = 0, sms = 0;
    FT_CUDA(cudaGetDevice(&dev));
    FT_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    FT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    p->tables_bytes = cfg.stage_tables ? staged_tables_bytes(t) : 0;
    if (p->algo == FT_ALGO_THREAD) {
        if (!thread_ok) return FT_EUNSUPPORTED;
        p->tw = (maxn + 31) / 32;
        p->tmaxn = maxn;
        const size_t per_warp = size_t(lane_words(maxn)) * 32 * 4;
        p->twarps = cfg.warps_per_cta > 0 ? cfg.warps_per_cta : 4;
        p->tsmem = size_t(p->tables_bytes) + size_t(p->twarps) * per_warp;
        if (p->tsmem > size_t(max_smem)) return FT_EUNSUPPORTED;
        int bps = 0;
        FT_TRY(ft_prepare_kernel(thread_kernel(save), p->twarps * 32, p->tsmem, &bps));
        if (bps < 1) return FT_EUNSUPPORTED;
        // resident blocks, but no more threads than pairs (each thread owns a
        // slice of residual words in the workspace)
        const int64_t need_blocks = (std::max<int64_t>(n_pairs, 1) + p->twarps * 32 - 1) / (p->twarps * 32);
        p->tblocks = int(std::min<int64_t>(int64_t(sms) * bps, need_blocks));
        return FT_OK;
    }
    if (p->algo == FT_ALGO_BLOCKED) {
        // the warp's staging: an odd number of items per lane, at most what the
        // longest pair needs; by default 13 per lane (pairs up to 416 items),
        // longer pairs go to a CTA each
        const int need = 32 * ((maxn / 32) | 1);
        int capw = cfg.stage_items > 0 ? 32 * (((cfg.stage_items + 31) / 32) | 1) : std::min(need, kWarpCapDefault);
        capw = std::min(std::min(capw, need), kBlockedCap);
        p->cap = capw;
        p->smem = size_t(p->tables_bytes) +
                  size_t(p->warps) * blockedbuf_bytes(p->cap, blocked_pt16(t), blocked_has_meta(blocked_pt16(t), save),
                                                      blocked_has_queue(mode));
        if (p->smem > size_t(max_smem)) return FT_EUNSUPPORTED;
        int bps = 0;
        p->kernel = blocked_kernel(t, mode, save);
        FT_TRY(ft_prepare_kernel(p->kernel, p->warps * 32, p->smem, &bps));
        if (bps < 1) return FT_EUNSUPPORTED;
        p->blocks = sms * bps;
        if (maxn > capw) {
            p->team_cap = kTeamThreads * (((maxn + kTeamThreads - 1) / kTeamThreads) | 1);
            p->team_smem = size_t(p->tables_bytes) + teambuf_bytes(p->team_cap);
            if (p->team_smem + sizeof(TeamScratch) > size_t(max_smem)) return FT_EUNSUPPORTED;
            p->team_kernel = team_kernel(mode, save);
            int tbps = 0;
            FT_TRY(ft_prepare_kernel(p->team_kernel, kTeamThreads, p->team_smem, &tbps));
            if (tbps < 1) return FT_EUNSUPPORTED;
            p->team_blocks = sms * tbps;
        }
        return FT_OK;
    }
    int cap = cfg.stage_items > 0 ? round32(cfg.stage_items) : std::min(maxn, 512);
    cap = std::min(cap, kMaxStage);
    p->cap = cap;
    p->smem = size_t(p->tables_bytes) + size_t(p->warps) * warpbuf_bytes(cap);
    if (p->smem > size_t(max_smem)) return FT_EUNSUPPORTED;
    p->deep = cfg.deep_loads != 0 && mode >= 1;
    void* fn = persistent_kernel(mode, save, p->deep);
    int bps = 0;
    FT_TRY(ft_prepare_kernel(fn, p->warps * 32, p->smem, &bps));
    if (bps < 1) return FT_EUNSUPPORTED;
    p->blocks = sms * bps;
    if (maxn > cap) {
        p->gscratch_items = maxn;
        p->gscratch_warp_bytes = (warpbuf_bytes(maxn) + 255) & ~size_t(255);
    }
    return FT_OK;
}

// AUTO: the blocked form (warp per pair, with a CTA per pair beyond the
// warp's staging) when the device can hold its buffers, else the compacting
// warp form.
ft_status make_plan(const ft_tree* t, const ft_docs* a, const ft_docs* b, int64_t n_pairs, int mode, bool save,
                    bool explicit_pairs, const ft_flowtree_config& cfg, Plan* p) {
    if (cfg.algo != FT_ALGO_AUTO) return make_plan_algo(t, a, b, n_pairs, mode, save, explicit_pairs, cfg, p);
    ft_flowtree_config c2 = cfg;
    c2.algo = FT_ALGO_BLOCKED;
    const ft_status st = make_plan_algo(t, a, b, n_pairs, mode, save, explicit_pairs, c2, p);
    if (st != FT_EUNSUPPORTED) return st;
    *p = Plan();
    c2.algo = FT_ALGO_WARP;
    return make_plan_algo(t, a, b, n_pairs, mode, save, explicit_pairs, c2, p);
}

struct WsLayout {
    unsigned int* queue;  // [0..1] pair counter, [2] long pairs listed, [3] long pairs taken
    uint32_t* long_list;  // blocked form with a team launch: [n_pairs]
    uint32_t* gres;       // thread algorithm: residuals of partly matched items, per thread
    uint32_t* order;
    uint32_t* keys;
    void* sort_tmp;
    uint8_t* gscratch;
};

size_t layout(const Plan& p, void* base, WsLayout* out) {
    WsCarver w(base);
    WsLayout l{};
    l.queue = w.take<unsigned int>(4);
    if (p.algo == FT_ALGO_THREAD) l.gres = w.take<uint32_t>(size_t(p.tblocks) * p.twarps * 32 * p.tmaxn);
    if (p.team_cap > 0) l.long_list = w.take<uint32_t>(size_t(p.n_pairs));
    if (p.need_order) {
        l.order = w.take<uint32_t>(size_t(p.n_pairs));
        l.keys = w.take<uint32_t>(size_t(p.n_pairs));
        l.sort_tmp = w.take<uint8_t>(ft_sort_tmp_bytes(p.n_pairs));
    }
    if (p.gscratch_items > 0)
        l.gscratch = w.take<uint8_t>(size_t(p.blocks) * p.warps * p.gscratch_warp_bytes);
    if (out) *out = l;
    return w.off + 256;
}

ft_status check_common(const ft_tree* t, const float* vocab, const ft_docs* a, const ft_docs* b,
                       const int32_t* pa, const int32_t* pb, int64_t n_pairs, const float* cost_out) {
    if (!t || !vocab || !a || !b || !cost_out || n_pairs < 0) return FT_EINVAL;
    if (a->tree != t || b->tree != t) return FT_EINVAL;
    if ((pa == nullptr) != (pb == nullptr)) return FT_EINVAL;
    if (!pa && n_pairs != a->n_docs * b->n_docs) return FT_EINVAL;
    if (n_pairs >= (int64_t(1) << 32)) return FT_EUNSUPPORTED;
    return FT_OK;
}

FlowCtx make_ctx(const ft_tree* t, const float* vocab, const ft_docs* a, const ft_docs* b, const int32_t* pa,
                 const int32_t* pb, int64_t n_pairs, float* cost_out) {
    FlowCtx c{};
    c.rmq = t->d_rmq;
    c.n_points = t->n;
    c.levels = t->levels;
    c.rmq_levels = t->rmq_levels;
    c.vocab = vocab;
    c.dim = t->dim;
    c.a_ptr = a->d_ptr;
    c.a_rank = a->d_rank;
    c.a_mass = a->d_mass;
    c.a_word = a->d_word;
    c.b_ptr = b->d_ptr;
    c.b_rank = b->d_rank;
    c.b_mass = b->d_mass;
    c.b_word = b->d_word;
    c.pair_a = pa;
    c.pair_b = pb;
    c.nb_cross = b->n_docs;
    c.n_pairs = n_pairs;
    c.na_docs = a->n_docs;
    c.nb_docs = b->n_docs;
    c.cost_out = cost_out;
    c.status = t->d_status;
    return c;
}

ft_status launch_warps(const Plan& p, const FlowCtx& c, bool save, cudaStream_t s) {
    const int64_t n_warps = int64_t(p.blocks) * p.warps;
    int64_t grab = c.n_pairs / (n_warps * 32);
    grab = std::max<int64_t>(1, std::min<int64_t>(grab, 16));
    FlowCtx cc = c;
    int cap = p.cap, g = int(grab), tbytes = p.tables_bytes;
    if (p.algo == FT_ALGO_BLOCKED) {
        void* args[] = {&cc, &g, &cap, &tbytes};
        FT_CUDA(cudaLaunchKernel(p.kernel, dim3(p.blocks), dim3(p.warps * 32), args, p.smem, s));
        if (p.team_cap > 0) {
            unsigned int* tq = c.queue + 3;
            int tcap = p.team_cap;
            void* targs[] = {&cc, &tq, &tcap, &tbytes};
            FT_CUDA(cudaLaunchKernel(p.team_kernel, dim3(p.team_blocks), dim3(kTeamThreads), targs, p.team_smem, s));
        }
        return FT_OK;
    }
    void* fn = persistent_kernel(p.mode, save, p.deep);
    void* args[] = {&cc, &cap, &g, &tbytes};
    FT_CUDA(cudaLaunchKernel(fn, dim3(p.blocks), dim3(p.warps * 32), args, p.smem, s));
    return FT_OK;
}

ft_status launch_persistent(const Plan& p, const WsLayout& l, FlowCtx c, bool save, cudaStream_t s) {
    FT_CUDA(cudaMemsetAsync(c.queue, 0, 16, s));
    if (p.algo != FT_ALGO_THREAD) return launch_warps(p, c, save, s);
    void* fn = thread_kernel(save);
    int tw = p.tw, tbytes = p.tables_bytes, nmax = p.tmaxn;
    uint32_t* gres = l.gres;
    void* args[] = {&c, &tw, &tbytes, &gres, &nmax};
    FT_CUDA(cudaLaunchKernel(fn, dim3(p.tblocks), dim3(p.twarps * 32), args, p.tsmem, s));
    return FT_OK;
}

ft_status run_batch(const ft_tree* t, const float* vocab, const ft_docs* a, const ft_docs* b, const int32_t* pa,
                    const int32_t* pb, int64_t n_pairs, float* cost_out, ft_flows* flows, void* ws, size_t ws_bytes,
                    cudaStream_t s, const ft_flowtree_config& cfg) {
    FT_TRY(check_common(t, vocab, a, b, pa, pb, n_pairs, cost_out));
    if (flows && (flows->n_pairs != n_pairs)) return FT_EINVAL;
    if (n_pairs == 0) return FT_OK;
    Plan p;
    const bool save = flows != nullptr;
    FT_TRY(make_plan(t, a, b, n_pairs, pick_mode(t, vocab), save, pa != nullptr, cfg, &p));
    const size_t need = layout(p, nullptr, nullptr);
    if (!ws || ws_bytes < need) return FT_EWORKSPACE;
    WsLayout l;
    layout(p, ws, &l);
    FlowCtx c = make_ctx(t, vocab, a, b, pa, pb, n_pairs, cost_out);
    c.queue = l.queue;
    c.gscratch = l.gscratch;
    if (p.team_cap > 0) {
        c.long_list = l.long_list;
        c.long_count = l.queue + 2;
    }
    c.gscratch_items = p.gscratch_items;
    c.gscratch_warp_bytes = p.gscratch_warp_bytes;
    if (p.need_order) {
        k_pair_len_key<<<grid_for(n_pairs, 256), 256, 0, s>>>(a->d_ptr, b->d_ptr, pa, pb, n_pairs, a->n_docs,
                                                             b->n_docs, l.keys, t->d_status);
        FT_TRY(ft_iota_u32(l.order, n_pairs, s));
        FT_TRY(ft_sort_perm_by_u32(l.keys, l.order, n_pairs, 16, l.sort_tmp, s));
        c.order = l.order;
    }
    if (save) {
        c.slot_ptr = flows->d_slot_ptr;
        c.count = flows->d_count;
        c.f_ia = flows->d_ia;
        c.f_ib = flows->d_ib;
        c.f_f = flows->d_f;
        c.f_depth = flows->d_depth;
        c.f_dist = flows->d_dist;
    }
    return launch_persistent(p, l, c, save, s);
}

template <class T>
ft_status dmalloc(T** p, size_t count) {
    if (count == 0) count = 1;
    if (cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return FT_ENOMEM;
    }
    return FT_OK;
}

void free_flows(ft_flows* f) {
    if (!f) return;
    cudaFree(f->d_pair_a);
    cudaFree(f->d_pair_b);
    cudaFree(f->d_slot_ptr);
    cudaFree(f->d_count);
    cudaFree(f->d_ia);
    cudaFree(f->d_ib);
    cudaFree(f->d_f);
    cudaFree(f->d_depth);
    cudaFree(f->d_dist);
    cudaFree(f->d_scan_tmp);
    delete f;
}

}  // namespace

// Workspace of the launch ft_flowtree_batch would make for these arguments
// without saved flows (the plan it runs: cross product or explicit pairs, the
// pricing mode of this vocabulary); the plan's own status on failure.
ft_status ft_flowtree_batch_need(const ft_tree* t, const float* vocab, const ft_docs* a, const ft_docs* b,
                                 const int32_t* pa, const int32_t* pb, int64_t n_pairs, size_t* need) {
    *need = 0;
    FT_TRY(check_common(t, vocab, a, b, pa, pb, n_pairs, vocab));
    if (n_pairs == 0) return FT_OK;
    Plan p;
    FT_TRY(make_plan(t, a, b, n_pairs, pick_mode(t, vocab), false, pa != nullptr, t->cfg, &p));
    *need = layout(p, nullptr, nullptr);
    return FT_OK;
}

extern "C" size_t ft_flowtree_batch_workspace_size(const ft_tree* t, const ft_docs* a, const ft_docs* b,
                                                   int64_t n_pairs) {
    if (!t || !a || !b || n_pairs < 0) return 0;
    Plan p;
    // the saving and non-saving kernels have the same footprint; size for the
    // explicit-pair case (a superset of the cross-product case)
    if (make_plan(t, a, b, n_pairs, 0, false, true, t->cfg, &p) != FT_OK) return 0;
    Plan p1 = p;
    if (t->dim > 8 && make_plan(t, a, b, n_pairs, 1, false, true, t->cfg, &p1) != FT_OK) return 0;
    Plan p2 = p;
    if (t->dim > 8 && make_plan(t, a, b, n_pairs, 2, true, true, t->cfg, &p2) != FT_OK) return 0;
    return std::max(layout(p, nullptr, nullptr), std::max(layout(p1, nullptr, nullptr), layout(p2, nullptr, nullptr)));
}

extern "C" ft_status ft_flowtree_batch(const ft_tree* t, const float* vocab_dev, const ft_docs* a, const ft_docs* b,
                                       const int32_t* pair_a_dev, const int32_t* pair_b_dev, int64_t n_pairs,
                                       float* cost_out_dev, ft_flows* flows_out, void* workspace, size_t ws_bytes,
                                       void* stream) {
    if (!t) return FT_EINVAL;
    return run_batch(t, vocab_dev, a, b, pair_a_dev, pair_b_dev, n_pairs, cost_out_dev, flows_out, workspace,
                     ws_bytes, static_cast<cudaStream_t>(stream), t->cfg);
}

extern "C" ft_status ft_flowtree_plain(const ft_tree* t, const float* vocab_dev, const ft_docs* a, const ft_docs* b,
                                       const int32_t* pair_a_dev, const int32_t* pair_b_dev, int64_t n_pairs,
                                       float* cost_out_dev, void* workspace, size_t ws_bytes, void* stream) {
    FT_TRY(check_common(t, vocab_dev, a, b, pair_a_dev, pair_b_dev, n_pairs, cost_out_dev));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int mode = pick_mode(t, vocab_dev);
    const int maxn = round32(std::max(a->max_support + b->max_support, 32));
    const int cap = std::min(maxn, kMaxStage);
    const size_t smem = warpbuf_bytes(cap);
    FlowCtx c = make_ctx(t, vocab_dev, a, b, pair_a_dev, pair_b_dev, n_pairs, cost_out_dev);
    if (maxn > cap) {
        const size_t need = (warpbuf_bytes(maxn) + 255) & ~size_t(255);
        if (!workspace || ws_bytes < need) return FT_EWORKSPACE;
        c.gscratch = static_cast<uint8_t*>(workspace);
        c.gscratch_items = maxn;
        c.gscratch_warp_bytes = need;
    }
    void* fn = mode == 0 ? reinterpret_cast<void*>(&k_flowtree_one<0>)
                         : (mode == 1 ? reinterpret_cast<void*>(&k_flowtree_one<1>)
                                      : reinterpret_cast<void*>(&k_flowtree_one<2>));
    int bps = 0;
    FT_TRY(ft_prepare_kernel(fn, 32, smem, &bps));
    if (bps < 1) return FT_EUNSUPPORTED;
    for (int64_t i = 0; i < n_pairs; ++i) {
        int cap_arg = cap;
        int64_t pair = i;
        void* args[] = {&c, &cap_arg, &pair};
        FT_CUDA(cudaLaunchKernel(fn, dim3(1), dim3(32), args, smem, s));
    }
    return FT_OK;
}

extern "C" ft_status ft_flowtree_autotune(ft_tree* t, const float* vocab_dev, const ft_docs* a, const ft_docs* b,
                                          const int32_t* pair_a_dev, const int32_t* pair_b_dev, int64_t n_pairs,
                                          float* cost_scratch_dev, void* workspace, size_t ws_bytes, void* stream,
                                          ft_flowtree_config* chosen) {
    FT_TRY(check_common(t, vocab_dev, a, b, pair_a_dev, pair_b_dev, n_pairs, cost_scratch_dev));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int maxn = round32(std::max(a->max_support + b->max_support, 32));
    std::vector<ft_flowtree_config> cands;
    const int caps[] = {maxn, 256, 384, 512, 768, 1024};
    const int warps[] = {3, 4, 5, 6, 7, 8};
    for (int cap : caps) {
        if (cap > maxn || cap > kMaxStage) continue;
        for (int w : warps)
            for (int st : {0, 1}) cands.push_back({w, cap, FT_ALGO_WARP, st, 0});
        if (t->dim > 8)  // the deep-loads build (8-lane-group pricing)
            for (int w : {2, 4, 7}) cands.push_back({w, cap, FT_ALGO_WARP, 0, 1});
    }
    // smaller stagings: more resident warps and a larger L1, longer pairs from the workspace
    for (int cap : {128, 160, 192, 224}) {
        if (cap >= maxn) continue;
        for (int w : {2, 4, 6}) cands.push_back({w, cap, FT_ALGO_WARP, 0, 0});
    }
    // the blocked form: warps per CTA x the warp's staging (0 = default; longer pairs take a CTA each)
    for (int w : {2, 3, 4, 6, 8}) {
        for (int st : {0, 1}) cands.push_back({w, 0, FT_ALGO_BLOCKED, st, 0});
        for (int stage : {224, 352, 480, 608})
            if (stage < maxn) cands.push_back({w, stage, FT_ALGO_BLOCKED, 0, 0});
    }
    if (t->dim <= 8 && maxn <= kThreadMaxItems) {
        // lane per pair: warps per block x item buffer entries per lane
        for (int w : {2, 4, 8}) cands.push_back({w, 0, FT_ALGO_THREAD, 0, 0});
    }
    if (cands.empty()) cands.push_back({kDefaultWarps, std::min(maxn, 512), FT_ALGO_WARP, 0, 0});
    cudaEvent_t e0, e1;
    FT_CUDA(cudaEventCreate(&e0));
    FT_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    ft_flowtree_config best_cfg = cands[0];
    for (const auto& cfg : cands) {
        Plan p;
        if (make_plan(t, a, b, n_pairs, pick_mode(t, vocab_dev), false, pair_a_dev != nullptr, cfg, &p) != FT_OK)
            continue;
        if (layout(p, nullptr, nullptr) > ws_bytes) continue;
        // warm-up, then one timed run
        ft_status st = run_batch(t, vocab_dev, a, b, pair_a_dev, pair_b_dev, n_pairs, cost_scratch_dev, nullptr,
                                 workspace, ws_bytes, s, cfg);
        if (st != FT_OK) continue;
        FT_CUDA(cudaEventRecord(e0, s));
        FT_TRY(run_batch(t, vocab_dev, a, b, pair_a_dev, pair_b_dev, n_pairs, cost_scratch_dev, nullptr, workspace,
                         ws_bytes, s, cfg));
        FT_CUDA(cudaEventRecord(e1, s));
        FT_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        FT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
            best = ms;
            best_cfg = cfg;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    t->cfg = best_cfg;
    if (chosen) *chosen = best_cfg;
    return FT_OK;
}

extern "C" ft_status ft_flows_create(const ft_tree* t, const ft_docs* a, const ft_docs* b, const int32_t* pair_a_dev,
                                     const int32_t* pair_b_dev, int64_t n_pairs, void* stream, ft_flows** out) {
    if (!out) return FT_EINVAL;
    *out = nullptr;
    if (!t || !a || !b || n_pairs < 0 || a->tree != t || b->tree != t) return FT_EINVAL;
    if ((pair_a_dev == nullptr) != (pair_b_dev == nullptr)) return FT_EINVAL;
    if (!pair_a_dev && n_pairs != a->n_docs * b->n_docs) return FT_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ft_flows* f = new ft_flows;
    f->n_pairs = n_pairs;
    f->cross = pair_a_dev == nullptr;
    f->nb_cross = b->n_docs;
    auto fail = [&](ft_status st) {
        free_flows(f);
        return st;
    };
    ft_status st;
    if (pair_a_dev) {
        if ((st = dmalloc(&f->d_pair_a, size_t(n_pairs))) != FT_OK) return fail(st);
        if ((st = dmalloc(&f->d_pair_b, size_t(n_pairs))) != FT_OK) return fail(st);
        if (cudaMemcpyAsync(f->d_pair_a, pair_a_dev, size_t(n_pairs) * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(f->d_pair_b, pair_b_dev, size_t(n_pairs) * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return fail(FT_ECUDA);
    }
    if ((st = dmalloc(&f->d_slot_ptr, size_t(n_pairs) + 1)) != FT_OK) return fail(st);
    if ((st = dmalloc(&f->d_count, size_t(n_pairs))) != FT_OK) return fail(st);
    int64_t* scan_tmp = nullptr;
    if ((st = dmalloc(&scan_tmp, ft_scan_tmp_elems(n_pairs + 1))) != FT_OK) return fail(st);
    k_slot_len<<<grid_for(std::max<int64_t>(n_pairs, 1), 256), 256, 0, s>>>(
        a->d_ptr, b->d_ptr, pair_a_dev, pair_b_dev, n_pairs, b->n_docs, a->n_docs, b->n_docs, f->d_slot_ptr,
        t->d_status);
    cudaMemsetAsync(f->d_slot_ptr + n_pairs, 0, 8, s);
    st = ft_exclusive_scan_i64(f->d_slot_ptr, f->d_slot_ptr, n_pairs + 1, scan_tmp, s);
    int64_t cap = 0;
    cudaMemcpyAsync(&cap, f->d_slot_ptr + n_pairs, 8, cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(scan_tmp);
    if (st != FT_OK) return fail(st);
    if (e != cudaSuccess) return fail(FT_ECUDA);
    uint32_t w = 0;
    cudaMemcpy(&w, t->d_status, 4, cudaMemcpyDeviceToHost);
    if (w & FT_DEV_EINVAL) {
        cudaMemset(t->d_status, 0, 4);
        return fail(FT_EINVAL);
    }
    f->capacity = cap;
    if ((st = dmalloc(&f->d_ia, size_t(cap))) != FT_OK) return fail(st);
    if ((st = dmalloc(&f->d_ib, size_t(cap))) != FT_OK) return fail(st);
    if ((st = dmalloc(&f->d_f, size_t(cap))) != FT_OK) return fail(st);
    if ((st = dmalloc(&f->d_depth, size_t(cap))) != FT_OK) return fail(st);
    if ((st = dmalloc(&f->d_dist, size_t(cap))) != FT_OK) return fail(st);
    if (cudaMemsetAsync(f->d_count, 0, size_t(std::max<int64_t>(n_pairs, 1)) * 4, s) != cudaSuccess) return fail(FT_ECUDA);
    *out = f;
    return FT_OK;
}

extern "C" void ft_flows_free(ft_flows* f) { free_flows(f); }

extern "C" ft_status ft_flows_capacity(const ft_flows* f, int64_t* n_pairs, int64_t* capacity) {
    if (!f) return FT_EINVAL;
    if (n_pairs) *n_pairs = f->n_pairs;
    if (capacity) *capacity = f->capacity;
    return FT_OK;
}

extern "C" ft_status ft_flows_export(const ft_flows* f, int64_t* slot_ptr_host, int32_t* count_host,
                                     uint32_t* item_a_host, uint32_t* item_b_host, uint32_t* flow_host,
                                     uint8_t* depth_host) {
    if (!f) return FT_EINVAL;
    const size_t np = size_t(f->n_pairs), cap = size_t(f->capacity);
    if (slot_ptr_host) FT_CUDA(cudaMemcpy(slot_ptr_host, f->d_slot_ptr, (np + 1) * 8, cudaMemcpyDeviceToHost));
    if (count_host) FT_CUDA(cudaMemcpy(count_host, f->d_count, np * 4, cudaMemcpyDeviceToHost));
    if (item_a_host) FT_CUDA(cudaMemcpy(item_a_host, f->d_ia, cap * 4, cudaMemcpyDeviceToHost));
    if (item_b_host) FT_CUDA(cudaMemcpy(item_b_host, f->d_ib, cap * 4, cudaMemcpyDeviceToHost));
    if (flow_host) FT_CUDA(cudaMemcpy(flow_host, f->d_f, cap * 4, cudaMemcpyDeviceToHost));
    if (depth_host) FT_CUDA(cudaMemcpy(depth_host, f->d_depth, cap, cudaMemcpyDeviceToHost));
    return FT_OK;
}

extern "C" ft_status ft_flows_create_capacity(const ft_tree* t, const ft_docs* a, const ft_docs* b, int64_t max_pairs,
                                              ft_flows** out) {
    if (!out) return FT_EINVAL;
    *out = nullptr;
    if (!t || !a || !b || max_pairs < 1 || a->tree != t || b->tree != t) return FT_EINVAL;
    const int64_t per_pair = int64_t(a->max_support) + b->max_support;
    const int64_t cap = std::max<int64_t>(max_pairs * per_pair, 1);
    ft_flows* f = new ft_flows;
    f->tree = t;
    f->a = a;
    f->b = b;
    f->max_pairs = max_pairs;
    f->capacity = cap;
    auto fail = [&](ft_status st) {
        free_flows(f);
        return st;
    };
    ft_status st;
    if ((st = dmalloc(&f->d_pair_a, size_t(max_pairs))) != FT_OK) return fail(st);
    if ((st = dmalloc(&f->d_pair_b, size_t(max_pairs))) != FT_OK) return fail(st);
    if ((st = dmalloc(&f->d_slot_ptr, size_t(max_pairs) + 1)) != FT_OK) return fail(st);
    if ((st = dmalloc(&f->d_count, size_t(max_pairs))) != FT_OK) return fail(st);
    if ((st = dmalloc(&f->d_scan_tmp, ft_scan_tmp_elems(max_pairs + 1))) != FT_OK) return fail(st);
    if ((st = dmalloc(&f->d_ia, size_t(cap))) != FT_OK) return fail(st);
    if ((st = dmalloc(&f->d_ib, size_t(cap))) != FT_OK) return fail(st);
    if ((st = dmalloc(&f->d_f, size_t(cap))) != FT_OK) return fail(st);
    if ((st = dmalloc(&f->d_depth, size_t(cap))) != FT_OK) return fail(st);
    if ((st = dmalloc(&f->d_dist, size_t(cap))) != FT_OK) return fail(st);
    *out = f;
    return FT_OK;
}

extern "C" ft_status ft_flows_bind(ft_flows* f, const int32_t* pair_a_dev, const int32_t* pair_b_dev, int64_t n_pairs,
                                   void* stream) {
    FtRange nvtx_range("ft_flows_bind");
    if (!f || f->max_pairs == 0 || n_pairs < 0 || n_pairs > f->max_pairs) return FT_EINVAL;
    if ((pair_a_dev == nullptr) != (pair_b_dev == nullptr)) return FT_EINVAL;
    if (!pair_a_dev && n_pairs != f->a->n_docs * f->b->n_docs) return FT_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    f->cross = pair_a_dev == nullptr;
    f->nb_cross = f->b->n_docs;
    f->n_pairs = n_pairs;
    if (n_pairs == 0) return FT_OK;
    // the pair list is copied (the caller may reuse its buffers); a cross
    // product keeps no list
    const int32_t* pa = nullptr;
    const int32_t* pb = nullptr;
    if (pair_a_dev) {
        FT_CUDA(cudaMemcpyAsync(f->d_pair_a, pair_a_dev, size_t(n_pairs) * 4, cudaMemcpyDeviceToDevice, s));
        FT_CUDA(cudaMemcpyAsync(f->d_pair_b, pair_b_dev, size_t(n_pairs) * 4, cudaMemcpyDeviceToDevice, s));
        pa = f->d_pair_a;
        pb = f->d_pair_b;
    }
    k_slot_len<<<grid_for(n_pairs, 256), 256, 0, s>>>(f->a->d_ptr, f->b->d_ptr, pa, pb, n_pairs, f->b->n_docs,
                                                      f->a->n_docs, f->b->n_docs, f->d_slot_ptr, f->tree->d_status);
    FT_CUDA(cudaMemsetAsync(f->d_slot_ptr + n_pairs, 0, 8, s));
    FT_TRY(ft_exclusive_scan_i64(f->d_slot_ptr, f->d_slot_ptr, n_pairs + 1, f->d_scan_tmp, s));
    FT_CUDA(cudaMemsetAsync(f->d_count, 0, size_t(n_pairs) * 4, s));
    return FT_OK;
}
