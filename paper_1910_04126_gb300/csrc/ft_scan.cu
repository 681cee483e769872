// Quadtree-W1 prefilter (Sec. 2 closed form), top-k selects, and the
// k-nearest-neighbour pipeline of Sec. 5.2 (quadtree -> Flowtree).
//
// Tree W1 between a query q and a document j:
//   L1 = sum_k w_k sum_v |mu_q(v) - mu_j(v)|
// Every level's masses sum to 2^24 on both sides, so with
//   S = sum_v w(v) min(mu_q(v), mu_j(v))   (over nodes both touch)
//   C = 2^24 sum_{k=1..L+1} w_k = 2^24 (2^(L+1) - 1)
// L1 = 2C - 2S exactly (int64, units of u * 2^-24).  S only needs the nodes
// both distributions touch, so the scan walks, for every node of the query,
// the database's posting list of that node (the inverted index built with
// the embedding): its cost is the number of (query node, document) matches,
// not the product of the two embedding sizes.
#include <algorithm>

#include "ft_internal.cuh"

extern "C" ft_status ft_flowtree_batch(const ft_tree* t, const float* vocab_dev, const ft_docs* a, const ft_docs* b,
                                       const int32_t* pair_a_dev, const int32_t* pair_b_dev, int64_t n_pairs,
                                       float* cost_out_dev, ft_flows* flows_out, void* workspace, size_t ws_bytes,
                                       void* stream);

namespace {

#ifndef FT_SCAN_THREADS
#define FT_SCAN_THREADS 512
#endif
#ifndef FT_SCAN_TILE
#define FT_SCAN_TILE 4096  // largest shared-memory tile, documents
#endif
#ifndef FT_SCAN_UNROLL
#define FT_SCAN_UNROLL 4   // warp loads of 32 postings in flight per step
#endif
constexpr int SCAN_THREADS = FT_SCAN_THREADS;
constexpr int SEL_THREADS = 512;  // two CTAs per SM: a 256-row select fits one wave
constexpr int MAX_K1 = 4096;

// edge weight carried by an embedding entry
__device__ __forceinline__ int64_t entry_weight(uint32_t key, int L) {
    if (key & 0x80000000u) {
        const int c = int((key >> 24) & 0x7Fu);
        return (int64_t(1) << (L + 1 - c)) - 1;
    }
    const int k = int(key >> 24);
    return int64_t(1) << (L + 1 - k);
}

struct ScanArgs {
    const int64_t* q_eptr;
    const uint32_t* q_ekey;
    const uint32_t* q_emass;
    int64_t nq;
    const uint32_t* ukey;   // database index: distinct keys, ascending
    const uint32_t* uoff;   // [n_ukeys+1] posting ranges
    int64_t n_ukeys;
    const uint2* post;      // postings {document, mass}, documents ascending within a key
    int64_t nd;
    int L;
    int tile;               // documents per shared-memory tile
    int ecap;               // entry slots (>= the longest query embedding)
    int64_t docs_per_range; // documents per block, a multiple of tile
    uint64_t* keys;         // [nq][nd] (L1 << 24) | doc, or NULL
    int64_t* l1_out;        // [nq][nd] or NULL
};

// The tile keeps two 32-bit counters per document, S = lo + 2^16 hi: lo sums
// the low 16 bits of each addend and hi the rest.  lo stays below 2^32 while a
// document matches at most 65,536 query entries, hi below 2^24 because
// S < 2^40.  (Two 32-bit shared-memory atomics measured faster than one
// 64-bit one.)
__device__ __forceinline__ void tile_add(uint32_t* S, int tile, uint32_t d, uint64_t v) {
    atomicAdd(S + d, uint32_t(v & 0xFFFFu));
    atomicAdd(S + tile + d, uint32_t(v >> 16));
}

__device__ __forceinline__ uint64_t tile_take(uint32_t* S, int tile, int d) {
    const uint64_t v = uint64_t(S[d]) + (uint64_t(S[tile + d]) << 16);
    S[d] = 0;
    S[tile + d] = 0;
    return v;
}

// Postings of [c, lim) with document < thi (documents ascend): galloping
// then binary search, so an entry with n postings in the tile costs about
// 2 log2(n) loads.
__device__ __forceinline__ uint32_t count_below(const uint2* __restrict__ post, uint32_t c, uint32_t lim,
                                                uint32_t thi) {
    uint32_t lo = c, hi = lim, step = 1;
    for (;;) {
        const uint32_t probe = lo + step - 1;
        if (probe >= lim) break;
        if (__ldg(&post[probe].x) >= thi) {
            hi = probe;
            break;
        }
        lo = probe + 1;
        step <<= 1;
    }
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(&post[mid].x) < thi) lo = mid + 1; else hi = mid;
    }
    return lo - c;
}

// exclusive scan of v[0..n) in place by the whole block; returns the total
__device__ uint32_t block_exclusive_scan(uint32_t* v, int n, uint32_t* warp_tot) {
    const int T = blockDim.x, per = (n + T - 1) / T;
    const int b = min(n, int(threadIdx.x) * per), e = min(n, b + per);
    uint32_t s = 0;
    for (int i = b; i < e; ++i) s += v[i];
    const uint32_t incl = warp_incl_scan_u32(s);
    const int warp = int(threadIdx.x >> 5), nw = T >> 5;
    if (lane_id() == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t x = lane_id() < unsigned(nw) ? warp_tot[lane_id()] : 0u;
        const uint32_t xi = warp_incl_scan_u32(x);
        if (lane_id() < unsigned(nw)) warp_tot[lane_id()] = xi - x;
        if (lane_id() == 31) warp_tot[32] = xi;
    }
    __syncthreads();
    uint32_t run = warp_tot[warp] + incl - s;
    for (int i = b; i < e; ++i) {
        const uint32_t x = v[i];
        v[i] = run;
        run += x;
    }
    const uint32_t total = warp_tot[32];
    __syncthreads();
    return total;
}

// One block per (document range, query); block b covers range b / nq of
// query b % nq, so blocks resident together read the same slice of the
// long posting lists.  Every query entry keeps a cursor into its posting
// list.  Per tile of documents [tlo, thi):
//   1. each entry counts its postings in the tile (galloping search);
//   2. a block scan lays those postings out as one flat range;
//   3. the warps split the flat range evenly (a contiguous share each) and
//      walk it entry by entry, FT_SCAN_UNROLL loads of 32 postings in flight
//      per warp, adding w(v) * min(mu_q(v), mu_doc(v)) to the document's
//      shared-memory counter;
//   4. the tile is written out as L1 = 2C - 2S and the cursors advance.
// The even split keeps the warps of a block busy alike however the work is
// spread over the entries (one node shared by every document holds as many
// postings per tile as all the rare words together).
__global__ void __launch_bounds__(SCAN_THREADS) k_qt_scan(ScanArgs a) {
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ uint32_t warp_tot[33];
    uint32_t* S = sm;  // [2][tile]
    uint32_t* ecur = S + 2 * a.tile;
    uint32_t* eend = ecur + a.ecap;
    uint32_t* ew = eend + a.ecap;       // edge weight
    uint32_t* emq = ew + a.ecap;        // query mass
    uint32_t* pre = emq + a.ecap;       // [ecap+1] flat offsets of the tile's postings
    const int64_t q = int64_t(blockIdx.x) % a.nq;
    const int64_t d_lo = (int64_t(blockIdx.x) / a.nq) * a.docs_per_range;
    const int64_t d_hi = min(a.nd, d_lo + a.docs_per_range);
    if (d_lo >= d_hi) return;  // uniform over the block
    const int64_t eb = a.q_eptr[q];
    const int E = int(a.q_eptr[q + 1] - eb);
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const uint32_t key = a.q_ekey[eb + e];
        int64_t lo = 0, hi = a.n_ukeys;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(a.ukey + mid) < key) lo = mid + 1; else hi = mid;
        }
        uint32_t c = 0, en = 0;
        if (lo < a.n_ukeys && __ldg(a.ukey + lo) == key) {
            c = __ldg(a.uoff + lo);
            en = __ldg(a.uoff + lo + 1);
            uint32_t h = en;  // first posting with doc >= d_lo
            while (c < h) {
                const uint32_t mid = c + ((h - c) >> 1);
                if (int64_t(__ldg(&a.post[mid].x)) < d_lo) c = mid + 1; else h = mid;
            }
        }
        ecur[e] = c;
        eend[e] = en;
        ew[e] = uint32_t(entry_weight(key, a.L));
        emq[e] = a.q_emass[eb + e];
    }
    for (int i = threadIdx.x; i < 2 * a.tile; i += blockDim.x) S[i] = 0;
    __syncthreads();
    const int64_t C2 = (int64_t(1) << 25) * ((int64_t(1) << (a.L + 1)) - 1);  // 2C
    const unsigned lane = lane_id();
    const int warp = int(threadIdx.x >> 5), nwarps = int(blockDim.x >> 5);
    constexpr int U = FT_SCAN_UNROLL;
    for (int64_t t_lo = d_lo; t_lo < d_hi; t_lo += a.tile) {
        const int64_t t_hi = min(d_hi, t_lo + a.tile);
        const uint32_t tlo = uint32_t(t_lo), thi = uint32_t(t_hi), n_t = thi - tlo;
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            const uint32_t c = ecur[e], en = eend[e];
            pre[e] = c < en ? count_below(a.post, c, min(en, c + n_t), thi) : 0u;
        }
        __syncthreads();
        const uint32_t P = block_exclusive_scan(pre, E, warp_tot);
        if (threadIdx.x == 0) pre[E] = P;
        __syncthreads();
        // each warp takes a contiguous share of the flat range (whole groups
        // of 32) and walks it entry piece by entry piece
        const uint32_t groups = (P + 31u) >> 5, per = (groups + uint32_t(nwarps) - 1u) / uint32_t(nwarps);
        uint32_t f = min(P, uint32_t(warp) * per * 32u);
        const uint32_t f_end = min(P, f + per * 32u);
        int e = 0;
        if (f < f_end) {
            int hi = E;  // last entry with pre[e] <= f
            while (e < hi) {
                const int mid = (e + hi + 1) >> 1;
                if (pre[mid] <= f) e = mid; else hi = mid - 1;
            }
        }
        while (f < f_end) {
            while (pre[e + 1] <= f) ++e;
            const uint32_t seg_end = min(pre[e + 1], f_end);
            const uint32_t base = ecur[e] - pre[e];  // posting index = base + flat index
            const uint64_t w = ew[e];
            const uint32_t mq = emq[e];
            for (; f + 32u * U <= seg_end; f += 32u * U) {
                uint2 p[U];
#pragma unroll
                for (int u = 0; u < U; ++u) p[u] = __ldg(a.post + base + f + lane + 32u * u);
#pragma unroll
                for (int u = 0; u < U; ++u) tile_add(S, a.tile, p[u].x - tlo, w * min(mq, p[u].y));
            }
            if (f < seg_end) {
                uint2 p[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t g = f + lane + 32u * u;
                    p[u] = g < seg_end ? __ldg(a.post + base + g) : make_uint2(0xFFFFFFFFu, 0u);
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (p[u].x != 0xFFFFFFFFu) tile_add(S, a.tile, p[u].x - tlo, w * min(mq, p[u].y));
                f = seg_end;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < int(n_t); i += blockDim.x) {
            const int64_t doc = t_lo + i;
            const int64_t l1 = C2 - 2 * int64_t(tile_take(S, a.tile, i));
            const int64_t o = q * a.nd + doc;
            if (a.keys) a.keys[o] = (uint64_t(l1) << 24) | uint64_t(doc);
            if (a.l1_out) a.l1_out[o] = l1;
        }
        for (int e = threadIdx.x; e < E; e += blockDim.x) ecur[e] += pre[e + 1] - pre[e];
        __syncthreads();
    }
}

// Per row: the k smallest of n unique u64 keys, ascending, by a radix select
// over 11-bit digits (most significant first) that stops as soon as the keys
// at or below the current prefix fit the candidate buffer (or at the exact
// k-th key), followed by a bitonic sort of the survivors.
// Quadtree keys (F32 = false): ids_out = low 24 bits, l1_out = key >> 24.
// Value keys (F32 = true): key = (float bits << 32) | column, ids_out = low 32
// bits, val_out = the float.
template <bool F32>
__global__ void __launch_bounds__(SEL_THREADS) k_select_u64(const uint64_t* __restrict__ keys, int64_t n, int k,
                                                            int32_t* __restrict__ ids_out, int64_t* __restrict__ l1_out,
                                                            float* __restrict__ val_out, uint32_t* status) {
    __shared__ uint32_t hist[2048];
    __shared__ uint64_t cand[MAX_K1];
    __shared__ uint64_t prefix_s, mask_s;
    __shared__ int krem_s, cnt_s, below_s, eq_s;
    const uint64_t* row = keys + int64_t(blockIdx.x) * n;
    if (threadIdx.x == 0) {
        prefix_s = 0;
        mask_s = 0;
        krem_s = k;
        cnt_s = 0;
        below_s = 0;
        eq_s = n < int64_t(0x7FFFFFFF) ? int(n) : 0x7FFFFFFF;
    }
    __syncthreads();
    bool exact = true;
    for (int dg = 0; dg < 6; ++dg) {
        if (below_s + eq_s <= MAX_K1) {
            exact = false;  // every key at or below the prefix fits the buffer
            break;
        }
        // digits: bits 63..53, 52..42, 41..31, 30..20, 19..9, 8..0
        const int sh = dg < 5 ? 53 - 11 * dg : 0, nb = dg < 5 ? 2048 : 512;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const uint64_t prefix = prefix_s, mask = mask_s;
        // eight independent key loads in flight per thread (the row streams
        // from L2/HBM once per digit); the loop is warp-uniform so that a warp
        // whose counted keys share one bucket adds them with one atomic
        const int lane = threadIdx.x & 31;
        const int64_t step = int64_t(blockDim.x) * 8;
        for (int64_t i0 = threadIdx.x - lane; i0 < n; i0 += step) {
            uint64_t kv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t i = i0 + lane + int64_t(u) * blockDim.x;
                kv[u] = i < n ? row[i] : ~uint64_t(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t i = i0 + lane + int64_t(u) * blockDim.x;
                const bool in = i < n && (kv[u] & mask) == prefix;
                const uint32_t bk = uint32_t(kv[u] >> sh) & uint32_t(nb - 1);
                const unsigned act = __ballot_sync(0xFFFFFFFFu, in);
                if (act == 0) continue;
                const int leader = __ffs(act) - 1;
                const uint32_t lb = __shfl_sync(0xFFFFFFFFu, bk, leader);
                const unsigned same = __ballot_sync(0xFFFFFFFFu, in && bk == lb);
                if (same == act) {
                    if (lane == leader) atomicAdd(&hist[lb], unsigned(__popc(act)));
                } else if (in) {
                    atomicAdd(&hist[bk], 1u);
                }
            }
        }
        __syncthreads();
        // warp 0 finds the bucket of the krem-th counted key: lane sums over
        // nb/32 buckets, a warp scan, then the owning lane walks its buckets
        if (threadIdx.x < 32) {
            const int per = nb >> 5;
            int sum = 0;
            for (int j = 0; j < per; ++j) sum += int(hist[lane * per + j]);
            int inc = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                if (lane >= o) inc += t;
            }
            const int krem0 = krem_s;
            const unsigned hit = __ballot_sync(0xFFFFFFFFu, inc >= krem0);
            const int owner = hit ? __ffs(hit) - 1 : 31;
            if (lane == owner) {
                if (!hit) ft_flag(status, FT_DEV_EINVAL);  // fewer than k keys: cannot happen for k <= n
                int krem = krem0 - (inc - sum), below = below_s + (inc - sum);
                int b = lane * per;
                for (; b < lane * per + per - 1; ++b) {
                    if (int(hist[b]) >= krem) break;
                    krem -= int(hist[b]);
                    below += int(hist[b]);
                }
                krem_s = krem;
                below_s = below;
                eq_s = int(hist[b]);
                prefix_s = prefix | (uint64_t(b) << sh);
                mask_s = mask | (uint64_t(nb - 1) << sh);
            }
        }
        __syncthreads();
    }
    // exact: the k-th smallest key; else every key whose digits so far are at
    // most the prefix (fewer than MAX_K1 of them)
    const uint64_t thr = exact ? prefix_s : (prefix_s | ~mask_s);
    for (int64_t i0 = threadIdx.x; i0 < n; i0 += int64_t(blockDim.x) * 8) {
        uint64_t kv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t i = i0 + int64_t(u) * blockDim.x;
            kv[u] = i < n ? row[i] : ~uint64_t(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (kv[u] <= thr && i0 + int64_t(u) * blockDim.x < n) {
                const int pos = atomicAdd(&cnt_s, 1);
                if (pos < MAX_K1) cand[pos] = kv[u];
            }
        }
    }
    __syncthreads();
    // exact: cnt == k; else k <= cnt <= MAX_K1 (MAX_K1 is a power of two)
    const int cnt = min(cnt_s, MAX_K1);
    int m = 1;
    while (m < cnt || m < k) m <<= 1;
    for (int i = cnt + threadIdx.x; i < m; i += blockDim.x) cand[i] = ~uint64_t(0);
    __syncthreads();
    for (int size = 2; size <= m; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const uint64_t x = cand[i], y = cand[j];
                    if ((x > y) == up) {
                        cand[i] = y;
                        cand[j] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const uint64_t key = cand[i];
        if (F32) {
            ids_out[int64_t(blockIdx.x) * k + i] = int32_t(key & 0xFFFFFFFFu);
            val_out[int64_t(blockIdx.x) * k + i] = __uint_as_float(uint32_t(key >> 32));
        } else {
            ids_out[int64_t(blockIdx.x) * k + i] = int32_t(key & 0xFFFFFFu);
            if (l1_out) l1_out[int64_t(blockIdx.x) * k + i] = int64_t(key >> 24);
        }
    }
}

// key = (bits of the value << 32) | column; values are non-negative costs,
// so their bit patterns order like the values (NaN sorts after +inf).
__global__ void k_f32_keys(const float* __restrict__ v, int64_t rows, int64_t cols, uint64_t* __restrict__ keys) {
    const int64_t n = rows * cols;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const float x = v[i];
        uint32_t bits = __float_as_uint(x);
        if (x != x) bits = 0x7FC00000u;
        else if (bits & 0x80000000u) bits = 0;  // -0.0 (and any negative) sorts first
        keys[i] = (uint64_t(bits) << 32) | uint64_t(i % cols);
    }
}

// final top-k of the Flowtree costs of each query's k1 candidates
__global__ void __launch_bounds__(SEL_THREADS) k_final_topk(const float* __restrict__ cost,
                                                            const int32_t* __restrict__ cand, int k1, int k,
                                                            int32_t* __restrict__ ids_out, float* __restrict__ dist_out) {
    __shared__ uint64_t v[MAX_K1];
    int m = 1;
    while (m < k1) m <<= 1;
    const int64_t base = int64_t(blockIdx.x) * k1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        if (i < k1) {
            float c = cost[base + i];
            uint32_t bits = __float_as_uint(c);
            if (c != c) bits = 0x7F800000u;  // NaN sorts last among finite
            v[i] = (uint64_t(bits) << 32) | uint32_t(cand[base + i]);
        } else {
            v[i] = ~uint64_t(0);
        }
    }
    __syncthreads();
    for (int size = 2; size <= m; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const uint64_t x = v[i], y = v[j];
                    if ((x > y) == up) {
                        v[i] = y;
                        v[j] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        ids_out[int64_t(blockIdx.x) * k + i] = int32_t(v[i] & 0xFFFFFFFFu);
        dist_out[int64_t(blockIdx.x) * k + i] = __uint_as_float(uint32_t(v[i] >> 32));
    }
}

__global__ void k_knn_pairs(const int32_t* __restrict__ cand, int64_t nq, int k1, int32_t* __restrict__ pa,
                            int32_t* __restrict__ pb) {
    const int64_t n = nq * k1;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        pa[i] = int32_t(i / k1);
        pb[i] = cand[i];
    }
}

int grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535 * 8) b = 65535 * 8;
    return int(b);
}

struct ScanPlan {
    int tile = 4096;
    int ecap = 1;
    int64_t docs_per_range = 0;
    int64_t blocks = 0;
    size_t smem = 0;
};

ft_status plan_scan(const ft_tree* t, const ft_docs* q, const ft_docs* d, ScanPlan* p) {
    int dev = 0, max_smem = 0;
    FT_CUDA(cudaGetDevice(&dev));
    FT_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    p->ecap = std::max(q->max_embed, 1);
    const size_t entry_bytes = size_t(20) * p->ecap + 4;
    // the largest tile (<= 4096 documents) that leaves room for three blocks
    // per SM, else for one
    const size_t room = size_t(max_smem) - 1024;  // less the block's static shared memory
    int tile = FT_SCAN_TILE;
    while (tile > 256 && 3 * (size_t(8) * tile + entry_bytes) > room) tile >>= 1;
    if (size_t(8) * tile + entry_bytes > room || p->ecap > 65536) return FT_EUNSUPPORTED;
    p->tile = tile;
    p->smem = size_t(8) * tile + entry_bytes;
    int bps = 0;
    FT_TRY(ft_prepare_kernel(reinterpret_cast<const void*>(&k_qt_scan), SCAN_THREADS, p->smem, &bps));
    if (bps < 1) return FT_EUNSUPPORTED;
    // split each query's documents into ranges until about four waves of
    // blocks exist; a range spans whole tiles
    const int64_t tiles = (d->n_docs + tile - 1) / tile;
    const int64_t want = int64_t(4) * t->num_sms * bps;
    int64_t ranges = std::min(tiles, std::max<int64_t>(1, (want + q->n_docs - 1) / q->n_docs));
    const int64_t tiles_per_range = (tiles + ranges - 1) / ranges;
    ranges = (tiles + tiles_per_range - 1) / tiles_per_range;
    p->docs_per_range = tiles_per_range * tile;
    p->blocks = ranges * q->n_docs;
    if (p->blocks > 0x7FFFFFFF) return FT_EUNSUPPORTED;
    return FT_OK;
}

ft_status launch_scan(const ft_tree* t, const ft_docs* q, const ft_docs* d, uint64_t* keys, int64_t* l1,
                      cudaStream_t s) {
    if (q->n_docs == 0) return FT_OK;
    ScanPlan p;
    FT_TRY(plan_scan(t, q, d, &p));
    ScanArgs a{};
    a.q_eptr = q->d_eptr;
    a.q_ekey = q->d_ekey;
    a.q_emass = q->d_emass;
    a.nq = q->n_docs;
    a.ukey = d->d_ukey;
    a.uoff = d->d_uoff;
    a.n_ukeys = d->n_ukeys;
    a.post = d->d_post;
    a.nd = d->n_docs;
    a.L = t->levels;
    a.tile = p.tile;
    a.ecap = p.ecap;
    a.docs_per_range = p.docs_per_range;
    a.keys = keys;
    a.l1_out = l1;
    k_qt_scan<<<unsigned(p.blocks), SCAN_THREADS, p.smem, s>>>(a);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

ft_status check_scan(const ft_tree* t, const ft_docs* q, const ft_docs* d, int32_t k1) {
    if (!t || !q || !d || q->tree != t || d->tree != t) return FT_EINVAL;
    if (k1 < 1 || k1 > MAX_K1 || int64_t(k1) > d->n_docs) return FT_EINVAL;
    if (t->levels > FT_MAX_LEVELS || d->n_docs > (int64_t(1) << 24)) return FT_EUNSUPPORTED;
    return FT_OK;
}

size_t scan_layout(const ft_docs* q, const ft_docs* d, void* base, uint64_t** keys) {
    WsCarver w(base);
    uint64_t* k = w.take<uint64_t>(size_t(q->n_docs) * d->n_docs);
    if (keys) *keys = k;
    return w.off + 256;
}

struct KnnLayout {
    uint64_t* keys;
    int32_t* cand;
    int32_t* pa;
    int32_t* pb;
    float* cost;
    void* fws;
    size_t fws_bytes;
};

}  // namespace

extern "C" size_t ft_quadtree_scan_workspace_size(const ft_tree* t, const ft_docs* queries, const ft_docs* db,
                                                  int32_t k1) {
    if (check_scan(t, queries, db, k1) != FT_OK) return 0;
    return scan_layout(queries, db, nullptr, nullptr);
}

extern "C" ft_status ft_quadtree_scan(const ft_tree* t, const ft_docs* queries, const ft_docs* db, int32_t k1,
                                      void* workspace, size_t ws_bytes, int32_t* cand_ids_out_dev,
                                      int64_t* cand_l1_out_dev, void* stream) {
    FtRange nvtx_range("ft_quadtree_scan");
    FT_TRY(check_scan(t, queries, db, k1));
    if (!cand_ids_out_dev) return FT_EINVAL;
    if (!workspace || ws_bytes < scan_layout(queries, db, nullptr, nullptr)) return FT_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t* keys = nullptr;
    scan_layout(queries, db, workspace, &keys);
    FT_TRY(launch_scan(t, queries, db, keys, nullptr, s));
    k_select_u64<false><<<unsigned(queries->n_docs), SEL_THREADS, 0, s>>>(keys, db->n_docs, k1, cand_ids_out_dev,
                                                                          cand_l1_out_dev, nullptr, t->d_status);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

extern "C" ft_status ft_quadtree_l1_dense(const ft_tree* t, const ft_docs* queries, const ft_docs* db,
                                          int64_t* l1_all_out_dev, void* stream) {
    FtRange nvtx_range("ft_quadtree_l1_dense");
    FT_TRY(check_scan(t, queries, db, 1));
    if (!l1_all_out_dev) return FT_EINVAL;
    return launch_scan(t, queries, db, nullptr, l1_all_out_dev, static_cast<cudaStream_t>(stream));
}

namespace {
// df of every query entry's node in the database index, summed
__global__ void k_scan_matches(const uint32_t* __restrict__ q_ekey, int64_t n, const uint32_t* __restrict__ ukey,
                               const uint32_t* __restrict__ uoff, int64_t n_ukeys,
                               unsigned long long* __restrict__ total) {
    unsigned long long acc = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t key = q_ekey[i];
        int64_t lo = 0, hi = n_ukeys;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (ukey[mid] < key) lo = mid + 1; else hi = mid;
        }
        if (lo < n_ukeys && ukey[lo] == key) acc += uoff[lo + 1] - uoff[lo];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL_MASK, acc, o);
    if (lane_id() == 0 && acc) atomicAdd(total, acc);
}
}  // namespace

extern "C" ft_status ft_quadtree_scan_matches(const ft_tree* t, const ft_docs* queries, const ft_docs* db,
                                              int64_t* matches_out_host) {
    if (!t || !queries || !db || queries->tree != t || db->tree != t || !matches_out_host) return FT_EINVAL;
    unsigned long long* d_total = nullptr;
    FT_CUDA(cudaMalloc(&d_total, sizeof(unsigned long long)));
    unsigned long long h = 0;
    cudaError_t e = cudaMemset(d_total, 0, sizeof(unsigned long long));
    if (e == cudaSuccess && queries->n_embed > 0) {
        k_scan_matches<<<grid_for(queries->n_embed, 256), 256>>>(queries->d_ekey, queries->n_embed, db->d_ukey,
                                                                 db->d_uoff, db->n_ukeys, d_total);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d_total, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d_total);
    if (e != cudaSuccess) {
        ft_note_cuda_error(e, "ft_quadtree_scan_matches", __FILE__, __LINE__);
        return FT_ECUDA;
    }
    *matches_out_host = int64_t(h);
    return FT_OK;
}

namespace {
size_t knn_layout(const ft_tree* t, const ft_docs* db, const ft_docs* q, int32_t k1, void* base, KnnLayout* out) {
    WsCarver w(base);
    KnnLayout l{};
    const int64_t np = q->n_docs * int64_t(k1);
    l.keys = w.take<uint64_t>(size_t(q->n_docs) * db->n_docs);
    l.cand = w.take<int32_t>(size_t(np));
    l.pa = w.take<int32_t>(size_t(np));
    l.pb = w.take<int32_t>(size_t(np));
    l.cost = w.take<float>(size_t(np));
    l.fws_bytes = ft_flowtree_batch_workspace_size(t, q, db, np);
    l.fws = w.take<uint8_t>(l.fws_bytes);
    if (out) *out = l;
    return w.off + 256;
}
}  // namespace

extern "C" size_t ft_knn_workspace_size(const ft_tree* t, const ft_docs* db, const ft_docs* queries, int32_t k1,
                                        int32_t k) {
    if (check_scan(t, queries, db, k1) != FT_OK || k < 1 || k > k1) return 0;
    return knn_layout(t, db, queries, k1, nullptr, nullptr);
}

extern "C" ft_status ft_knn(const ft_tree* t, const float* vocab_dev, const ft_docs* db, const ft_docs* queries,
                            int32_t k1, int32_t k, void* workspace, size_t ws_bytes, int32_t* ids_out_dev,
                            float* dist_out_dev, void* stream) {
    FtRange nvtx_range("ft_knn");
    FT_TRY(check_scan(t, queries, db, k1));
    if (!vocab_dev || !ids_out_dev || !dist_out_dev || k < 1 || k > k1) return FT_EINVAL;
    if (!workspace || ws_bytes < knn_layout(t, db, queries, k1, nullptr, nullptr)) return FT_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    KnnLayout l;
    knn_layout(t, db, queries, k1, workspace, &l);
    const int64_t nq = queries->n_docs, np = nq * int64_t(k1);
    FT_TRY(launch_scan(t, queries, db, l.keys, nullptr, s));
    k_select_u64<false><<<unsigned(nq), SEL_THREADS, 0, s>>>(l.keys, db->n_docs, k1, l.cand, nullptr, nullptr, t->d_status);
    k_knn_pairs<<<grid_for(np, 256), 256, 0, s>>>(l.cand, nq, k1, l.pa, l.pb);
    FT_CUDA(cudaGetLastError());
    FT_TRY(ft_flowtree_batch(t, vocab_dev, queries, db, l.pa, l.pb, np, l.cost, nullptr, l.fws, l.fws_bytes, s));
    k_final_topk<<<unsigned(nq), SEL_THREADS, 0, s>>>(l.cost, l.cand, k1, k, ids_out_dev, dist_out_dev);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

namespace {
struct KnnExactLayout {
    KnnLayout knn;
    int32_t* ids2;   // [nq][k2] Flowtree survivors
    float* dist2;    // [nq][k2] their Flowtree values (unused downstream)
    int32_t* pa2;    // [nq * k2] exact-stage pairs
    int32_t* pb2;
    float* cost2;    // [nq * k2] exact W1
    void* ews;
    size_t ews_bytes;
};

size_t knn_exact_layout(const ft_tree* t, const ft_docs* db, const ft_docs* q, int32_t k1, int32_t k2, void* base,
                        KnnExactLayout* out) {
    KnnExactLayout l{};
    const size_t knn_bytes = (knn_layout(t, db, q, k1, base, base ? &l.knn : nullptr) + 255) & ~size_t(255);
    WsCarver w(base ? static_cast<char*>(base) + knn_bytes : nullptr);  // 256-byte aligned like the rest
    const int64_t np2 = q->n_docs * int64_t(k2);
    l.ids2 = w.take<int32_t>(size_t(np2));
    l.dist2 = w.take<float>(size_t(np2));
    l.pa2 = w.take<int32_t>(size_t(np2));
    l.pb2 = w.take<int32_t>(size_t(np2));
    l.cost2 = w.take<float>(size_t(np2));
    l.ews_bytes = ft_exact_w1_workspace_size(q, db, np2);
    l.ews = w.take<uint8_t>(l.ews_bytes);
    if (out) *out = l;
    return knn_bytes + w.off + 256;
}
}  // namespace

extern "C" size_t ft_knn_exact_workspace_size(const ft_tree* t, const ft_docs* db, const ft_docs* queries, int32_t k1,
                                              int32_t k2, int32_t k) {
    if (check_scan(t, queries, db, k1) != FT_OK || k < 1 || k > k2 || k2 > k1) return 0;
    if (ft_exact_w1_workspace_size(queries, db, queries->n_docs * int64_t(k2)) == 0) return 0;
    return knn_exact_layout(t, db, queries, k1, k2, nullptr, nullptr);
}

extern "C" ft_status ft_knn_exact(const ft_tree* t, const float* vocab_dev, const ft_docs* db, const ft_docs* queries,
                                  int32_t k1, int32_t k2, int32_t k, void* workspace, size_t ws_bytes,
                                  int32_t* ids_out_dev, float* dist_out_dev, void* stream) {
    FtRange nvtx_range("ft_knn_exact");
    FT_TRY(check_scan(t, queries, db, k1));
    if (!vocab_dev || !ids_out_dev || !dist_out_dev || k < 1 || k > k2 || k2 > k1) return FT_EINVAL;
    if (ft_exact_w1_workspace_size(queries, db, queries->n_docs * int64_t(k2)) == 0) return FT_EUNSUPPORTED;
    if (!workspace || ws_bytes < knn_exact_layout(t, db, queries, k1, k2, nullptr, nullptr)) return FT_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    KnnExactLayout l;
    knn_exact_layout(t, db, queries, k1, k2, workspace, &l);
    const int64_t nq = queries->n_docs, np = nq * int64_t(k1), np2 = nq * int64_t(k2);
    // stage 1: quadtree scan -> top-k1
    FT_TRY(launch_scan(t, queries, db, l.knn.keys, nullptr, s));
    k_select_u64<false><<<unsigned(nq), SEL_THREADS, 0, s>>>(l.knn.keys, db->n_docs, k1, l.knn.cand, nullptr, nullptr,
                                                             t->d_status);
    // stage 2: Flowtree on the k1 candidates -> top-k2
    k_knn_pairs<<<grid_for(np, 256), 256, 0, s>>>(l.knn.cand, nq, k1, l.knn.pa, l.knn.pb);
    FT_CUDA(cudaGetLastError());
    FT_TRY(ft_flowtree_batch(t, vocab_dev, queries, db, l.knn.pa, l.knn.pb, np, l.knn.cost, nullptr, l.knn.fws,
                             l.knn.fws_bytes, s));
    k_final_topk<<<unsigned(nq), SEL_THREADS, 0, s>>>(l.knn.cost, l.knn.cand, k1, k2, l.ids2, l.dist2);
    // stage 3: exact W1 on the k2 survivors -> top-k
    k_knn_pairs<<<grid_for(np2, 256), 256, 0, s>>>(l.ids2, nq, k2, l.pa2, l.pb2);
    FT_CUDA(cudaGetLastError());
    FT_TRY(ft_exact_w1_batch(vocab_dev, queries, db, l.pa2, l.pb2, np2, l.cost2, l.ews, l.ews_bytes, s));
    k_final_topk<<<unsigned(nq), SEL_THREADS, 0, s>>>(l.cost2, l.ids2, k2, k, ids_out_dev, dist_out_dev);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

extern "C" size_t ft_topk_f32_workspace_size(int64_t n_rows, int64_t n_cols) {
    if (n_rows < 1 || n_cols < 1) return 0;
    WsCarver w(nullptr);
    w.take<uint64_t>(size_t(n_rows) * n_cols);
    return w.off + 256;
}

extern "C" ft_status ft_topk_f32(const float* values_dev, int64_t n_rows, int64_t n_cols, int32_t k, void* workspace,
                                 size_t ws_bytes, int32_t* ids_out_dev, float* vals_out_dev, void* stream) {
    FtRange nvtx_range("ft_topk_f32");
    if (!values_dev || !ids_out_dev || !vals_out_dev || n_rows < 1 || n_cols < 1 || k < 1 || k > MAX_K1 ||
        int64_t(k) > n_cols || n_cols >= (int64_t(1) << 32) || n_rows > 0x7FFFFFFF)
        return FT_EINVAL;
    if (!workspace || ws_bytes < ft_topk_f32_workspace_size(n_rows, n_cols)) return FT_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t* keys = static_cast<uint64_t*>(workspace);
    k_f32_keys<<<grid_for(n_rows * n_cols, 256), 256, 0, s>>>(values_dev, n_rows, n_cols, keys);
    k_select_u64<true><<<unsigned(n_rows), SEL_THREADS, 0, s>>>(keys, n_cols, k, ids_out_dev, nullptr, vals_out_dev,
                                                                nullptr);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}
