// Quadtree-W1 prefilter (Sec. 2 closed form), top-k selects, and the
// k-nearest-neighbour pipeline of Sec. 5.2 (quadtree -> Flowtree).
//
// Tree W1 between a query q and a document j:
//   L1 = sum_k w_k sum_v |mu_q(v) - mu_j(v)|
// Every level's masses sum to 2^24 on both sides, so with
//   S = sum_v w(v) min(mu_q(v), mu_j(v))   (over nodes both touch)
//   C = 2^24 sum_{k=1..L+1} w_k = 2^24 (2^(L+1) - 1)
// L1 = 2C - 2S exactly (int64, units of u * 2^-24).  S only needs the nodes
// both distributions touch: query embeddings sit in shared-memory hash
// tables, document embeddings are streamed past them.
#include <algorithm>

#include "ft_internal.cuh"

extern "C" ft_status ft_flowtree_batch(const ft_tree* t, const float* vocab_dev, const ft_docs* a, const ft_docs* b,
                                       const int32_t* pair_a_dev, const int32_t* pair_b_dev, int64_t n_pairs,
                                       float* cost_out_dev, ft_flows* flows_out, void* workspace, size_t ws_bytes,
                                       void* stream);

namespace {

constexpr uint32_t EMPTY = 0xFFFFFFFFu;
constexpr int SCAN_THREADS = 256;
constexpr int SEL_THREADS = 1024;
constexpr int MAX_K1 = 4096;

__device__ __forceinline__ uint32_t hslot(uint32_t key, int log2cap) {
    return (key * 0x9E3779B1u) >> (32 - log2cap);
}

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
    const int64_t* d_eptr;
    const uint32_t* d_ekey;
    const uint32_t* d_emass;
    int64_t nd;
    int L;
    int qb;         // queries per block
    int log2cap;    // hash capacity per query
    int docs_per_block;
    uint64_t* keys;     // [nq][nd] (L1 << 24) | doc, or NULL
    int64_t* l1_out;    // [nq][nd] or NULL
};

// grid: (query groups, document tiles)
template <int QB>
__global__ void __launch_bounds__(SCAN_THREADS) k_qt_scan(ScanArgs a) {
    extern __shared__ __align__(16) uint32_t tab[];  // [QB][cap] keys then [QB][cap] masses
    const int cap = 1 << a.log2cap;
    uint32_t* tkey = tab;
    uint32_t* tmass = tab + size_t(QB) * cap;
    const int64_t q0 = int64_t(blockIdx.x) * QB;
    const int nqb = int(min(int64_t(QB), a.nq - q0));
    for (int i = threadIdx.x; i < QB * cap; i += blockDim.x) tkey[i] = EMPTY;
    __syncthreads();
    for (int qi = 0; qi < nqb; ++qi) {
        const int64_t b = a.q_eptr[q0 + qi], e = a.q_eptr[q0 + qi + 1];
        for (int64_t j = b + threadIdx.x; j < e; j += blockDim.x) {
            const uint32_t key = a.q_ekey[j];
            uint32_t s = hslot(key, a.log2cap);
            for (;;) {
                const uint32_t old = atomicCAS(&tkey[qi * cap + s], EMPTY, key);
                if (old == EMPTY) {
                    tmass[qi * cap + s] = a.q_emass[j];
                    break;
                }
                s = (s + 1) & uint32_t(cap - 1);
            }
        }
    }
    __syncthreads();
    const int64_t C2 = (int64_t(1) << 25) * ((int64_t(1) << (a.L + 1)) - 1);  // 2C
    const unsigned lane = lane_id();
    const int warp = int(threadIdx.x >> 5), nwarps = int(blockDim.x >> 5);
    const int64_t d_begin = int64_t(blockIdx.y) * a.docs_per_block;
    const int64_t d_end = min(a.nd, d_begin + int64_t(a.docs_per_block));
    for (int64_t doc = d_begin + warp; doc < d_end; doc += nwarps) {
        int64_t acc[QB];
#pragma unroll
        for (int qi = 0; qi < QB; ++qi) acc[qi] = 0;
        const int64_t b = a.d_eptr[doc], e = a.d_eptr[doc + 1];
        for (int64_t j = b + lane; j < e; j += 32) {
            const uint32_t key = __ldg(a.d_ekey + j);
            const uint32_t m = __ldg(a.d_emass + j);
            const int64_t w = entry_weight(key, a.L);
            const uint32_t s0 = hslot(key, a.log2cap);
#pragma unroll
            for (int qi = 0; qi < QB; ++qi) {
                uint32_t s = s0;
                for (;;) {
                    const uint32_t k2 = tkey[qi * cap + s];
                    if (k2 == key) {
                        acc[qi] += w * int64_t(min(m, tmass[qi * cap + s]));
                        break;
                    }
                    if (k2 == EMPTY) break;
                    s = (s + 1) & uint32_t(cap - 1);
                }
            }
        }
#pragma unroll
        for (int qi = 0; qi < QB; ++qi) {
            const int64_t S = warp_sum_i64(acc[qi]);
            if (lane == 0 && qi < nqb) {
                const int64_t l1 = C2 - 2 * S;
                const int64_t o = (q0 + qi) * a.nd + doc;
                if (a.keys) a.keys[o] = (uint64_t(l1) << 24) | uint64_t(doc);
                if (a.l1_out) a.l1_out[o] = l1;
            }
        }
    }
}

// Per row: the k smallest of n unique u64 keys, ascending, by an 8-bit
// radix select (MSB first) followed by a bitonic sort of the k survivors.
// Quadtree keys (F32 = false): ids_out = low 24 bits, l1_out = key >> 24.
// Value keys (F32 = true): key = (float bits << 32) | column, ids_out = low 32
// bits, val_out = the float.
template <bool F32>
__global__ void __launch_bounds__(SEL_THREADS) k_select_u64(const uint64_t* __restrict__ keys, int64_t n, int k,
                                                            int32_t* __restrict__ ids_out, int64_t* __restrict__ l1_out,
                                                            float* __restrict__ val_out, uint32_t* status) {
    __shared__ uint32_t hist[256];
    __shared__ uint64_t cand[MAX_K1];
    __shared__ uint64_t prefix_s, mask_s;
    __shared__ int krem_s, cnt_s;
    const uint64_t* row = keys + int64_t(blockIdx.x) * n;
    if (threadIdx.x == 0) {
        prefix_s = 0;
        mask_s = 0;
        krem_s = k;
        cnt_s = 0;
    }
    __syncthreads();
    for (int dg = 7; dg >= 0; --dg) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const uint64_t prefix = prefix_s, mask = mask_s;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const uint64_t key = row[i];
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> (8 * dg)) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int krem = krem_s;
            int b = 0;
            for (; b < 256; ++b) {
                if (int(hist[b]) >= krem) break;
                krem -= int(hist[b]);
            }
            if (b == 256) {  // fewer than k keys: cannot happen for k <= n
                ft_flag(status, FT_DEV_EINVAL);
                b = 255;
            }
            krem_s = krem;
            prefix_s = prefix | (uint64_t(b) << (8 * dg));
            mask_s = mask | (uint64_t(255) << (8 * dg));
        }
        __syncthreads();
    }
    const uint64_t thr = prefix_s;  // the k-th smallest key
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint64_t key = row[i];
        if (key <= thr) {
            const int pos = atomicAdd(&cnt_s, 1);
            if (pos < MAX_K1) cand[pos] = key;
        }
    }
    __syncthreads();
    int m = 1;
    while (m < k) m <<= 1;
    for (int i = k + threadIdx.x; i < m; i += blockDim.x) cand[i] = ~uint64_t(0);
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
    int qb = 16;
    int log2cap = 6;
    size_t smem = 0;
    int docs_per_block = 256;
};

ft_status plan_scan(const ft_docs* queries, ScanPlan* p) {
    int log2cap = 5;
    while ((1 << log2cap) < 2 * std::max(queries->max_embed, 1)) ++log2cap;
    p->log2cap = log2cap;
    int dev = 0, max_smem = 0;
    FT_CUDA(cudaGetDevice(&dev));
    FT_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t per_q = size_t(8) << log2cap;
    int qb = 16;
    while (qb > 1 && per_q * qb > size_t(max_smem) / 2) qb >>= 1;
    if (per_q * qb > size_t(max_smem)) return FT_EUNSUPPORTED;
    p->qb = qb;
    p->smem = per_q * qb;
    return FT_OK;
}

template <int QB>
ft_status launch_scan_q(const ScanPlan& p, ScanArgs a, cudaStream_t s) {
    auto fn = &k_qt_scan<QB>;
    int bps = 0;
    FT_TRY(ft_prepare_kernel(reinterpret_cast<const void*>(fn), SCAN_THREADS, p.smem, &bps));
    if (bps < 1) return FT_EUNSUPPORTED;
    dim3 grid(unsigned((a.nq + QB - 1) / QB), unsigned((a.nd + p.docs_per_block - 1) / p.docs_per_block));
    fn<<<grid, SCAN_THREADS, p.smem, s>>>(a);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

ft_status launch_scan(const ft_tree* t, const ft_docs* q, const ft_docs* d, uint64_t* keys, int64_t* l1,
                      cudaStream_t s) {
    ScanPlan p;
    FT_TRY(plan_scan(q, &p));
    ScanArgs a{};
    a.q_eptr = q->d_eptr;
    a.q_ekey = q->d_ekey;
    a.q_emass = q->d_emass;
    a.nq = q->n_docs;
    a.d_eptr = d->d_eptr;
    a.d_ekey = d->d_ekey;
    a.d_emass = d->d_emass;
    a.nd = d->n_docs;
    a.L = t->levels;
    a.qb = p.qb;
    a.log2cap = p.log2cap;
    a.docs_per_block = p.docs_per_block;
    a.keys = keys;
    a.l1_out = l1;
    switch (p.qb) {
        case 16: return launch_scan_q<16>(p, a, s);
        case 8: return launch_scan_q<8>(p, a, s);
        case 4: return launch_scan_q<4>(p, a, s);
        case 2: return launch_scan_q<2>(p, a, s);
        default: return launch_scan_q<1>(p, a, s);
    }
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
    FT_TRY(check_scan(t, queries, db, 1));
    if (!l1_all_out_dev) return FT_EINVAL;
    return launch_scan(t, queries, db, nullptr, l1_all_out_dev, static_cast<cudaStream_t>(stream));
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

extern "C" size_t ft_topk_f32_workspace_size(int64_t n_rows, int64_t n_cols) {
    if (n_rows < 1 || n_cols < 1) return 0;
    WsCarver w(nullptr);
    w.take<uint64_t>(size_t(n_rows) * n_cols);
    return w.off + 256;
}

extern "C" ft_status ft_topk_f32(const float* values_dev, int64_t n_rows, int64_t n_cols, int32_t k, void* workspace,
                                 size_t ws_bytes, int32_t* ids_out_dev, float* vals_out_dev, void* stream) {
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
