// Adjoint of the batched Flowtree estimate for the frozen tree flow.
//
// The paper prices the tree flow f with Euclidean distances (Sec. 3):
// W~ = sum f(x, y) ||x - y||.  The flow depends on the quadtree cells only,
// so for fixed cells dW~/dx = sum_y f(x, y) (x - y)/||x - y|| and the
// opposite sign for y.  With upstream gradients g_i per pair:
//   grad[x] += g_i f/2^24 (x - y)/||x - y||,  grad[y] -= the same.
// Deterministic, no floating-point atomics:
//   1. one coefficient per saved flow record, two contributions per record
//      (one per endpoint), keyed by the point they update;
//   2. stable radix sort of the contributions by point;
//   3. a warp per chunk of CHUNK sorted contributions sums every run of
//      equal points in order.  A run that lies inside the chunk holds all of
//      its point's contributions: the warp adds it to grad directly.  A run
//      cut by a chunk boundary goes to one of the chunk's two partial slots
//      (A: the run that continues from the previous chunk, B: the run that
//      starts in this chunk and continues into the next);
//   4. every B slot starts a chain B(c), A(c+1), A(c+2), ... of one point.
//      A warp sums a chain of at most 16 elements in order; a longer chain
//      gets a CTA, whose warp r sums elements r, r + 8, ... and whose eight
//      warp sums are then added in warp order.  The total goes to grad.
// Rows are read as float4 when the dimension and the pointers allow it.
#include <algorithm>
#include <cstdint>

#include "ft_internal.cuh"

namespace {

constexpr int CHUNK = 64;       // sorted contributions per warp
constexpr int COLS = 3;         // row vectors per lane in one column block (block = 96 vectors)
constexpr int CHAIN_WARPS = 8;  // warps per CTA of a long chain
constexpr int SHORT_CHAIN = 16; // longest chain one warp sums alone
constexpr int BATCH = 2;        // contributions whose rows are loaded together

__device__ __forceinline__ void vzero(float& a) { a = 0.0f; }
__device__ __forceinline__ void vzero(float4& a) { a = make_float4(0.0f, 0.0f, 0.0f, 0.0f); }
__device__ __forceinline__ void vfma_diff(float& a, float c, float x, float y) { a = fmaf(c, x - y, a); }
__device__ __forceinline__ void vfma_diff(float4& a, float c, const float4& x, const float4& y) {
    a.x = fmaf(c, x.x - y.x, a.x);
    a.y = fmaf(c, x.y - y.y, a.y);
    a.z = fmaf(c, x.z - y.z, a.z);
    a.w = fmaf(c, x.w - y.w, a.w);
}
__device__ __forceinline__ void vadd(float& a, float b) { a += b; }
__device__ __forceinline__ void vadd(float4& a, const float4& b) {
    a.x += b.x;
    a.y += b.y;
    a.z += b.z;
    a.w += b.w;
}

template <int VEC>
struct VecOf;
template <>
struct VecOf<1> {
    using T = float;
};
template <>
struct VecOf<4> {
    using T = float4;
};

__global__ void k_bwd_slots(const int64_t* __restrict__ slot_ptr, const int32_t* __restrict__ count,
                            const uint32_t* __restrict__ f_ia, const uint32_t* __restrict__ f_ib,
                            const uint32_t* __restrict__ f_f, const uint8_t* __restrict__ f_depth,
                            const float* __restrict__ f_dist, const int32_t* __restrict__ pair_a,
                            const int32_t* __restrict__ pair_b, int64_t nb_cross, int64_t n_pairs,
                            const int64_t* __restrict__ a_ptr, const uint32_t* __restrict__ a_word,
                            const int64_t* __restrict__ b_ptr, const uint32_t* __restrict__ b_word,
                            const float* __restrict__ grad_cost, int levels, uint32_t sentinel,
                            uint32_t* __restrict__ key, uint32_t* __restrict__ s_wa, uint32_t* __restrict__ s_wb,
                            float* __restrict__ s_coef, int64_t capacity) {
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x / 32);
    const unsigned lane = lane_id();
    // slots past the bound pairs' total (flows sized for more pairs than
    // they hold) take no part: sentinel keys sort them last
    for (int64_t s = slot_ptr[n_pairs] + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < capacity;
         s += int64_t(gridDim.x) * blockDim.x) {
        key[2 * s] = sentinel;
        key[2 * s + 1] = sentinel;
        s_wa[s] = 0;
        s_wb[s] = 0;
        s_coef[s] = 0.0f;
    }
    for (int64_t p = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32; p < n_pairs; p += warps) {
        int64_t da, db;
        if (pair_a) {
            da = pair_a[p];
            db = pair_b[p];
        } else {
            da = p / nb_cross;
            db = p - da * nb_cross;
        }
        const int64_t s0 = slot_ptr[p], s1 = slot_ptr[p + 1];
        const int64_t cnt = count[p];
        const float g = grad_cost[p];
        const int64_t ao = a_ptr[da], bo = b_ptr[db];
        for (int64_t s = s0 + lane; s < s1; s += 32) {
            bool valid = false;
            uint32_t wa = 0, wb = 0;
            float coef = 0.0f;
            if (s - s0 < cnt) {
                wa = a_word[ao + f_ia[s]];
                wb = b_word[bo + f_ib[s]];
                const float dist = f_dist[s];
                valid = int(f_depth[s]) <= levels && dist > 0.0f;
                if (valid) coef = g * (float(f_f[s]) * (1.0f / 16777216.0f)) / dist;
            }
            key[2 * s] = valid ? wa : sentinel;
            key[2 * s + 1] = valid ? wb : sentinel;
            s_wa[s] = wa;
            s_wb[s] = wb;
            s_coef[s] = coef;
        }
    }
}

// A chunk of sorted contributions: its range, the keys just outside it and
// the points that went to its two partial slots (sentinel = unused).
struct RunChunk {
    int64_t c, j0, j1;
    uint32_t k_before, k_after, sentinel;
    uint32_t used_a, used_b;
};

// Adds the run [rs, re) of point cur (column block cb) to grad when the run
// holds all of the point's contributions, else to the chunk's partial slot
// (A when it continues from the previous chunk, B when it continues into the
// next one); clears the accumulators.
template <class V>
__device__ __forceinline__ void flush_run(V (&acc)[COLS], uint32_t cur, int64_t rs, int64_t re, RunChunk& rc, int cb,
                                          int nv, unsigned lane, V* __restrict__ gv, V* __restrict__ pv) {
    if (cur == rc.sentinel) return;
    const bool from_prev = rs == rc.j0 && rc.k_before == cur;
    const bool to_next = re == rc.j1 && rc.k_after == cur;
    if (!from_prev && !to_next) {
#pragma unroll
        for (int t = 0; t < COLS; ++t) {
            const int x = cb + t * 32 + int(lane);
            if (x < nv) {
                V g = gv[size_t(cur) * nv + x];
                vadd(g, acc[t]);
                gv[size_t(cur) * nv + x] = g;
            }
        }
    } else {
        const int64_t slot = 2 * rc.c + (from_prev ? 0 : 1);
#pragma unroll
        for (int t = 0; t < COLS; ++t) {
            const int x = cb + t * 32 + int(lane);
            if (x < nv) pv[size_t(slot) * nv + x] = acc[t];
        }
        if (from_prev) rc.used_a = cur; else rc.used_b = cur;
    }
#pragma unroll
    for (int t = 0; t < COLS; ++t) vzero(acc[t]);
}

// Step 3: one warp per chunk of CHUNK sorted contributions.  Every
// contribution of a run updates the run's own point w, and for both
// endpoints it is coef * (x_w - x_other) (for the nu endpoint,
// -coef (x_a - x_b) = coef (x_b - x_a), the same floating-point value), so
// each contribution gathers only the other endpoint's row; x_w is loaded once
// per run.  Lane q of a 32-entry window holds contribution q (point, other
// point, coefficient); the warp walks the window in order, BATCH
// contributions at a time with their row loads in flight together.
// Three resident CTAs per SM (at most 80 registers per thread): more warps
// waiting on the row gathers beat more rows in flight per warp.
template <int VEC>
__global__ void __launch_bounds__(256, 3) k_bwd_runs(const uint32_t* __restrict__ key, const uint32_t* __restrict__ perm,
                                                  int64_t n, uint32_t sentinel, const uint32_t* __restrict__ s_wa,
                                                  const uint32_t* __restrict__ s_wb, const float* __restrict__ s_coef,
                                                  const float* __restrict__ vocab, int dim, float* __restrict__ grad,
                                                  uint32_t* __restrict__ part_word, float* __restrict__ part,
                                                  uint32_t* __restrict__ heads, uint32_t* __restrict__ n_heads) {
    using V = typename VecOf<VEC>::T;
    const int nv = dim / VEC;  // vectors per row
    const int64_t n_chunks = (n + CHUNK - 1) / CHUNK;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x / 32);
    const unsigned lane = lane_id();
    const V* vv = reinterpret_cast<const V*>(vocab);
    V* gv = reinterpret_cast<V*>(grad);
    V* pv = reinterpret_cast<V*>(part);
    for (int64_t c = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32; c < n_chunks; c += warps) {
        const int64_t j0 = c * CHUNK, j1 = min(n, j0 + CHUNK);
        const uint32_t k_before = j0 > 0 ? key[perm[j0 - 1]] : sentinel;
        const uint32_t k_after = j1 < n ? key[perm[j1]] : sentinel;
        RunChunk rc{c, j0, j1, k_before, k_after, sentinel, sentinel, sentinel};
        for (int cb = 0; cb < nv; cb += 32 * COLS) {
            V acc[COLS], xw[COLS];
#pragma unroll
            for (int t = 0; t < COLS; ++t) {
                vzero(acc[t]);
                vzero(xw[t]);
            }
            uint32_t cur = sentinel;  // point of the open run
            int64_t rs = j0;          // where it started
            int64_t end = j1;         // first sentinel (sentinels sort last)
            for (int64_t jb = j0; jb < end; jb += 32) {
                const int64_t j = jb + lane;
                uint32_t k = sentinel, o = 0;
                float cf = 0.0f;
                if (j < end) {
                    const uint32_t e = perm[j];
                    k = key[e];
                    if (k != sentinel) {
                        const uint32_t s = e >> 1;
                        o = (e & 1u) ? s_wa[s] : s_wb[s];
                        cf = s_coef[s];
                    }
                }
                const unsigned vm = __ballot_sync(FULL_MASK, k != sentinel);
                const int cnt = __popc(vm);  // valid keys are a prefix of the window
                if (cnt < 32) end = jb + cnt;
                for (int q = 0; q < cnt; q += BATCH) {
                    // the other endpoints' rows of BATCH contributions in flight
                    V xo[BATCH][COLS];
#pragma unroll
                    for (int u = 0; u < BATCH; ++u) {
                        const uint32_t ou = __shfl_sync(FULL_MASK, o, (q + u) & 31);
#pragma unroll
                        for (int t = 0; t < COLS; ++t) {
                            const int x = cb + t * 32 + int(lane);
                            vzero(xo[u][t]);
                            if (x < nv && q + u < cnt) xo[u][t] = __ldg(vv + size_t(ou) * nv + x);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < BATCH; ++u) {
                        const uint32_t ku = __shfl_sync(FULL_MASK, k, (q + u) & 31);
                        const float cu = __shfl_sync(FULL_MASK, cf, (q + u) & 31);
                        if (q + u < cnt) {
                            if (ku != cur) {  // a run starts: load its own row
                                flush_run<V>(acc, cur, rs, jb + q + u, rc, cb, nv, lane, gv, pv);
                                cur = ku;
                                rs = jb + q + u;
#pragma unroll
                                for (int t = 0; t < COLS; ++t) {
                                    const int x = cb + t * 32 + int(lane);
                                    if (x < nv) xw[t] = __ldg(vv + size_t(ku) * nv + x);
                                }
                            }
#pragma unroll
                            for (int t = 0; t < COLS; ++t) vfma_diff(acc[t], cu, xw[t], xo[u][t]);
                        }
                    }
                }
            }
            flush_run<V>(acc, cur, rs, end, rc, cb, nv, lane, gv, pv);
        }
        if (lane == 0) {
            part_word[2 * c] = rc.used_a;
            part_word[2 * c + 1] = rc.used_b;
            if (rc.used_b != sentinel) heads[atomicAdd(n_heads, 1u)] = uint32_t(c);
        }
    }
}

// Length of the chain that starts at B(c0) of point w: B(c0) plus the A
// slots of w that follow (whole warp; the result is on every lane).
__device__ __forceinline__ int chain_length(const uint32_t* __restrict__ part_word, int64_t n_chunks, int64_t c0,
                                            uint32_t w) {
    const unsigned lane = lane_id();
    int m = 1;
    for (int64_t base = c0 + 1; base < n_chunks; base += 32) {
        const int64_t cc = base + lane;
        const bool same = cc < n_chunks && part_word[2 * cc] == w;
        const unsigned b = __ballot_sync(FULL_MASK, same);
        const int run = __ffs(~b) - 1;  // leading matches (b == all ones -> -1)
        m += run < 0 ? 32 : run;
        if (run >= 0) break;
    }
    return m;
}

__device__ __forceinline__ int64_t chain_slot(int64_t c0, int i) { return i == 0 ? 2 * c0 + 1 : 2 * (c0 + i); }

// Step 4a: a warp per chain head.  A chain of at most SHORT_CHAIN elements is
// summed by the warp in order and added to grad; a longer one goes to the
// list of long chains.
template <int VEC>
__global__ void __launch_bounds__(256) k_bwd_chains(const uint32_t* __restrict__ heads,
                                                    const uint32_t* __restrict__ counters,
                                                    const uint32_t* __restrict__ part_word,
                                                    const float* __restrict__ part, int64_t n_chunks, int dim,
                                                    float* __restrict__ grad, uint32_t* __restrict__ long_heads,
                                                    uint32_t* __restrict__ n_long) {
    using V = typename VecOf<VEC>::T;
    const int nv = dim / VEC;
    const unsigned lane = lane_id();
    const V* pv = reinterpret_cast<const V*>(part);
    V* gv = reinterpret_cast<V*>(grad);
    const uint32_t nh = counters[0];
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t h = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; h < nh; h += warps) {
        const int64_t c0 = heads[h];
        const uint32_t w = part_word[2 * c0 + 1];
        const int m = chain_length(part_word, n_chunks, c0, w);
        if (m > SHORT_CHAIN) {
            if (lane == 0) long_heads[atomicAdd(n_long, 1u)] = uint32_t(c0);
            continue;
        }
        for (int cb = 0; cb < nv; cb += 32 * COLS) {
            V acc[COLS];
#pragma unroll
            for (int t = 0; t < COLS; ++t) vzero(acc[t]);
            for (int i = 0; i < m; ++i) {
                const int64_t slot = chain_slot(c0, i);
#pragma unroll
                for (int t = 0; t < COLS; ++t) {
                    const int x = cb + t * 32 + int(lane);
                    if (x < nv) vadd(acc[t], pv[size_t(slot) * nv + x]);
                }
            }
#pragma unroll
            for (int t = 0; t < COLS; ++t) {
                const int x = cb + t * 32 + int(lane);
                if (x < nv) {
                    V g = gv[size_t(w) * nv + x];
                    vadd(g, acc[t]);
                    gv[size_t(w) * nv + x] = g;
                }
            }
        }
    }
}

// Step 4b: a CTA per long chain (persistent over the list): warp r sums
// elements r, r + CHAIN_WARPS, ... in order, then the warp sums are added in
// warp order.
template <int VEC>
__global__ void __launch_bounds__(CHAIN_WARPS * 32) k_bwd_long_chains(const uint32_t* __restrict__ long_heads,
                                                                      const uint32_t* __restrict__ n_long,
                                                                      const uint32_t* __restrict__ part_word,
                                                                      const float* __restrict__ part,
                                                                      int64_t n_chunks, int dim,
                                                                      float* __restrict__ grad) {
    using V = typename VecOf<VEC>::T;
    __shared__ V red[CHAIN_WARPS][32 * COLS];
    const int nv = dim / VEC;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const V* pv = reinterpret_cast<const V*>(part);
    V* gv = reinterpret_cast<V*>(grad);
    const uint32_t nl = *n_long;
    for (uint32_t h = blockIdx.x; h < nl; h += gridDim.x) {
        const int64_t c0 = long_heads[h];
        const uint32_t w = part_word[2 * c0 + 1];
        const int m = chain_length(part_word, n_chunks, c0, w);  // every warp, same value
        for (int cb = 0; cb < nv; cb += 32 * COLS) {
            V acc[COLS];
#pragma unroll
            for (int t = 0; t < COLS; ++t) vzero(acc[t]);
            for (int i = int(warp); i < m; i += CHAIN_WARPS) {
                const int64_t slot = chain_slot(c0, i);
#pragma unroll
                for (int t = 0; t < COLS; ++t) {
                    const int x = cb + t * 32 + int(lane);
                    if (x < nv) vadd(acc[t], pv[size_t(slot) * nv + x]);
                }
            }
#pragma unroll
            for (int t = 0; t < COLS; ++t) red[warp][t * 32 + lane] = acc[t];
            __syncthreads();
            if (warp == 0) {
#pragma unroll
                for (int t = 0; t < COLS; ++t) {
                    const int x = cb + t * 32 + int(lane);
                    V s = red[0][t * 32 + lane];
#pragma unroll
                    for (int r = 1; r < CHAIN_WARPS; ++r) vadd(s, red[r][t * 32 + lane]);
                    if (x < nv) {
                        V g = gv[size_t(w) * nv + x];
                        vadd(g, s);
                        gv[size_t(w) * nv + x] = g;
                    }
                }
            }
            __syncthreads();
        }
    }
}

int grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535 * 8) b = 65535 * 8;
    return int(b);
}

struct BwdLayout {
    uint32_t* key;
    uint32_t* perm;
    void* sort_tmp;
    uint32_t* s_wa;
    uint32_t* s_wb;
    float* s_coef;
    uint32_t* part_word;
    float* part;
    uint32_t* heads;
    uint32_t* long_heads;
    uint32_t* counters;  // [0] chain heads, [1] long chains
};

size_t bwd_layout(const ft_tree* t, const ft_flows* f, void* base, BwdLayout* out) {
    WsCarver w(base);
    BwdLayout l{};
    const int64_t ne = 2 * f->capacity;
    const int64_t n_chunks = (ne + CHUNK - 1) / CHUNK;
    l.key = w.take<uint32_t>(size_t(ne));
    l.perm = w.take<uint32_t>(size_t(ne));
    l.sort_tmp = w.take<uint8_t>(ft_sort_tmp_bytes(ne));
    l.s_wa = w.take<uint32_t>(size_t(f->capacity));
    l.s_wb = w.take<uint32_t>(size_t(f->capacity));
    l.s_coef = w.take<float>(size_t(f->capacity));
    l.part_word = w.take<uint32_t>(size_t(2 * n_chunks));
    l.part = w.take<float>(size_t(2 * n_chunks) * t->dim);
    l.heads = w.take<uint32_t>(size_t(n_chunks));
    l.long_heads = w.take<uint32_t>(size_t(n_chunks));
    l.counters = w.take<uint32_t>(2);
    if (out) *out = l;
    return w.off + 256;
}

}  // namespace

extern "C" size_t ft_flowtree_backward_workspace_size(const ft_tree* t, const ft_flows* flows) {
    if (!t || !flows) return 0;
    return bwd_layout(t, flows, nullptr, nullptr);
}

extern "C" ft_status ft_flowtree_backward(const ft_tree* t, const ft_docs* a, const ft_docs* b, const ft_flows* flows,
                                          const float* vocab_dev, const float* grad_cost_dev, float* grad_vocab_dev,
                                          void* workspace, size_t ws_bytes, void* stream) {
    FtRange nvtx_range("ft_flowtree_backward");
    if (!t || !a || !b || !flows || !vocab_dev || !grad_cost_dev || !grad_vocab_dev) return FT_EINVAL;
    if (a->tree != t || b->tree != t) return FT_EINVAL;
    if (flows->cross && flows->nb_cross != b->n_docs) return FT_EINVAL;
    const size_t need = bwd_layout(t, flows, nullptr, nullptr);
    if (!workspace || ws_bytes < need) return FT_EWORKSPACE;
    if (flows->n_pairs == 0 || flows->capacity == 0) return FT_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BwdLayout l;
    bwd_layout(t, flows, workspace, &l);
    const int64_t ne = 2 * flows->capacity;
    const int64_t n_chunks = (ne + CHUNK - 1) / CHUNK;
    const uint32_t sentinel = uint32_t(t->n);
    int key_bits = 1;
    while ((int64_t(1) << key_bits) <= t->n) ++key_bits;

    k_bwd_slots<<<grid_for(flows->n_pairs * 32, 256), 256, 0, s>>>(
        flows->d_slot_ptr, flows->d_count, flows->d_ia, flows->d_ib, flows->d_f, flows->d_depth, flows->d_dist,
        flows->cross ? nullptr : flows->d_pair_a, flows->cross ? nullptr : flows->d_pair_b, flows->nb_cross,
        flows->n_pairs, a->d_ptr, a->d_word, b->d_ptr, b->d_word, grad_cost_dev, t->levels, sentinel, l.key, l.s_wa,
        l.s_wb, l.s_coef, flows->capacity);
    FT_TRY(ft_iota_u32(l.perm, ne, s));
    FT_TRY(ft_sort_perm_by_u32(l.key, l.perm, ne, key_bits, l.sort_tmp, s));
    FT_CUDA(cudaMemsetAsync(l.counters, 0, 2 * sizeof(uint32_t), s));
    const int dim = t->dim;
    const bool vec4 = dim % 4 == 0 && (reinterpret_cast<uintptr_t>(vocab_dev) & 15u) == 0 &&
                      (reinterpret_cast<uintptr_t>(grad_vocab_dev) & 15u) == 0;
    const int grid_runs = grid_for(n_chunks * 32, 256);
    const int grid_chains = int(std::max<int64_t>(1, std::min<int64_t>((n_chunks + 7) / 8, int64_t(t->num_sms) * 8)));
    const int grid_long = std::max(1, t->num_sms * 2);
    if (vec4) {
        k_bwd_runs<4><<<grid_runs, 256, 0, s>>>(l.key, l.perm, ne, sentinel, l.s_wa, l.s_wb, l.s_coef, vocab_dev, dim,
                                                grad_vocab_dev, l.part_word, l.part, l.heads, l.counters);
        k_bwd_chains<4><<<grid_chains, 256, 0, s>>>(l.heads, l.counters, l.part_word, l.part, n_chunks, dim,
                                                    grad_vocab_dev, l.long_heads, l.counters + 1);
        k_bwd_long_chains<4><<<grid_long, CHAIN_WARPS * 32, 0, s>>>(l.long_heads, l.counters + 1, l.part_word, l.part,
                                                                    n_chunks, dim, grad_vocab_dev);
    } else {
        k_bwd_runs<1><<<grid_runs, 256, 0, s>>>(l.key, l.perm, ne, sentinel, l.s_wa, l.s_wb, l.s_coef, vocab_dev, dim,
                                                grad_vocab_dev, l.part_word, l.part, l.heads, l.counters);
        k_bwd_chains<1><<<grid_chains, 256, 0, s>>>(l.heads, l.counters, l.part_word, l.part, n_chunks, dim,
                                                    grad_vocab_dev, l.long_heads, l.counters + 1);
        k_bwd_long_chains<1><<<grid_long, CHAIN_WARPS * 32, 0, s>>>(l.long_heads, l.counters + 1, l.part_word, l.part,
                                                                    n_chunks, dim, grad_vocab_dev);
    }
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}
