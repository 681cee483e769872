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
//   3. chunks of 32 sorted contributions -> one partial vector per run of
//      equal points inside a chunk;
//   4. per point, its partials (contiguous, in sorted order) are summed in
//      order and added to grad.
#include "ft_internal.cuh"

namespace {

constexpr int CHUNK = 32;
constexpr int COORD_BLOCK = 256;  // coordinates per pass: 8 per lane

__global__ void k_bwd_slots(const int64_t* __restrict__ slot_ptr, const int32_t* __restrict__ count,
                            const uint32_t* __restrict__ f_ia, const uint32_t* __restrict__ f_ib,
                            const uint32_t* __restrict__ f_f, const uint8_t* __restrict__ f_depth,
                            const float* __restrict__ f_dist, const int32_t* __restrict__ pair_a,
                            const int32_t* __restrict__ pair_b, int64_t nb_cross, int64_t n_pairs,
                            const int64_t* __restrict__ a_ptr, const uint32_t* __restrict__ a_word,
                            const int64_t* __restrict__ b_ptr, const uint32_t* __restrict__ b_word,
                            const float* __restrict__ grad_cost, int levels, uint32_t sentinel,
                            uint32_t* __restrict__ key, uint32_t* __restrict__ s_wa, uint32_t* __restrict__ s_wb,
                            float* __restrict__ s_coef) {
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x / 32);
    const unsigned lane = lane_id();
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

// runs of equal non-sentinel keys inside each chunk of 32 sorted entries
__global__ void k_bwd_chunk_runs(const uint32_t* __restrict__ key, const uint32_t* __restrict__ perm, int64_t n,
                                 uint32_t sentinel, int64_t n_chunks, int64_t* __restrict__ runs) {
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < n_chunks; c += int64_t(gridDim.x) * blockDim.x) {
        int64_t r = 0;
        uint32_t prev = sentinel;
        const int64_t e1 = min(n, (c + 1) * CHUNK);
        for (int64_t j = c * CHUNK; j < e1; ++j) {
            const uint32_t k = key[perm[j]];
            if (k != sentinel && (j == c * CHUNK || k != prev)) ++r;
            prev = k;
        }
        runs[c] = r;
    }
}

__global__ void k_bwd_partials(const uint32_t* __restrict__ key, const uint32_t* __restrict__ perm, int64_t n,
                               uint32_t sentinel, int64_t n_chunks, const int64_t* __restrict__ run_off,
                               const uint32_t* __restrict__ s_wa, const uint32_t* __restrict__ s_wb,
                               const float* __restrict__ s_coef, const float* __restrict__ vocab, int dim,
                               uint32_t* __restrict__ part_word, float* __restrict__ part) {
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x / 32);
    const unsigned lane = lane_id();
    for (int64_t c = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32; c < n_chunks; c += warps) {
        const int64_t j = c * CHUNK + lane;
        const uint32_t e = j < n ? perm[j] : 0u;
        const uint32_t k = j < n ? key[e] : sentinel;
        for (int cb = 0; cb < dim; cb += COORD_BLOCK) {
            float acc[COORD_BLOCK / 32];
#pragma unroll
            for (int t = 0; t < COORD_BLOCK / 32; ++t) acc[t] = 0.0f;
            int64_t slot = run_off[c] - 1;
            uint32_t prev = sentinel;
            for (int q = 0; q < CHUNK; ++q) {
                const uint32_t kq = __shfl_sync(FULL_MASK, k, q);
                if (kq == sentinel) break;
                const uint32_t eq = __shfl_sync(FULL_MASK, e, q);
                if (q == 0 || kq != prev) {
                    if (slot >= run_off[c]) {
#pragma unroll
                        for (int t = 0; t < COORD_BLOCK / 32; ++t) {
                            const int x = cb + t * 32 + int(lane);
                            if (x < dim) part[size_t(slot) * dim + x] = acc[t];
                            acc[t] = 0.0f;
                        }
                    }
                    ++slot;
                    if (lane == 0 && cb == 0) part_word[slot] = kq;
                    prev = kq;
                }
                const uint32_t s = eq >> 1;
                const float coef = (eq & 1u) ? -s_coef[s] : s_coef[s];
                const float* xa = vocab + size_t(s_wa[s]) * dim;
                const float* xb = vocab + size_t(s_wb[s]) * dim;
#pragma unroll
                for (int t = 0; t < COORD_BLOCK / 32; ++t) {
                    const int x = cb + t * 32 + int(lane);
                    if (x < dim) acc[t] = fmaf(coef, __ldg(xa + x) - __ldg(xb + x), acc[t]);
                }
            }
            if (slot >= run_off[c]) {
#pragma unroll
                for (int t = 0; t < COORD_BLOCK / 32; ++t) {
                    const int x = cb + t * 32 + int(lane);
                    if (x < dim) part[size_t(slot) * dim + x] = acc[t];
                }
            }
        }
    }
}

__global__ void k_bwd_finalize(const uint32_t* __restrict__ part_word, const float* __restrict__ part,
                               const int64_t* __restrict__ n_part_dev, int dim, float* __restrict__ grad) {
    const int64_t n_part = *n_part_dev;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x / 32);
    const unsigned lane = lane_id();
    for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32; i < n_part; i += warps) {
        const uint32_t w = part_word[i];
        if (i > 0 && part_word[i - 1] == w) continue;
        int64_t end = i + 1;
        while (end < n_part && part_word[end] == w) ++end;
        for (int x = lane; x < dim; x += 32) {
            float s = 0.0f;
            for (int64_t j = i; j < end; ++j) s += part[size_t(j) * dim + x];
            grad[size_t(w) * dim + x] += s;
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
    int64_t* runs;
    int64_t* scan_tmp;
    uint32_t* part_word;
    float* part;
    int64_t max_part;
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
    l.runs = w.take<int64_t>(size_t(n_chunks) + 1);
    l.scan_tmp = w.take<int64_t>(ft_scan_tmp_elems(n_chunks + 1));
    l.max_part = std::min<int64_t>(ne, n_chunks + t->n + 1);
    l.part_word = w.take<uint32_t>(size_t(l.max_part));
    l.part = w.take<float>(size_t(l.max_part) * t->dim);
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
        flows->d_pair_a, flows->d_pair_b, flows->nb_cross, flows->n_pairs, a->d_ptr, a->d_word, b->d_ptr, b->d_word,
        grad_cost_dev, t->levels, sentinel, l.key, l.s_wa, l.s_wb, l.s_coef);
    FT_TRY(ft_iota_u32(l.perm, ne, s));
    FT_TRY(ft_sort_perm_by_u32(l.key, l.perm, ne, key_bits, l.sort_tmp, s));
    k_bwd_chunk_runs<<<grid_for(n_chunks, 256), 256, 0, s>>>(l.key, l.perm, ne, sentinel, n_chunks, l.runs);
    FT_CUDA(cudaMemsetAsync(l.runs + n_chunks, 0, 8, s));
    FT_TRY(ft_exclusive_scan_i64(l.runs, l.runs, n_chunks + 1, l.scan_tmp, s));
    k_bwd_partials<<<grid_for(n_chunks * 32, 256), 256, 0, s>>>(l.key, l.perm, ne, sentinel, n_chunks, l.runs,
                                                                l.s_wa, l.s_wb, l.s_coef, vocab_dev, t->dim,
                                                                l.part_word, l.part);
    k_bwd_finalize<<<grid_for(l.max_part * 32, 256), 256, 0, s>>>(l.part_word, l.part, l.runs + n_chunks, t->dim,
                                                                  grad_vocab_dev);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}
