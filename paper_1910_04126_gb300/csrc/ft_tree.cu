// Quadtree build (Sec. 2 "Generic Quadtree") on the GPU.
//
// The tree is never materialised as nodes.  Every quadtree node is a
// contiguous interval of the "rank" order (depth-first order of the halving
// with children ordered by their bit vector, dimension 0 most significant),
// so the tree is fully described by
//   rank_of_point / point_of_rank,
//   lcp[r]    = depth of the lowest common ancestor of ranks r and r+1,
//   rmq[j][r] = min(lcp[r .. r + 2^j - 1])  (LCA depth of any two ranks),
//   chain[r]  = deepest depth at which rank r shares a cell with another
//               point (below it the point is alone: the paper's leaf),
//   node_id[k][r] = dense id of the depth-k node holding rank r.
// Build: quantise once (40-bit integer grid, random shift) -> per-point cell
// code at depth L -> Morton byte keys (bit-plane major) -> stable LSD radix
// sort -> lcp -> tables.
#include <cmath>
#include <cstring>

#include "ft_internal.cuh"

namespace {

constexpr uint64_t kOneB = uint64_t(1) << FT_LEAF_BITS;

__global__ void k_minmax_partial(const float* __restrict__ pts, int64_t n, int d, int rows_per_block,
                                 float* __restrict__ pmin, float* __restrict__ pmax, uint32_t* status) {
    const int64_t r0 = int64_t(blockIdx.x) * rows_per_block;
    const int64_t r1 = min(n, r0 + rows_per_block);
    for (int c = threadIdx.x; c < d; c += blockDim.x) {
        float mn = INFINITY, mx = -INFINITY;
        bool bad = false;
        for (int64_t r = r0; r < r1; ++r) {
            float v = pts[r * d + c];
            bad |= !isfinite(v);
            mn = fminf(mn, v);
            mx = fmaxf(mx, v);
        }
        if (bad) ft_flag(status, FT_DEV_EINVAL);
        pmin[int64_t(blockIdx.x) * d + c] = mn;
        pmax[int64_t(blockIdx.x) * d + c] = mx;
    }
}

__global__ void k_minmax_final(const float* __restrict__ pmin, const float* __restrict__ pmax, int nblk, int d,
                               float* __restrict__ lo, float* __restrict__ hi) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d) return;
    float mn = INFINITY, mx = -INFINITY;
    for (int b = 0; b < nblk; ++b) {
        mn = fminf(mn, pmin[int64_t(b) * d + c]);
        mx = fmaxf(mx, pmax[int64_t(b) * d + c]);
    }
    lo[c] = mn;
    hi[c] = mx;
}

// Cell code at depth L of every coordinate: z >> (B + 1 - L), where
// q = min(2^B, floor((x - lo) * 2^B / Phi)) and z = min(q + 2^B - s, 2^(B+1) - 1).
__global__ void k_quantize(const float* __restrict__ pts, int64_t n, int d, int L, double scale,
                           const float* __restrict__ lo, const uint64_t* __restrict__ shift,
                           uint16_t* __restrict__ cell) {
    const int64_t total = n * d;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(i % d);
        const double diff = __dsub_rn(double(pts[i]), double(lo[c]));
        const double scaled = __dmul_rn(diff, scale);
        uint64_t q = uint64_t(floor(scaled));
        if (q > kOneB) q = kOneB;
        uint64_t z = q + kOneB - shift[c];
        if (z > 2 * kOneB - 1) z = 2 * kOneB - 1;
        cell[i] = uint16_t(z >> (FT_LEAF_BITS + 1 - L));
    }
}

// Morton key as a byte string, most significant first: bit j = (k-1)*d + c
// (k = 1..L, c = 0..d-1) is bit (L-k) of the depth-L cell code of dim c.
__global__ void k_morton_bytes(const uint16_t* __restrict__ cell, int64_t n, int d, int L, int key_bytes,
                               uint8_t* __restrict__ keys) {
    const int64_t total = n * key_bytes;
    const int nbits = L * d;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t p = i / key_bytes;
        const int b = int(i % key_bytes);
        uint32_t byte = 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int j = b * 8 + t;
            uint32_t bit = 0;
            if (j < nbits) {
                const int k = j / d + 1;
                const int c = j % d;
                bit = (cell[p * d + c] >> (L - k)) & 1u;
            }
            byte = (byte << 1) | bit;
        }
        keys[i] = uint8_t(byte);
    }
}

// varying[b] |= key[p][b] ^ key[0][b]  (byte positions where points differ)
__global__ void k_key_varying(const uint8_t* __restrict__ keys, int64_t n, int key_bytes, uint32_t* __restrict__ var) {
    const int64_t total = n * key_bytes;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int b = int(i % key_bytes);
        if (keys[i] != keys[b]) atomicOr(&var[b], 1u);
    }
}

__global__ void k_iota(uint32_t* __restrict__ a, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        a[i] = uint32_t(i);
}

__global__ void k_invert(const uint32_t* __restrict__ por, uint32_t* __restrict__ rop, int64_t n) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x)
        rop[por[r]] = uint32_t(r);
}

// lcp[r] = L - bitlen(OR_c (cell_p[c] ^ cell_q[c])) for p, q at ranks r, r+1:
// the deepest common cell is where all coordinates still agree.  One warp per r.
__global__ void k_lcp(const uint16_t* __restrict__ cell, const uint32_t* __restrict__ por, int64_t n, int d, int L,
                      uint8_t* __restrict__ lcp) {
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x / 32);
    const unsigned lane = lane_id();
    for (int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32; r < n; r += warps) {
        if (r == n - 1) {
            if (lane == 0) lcp[r] = 0;
            continue;
        }
        const int64_t p = por[r], q = por[r + 1];
        uint32_t x = 0;
        for (int c = lane; c < d; c += 32) x |= uint32_t(cell[p * d + c] ^ cell[q * d + c]);
        x = __reduce_or_sync(FULL_MASK, x);
        if (lane == 0) {
            const int bitlen = x ? 32 - __clz(x) : 0;
            lcp[r] = uint8_t(L - bitlen);
        }
    }
}

__global__ void k_rmq_level(const uint8_t* __restrict__ prev, uint8_t* __restrict__ next, int64_t n, int64_t half) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
        uint8_t v = prev[r];
        if (r + half < n) v = min(v, prev[r + half]);
        next[r] = v;
    }
}

__global__ void k_chain(const uint8_t* __restrict__ lcp, int64_t n, uint8_t* __restrict__ chain) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
        uint8_t m = 0;
        if (r > 0) m = lcp[r - 1];
        if (r + 1 < n) m = max(m, lcp[r]);
        chain[r] = m;
    }
}

// flag[r] = 1 if rank r starts a new depth-k node
__global__ void k_node_start(const uint8_t* __restrict__ lcp, int64_t n, int k, int64_t* __restrict__ flag) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x)
        flag[r] = (r == 0 || lcp[r - 1] < k) ? 1 : 0;
}

__global__ void k_node_id(const int64_t* __restrict__ excl, const uint8_t* __restrict__ lcp, int64_t n, int k,
                          uint32_t* __restrict__ id) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
        const int64_t f = (r == 0 || lcp[r - 1] < k) ? 1 : 0;
        id[r] = uint32_t(excl[r] + f - 1);
    }
}

uint64_t splitmix64_next(uint64_t* state) {
    // S. Vigna's splitmix64 (public-domain reference definition).
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int phi_log2_for(double range) {
    if (!(range > 0.0)) return 0;
    int ex = 0;
    double m = std::frexp(range, &ex);
    return (m == 0.5) ? ex - 1 : ex;
}

int grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535 * 8) b = 65535 * 8;
    return int(b);
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

struct TmpBufs {
    std::vector<void*> ptrs;
    ~TmpBufs() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <class T>
    ft_status get(T** p, size_t count) {
        FT_TRY(dmalloc(p, count));
        ptrs.push_back(*p);
        return FT_OK;
    }
};

void free_tree(ft_tree* t) {
    if (!t) return;
    cudaFree(t->d_rank_of_point);
    cudaFree(t->d_point_of_rank);
    cudaFree(t->d_lcp);
    cudaFree(t->d_rmq);
    cudaFree(t->d_chain);
    cudaFree(t->d_node_id);
    cudaFree(t->d_status);
    delete t;
}

ft_status build(const float* pts, int64_t n, int d, int L, const uint64_t* shift_host, uint64_t seed,
                cudaStream_t s, ft_tree* t) {
    TmpBufs tmp;
    t->n = n;
    t->dim = d;
    t->levels = L;
    FT_CUDA(cudaGetDevice(&t->device));
    FT_TRY(ft_device_sms(&t->num_sms));
    t->shift.resize(size_t(d));
    if (shift_host) {
        for (int c = 0; c < d; ++c) t->shift[size_t(c)] = shift_host[c];
    } else {
        uint64_t st = seed;
        for (int c = 0; c < d; ++c) t->shift[size_t(c)] = splitmix64_next(&st) % (kOneB + 1);
    }
    FT_TRY(dmalloc(&t->d_status, 1));
    FT_CUDA(cudaMemsetAsync(t->d_status, 0, 4, s));

    // 1. per-dimension min / max
    const int rows_per_block = 256;
    const int nblk = ft_ceil_div(n, rows_per_block);
    float *pmin, *pmax, *dlo, *dhi;
    FT_TRY(tmp.get(&pmin, size_t(nblk) * d));
    FT_TRY(tmp.get(&pmax, size_t(nblk) * d));
    FT_TRY(tmp.get(&dlo, size_t(d)));
    FT_TRY(tmp.get(&dhi, size_t(d)));
    k_minmax_partial<<<nblk, 128, 0, s>>>(pts, n, d, rows_per_block, pmin, pmax, t->d_status);
    k_minmax_final<<<ft_ceil_div(d, 128), 128, 0, s>>>(pmin, pmax, nblk, d, dlo, dhi);
    FT_CUDA(cudaGetLastError());
    std::vector<float> hlo(static_cast<size_t>(d)), hhi(static_cast<size_t>(d));
    uint32_t st_word = 0;
    FT_CUDA(cudaMemcpyAsync(hlo.data(), dlo, size_t(d) * 4, cudaMemcpyDeviceToHost, s));
    FT_CUDA(cudaMemcpyAsync(hhi.data(), dhi, size_t(d) * 4, cudaMemcpyDeviceToHost, s));
    FT_CUDA(cudaMemcpyAsync(&st_word, t->d_status, 4, cudaMemcpyDeviceToHost, s));
    FT_CUDA(cudaStreamSynchronize(s));
    if (st_word) return FT_EINVAL;  // non-finite coordinate
    t->lo = hlo;
    double range = 0.0;
    for (int c = 0; c < d; ++c) range = std::max(range, double(hhi[size_t(c)]) - double(hlo[size_t(c)]));
    t->phi_log2 = phi_log2_for(range);
    const double scale = std::ldexp(1.0, FT_LEAF_BITS - t->phi_log2);

    // 2. quantise to depth-L cell codes
    uint64_t* dshift;
    uint16_t* cell;
    FT_TRY(tmp.get(&dshift, size_t(d)));
    FT_TRY(tmp.get(&cell, size_t(n) * d));
    FT_CUDA(cudaMemcpyAsync(dshift, t->shift.data(), size_t(d) * 8, cudaMemcpyHostToDevice, s));
    k_quantize<<<grid_for(n * d, 256), 256, 0, s>>>(pts, n, d, L, scale, dlo, dshift, cell);

    // 3. Morton byte keys and the byte positions that vary
    const int key_bytes = (L * d + 7) / 8;
    uint8_t* keys;
    uint32_t* var;
    FT_TRY(tmp.get(&keys, size_t(n) * key_bytes));
    FT_TRY(tmp.get(&var, size_t(key_bytes)));
    k_morton_bytes<<<grid_for(n * key_bytes, 256), 256, 0, s>>>(cell, n, d, L, key_bytes, keys);
    FT_CUDA(cudaMemsetAsync(var, 0, size_t(key_bytes) * 4, s));
    k_key_varying<<<grid_for(n * key_bytes, 256), 256, 0, s>>>(keys, n, key_bytes, var);
    FT_CUDA(cudaGetLastError());
    std::vector<uint32_t> hvar(static_cast<size_t>(key_bytes));
    FT_CUDA(cudaMemcpyAsync(hvar.data(), var, size_t(key_bytes) * 4, cudaMemcpyDeviceToHost, s));
    FT_CUDA(cudaStreamSynchronize(s));
    std::vector<uint8_t> varying(static_cast<size_t>(key_bytes));
    for (int b = 0; b < key_bytes; ++b) varying[size_t(b)] = hvar[size_t(b)] ? 1 : 0;

    // 4. rank order: stable sort of point ids by key (ties keep id order)
    FT_TRY(dmalloc(&t->d_point_of_rank, size_t(n)));
    FT_TRY(dmalloc(&t->d_rank_of_point, size_t(n)));
    void* sort_tmp;
    FT_TRY(tmp.get(reinterpret_cast<char**>(&sort_tmp), ft_sort_tmp_bytes(n)));
    k_iota<<<grid_for(n, 256), 256, 0, s>>>(t->d_point_of_rank, n);
    FT_TRY(ft_sort_perm_by_bytes(keys, key_bytes, varying, t->d_point_of_rank, n, sort_tmp, s));
    k_invert<<<grid_for(n, 256), 256, 0, s>>>(t->d_point_of_rank, t->d_rank_of_point, n);

    // 5. lcp, range-minimum table, chain depth
    FT_TRY(dmalloc(&t->d_lcp, size_t(n)));
    k_lcp<<<grid_for(n * 32, 256), 256, 0, s>>>(cell, t->d_point_of_rank, n, d, L, t->d_lcp);
    int rl = 1;
    while ((int64_t(1) << rl) <= n) ++rl;  // rows j with 2^j <= n
    t->rmq_levels = rl;
    FT_TRY(dmalloc(&t->d_rmq, size_t(rl) * n));
    FT_CUDA(cudaMemcpyAsync(t->d_rmq, t->d_lcp, size_t(n), cudaMemcpyDeviceToDevice, s));
    for (int j = 1; j < rl; ++j)
        k_rmq_level<<<grid_for(n, 256), 256, 0, s>>>(t->d_rmq + size_t(j - 1) * n, t->d_rmq + size_t(j) * n, n,
                                                     int64_t(1) << (j - 1));
    FT_TRY(dmalloc(&t->d_chain, size_t(n)));
    k_chain<<<grid_for(n, 256), 256, 0, s>>>(t->d_lcp, n, t->d_chain);

    // 6. dense node ids per depth 1..L
    FT_TRY(dmalloc(&t->d_node_id, size_t(L) * n));
    int64_t *flag, *scan_tmp;
    FT_TRY(tmp.get(&flag, size_t(n)));
    FT_TRY(tmp.get(&scan_tmp, ft_scan_tmp_elems(n)));
    for (int k = 1; k <= L; ++k) {
        k_node_start<<<grid_for(n, 256), 256, 0, s>>>(t->d_lcp, n, k, flag);
        FT_TRY(ft_exclusive_scan_i64(flag, flag, n, scan_tmp, s));
        k_node_id<<<grid_for(n, 256), 256, 0, s>>>(flag, t->d_lcp, n, k, t->d_node_id + size_t(k - 1) * n);
    }
    FT_CUDA(cudaGetLastError());
    FT_CUDA(cudaStreamSynchronize(s));
    return FT_OK;
}

}  // namespace

extern "C" ft_status ft_build_quadtree(const float* points_dev, int64_t n_points, int32_t dim, int32_t levels,
                                       const uint64_t* shift_host, uint64_t seed, void* stream, ft_tree** out) {
    FtRange nvtx_range("ft_build_quadtree");
    if (!out) return FT_EINVAL;
    *out = nullptr;
    if (!points_dev || n_points < 1 || n_points >= (int64_t(1) << 24) || dim < 1 || levels < 1 ||
        levels > FT_MAX_LEVELS)
        return FT_EINVAL;
    if (shift_host)
        for (int c = 0; c < dim; ++c)
            if (shift_host[c] > kOneB) return FT_EINVAL;
    ft_tree* t = new ft_tree;
    ft_status st = build(points_dev, n_points, dim, levels, shift_host, seed, static_cast<cudaStream_t>(stream), t);
    if (st != FT_OK) {
        free_tree(t);
        return st;
    }
    *out = t;
    return FT_OK;
}

extern "C" void ft_tree_free(ft_tree* t) { free_tree(t); }

extern "C" ft_status ft_tree_get_info(const ft_tree* t, ft_tree_info* info) {
    if (!t || !info) return FT_EINVAL;
    info->n_points = t->n;
    info->dim = t->dim;
    info->levels = t->levels;
    info->phi_log2 = t->phi_log2;
    info->rmq_levels = t->rmq_levels;
    return FT_OK;
}

extern "C" ft_status ft_tree_export(const ft_tree* t, uint32_t* rank_of_point_host, uint32_t* point_of_rank_host,
                                    uint8_t* lcp_host, uint64_t* shift_host) {
    if (!t) return FT_EINVAL;
    if (rank_of_point_host) FT_CUDA(cudaMemcpy(rank_of_point_host, t->d_rank_of_point, size_t(t->n) * 4, cudaMemcpyDeviceToHost));
    if (point_of_rank_host) FT_CUDA(cudaMemcpy(point_of_rank_host, t->d_point_of_rank, size_t(t->n) * 4, cudaMemcpyDeviceToHost));
    if (lcp_host && t->n > 1) FT_CUDA(cudaMemcpy(lcp_host, t->d_lcp, size_t(t->n - 1), cudaMemcpyDeviceToHost));
    if (shift_host) std::memcpy(shift_host, t->shift.data(), t->shift.size() * 8);
    return FT_OK;
}

extern "C" ft_status ft_tree_status(const ft_tree* t, void* stream) {
    if (!t) return FT_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t w = 0;
    FT_CUDA(cudaMemcpyAsync(&w, t->d_status, 4, cudaMemcpyDeviceToHost, s));
    FT_CUDA(cudaMemsetAsync(t->d_status, 0, 4, s));
    FT_CUDA(cudaStreamSynchronize(s));
    if (w & FT_DEV_EINVAL) return FT_EINVAL;
    if (w & FT_DEV_EOVERFLOW) return FT_EOVERFLOW;
    if (w & FT_DEV_EUNSUPPORTED) return FT_EUNSUPPORTED;
    if (w & FT_DEV_ETIMEOUT) return FT_ETIMEOUT;
    return FT_OK;
}

extern "C" ft_status ft_flowtree_set_config(ft_tree* t, const ft_flowtree_config* cfg) {
    if (!t || !cfg) return FT_EINVAL;
    if (cfg->warps_per_cta < 0 || cfg->warps_per_cta > 8 || cfg->stage_items < 0 || cfg->stage_items > 16384 ||
        cfg->algo < FT_ALGO_AUTO || cfg->algo > FT_ALGO_BLOCKED || cfg->stage_tables < 0 || cfg->stage_tables > 1 ||
        cfg->deep_loads < 0 || cfg->deep_loads > 1)
        return FT_EINVAL;
    if (cfg->algo == FT_ALGO_THREAD && t->dim > 8) return FT_EUNSUPPORTED;
    t->cfg = *cfg;
    return FT_OK;
}

extern "C" ft_status ft_flowtree_get_config(const ft_tree* t, ft_flowtree_config* cfg) {
    if (!t || !cfg) return FT_EINVAL;
    *cfg = t->cfg;
    return FT_OK;
}
