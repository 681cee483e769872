// Mean-distance prefilter: the "Mean" method of Sec. 5 (the Euclidean
// distance between the two distributions' mass-weighted centroids, a lower
// bound on W1 by Jensen's inequality), as a first stage that ranks a whole
// database for a batch of queries.
//
//   centroid(mu) = sum_i mu_i x_i          (masses mu_i = m_i / 2^24)
//   Mean(q, d)^2 = |c_q|^2 + |c_d|^2 - 2 c_q . c_d
//
// Three kernels, all FP32 (TF32 or BF16 products would move the ranking):
//   k_centroids   a warp per distribution: centroid row and squared norm;
//   k_mean_gemm   the cross terms c_q . c_d of all (query, document) pairs,
//                 128 x 128 output tiles per CTA, 8 x 8 per thread, the
//                 centroid tiles staged through shared memory 16 dimensions
//                 at a time (double-buffered, the next tile prefetched into
//                 registers), with the distance epilogue fused: the kernel
//                 writes sqrt(max(0, |c_q|^2 + |c_d|^2 - 2 c_q . c_d));
//   k_select_rows_f32  per query the k1 smallest distances, ties to the
//                 smaller document id: a radix select over the distance bits
//                 read straight from the distance row (11, 11 and 10 bits),
//                 then over the document ids only when ties at the threshold
//                 overflow the candidate buffer, and a bitonic sort of the
//                 survivors.
#include <algorithm>
#include <type_traits>

#include "ft_internal.cuh"

namespace {

// One warp per document: centroid row and squared norm.  The lanes hold the
// whole centroid in registers (lane l owns vectors l, l + 32, ... of VW
// floats, NV of them); the document's (word, mass) pairs are read 32 at a
// time, one per lane, and broadcast, and every word row is read once,
// coalesced, four rows in flight.
template <int VW, int NV>
__global__ void __launch_bounds__(256) k_centroids(const int64_t* __restrict__ ptr, const uint32_t* __restrict__ mass,
                                                   const uint32_t* __restrict__ word, int64_t n_docs,
                                                   const float* __restrict__ vocab, int dim,
                                                   float* __restrict__ cent, float* __restrict__ norm2) {
    using V = typename std::conditional<VW == 4, float4, float>::type;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    const unsigned lane = lane_id();
    const int nvec = dim / VW;
    const V* vv = reinterpret_cast<const V*>(vocab);
    for (int64_t d = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; d < n_docs; d += warps) {
        const int64_t b = ptr[d], e = ptr[d + 1];
        float acc[NV][VW];
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int c = 0; c < VW; ++c) acc[v][c] = 0.f;
        for (int64_t i0 = b; i0 < e; i0 += 32) {
            const int cnt = int(e - i0 < 32 ? e - i0 : 32);
            uint32_t my_w = 0;
            float my_m = 0.f;
            if (int(lane) < cnt) {
                my_w = word[i0 + lane];
                my_m = float(mass[i0 + lane]) * (1.0f / 16777216.0f);
            }
#pragma unroll 4
            for (int j = 0; j < cnt; ++j) {
                const uint32_t w = __shfl_sync(FULL_MASK, my_w, j);
                const float m = __shfl_sync(FULL_MASK, my_m, j);
                const V* row = vv + size_t(w) * nvec;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const int x = int(lane) + 32 * v;
                    if (x < nvec) {
                        const V r = __ldg(row + x);
                        const float* rf = reinterpret_cast<const float*>(&r);
#pragma unroll
                        for (int c = 0; c < VW; ++c) acc[v][c] = fmaf(m, rf[c], acc[v][c]);
                    }
                }
            }
        }
        float nrm = 0.f;
        V* out = reinterpret_cast<V*>(cent + size_t(d) * dim);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int x = int(lane) + 32 * v;
            if (x < nvec) {
                V o;
                float* of = reinterpret_cast<float*>(&o);
#pragma unroll
                for (int c = 0; c < VW; ++c) {
                    of[c] = acc[v][c];
                    nrm = fmaf(acc[v][c], acc[v][c], nrm);
                }
                out[x] = o;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(FULL_MASK, nrm, o);
        if (lane == 0) norm2[d] = nrm;
    }
}

using CentroidFn = void (*)(const int64_t*, const uint32_t*, const uint32_t*, int64_t, const float*, int, float*,
                            float*);

// the instantiation for this dimension (vectors of 4 when dim % 4 == 0), or
// nullptr beyond 32 x 8 vectors per row
CentroidFn centroid_kernel(int dim) {
    if (dim % 4 == 0) {
        const int nv = (dim / 4 + 31) / 32;
        switch (nv) {
            case 1: return &k_centroids<4, 1>;
            case 2: return &k_centroids<4, 2>;
            case 3: return &k_centroids<4, 3>;
            case 4: return &k_centroids<4, 4>;
            case 5: case 6: return &k_centroids<4, 6>;
            case 7: case 8: return &k_centroids<4, 8>;
            default: return nullptr;
        }
    }
    const int nv = (dim + 31) / 32;
    switch (nv) {
        case 1: return &k_centroids<1, 1>;
        case 2: return &k_centroids<1, 2>;
        case 3: case 4: return &k_centroids<1, 4>;
        case 5: case 6: case 7: case 8: return &k_centroids<1, 8>;
        case 9: case 10: case 11: case 12: return &k_centroids<1, 12>;
        default: return nullptr;
    }
}

int grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    return int(std::max<int64_t>(1, std::min<int64_t>(b, 65535 * 8)));
}

// ---------------------------------------------------------------------------
// cross terms with the distance epilogue: dist[q][d] for q < nq, d < nd
// ---------------------------------------------------------------------------
constexpr int GM = 128, GN = 128, GK = 16, GPAD = 4, GTHREADS = 256;

// Loads the k-chunk [k0, k0 + GK) of rows [r0, r0 + 128) of a row-major
// [rows][dim] table: two float4 (VEC) or eight scalars per thread, zero
// outside the table.
template <bool VEC>
__device__ __forceinline__ void gemm_load(const float* __restrict__ x, int64_t rows, int dim, int64_t r0, int k0,
                                          float (&v)[8]) {
    const int t = threadIdx.x;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int f = t + h * GTHREADS;  // float4 slot: row f / 4, k quad f % 4
        const int64_t r = r0 + (f >> 2);
        const int kk = k0 + (f & 3) * 4;
        if (VEC) {
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < rows && kk < dim) q = __ldg(reinterpret_cast<const float4*>(x + r * dim + kk));
            v[4 * h] = q.x;
            v[4 * h + 1] = q.y;
            v[4 * h + 2] = q.z;
            v[4 * h + 3] = q.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) v[4 * h + j] = (r < rows && kk + j < dim) ? __ldg(x + r * dim + kk + j) : 0.f;
        }
    }
}

// stores the chunk transposed: s[k][row]
__device__ __forceinline__ void gemm_store(float (*s)[GM + GPAD], const float (&v)[8]) {
    const int t = threadIdx.x;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int f = t + h * GTHREADS;
        const int row = f >> 2, kq = (f & 3) * 4;
#pragma unroll
        for (int j = 0; j < 4; ++j) s[kq + j][row] = v[4 * h + j];
    }
}

template <bool VEC>
__global__ void __launch_bounds__(GTHREADS) k_mean_gemm(const float* __restrict__ cq, const float* __restrict__ cd,
                                                       const float* __restrict__ nq2, const float* __restrict__ nd2,
                                                       int64_t nq, int64_t nd, int dim, float* __restrict__ dist) {
    __shared__ __align__(16) float As[2][GK][GM + GPAD];
    __shared__ __align__(16) float Bs[2][GK][GN + GPAD];
    const int t = threadIdx.x;
    const int tx = t & 15, ty = t >> 4;
    const int64_t m0 = int64_t(blockIdx.y) * GM, n0 = int64_t(blockIdx.x) * GN;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    float va[8], vb[8];
    gemm_load<VEC>(cq, nq, dim, m0, 0, va);
    gemm_load<VEC>(cd, nd, dim, n0, 0, vb);
    gemm_store(As[0], va);
    gemm_store(Bs[0], vb);
    __syncthreads();
    const int nk = (dim + GK - 1) / GK;
    for (int kc = 0; kc < nk; ++kc) {
        const int buf = kc & 1;
        if (kc + 1 < nk) {  // the next chunk in flight while this one is used
            gemm_load<VEC>(cq, nq, dim, m0, (kc + 1) * GK, va);
            gemm_load<VEC>(cd, nd, dim, n0, (kc + 1) * GK, vb);
        }
#pragma unroll
        for (int k = 0; k < GK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (kc + 1 < nk) {
            gemm_store(As[buf ^ 1], va);
            gemm_store(Bs[buf ^ 1], vb);
        }
        __syncthreads();
    }
    // epilogue: rows ty*4 + {0..3} and 64 + ty*4 + {0..3}, columns likewise with tx
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (m >= nq) continue;
        const float qn = nq2[m];
        float* row = dist + m * nd;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t n = n0 + h * 64 + tx * 4;
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float dn = (n + j < nd) ? nd2[n + j] : 0.f;
                o[j] = sqrtf(fmaxf(0.f, qn + dn - 2.f * acc[i][4 * h + j]));
            }
            if (n + 3 < nd && (nd & 3) == 0) {
                *reinterpret_cast<float4*>(row + n) = make_float4(o[0], o[1], o[2], o[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (n + j < nd) row[n + j] = o[j];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// per row: the k smallest (distance, column), ascending
// ---------------------------------------------------------------------------
constexpr int SR_THREADS = 512;
constexpr int SR_MAX = 4096;  // candidate buffer (k1 <= 4096)

// 64-bit select key of a non-negative distance: its bits, then the column
__device__ __forceinline__ uint64_t dist_key(float x, int64_t col) {
    uint32_t b = __float_as_uint(x);
    if (x != x) b = 0x7FC00000u;          // NaN after +inf
    else if (b & 0x80000000u) b = 0;      // -0.0 first
    return (uint64_t(b) << 32) | uint64_t(uint32_t(col));
}

__global__ void __launch_bounds__(SR_THREADS) k_select_rows_f32(const float* __restrict__ v, int64_t n, int k,
                                                               int32_t* __restrict__ ids_out,
                                                               float* __restrict__ val_out) {
    __shared__ uint32_t hist[2048];
    __shared__ uint64_t cand[SR_MAX];
    __shared__ uint64_t prefix_s, mask_s;
    __shared__ int krem_s, below_s, eq_s, cnt_s;
    const float* row = v + int64_t(blockIdx.x) * n;
    if (threadIdx.x == 0) {
        prefix_s = 0;
        mask_s = 0;
        krem_s = k;
        below_s = 0;
        cnt_s = 0;
    }
    __syncthreads();
    // digits of the key, most significant first: the distance bits (11, 11,
    // 10), then the column bits (11, 11, 10), the latter only when the keys
    // tied with the threshold distance overflow the candidate buffer
    const int shifts[6] = {53, 42, 32, 21, 10, 0};
    const int widths[6] = {11, 11, 10, 11, 11, 10};
    bool exact = true;
    for (int dg = 0; dg < 6; ++dg) {
        if (dg == 3 && below_s + eq_s <= SR_MAX) {
            exact = false;  // collect every key tied with the threshold distance
            break;
        }
        const int sh = shifts[dg], nb = 1 << widths[dg];
        for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const uint64_t prefix = prefix_s, mask = mask_s;
        for (int64_t i0 = threadIdx.x; i0 < n; i0 += int64_t(blockDim.x) * 8) {
            float x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t i = i0 + int64_t(u) * blockDim.x;
                x[u] = i < n ? __ldg(row + i) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t i = i0 + int64_t(u) * blockDim.x;
                if (i < n) {
                    const uint64_t key = dist_key(x[u], i);
                    if ((key & mask) == prefix) atomicAdd(&hist[(key >> sh) & uint64_t(nb - 1)], 1u);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int krem = krem_s, below = below_s, b = 0;
            for (; b < nb - 1; ++b) {
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
        __syncthreads();
    }
    // exact: the k-th smallest key itself; else every key whose distance is
    // at most the k-th smallest distance (fewer than SR_MAX)
    const uint64_t thr = exact ? prefix_s : (prefix_s | 0xFFFFFFFFull);
    for (int64_t i0 = threadIdx.x; i0 < n; i0 += int64_t(blockDim.x) * 8) {
        float x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t i = i0 + int64_t(u) * blockDim.x;
            x[u] = i < n ? __ldg(row + i) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t i = i0 + int64_t(u) * blockDim.x;
            if (i < n) {
                const uint64_t key = dist_key(x[u], i);
                if (key <= thr) {
                    const int pos = atomicAdd(&cnt_s, 1);
                    if (pos < SR_MAX) cand[pos] = key;
                }
            }
        }
    }
    __syncthreads();
    const int c = min(cnt_s, SR_MAX);
    int m = 1;
    while (m < c) m <<= 1;
    for (int i = c + threadIdx.x; i < m; i += blockDim.x) cand[i] = ~uint64_t(0);
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
        ids_out[int64_t(blockIdx.x) * k + i] = int32_t(key & 0xFFFFFFFFu);
        val_out[int64_t(blockIdx.x) * k + i] = __uint_as_float(uint32_t(key >> 32));
    }
}

struct MeanLayout {
    float* cq;
    float* cd;
    float* nq2;
    float* nd2;
    float* dist;
};

size_t mean_layout(const ft_docs* q, const ft_docs* d, void* base, MeanLayout* out) {
    WsCarver w(base);
    MeanLayout l{};
    const int dim = q->tree->dim;
    l.cq = w.take<float>(size_t(q->n_docs) * dim);
    l.cd = w.take<float>(size_t(d->n_docs) * dim);
    l.nq2 = w.take<float>(size_t(q->n_docs));
    l.nd2 = w.take<float>(size_t(d->n_docs));
    l.dist = w.take<float>(size_t(q->n_docs) * d->n_docs);
    if (out) *out = l;
    return w.off + 256;
}

ft_status check_mean(const float* vocab, const ft_docs* q, const ft_docs* d, int32_t k1) {
    if (!vocab || !q || !d || !q->tree || q->tree != d->tree) return FT_EINVAL;
    if (q->n_docs < 1 || d->n_docs < 1 || k1 < 1 || k1 > 4096 || int64_t(k1) > d->n_docs) return FT_EINVAL;
    if (q->n_docs > int64_t(65535) * 128 || d->n_docs > 0x7FFFFFFF) return FT_EUNSUPPORTED;
    if (!centroid_kernel(q->tree->dim)) return FT_EUNSUPPORTED;  // dim > 1024 (or > 384 when dim % 4 != 0)
    if (q->tree->dim % 4 == 0 && (reinterpret_cast<uintptr_t>(vocab) & 15u) != 0) return FT_EINVAL;
    return FT_OK;
}

}  // namespace

extern "C" size_t ft_mean_scan_workspace_size(const ft_docs* queries, const ft_docs* db, int32_t k1) {
    if (!queries || !db || !queries->tree || queries->tree != db->tree || k1 < 1) return 0;
    return mean_layout(queries, db, nullptr, nullptr);
}

extern "C" ft_status ft_mean_scan(const float* vocab_dev, const ft_docs* queries, const ft_docs* db, int32_t k1,
                                  void* workspace, size_t ws_bytes, int32_t* cand_ids_out_dev,
                                  float* cand_dist_out_dev, void* stream) {
    FtRange nvtx_range("ft_mean_scan");
    FT_TRY(check_mean(vocab_dev, queries, db, k1));
    if (!cand_ids_out_dev || !cand_dist_out_dev) return FT_EINVAL;
    if (!workspace || ws_bytes < mean_layout(queries, db, nullptr, nullptr)) return FT_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MeanLayout l;
    mean_layout(queries, db, workspace, &l);
    const int dim = queries->tree->dim;
    const int64_t nq = queries->n_docs, nd = db->n_docs;
    CentroidFn cent = centroid_kernel(dim);
    cent<<<grid_for(nq * 32, 256), 256, 0, s>>>(queries->d_ptr, queries->d_mass, queries->d_word, nq, vocab_dev, dim,
                                                l.cq, l.nq2);
    cent<<<grid_for(nd * 32, 256), 256, 0, s>>>(db->d_ptr, db->d_mass, db->d_word, nd, vocab_dev, dim, l.cd, l.nd2);
    const dim3 grid(unsigned((nd + GN - 1) / GN), unsigned((nq + GM - 1) / GM));
    if (dim % 4 == 0)
        k_mean_gemm<true><<<grid, GTHREADS, 0, s>>>(l.cq, l.cd, l.nq2, l.nd2, nq, nd, dim, l.dist);
    else
        k_mean_gemm<false><<<grid, GTHREADS, 0, s>>>(l.cq, l.cd, l.nq2, l.nd2, nq, nd, dim, l.dist);
    k_select_rows_f32<<<unsigned(nq), SR_THREADS, 0, s>>>(l.dist, nd, k1, cand_ids_out_dev, cand_dist_out_dev);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}
