// Distributions on the quadtree (Sec. 5 datasets; Sec. 2 l1 embedding).
//
// CSR (doc -> (word, weight)) becomes, per document,
//   * a support sorted by quadtree rank with integer masses summing to 2^24
//     (W = FP64 sum of the weights in CSR order; m_i = floor(w_i/W * 2^24);
//     the remaining units go to the largest fractional parts, ties to the
//     smaller rank; duplicates merged in CSR order; zeros dropped);
//   * its sparse quadtree embedding: one entry per node touched, holding the
//     document's mass under that node.  Nodes that hold a single ground
//     point from some depth c+1 down to the point level form a chain with
//     identical masses; each chain is stored once, keyed by the point, and
//     weighted by the sum of its edge weights 2^(L+1-c) - 1 (the paper's
//     singleton leaves, Sec. 2).  Internal nodes at depth k weigh 2^(L+1-k).
//     Key layout: internal = (k << 24) | node_id, chain = 2^31 | (c << 24) | rank.
#include <cstring>

#include "ft_internal.cuh"

namespace {

constexpr double kMassOneD = 16777216.0;

__global__ void k_check_rowptr(const int64_t* __restrict__ row_ptr, int64_t n_docs, uint32_t* status) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_docs; i += int64_t(gridDim.x) * blockDim.x) {
        if (i == 0 && row_ptr[0] != 0) ft_flag(status, FT_DEV_EINVAL);
        if (row_ptr[i + 1] < row_ptr[i]) ft_flag(status, FT_DEV_EINVAL);
    }
}

// entry checks + sort keys: rank of the entry's word, and its document
__global__ void k_entry_keys(const int64_t* __restrict__ row_ptr, int64_t n_docs, const int32_t* __restrict__ word,
                             const float* __restrict__ weight, const uint32_t* __restrict__ rank_of_point,
                             int64_t n_points, uint32_t* __restrict__ rank_key, uint32_t* __restrict__ doc_key,
                             uint32_t* status) {
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x / 32);
    for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32; i < n_docs; i += warps) {
        const int64_t b = row_ptr[i], e = row_ptr[i + 1];
        for (int64_t j = b + lane_id(); j < e; j += 32) {
            const int32_t w = word[j];
            const float g = weight[j];
            uint32_t r = 0;
            if (w < 0 || int64_t(w) >= n_points) ft_flag(status, FT_DEV_EINVAL);
            else r = rank_of_point[w];
            if (!isfinite(g) || g < 0.0f) ft_flag(status, FT_DEV_EINVAL);
            rank_key[j] = r;
            doc_key[j] = uint32_t(i);
        }
    }
}

// One warp per document.  perm: CSR entry indices sorted by (doc, rank),
// duplicates in CSR order.  Writes the final support at the doc's CSR
// offset in tmp arrays and its length to count[i].
__global__ void k_doc_masses(const int64_t* __restrict__ row_ptr, int64_t n_docs, const int32_t* __restrict__ word,
                             const float* __restrict__ weight, const uint32_t* __restrict__ perm,
                             const uint32_t* __restrict__ rank_key, uint32_t* __restrict__ t_rank,
                             uint32_t* __restrict__ t_word, double* __restrict__ t_x, uint32_t* __restrict__ t_mass,
                             int64_t* __restrict__ count, uint32_t* status) {
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x / 32);
    const unsigned lane = lane_id();
    for (int64_t doc = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32; doc < n_docs; doc += warps) {
        const int64_t b = row_ptr[doc], e = row_ptr[doc + 1];
        // W: FP64 sum of the positive weights in CSR order (one lane)
        double W = 0.0;
        if (lane == 0)
            for (int64_t j = b; j < e; ++j) {
                const float g = weight[j];
                if (g > 0.0f) W = __dadd_rn(W, double(g));
            }
        W = __shfl_sync(FULL_MASK, W, 0);
        if (!(W > 0.0)) {
            if (lane == 0) {
                ft_flag(status, FT_DEV_EINVAL);
                count[doc] = 0;
            }
            continue;
        }
        // items: first positive entry of each rank group; merged weight summed
        // in CSR order over the group's positive entries
        int n_items = 0;
        for (int64_t base = b; base < e; base += 32) {
            const int64_t j = base + lane;
            bool head = false;
            uint32_t r = 0;
            double wsum = 0.0;
            uint32_t wd = 0;
            if (j < e) {
                const uint32_t src = perm[j];
                r = rank_key[src];
                if (weight[src] > 0.0f) {
                    head = true;
                    for (int64_t t = j - 1; t >= b; --t) {
                        const uint32_t s2 = perm[t];
                        if (rank_key[s2] != r) break;
                        if (weight[s2] > 0.0f) { head = false; break; }
                    }
                    if (head) {
                        wd = uint32_t(word[src]);
                        for (int64_t t = j; t < e; ++t) {
                            const uint32_t s2 = perm[t];
                            if (rank_key[s2] != r) break;
                            const float g = weight[s2];
                            if (g > 0.0f) wsum = __dadd_rn(wsum, double(g));
                        }
                    }
                }
            }
            const unsigned hm = __ballot_sync(FULL_MASK, head);
            if (head) {
                const int64_t o = b + n_items + __popc(hm & lanemask_lt());
                t_rank[o] = r;
                t_word[o] = wd;
                t_x[o] = __dmul_rn(__ddiv_rn(wsum, W), kMassOneD);
            }
            n_items += __popc(hm);
        }
        __syncwarp();
        if (n_items > FT_MAX_SUPPORT) {
            if (lane == 0) {
                ft_flag(status, FT_DEV_EUNSUPPORTED);
                count[doc] = 0;
            }
            continue;
        }
        // floors, remainder, fractional parts
        int64_t msum = 0;
        double fmin = 2.0, fmax = -1.0;
        for (int i = lane; i < n_items; i += 32) {
            const double x = t_x[b + i];
            const double m = floor(x);
            msum += int64_t(m);
            const double fr = __dsub_rn(x, m);
            fmin = fmin < fr ? fmin : fr;
            fmax = fmax > fr ? fmax : fr;
        }
        msum = warp_sum_i64(msum);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double omin = __shfl_xor_sync(FULL_MASK, fmin, o);
            const double omax = __shfl_xor_sync(FULL_MASK, fmax, o);
            fmin = fmin < omin ? fmin : omin;
            fmax = fmax > omax ? fmax : omax;
        }
        const int64_t R = int64_t(16777216) - msum;
        if (R < 0 || R > n_items) ft_flag(status, FT_DEV_EOVERFLOW);
        const bool all_equal = (fmin == fmax);
        for (int i = lane; i < n_items; i += 32) {
            const double x = t_x[b + i];
            const double m = floor(x);
            const double fr = __dsub_rn(x, m);
            int64_t pos;
            if (all_equal) {
                pos = i;  // ties everywhere: rank order (items are rank-sorted)
            } else {
                pos = 0;
                for (int j2 = 0; j2 < n_items; ++j2) {
                    const double x2 = t_x[b + j2];
                    const double f2 = __dsub_rn(x2, floor(x2));
                    pos += (f2 > fr || (f2 == fr && j2 < i)) ? 1 : 0;
                }
            }
            t_mass[b + i] = uint32_t(int64_t(m) + (pos < R ? 1 : 0));
        }
        __syncwarp();
        // drop zero masses (stable compaction in place)
        int kept = 0;
        for (int base = 0; base < n_items; base += 32) {
            const int i = base + int(lane);
            uint32_t r = 0, wd = 0, m = 0;
            if (i < n_items) {
                r = t_rank[b + i];
                wd = t_word[b + i];
                m = t_mass[b + i];
            }
            const bool keep = i < n_items && m > 0;
            const unsigned km = __ballot_sync(FULL_MASK, keep);
            __syncwarp();
            if (keep) {
                const int64_t o = b + kept + __popc(km & lanemask_lt());
                t_rank[o] = r;
                t_word[o] = wd;
                t_mass[o] = m;
            }
            kept += __popc(km);
            __syncwarp();
        }
        if (lane == 0) count[doc] = kept;
    }
}

__global__ void k_compact_support(const int64_t* __restrict__ row_ptr, int64_t n_docs, const int64_t* __restrict__ ptr,
                                  const uint32_t* __restrict__ t_rank, const uint32_t* __restrict__ t_word,
                                  const uint32_t* __restrict__ t_mass, uint32_t* __restrict__ rank,
                                  uint32_t* __restrict__ word, uint32_t* __restrict__ mass) {
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x / 32);
    for (int64_t doc = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32; doc < n_docs; doc += warps) {
        const int64_t src = row_ptr[doc], dst = ptr[doc], len = ptr[doc + 1] - ptr[doc];
        for (int64_t i = lane_id(); i < len; i += 32) {
            rank[dst + i] = t_rank[src + i];
            word[dst + i] = t_word[src + i];
            mass[dst + i] = t_mass[src + i];
        }
    }
}

// Sparse quadtree embedding.  pass 0 counts entries per doc, pass 1 writes.
template <bool WRITE>
__global__ void k_embed(const int64_t* __restrict__ ptr, int64_t n_docs, const uint32_t* __restrict__ rank,
                        const uint32_t* __restrict__ mass, const uint8_t* __restrict__ chain,
                        const uint32_t* __restrict__ node_id, int64_t n_points, int L,
                        int64_t* __restrict__ ecount, const int64_t* __restrict__ eptr, uint32_t* __restrict__ ekey,
                        uint32_t* __restrict__ emass) {
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x / 32);
    const unsigned lane = lane_id();
    for (int64_t doc = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32; doc < n_docs; doc += warps) {
        const int64_t b = ptr[doc];
        const int s = int(ptr[doc + 1] - b);
        int64_t out = WRITE ? eptr[doc] : 0;
        int64_t cnt = 0;
        // internal nodes, depth 1..L: runs of items sharing node_id_k among
        // items whose chain depth reaches k
        for (int k = 1; k <= L; ++k) {
            const uint32_t* idk = node_id + size_t(k - 1) * n_points;
            for (int base = 0; base < s; base += 32) {
                const int i = base + int(lane);
                bool head = false;
                uint32_t key = 0, msum = 0;
                if (i < s) {
                    const uint32_t r = rank[b + i];
                    if (chain[r] >= k) {
                        const uint32_t id = idk[r];
                        head = true;
                        if (i > 0) {
                            const uint32_t rp = rank[b + i - 1];
                            if (chain[rp] >= k && idk[rp] == id) head = false;
                        }
                        if (head && WRITE) {
                            key = (uint32_t(k) << 24) | id;
                            for (int t = i; t < s; ++t) {
                                const uint32_t rt = rank[b + t];
                                if (chain[rt] < k || idk[rt] != id) break;
                                msum += mass[b + t];
                            }
                        }
                    }
                }
                const unsigned hm = __ballot_sync(FULL_MASK, head);
                if (WRITE && head) {
                    const int64_t o = out + cnt + __popc(hm & lanemask_lt());
                    ekey[o] = key;
                    emass[o] = msum;
                }
                cnt += __popc(hm);
            }
        }
        // chains: one per item
        if (WRITE)
            for (int i = lane; i < s; i += 32) {
                const uint32_t r = rank[b + i];
                const int64_t o = out + cnt + i;
                ekey[o] = 0x80000000u | (uint32_t(chain[r]) << 24) | r;
                emass[o] = mass[b + i];
            }
        cnt += s;
        if (!WRITE && lane == 0) ecount[doc] = cnt;
    }
}

__global__ void k_max_len(const int64_t* __restrict__ ptr, int64_t n, unsigned* __restrict__ out) {
    unsigned m = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        m = max(m, unsigned(ptr[i + 1] - ptr[i]));
    m = __reduce_max_sync(FULL_MASK, m);
    if (lane_id() == 0) atomicMax(out, m);
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

void free_docs(ft_docs* d) {
    if (!d) return;
    cudaFree(d->d_ptr);
    cudaFree(d->d_rank);
    cudaFree(d->d_mass);
    cudaFree(d->d_word);
    cudaFree(d->d_eptr);
    cudaFree(d->d_ekey);
    cudaFree(d->d_emass);
    cudaFree(d->d_ukey);
    cudaFree(d->d_uoff);
    cudaFree(d->d_post);
    delete d;
}

// ---------------------------------------------------------------------------
// inverted index of the embeddings (node key -> documents), for the scan
// ---------------------------------------------------------------------------
__global__ void k_entry_doc(const int64_t* __restrict__ eptr, int64_t n_docs, uint32_t* __restrict__ edoc) {
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x / 32);
    for (int64_t doc = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32; doc < n_docs; doc += warps)
        for (int64_t j = eptr[doc] + lane_id(); j < eptr[doc + 1]; j += 32) edoc[j] = uint32_t(doc);
}

// postings in key order (documents ascending within a key: the sort is
// stable and entries are laid out document by document); flag[i] = 1 where
// a new key starts
__global__ void k_postings(const uint32_t* __restrict__ perm, const uint32_t* __restrict__ ekey,
                           const uint32_t* __restrict__ emass, const uint32_t* __restrict__ edoc, int64_t n,
                           uint32_t* __restrict__ skey, uint2* __restrict__ post, int64_t* __restrict__ flag) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t e = perm[i];
        const uint32_t k = ekey[e];
        skey[i] = k;
        post[i] = make_uint2(edoc[e], emass[e]);
        flag[i] = (i == 0 || ekey[perm[i - 1]] != k) ? 1 : 0;
    }
}

__global__ void k_unique_keys(const uint32_t* __restrict__ skey, const int64_t* __restrict__ excl, int64_t n,
                              uint32_t* __restrict__ ukey, uint32_t* __restrict__ uoff) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const bool start = (i == 0) || (skey[i] != skey[i - 1]);
        if (start) {
            const int64_t id = excl[i];
            ukey[id] = skey[i];
            uoff[id] = uint32_t(i);
        }
    }
}

ft_status build_index(ft_docs* d, cudaStream_t s) {
    const int64_t n = d->n_embed;
    if (n >= (int64_t(1) << 32)) return FT_EUNSUPPORTED;
    TmpBufs tmp;
    uint32_t *perm, *edoc, *skey;
    int64_t *flag, *scan_tmp;
    void* sort_tmp;
    FT_TRY(tmp.get(&perm, size_t(n)));
    FT_TRY(tmp.get(&edoc, size_t(n)));
    FT_TRY(tmp.get(&skey, size_t(n)));
    FT_TRY(tmp.get(&flag, size_t(n) + 1));
    FT_TRY(tmp.get(&scan_tmp, ft_scan_tmp_elems(n + 1)));
    FT_TRY(tmp.get(reinterpret_cast<char**>(&sort_tmp), ft_sort_tmp_bytes(n)));
    FT_TRY(dmalloc(&d->d_post, size_t(n)));
    k_entry_doc<<<grid_for(d->n_docs * 32, 256), 256, 0, s>>>(d->d_eptr, d->n_docs, edoc);
    FT_TRY(ft_iota_u32(perm, n, s));
    FT_TRY(ft_sort_perm_by_u32(d->d_ekey, perm, n, 32, sort_tmp, s));
    k_postings<<<grid_for(n, 256), 256, 0, s>>>(perm, d->d_ekey, d->d_emass, edoc, n, skey, d->d_post, flag);
    FT_CUDA(cudaMemsetAsync(flag + n, 0, 8, s));
    FT_TRY(ft_exclusive_scan_i64(flag, flag, n + 1, scan_tmp, s));
    FT_CUDA(cudaMemcpyAsync(&d->n_ukeys, flag + n, 8, cudaMemcpyDeviceToHost, s));
    FT_CUDA(cudaStreamSynchronize(s));
    FT_TRY(dmalloc(&d->d_ukey, size_t(d->n_ukeys)));
    FT_TRY(dmalloc(&d->d_uoff, size_t(d->n_ukeys) + 1));
    k_unique_keys<<<grid_for(n, 256), 256, 0, s>>>(skey, flag, n, d->d_ukey, d->d_uoff);
    const uint32_t end = uint32_t(n);
    FT_CUDA(cudaMemcpyAsync(d->d_uoff + d->n_ukeys, &end, 4, cudaMemcpyHostToDevice, s));
    FT_CUDA(cudaGetLastError());
    FT_CUDA(cudaStreamSynchronize(s));
    return FT_OK;
}

ft_status read_status(const ft_tree* t, cudaStream_t s) {
    uint32_t w = 0;
    FT_CUDA(cudaMemcpyAsync(&w, t->d_status, 4, cudaMemcpyDeviceToHost, s));
    FT_CUDA(cudaMemsetAsync(t->d_status, 0, 4, s));
    FT_CUDA(cudaStreamSynchronize(s));
    if (w & FT_DEV_EINVAL) return FT_EINVAL;
    if (w & FT_DEV_EUNSUPPORTED) return FT_EUNSUPPORTED;
    if (w & FT_DEV_EOVERFLOW) return FT_EOVERFLOW;
    return FT_OK;
}

ft_status embed(const ft_tree* t, const int64_t* row_ptr, const int32_t* word, const float* weight, int64_t n_docs,
                cudaStream_t s, ft_docs* d) {
    TmpBufs tmp;
    d->tree = t;
    d->n_docs = n_docs;
    FT_TRY(read_status(t, s));  // start from a clean status word
    k_check_rowptr<<<grid_for(n_docs, 256), 256, 0, s>>>(row_ptr, n_docs, t->d_status);
    FT_CUDA(cudaGetLastError());
    FT_TRY(read_status(t, s));
    int64_t nnz = 0;
    FT_CUDA(cudaMemcpyAsync(&nnz, row_ptr + n_docs, 8, cudaMemcpyDeviceToHost, s));
    FT_CUDA(cudaStreamSynchronize(s));
    if (nnz < n_docs || nnz >= (int64_t(1) << 32)) return nnz < n_docs ? FT_EINVAL : FT_EUNSUPPORTED;

    // sort entries by (doc, rank), CSR order among equals
    uint32_t *rank_key, *doc_key, *perm;
    void* sort_tmp;
    FT_TRY(tmp.get(&rank_key, size_t(nnz)));
    FT_TRY(tmp.get(&doc_key, size_t(nnz)));
    FT_TRY(tmp.get(&perm, size_t(nnz)));
    FT_TRY(tmp.get(reinterpret_cast<char**>(&sort_tmp), ft_sort_tmp_bytes(nnz)));
    k_entry_keys<<<grid_for(n_docs * 32, 256), 256, 0, s>>>(row_ptr, n_docs, word, weight, t->d_rank_of_point, t->n,
                                                            rank_key, doc_key, t->d_status);
    FT_CUDA(cudaGetLastError());
    FT_TRY(read_status(t, s));
    int rank_bits = 1;
    while ((int64_t(1) << rank_bits) < t->n) ++rank_bits;
    int doc_bits = 1;
    while ((int64_t(1) << doc_bits) < n_docs) ++doc_bits;
    FT_TRY(ft_iota_u32(perm, nnz, s));
    FT_TRY(ft_sort_perm_by_u32(rank_key, perm, nnz, rank_bits, sort_tmp, s));
    FT_TRY(ft_sort_perm_by_u32(doc_key, perm, nnz, doc_bits, sort_tmp, s));

    // per-document masses
    uint32_t *t_rank, *t_word, *t_mass;
    double* t_x;
    int64_t *count, *scan_tmp;
    FT_TRY(tmp.get(&t_rank, size_t(nnz)));
    FT_TRY(tmp.get(&t_word, size_t(nnz)));
    FT_TRY(tmp.get(&t_mass, size_t(nnz)));
    FT_TRY(tmp.get(&t_x, size_t(nnz)));
    FT_TRY(tmp.get(&count, size_t(n_docs) + 1));
    FT_TRY(tmp.get(&scan_tmp, ft_scan_tmp_elems(n_docs + 1)));
    k_doc_masses<<<grid_for(n_docs * 32, 256), 256, 0, s>>>(row_ptr, n_docs, word, weight, perm, rank_key, t_rank,
                                                            t_word, t_x, t_mass, count, t->d_status);
    FT_CUDA(cudaGetLastError());
    FT_TRY(read_status(t, s));
    FT_TRY(dmalloc(&d->d_ptr, size_t(n_docs) + 1));
    FT_CUDA(cudaMemsetAsync(count + n_docs, 0, 8, s));
    FT_TRY(ft_exclusive_scan_i64(count, d->d_ptr, n_docs + 1, scan_tmp, s));
    FT_CUDA(cudaMemcpyAsync(&d->n_items, d->d_ptr + n_docs, 8, cudaMemcpyDeviceToHost, s));
    FT_CUDA(cudaStreamSynchronize(s));
    FT_TRY(dmalloc(&d->d_rank, size_t(d->n_items)));
    FT_TRY(dmalloc(&d->d_word, size_t(d->n_items)));
    FT_TRY(dmalloc(&d->d_mass, size_t(d->n_items)));
    k_compact_support<<<grid_for(n_docs * 32, 256), 256, 0, s>>>(row_ptr, n_docs, d->d_ptr, t_rank, t_word, t_mass,
                                                                 d->d_rank, d->d_word, d->d_mass);
    unsigned* dmax;
    FT_TRY(tmp.get(&dmax, 2));
    FT_CUDA(cudaMemsetAsync(dmax, 0, 8, s));
    k_max_len<<<grid_for(n_docs, 256), 256, 0, s>>>(d->d_ptr, n_docs, dmax);

    // sparse embedding
    FT_TRY(dmalloc(&d->d_eptr, size_t(n_docs) + 1));
    k_embed<false><<<grid_for(n_docs * 32, 256), 256, 0, s>>>(d->d_ptr, n_docs, d->d_rank, d->d_mass, t->d_chain,
                                                              t->d_node_id, t->n, t->levels, count, nullptr, nullptr,
                                                              nullptr);
    FT_TRY(ft_exclusive_scan_i64(count, d->d_eptr, n_docs + 1, scan_tmp, s));
    FT_CUDA(cudaMemcpyAsync(&d->n_embed, d->d_eptr + n_docs, 8, cudaMemcpyDeviceToHost, s));
    FT_CUDA(cudaStreamSynchronize(s));
    FT_TRY(dmalloc(&d->d_ekey, size_t(d->n_embed)));
    FT_TRY(dmalloc(&d->d_emass, size_t(d->n_embed)));
    k_embed<true><<<grid_for(n_docs * 32, 256), 256, 0, s>>>(d->d_ptr, n_docs, d->d_rank, d->d_mass, t->d_chain,
                                                             t->d_node_id, t->n, t->levels, nullptr, d->d_eptr,
                                                             d->d_ekey, d->d_emass);
    // longest embedding
    FT_CUDA(cudaMemsetAsync(dmax + 1, 0, 4, s));
    k_max_len<<<grid_for(n_docs, 256), 256, 0, s>>>(d->d_eptr, n_docs, dmax + 1);
    FT_CUDA(cudaGetLastError());
    unsigned hmax[2] = {0, 0};
    FT_CUDA(cudaMemcpyAsync(hmax, dmax, 8, cudaMemcpyDeviceToHost, s));
    FT_CUDA(cudaStreamSynchronize(s));
    d->max_support = int(hmax[0]);
    d->max_embed = int(hmax[1]);
    d->h_eptr.resize(size_t(n_docs) + 1);
    FT_CUDA(cudaMemcpy(d->h_eptr.data(), d->d_eptr, size_t(n_docs + 1) * 8, cudaMemcpyDeviceToHost));
    FT_TRY(build_index(d, s));
    return read_status(t, s);
}

}  // namespace

extern "C" ft_status ft_embed_docs(const ft_tree* t, const int64_t* row_ptr_dev, const int32_t* word_dev,
                                   const float* weight_dev, int64_t n_docs, void* stream, ft_docs** out) {
    FtRange nvtx_range("ft_embed_docs");
    if (!out) return FT_EINVAL;
    *out = nullptr;
    if (!t || !row_ptr_dev || !word_dev || !weight_dev || n_docs < 1 || n_docs >= (int64_t(1) << 31)) return FT_EINVAL;
    ft_docs* d = new ft_docs;
    ft_status st = embed(t, row_ptr_dev, word_dev, weight_dev, n_docs, static_cast<cudaStream_t>(stream), d);
    if (st != FT_OK) {
        free_docs(d);
        return st;
    }
    *out = d;
    return FT_OK;
}

extern "C" void ft_docs_free(ft_docs* d) { free_docs(d); }

extern "C" ft_status ft_docs_get_info(const ft_docs* d, ft_docs_info* info) {
    if (!d || !info) return FT_EINVAL;
    info->n_docs = d->n_docs;
    info->n_items = d->n_items;
    info->max_support = d->max_support;
    info->n_embed = d->n_embed;
    return FT_OK;
}

extern "C" ft_status ft_docs_export(const ft_docs* d, int64_t* sup_ptr_host, uint32_t* sup_point_host,
                                    uint32_t* sup_mass_host) {
    if (!d) return FT_EINVAL;
    if (sup_ptr_host) FT_CUDA(cudaMemcpy(sup_ptr_host, d->d_ptr, size_t(d->n_docs + 1) * 8, cudaMemcpyDeviceToHost));
    if (sup_point_host) FT_CUDA(cudaMemcpy(sup_point_host, d->d_word, size_t(d->n_items) * 4, cudaMemcpyDeviceToHost));
    if (sup_mass_host) FT_CUDA(cudaMemcpy(sup_mass_host, d->d_mass, size_t(d->n_items) * 4, cudaMemcpyDeviceToHost));
    return FT_OK;
}
