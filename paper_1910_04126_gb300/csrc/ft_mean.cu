// Mean-distance prefilter: the "Mean" method of Sec. 5 (the Euclidean
// distance between the two distributions' mass-weighted centroids, a lower
// bound on W1 by Jensen's inequality), as a first stage that ranks a whole
// database for a batch of queries.
//
//   centroid(mu) = sum_i mu_i x_i          (masses mu_i = m_i / 2^24)
//   Mean(q, d)^2 = |c_q|^2 + |c_d|^2 - 2 c_q . c_d
//
// The cross term for all (query, document) pairs is one plain FP32 GEMM of
// the two centroid tables (cuBLAS SGEMM: a library GEMM on the CUDA cores,
// FP32 so that the ranking keeps FP32 accuracy); a fused epilogue adds the
// norms and takes the square root, and the per-query top-k1 reuses the value
// select of ft_topk_f32.
#include <cublas_v2.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "ft_internal.cuh"

namespace {

// one warp per document: centroid row and squared norm
__global__ void k_centroids(const int64_t* __restrict__ ptr, const uint32_t* __restrict__ mass,
                            const uint32_t* __restrict__ word, int64_t n_docs, const float* __restrict__ vocab,
                            int dim, float* __restrict__ cent, float* __restrict__ norm2) {
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    const unsigned lane = lane_id();
    for (int64_t d = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; d < n_docs; d += warps) {
        const int64_t b = ptr[d], e = ptr[d + 1];
        float nrm = 0.0f;
        for (int t = int(lane); t < dim; t += 32) {
            float acc = 0.0f;
            for (int64_t i = b; i < e; ++i)
                acc = fmaf(float(mass[i]) * (1.0f / 16777216.0f), __ldg(vocab + size_t(word[i]) * dim + t), acc);
            cent[size_t(d) * dim + t] = acc;
            nrm = fmaf(acc, acc, nrm);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(FULL_MASK, nrm, o);
        if (lane == 0) norm2[d] = nrm;
    }
}

// dist[q][d] = sqrt(max(0, |c_q|^2 + |c_d|^2 - 2 G[q][d])), in place over G
__global__ void k_mean_epilogue(float* __restrict__ g, const float* __restrict__ nq2, const float* __restrict__ nd2,
                                int64_t nq, int64_t nd) {
    const int64_t n = nq * nd;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t q = i / nd, d = i - q * nd;
        g[i] = sqrtf(fmaxf(0.0f, nq2[q] + nd2[d] - 2.0f * g[i]));
    }
}

int grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    return int(std::max<int64_t>(1, std::min<int64_t>(b, 65535 * 8)));
}

// one cuBLAS handle per device, created on first use (outside any capture)
ft_status cublas_handle(cublasHandle_t* out) {
    static std::mutex mu;
    static std::unordered_map<int, cublasHandle_t> handles;
    int dev = 0;
    FT_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    auto it = handles.find(dev);
    if (it == handles.end()) {
        cublasHandle_t h = nullptr;
        if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return FT_ECUDA;
        it = handles.emplace(dev, h).first;
    }
    *out = it->second;
    return FT_OK;
}

struct MeanLayout {
    float* cq;
    float* cd;
    float* nq2;
    float* nd2;
    float* dist;
    void* topk_ws;
    size_t topk_bytes;
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
    l.topk_bytes = ft_topk_f32_workspace_size(q->n_docs, d->n_docs);
    l.topk_ws = w.take<uint8_t>(l.topk_bytes);
    if (out) *out = l;
    return w.off + 256;
}

ft_status check_mean(const float* vocab, const ft_docs* q, const ft_docs* d, int32_t k1) {
    if (!vocab || !q || !d || !q->tree || q->tree != d->tree) return FT_EINVAL;
    if (q->n_docs < 1 || d->n_docs < 1 || k1 < 1 || k1 > 4096 || int64_t(k1) > d->n_docs) return FT_EINVAL;
    if (q->n_docs > 0x7FFFFFFF || d->n_docs > 0x7FFFFFFF) return FT_EUNSUPPORTED;
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
    k_centroids<<<grid_for(nq * 32, 256), 256, 0, s>>>(queries->d_ptr, queries->d_mass, queries->d_word, nq,
                                                       vocab_dev, dim, l.cq, l.nq2);
    k_centroids<<<grid_for(nd * 32, 256), 256, 0, s>>>(db->d_ptr, db->d_mass, db->d_word, nd, vocab_dev, dim, l.cd,
                                                       l.nd2);
    FT_CUDA(cudaGetLastError());
    cublasHandle_t h;
    FT_TRY(cublas_handle(&h));
    if (cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS) return FT_ECUDA;
    if (cublasSetMathMode(h, CUBLAS_DEFAULT_MATH) != CUBLAS_STATUS_SUCCESS) return FT_ECUDA;  // FP32, no TF32
    // row-major dist[nq][nd] = Cq [nq][dim] x Cd^T: column-major Cd^T-view x Cq
    const float one = 1.0f, zero = 0.0f;
    if (cublasSgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, int(nd), int(nq), dim, &one, l.cd, dim, l.cq, dim, &zero, l.dist,
                    int(nd)) != CUBLAS_STATUS_SUCCESS)
        return FT_ECUDA;
    k_mean_epilogue<<<grid_for(nq * nd, 256), 256, 0, s>>>(l.dist, l.nq2, l.nd2, nq, nd);
    FT_CUDA(cudaGetLastError());
    return ft_topk_f32(l.dist, nq, nd, k1, l.topk_ws, l.topk_bytes, cand_ids_out_dev, cand_dist_out_dev, s);
}
