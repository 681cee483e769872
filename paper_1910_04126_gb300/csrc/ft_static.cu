// ft_flowtree_batch_static: the batched Flowtree for callers that cannot
// allocate device memory.
//
// ft_flowtree_batch itself allocates nothing, but it needs a caller-provided
// workspace (work-queue counter, longest-first pair order and its sort
// buffers, and shared-memory overflow space for unusually long pairs).  Some
// callers have no way to provide one: a host whose device memory is owned by
// its own pooled allocator that exposes no allocation to plug-ins, or code
// that must not call cudaMalloc because it would implicitly synchronise the
// device inside a latency-bound loop.  This entry point takes
// the same inputs and outputs but carves the workspace out of a fixed device
// array compiled into the library.
//
// The array (FT_STATIC_SCRATCH_BYTES) lives in every GPU that loads the
// library, for as long as the library stays loaded.  Its device address is
// looked up once per device, on the first call made with that device
// current (cudaGetSymbolAddress, on that call only).  All calls share
// the array: two calls whose work overlaps on the GPU (different streams, or
// different host threads, without ordering between them) race on it and give
// undefined results.  Serialise them on one stream.
#include <mutex>

#include "ft_internal.cuh"

static __device__ __align__(256) uint8_t g_ft_static_scratch[FT_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

// Device address of the fixed scratch for the current device (set-up on the
// first call per device).
ft_status static_scratch(void** out) {
    int dev = 0;
    FT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return FT_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_ft_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            ft_note_cuda_error(e, "cudaGetSymbolAddress(g_ft_static_scratch)", __FILE__, __LINE__);
            return FT_ECUDA;
        }
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return FT_OK;
}
}  // namespace

extern "C" ft_status ft_flowtree_batch_static(const ft_tree* t, const float* vocab_dev, const ft_docs* a,
                                              const ft_docs* b, const int32_t* pair_a_dev, const int32_t* pair_b_dev,
                                              int64_t n_pairs, float* cost_out_dev, void* stream) {
    FtRange nvtx_range("ft_flowtree_batch_static");
    if (!t || !a || !b || !vocab_dev || !cost_out_dev || n_pairs < 0) return FT_EINVAL;
    if (n_pairs == 0) return FT_OK;
    // the scratch this call's own plan needs (a cross product needs no pair
    // order, an explicit pair list does); planning errors pass through
    size_t need = 0;
    FT_TRY(ft_flowtree_batch_need(t, vocab_dev, a, b, pair_a_dev, pair_b_dev, n_pairs, &need));
    if (need > size_t(FT_STATIC_SCRATCH_BYTES)) return FT_ETOOBIG;
    void* scratch = nullptr;
    FT_TRY(static_scratch(&scratch));
    return ft_flowtree_batch(t, vocab_dev, a, b, pair_a_dev, pair_b_dev, n_pairs, cost_out_dev, nullptr, scratch,
                             size_t(FT_STATIC_SCRATCH_BYTES), stream);
}
