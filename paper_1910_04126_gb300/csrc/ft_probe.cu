// Read-bandwidth probe: the measured denominator of the L2 (and HBM)
// roofline of the row-gathering kernels.  Every SM streams the buffer with
// independent 16-byte loads that bypass L1 (ld.global.cg), so a buffer that
// fits in L2 measures L2 read bandwidth and a larger one measures HBM.  The
// loaded words are XOR-folded into one word per warp and then into *sink,
// so no load can be dropped.
#include <algorithm>

#include "ft_internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_UNROLL = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_read_probe(const uint4* __restrict__ p, int64_t n16, int passes,
                                                             unsigned int* __restrict__ sink) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    unsigned int acc = 0;
    for (int r = 0; r < passes; ++r) {
        for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n16; i += stride * PROBE_UNROLL) {
            uint4 v[PROBE_UNROLL];
#pragma unroll
            for (int u = 0; u < PROBE_UNROLL; ++u) {
                const int64_t j = i + u * stride;
                v[u] = j < n16 ? __ldcg(p + j) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < PROBE_UNROLL; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(FULL_MASK, acc, o);
    if (lane_id() == 0) atomicXor(sink, acc);
}

}  // namespace

extern "C" ft_status ft_read_probe(const void* buf_dev, size_t bytes, int32_t passes, uint32_t* sink_dev,
                                   void* stream) {
    if (!buf_dev || !sink_dev || passes < 1 || bytes < 16) return FT_EINVAL;
    if ((reinterpret_cast<uintptr_t>(buf_dev) & 15u) != 0 || (bytes & 15u) != 0) return FT_EINVAL;
    int dev = 0, sms = 0;
    FT_CUDA(cudaGetDevice(&dev));
    FT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t n16 = int64_t(bytes / 16);
    const int64_t want = (n16 + PROBE_THREADS - 1) / PROBE_THREADS;
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(sms) * (2048 / PROBE_THREADS))));
    k_read_probe<<<blocks, PROBE_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const uint4*>(buf_dev), n16, passes, reinterpret_cast<unsigned int*>(sink_dev));
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}
