// Device-wide exclusive scan, stable LSD radix sort of permutations, status
// strings and CUDA-error notes.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>

#include "ft_internal.cuh"

namespace {
thread_local char g_last_cuda_error[256] = {0};
}

void ft_note_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s:%d %s: %s", file, line, what, cudaGetErrorString(e));
    if (getenv("FT_VERBOSE")) fprintf(stderr, "[flowtree] %s\n", g_last_cuda_error);
}

extern "C" const char* ft_last_cuda_error(void) { return g_last_cuda_error; }

extern "C" const char* ft_status_string(ft_status s) {
    switch (s) {
        case FT_OK: return "FT_OK";
        case FT_EINVAL: return "FT_EINVAL: invalid argument or malformed input";
        case FT_ENOMEM: return "FT_ENOMEM: device allocation failed";
        case FT_ECUDA: return "FT_ECUDA: CUDA runtime error";
        case FT_ETIMEOUT: return "FT_ETIMEOUT: bounded device wait gave up";
        case FT_EOVERFLOW: return "FT_EOVERFLOW: device-side capacity exceeded";
        case FT_EUNSUPPORTED: return "FT_EUNSUPPORTED: outside the compiled limits";
        case FT_EWORKSPACE: return "FT_EWORKSPACE: workspace missing or too small";
        case FT_ETOOBIG: return "FT_ETOOBIG: batch needs more than the fixed static scratch";
    }
    return "unknown ft_status";
}

ft_status ft_device_sms(int* sms) {
    int dev = 0;
    FT_CUDA(cudaGetDevice(&dev));
    FT_CUDA(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
    return FT_OK;
}

namespace {
struct KernelKey {
    const void* fn;
    int dev, threads;
    size_t smem;
    bool operator<(const KernelKey& o) const {
        if (fn != o.fn) return fn < o.fn;
        if (dev != o.dev) return dev < o.dev;
        if (threads != o.threads) return threads < o.threads;
        return smem < o.smem;
    }
};
std::mutex g_kernel_mu;
std::map<KernelKey, int> g_occupancy;
std::map<std::pair<const void*, int>, bool> g_attr_set;
}  // namespace

ft_status ft_prepare_kernel(const void* fn, int threads, size_t smem, int* blocks_per_sm) {
    int dev = 0;
    FT_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_kernel_mu);
    const KernelKey key{fn, dev, threads, smem};
    auto it = g_occupancy.find(key);
    if (it != g_occupancy.end()) {
        *blocks_per_sm = it->second;
        return FT_OK;
    }
    if (!g_attr_set[{fn, dev}]) {
        int max_smem = 0;
        FT_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        cudaFuncAttributes fa{};
        FT_CUDA(cudaFuncGetAttributes(&fa, fn));  // static shared memory counts against the same limit
        FT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     max_smem - int(fa.sharedSizeBytes)));
        g_attr_set[{fn, dev}] = true;
    }
    int bps = 0;
    FT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, threads, smem));
    g_occupancy[key] = bps;
    *blocks_per_sm = bps;
    return FT_OK;
}

// ---------------------------------------------------------------------------
// exclusive scan of int64 values: tile sums -> scan of tile sums -> tiles
// ---------------------------------------------------------------------------
namespace {
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// exclusive block scan of one int64 per thread; returns the block total
template <int THREADS>
__device__ int64_t block_excl_scan_i64(int64_t v, int64_t* excl) {
    constexpr int NW = THREADS / 32;
    __shared__ int64_t warp_off[NW];
    __shared__ int64_t total_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(FULL_MASK, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_off[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < NW ? warp_off[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(FULL_MASK, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < NW) warp_off[lane] = wi - w;
        if (lane == 31) total_s = wi;
    }
    __syncthreads();
    *excl = warp_off[warp] + inc - v;
    const int64_t total = total_s;
    __syncthreads();
    return total;
}

__global__ void k_scan_reduce(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
    __shared__ int64_t red[SCAN_THREADS / 32];
    const int64_t tile0 = int64_t(blockIdx.x) * SCAN_TILE;
    int64_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        int64_t i = tile0 + int64_t(j) * SCAN_THREADS + threadIdx.x;
        if (i < n) s += in[i];
    }
    s = warp_sum_i64(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t v = threadIdx.x < SCAN_THREADS / 32 ? red[threadIdx.x] : 0;
        v = warp_sum_i64(v);
        if (threadIdx.x == 0) sums[blockIdx.x] = v;
    }
}

__global__ void k_scan_single(int64_t* sums, int64_t nb) {
    __shared__ int64_t carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += SCAN_THREADS) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < nb ? sums[i] : 0;
        int64_t excl;
        const int64_t tot = block_excl_scan_i64<SCAN_THREADS>(v, &excl);
        const int64_t carry = carry_s;
        if (i < nb) sums[i] = carry + excl;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + tot;
        __syncthreads();
    }
}

__global__ void k_scan_down(const int64_t* in, int64_t* out, int64_t n, const int64_t* __restrict__ sums) {
    const int64_t tile0 = int64_t(blockIdx.x) * SCAN_TILE;
    const int64_t my0 = tile0 + int64_t(threadIdx.x) * SCAN_ITEMS;  // thread-contiguous items
    int64_t v[SCAN_ITEMS];
    int64_t t = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        int64_t i = my0 + j;
        v[j] = i < n ? in[i] : 0;
        t += v[j];
    }
    int64_t excl;
    block_excl_scan_i64<SCAN_THREADS>(t, &excl);
    int64_t run = sums[blockIdx.x] + excl;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        int64_t i = my0 + j;
        if (i < n) out[i] = run;
        run += v[j];
    }
}
}  // namespace

size_t ft_scan_tmp_elems(int64_t n) { return size_t(ft_ceil_div(n > 0 ? n : 1, SCAN_TILE)) + 1; }

ft_status ft_exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s) {
    if (n <= 0) return FT_OK;
    const int nb = ft_ceil_div(n, SCAN_TILE);
    k_scan_reduce<<<nb, SCAN_THREADS, 0, s>>>(in, n, tmp);
    k_scan_single<<<1, SCAN_THREADS, 0, s>>>(tmp, nb);
    k_scan_down<<<nb, SCAN_THREADS, 0, s>>>(in, out, n, tmp);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

namespace {
__global__ void k_iota_u32(uint32_t* __restrict__ a, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        a[i] = uint32_t(i);
}
}  // namespace

ft_status ft_iota_u32(uint32_t* a, int64_t n, cudaStream_t s) {
    if (n <= 0) return FT_OK;
    int64_t b = (n + 255) / 256;
    if (b > 65535 * 8) b = 65535 * 8;
    k_iota_u32<<<int(b), 256, 0, s>>>(a, n);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of a permutation, 8-bit digits
// ---------------------------------------------------------------------------
namespace {
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

struct U32Digit {
    const uint32_t* keys;
    int shift;
    __device__ __forceinline__ uint32_t operator()(uint32_t e) const { return (keys[e] >> shift) & 0xFFu; }
};

struct ByteDigit {
    const uint8_t* keys;
    int key_bytes;
    int b;
    __device__ __forceinline__ uint32_t operator()(uint32_t e) const { return keys[size_t(e) * key_bytes + b]; }
};

template <class DigitFn>
__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const uint32_t* __restrict__ perm, int64_t n,
                                                           int64_t* __restrict__ hist, int nblocks, DigitFn digit) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t tile0 = int64_t(blockIdx.x) * RS_TILE;
    // all of the tile's loads first (the digit is a gather through perm)
    uint32_t ev[RS_ITEMS], dv[RS_ITEMS];
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = tile0 + int64_t(r) * RS_THREADS + threadIdx.x;
        ev[r] = i < n ? perm[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = tile0 + int64_t(r) * RS_THREADS + threadIdx.x;
        dv[r] = i < n ? digit(ev[r]) : 0u;
    }
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = tile0 + int64_t(r) * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&cnt[dv[r]], 1u);
    }
    __syncthreads();
    hist[int64_t(threadIdx.x) * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

template <class DigitFn>
__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(const uint32_t* __restrict__ perm_in,
                                                              uint32_t* __restrict__ perm_out, int64_t n,
                                                              const int64_t* __restrict__ offsets, int nblocks,
                                                              DigitFn digit) {
    __shared__ uint32_t base[256];
    __shared__ int64_t boff[256];  // this tile's first output position per digit
    __shared__ uint32_t wcnt[RS_THREADS / 32][256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t tile0 = int64_t(blockIdx.x) * RS_TILE;
    base[tid] = 0;
    boff[tid] = offsets[int64_t(tid) * nblocks + blockIdx.x];
    // all of the tile's loads first (the digit is a gather through perm); the
    // ranking rounds below then work from registers and shared memory
    uint32_t ev[RS_ITEMS], dv[RS_ITEMS];
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = tile0 + int64_t(r) * RS_THREADS + tid;
        ev[r] = i < n ? perm_in[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = tile0 + int64_t(r) * RS_THREADS + tid;
        dv[r] = i < n ? digit(ev[r]) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = tile0 + int64_t(r) * RS_THREADS + tid;
        const bool valid = i < n;
        const uint32_t e = ev[r];
        const uint32_t d = dv[r];
        for (int j = tid; j < (RS_THREADS / 32) * 256; j += RS_THREADS) (&wcnt[0][0])[j] = 0;
        __syncthreads();
        const unsigned peers = __match_any_sync(FULL_MASK, d);
        const int rank_in_warp = __popc(peers & lanemask_lt());
        const int leader = __ffs(peers) - 1;
        if (valid && lane == leader) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t run = base[tid];
#pragma unroll
            for (int w = 0; w < RS_THREADS / 32; ++w) {
                uint32_t t = wcnt[w][tid];
                wcnt[w][tid] = run;
                run += t;
            }
            base[tid] = run;
        }
        __syncthreads();
        if (valid) {
            uint32_t local = wcnt[warp][d] + uint32_t(rank_in_warp);
            perm_out[boff[d] + local] = e;
        }
        __syncthreads();
    }
}

template <class DigitFn>
ft_status radix_pass(const uint32_t* in, uint32_t* out, int64_t n, int64_t* hist, int64_t* scan_tmp,
                     DigitFn digit, cudaStream_t s) {
    const int nb = ft_ceil_div(n, RS_TILE);
    k_radix_hist<<<nb, RS_THREADS, 0, s>>>(in, n, hist, nb, digit);
    FT_TRY(ft_exclusive_scan_i64(hist, hist, int64_t(nb) * 256, scan_tmp, s));
    k_radix_scatter<<<nb, RS_THREADS, 0, s>>>(in, out, n, hist, nb, digit);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

struct SortTmp {
    uint32_t* alt;
    int64_t* hist;
    int64_t* scan_tmp;
};

SortTmp carve_sort_tmp(void* tmp, int64_t n) {
    WsCarver w(tmp);
    SortTmp t;
    const int nb = ft_ceil_div(n > 0 ? n : 1, RS_TILE);
    t.alt = w.take<uint32_t>(size_t(n));
    t.hist = w.take<int64_t>(size_t(nb) * 256);
    t.scan_tmp = w.take<int64_t>(ft_scan_tmp_elems(int64_t(nb) * 256));
    return t;
}
}  // namespace

size_t ft_sort_tmp_bytes(int64_t n) {
    WsCarver w(nullptr);
    const int nb = ft_ceil_div(n > 0 ? n : 1, RS_TILE);
    w.take<uint32_t>(size_t(n));
    w.take<int64_t>(size_t(nb) * 256);
    w.take<int64_t>(ft_scan_tmp_elems(int64_t(nb) * 256));
    return w.off + 256;
}

ft_status ft_sort_perm_by_u32(const uint32_t* keys, uint32_t* perm, int64_t n, int key_bits, void* tmp,
                              cudaStream_t s) {
    if (n <= 1) return FT_OK;
    SortTmp t = carve_sort_tmp(tmp, n);
    uint32_t* cur = perm;
    uint32_t* nxt = t.alt;
    for (int shift = 0; shift < key_bits; shift += 8) {
        FT_TRY(radix_pass(cur, nxt, n, t.hist, t.scan_tmp, U32Digit{keys, shift}, s));
        uint32_t* x = cur;
        cur = nxt;
        nxt = x;
    }
    if (cur != perm) FT_CUDA(cudaMemcpyAsync(perm, cur, size_t(n) * 4, cudaMemcpyDeviceToDevice, s));
    return FT_OK;
}

ft_status ft_sort_perm_by_bytes(const uint8_t* keys, int key_bytes, const std::vector<uint8_t>& varying,
                                uint32_t* perm, int64_t n, void* tmp, cudaStream_t s) {
    if (n <= 1) return FT_OK;
    SortTmp t = carve_sort_tmp(tmp, n);
    uint32_t* cur = perm;
    uint32_t* nxt = t.alt;
    for (int b = key_bytes - 1; b >= 0; --b) {
        if (!varying[size_t(b)]) continue;
        FT_TRY(radix_pass(cur, nxt, n, t.hist, t.scan_tmp, ByteDigit{keys, key_bytes, b}, s));
        uint32_t* x = cur;
        cur = nxt;
        nxt = x;
    }
    if (cur != perm) FT_CUDA(cudaMemcpyAsync(perm, cur, size_t(n) * 4, cudaMemcpyDeviceToDevice, s));
    return FT_OK;
}
