// Internal definitions shared by the CUDA translation units of libflowtree.
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "flowtree.h"

#define FT_LEAF_BITS 40  // coordinate quantisation bits (B)

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
#define FT_CUDA(call)                                  \
    do {                                               \
        cudaError_t e__ = (call);                      \
        if (e__ != cudaSuccess) {                      \
            ft_note_cuda_error(e__, #call, __FILE__, __LINE__); \
            return FT_ECUDA;                           \
        }                                              \
    } while (0)

#define FT_TRY(expr)                      \
    do {                                  \
        ft_status s__ = (expr);           \
        if (s__ != FT_OK) return s__;     \
    } while (0)

void ft_note_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// Device status word codes (bit flags, OR-ed by kernels).
enum : uint32_t {
    FT_DEV_EINVAL = 1u,
    FT_DEV_EOVERFLOW = 2u,
    FT_DEV_EUNSUPPORTED = 4u,
    FT_DEV_ETIMEOUT = 8u,
};

__device__ __forceinline__ void ft_flag(uint32_t* status, uint32_t code) {
    if (status) atomicOr(status, code);
}

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
struct ft_tree {
    int device = 0;
    int num_sms = 0;
    int64_t n = 0;
    int dim = 0;
    int levels = 0;
    int phi_log2 = 0;
    int rmq_levels = 0;
    std::vector<float> lo;
    std::vector<uint64_t> shift;
    uint32_t* d_rank_of_point = nullptr;  // [n]
    uint32_t* d_point_of_rank = nullptr;  // [n]
    uint8_t* d_lcp = nullptr;             // [n]   lcp[r] = depth of LCA(rank r, rank r+1); lcp[n-1] = 0
    uint8_t* d_rmq = nullptr;             // [rmq_levels][n] sparse table of minima over lcp
    uint8_t* d_chain = nullptr;           // [n]   deepest depth at which rank r shares a cell
    uint32_t* d_node_id = nullptr;        // [L][n] dense node id of rank r at depth k (row k-1)
    uint32_t* d_status = nullptr;         // device status word
    ft_flowtree_config cfg{0, 0, 0, 0, 0};
};

struct ft_docs {
    const ft_tree* tree = nullptr;
    int64_t n_docs = 0;
    int64_t n_items = 0;
    int64_t n_embed = 0;
    int max_support = 0;
    int max_embed = 0;
    int64_t* d_ptr = nullptr;    // [n_docs+1] support offsets
    uint32_t* d_rank = nullptr;  // [n_items] quadtree rank, ascending within a doc
    uint32_t* d_mass = nullptr;  // [n_items]
    uint32_t* d_word = nullptr;  // [n_items] ground-point id
    int64_t* d_eptr = nullptr;   // [n_docs+1] embedding offsets
    uint32_t* d_ekey = nullptr;  // [n_embed] node key
    uint32_t* d_emass = nullptr; // [n_embed] node mass
    std::vector<int64_t> h_eptr; // host copy of d_eptr (launch planning without a device read)
    // inverted index of the embedding: for every distinct node key, the
    // documents holding it (ascending) and their masses
    int64_t n_ukeys = 0;
    uint32_t* d_ukey = nullptr;  // [n_ukeys] distinct keys, ascending
    uint32_t* d_uoff = nullptr;  // [n_ukeys+1] posting ranges
    uint2* d_post = nullptr;     // [n_embed] postings {document, mass}
};

struct ft_flows {
    int64_t n_pairs = 0;
    int64_t capacity = 0;
    bool cross = false;
    int64_t nb_cross = 0;
    int32_t* d_pair_a = nullptr;  // [n_pairs] (copies; NULL for a cross product)
    int32_t* d_pair_b = nullptr;
    int64_t* d_slot_ptr = nullptr;  // [n_pairs+1]
    int32_t* d_count = nullptr;     // [n_pairs]
    uint32_t* d_ia = nullptr;       // [capacity]
    uint32_t* d_ib = nullptr;
    uint32_t* d_f = nullptr;
    uint8_t* d_depth = nullptr;
    float* d_dist = nullptr;        // Euclidean distance of the pair (FP32)
    // rebindable flows (ft_flows_create_capacity): capacity for any max_pairs
    // pairs of these document sets, rebound to a pair list by ft_flows_bind
    const ft_tree* tree = nullptr;
    const ft_docs* a = nullptr;
    const ft_docs* b = nullptr;
    int64_t max_pairs = 0;          // 0: fixed pair list (ft_flows_create)
    int64_t* d_scan_tmp = nullptr;  // [ft_scan_tmp_elems(max_pairs + 1)]
};

// ---------------------------------------------------------------------------
// workspace carving (256-byte aligned sub-buffers)
// ---------------------------------------------------------------------------
struct WsCarver {
    char* base;
    size_t off = 0;
    explicit WsCarver(void* b) : base(static_cast<char*>(b)) {}
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

// NVTX range over a host entry point: names the call in a profiler's
// timeline (a no-op unless a profiling tool is attached).
struct FtRange {
    explicit FtRange(const char* name) { nvtxRangePushA(name); }
    ~FtRange() { nvtxRangePop(); }
    FtRange(const FtRange&) = delete;
    FtRange& operator=(const FtRange&) = delete;
};

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
constexpr unsigned FULL_MASK = 0xffffffffu;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// inclusive warp scan (sum) of a 64-bit value
__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(FULL_MASK, v, o);
        if (lane >= (unsigned)o) v += t;
    }
    return v;
}

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(FULL_MASK, v, o);
        if (lane >= (unsigned)o) v += t;
    }
    return v;
}

// inclusive warp max-scan of a signed int
__device__ __forceinline__ int warp_incl_max_i32(int v) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL_MASK, v, o);
        if (lane >= (unsigned)o) v = max(v, t);
    }
    return v;
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

__device__ __forceinline__ int64_t warp_sum_i64(int64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// number of elements of sorted a[0..n) that are < key (lower_bound)
template <class T>
__device__ __forceinline__ int lower_bound_dev(const T* a, int n, T key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// number of elements of sorted a[0..n) that are <= key (upper_bound)
template <class T>
__device__ __forceinline__ int upper_bound_dev(const T* a, int n, T key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

inline int ft_ceil_div(int64_t a, int64_t b) { return int((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// host-side helpers implemented in ft_util.cu
// ---------------------------------------------------------------------------
ft_status ft_device_sms(int* sms);
// First use of a kernel on a device: raise its dynamic shared-memory limit to
// the device maximum and record its occupancy for (threads, smem).  Later
// calls only read the cache, so launches inside stream capture make no
// attribute or occupancy calls once the same configuration has run before.
ft_status ft_prepare_kernel(const void* fn, int threads, size_t smem, int* blocks_per_sm);
// exclusive scan (int64) of n values; in and out may alias.  tmp must hold
// ft_scan_tmp_elems(n) int64 values.
size_t ft_scan_tmp_elems(int64_t n);
ft_status ft_exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s);
// a[i] = i
ft_status ft_iota_u32(uint32_t* a, int64_t n, cudaStream_t s);
// stable LSD radix sort of a permutation by 8-bit digits of u32 keys:
// perm (initially any order) is reordered so that keys[perm[i]] ascend, ties
// keeping their current relative order.  Only `key_bits` low bits are used.
size_t ft_sort_tmp_bytes(int64_t n);
ft_status ft_sort_perm_by_u32(const uint32_t* keys, uint32_t* perm, int64_t n, int key_bits, void* tmp,
                              cudaStream_t s);
// the same for byte-string keys: keys[e * key_bytes + b], byte 0 most significant.
// Only byte positions with varying[b] != 0 are sorted on (host array).
ft_status ft_sort_perm_by_bytes(const uint8_t* keys, int key_bytes, const std::vector<uint8_t>& varying,
                                uint32_t* perm, int64_t n, void* tmp, cudaStream_t s);

// Workspace bytes of the launch ft_flowtree_batch makes for these arguments
// without saved flows (ft_flow.cu); returns the planning status.
ft_status ft_flowtree_batch_need(const ft_tree* t, const float* vocab, const ft_docs* a, const ft_docs* b,
                                 const int32_t* pa, const int32_t* pb, int64_t n_pairs, size_t* need);
