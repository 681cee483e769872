/*
 * flowtree.h -- C ABI of the GB300-native batched Flowtree library.
 *
 * Flowtree (Backurs, Dong, Indyk, Razenshteyn, Wagner, arXiv 1910.04126)
 * estimates the Wasserstein-1 distance between two distributions over a
 * ground set X in R^d: build a randomly shifted quadtree over X (Sec. 2),
 * compute the optimal flow between the two distributions for the tree
 * metric with the bottom-up greedy of App. A.1, and price that flow with
 * true Euclidean distances (Sec. 3).  The same tree also gives the classic
 * quadtree W1 as an l1 distance between sparse embeddings (Sec. 2,
 * "Wasserstein-1 on Quadtree"), used here as the prefilter of the
 * nearest-neighbour pipeline (Sec. 5.2, "prefetch and prune").
 *
 * Conventions shared by every entry point:
 *   - All pointers named *_dev are CUDA device pointers on the current
 *     device; *_host are host pointers.  The caller owns every pointer it
 *     passes; the library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered unless stated otherwise.  Calls
 *     documented as "synchronous" block the host until their work is done.
 *   - Errors are returned as ft_status values, never thrown.  Argument
 *     errors are detected on the host before any launch.  Errors detected
 *     inside kernels (overflow, malformed input found on the device) are
 *     recorded in a per-tree device status word, read and cleared by
 *     ft_tree_status().
 *   - Handles (ft_tree, ft_docs, ft_flows) are created by the library
 *     (device memory is allocated at creation, never later) and released by
 *     the matching *_free call.  Workspaces are caller-allocated device
 *     buffers whose size comes from the matching *_workspace_size call, so
 *     that the hot entry points allocate nothing.
 *
 * Fixed readings of the paper (where it is silent or ambiguous):
 *   - levels L: depths 1..L are subdivided cells below the root (depth 0);
 *     depth L+1 is the point level (the paper's singleton leaves).
 *   - coordinates are quantised once to 40 bits: with lo_c the per-dimension
 *     minimum and Phi the smallest power of two >= the largest coordinate
 *     range, q = min(2^40, floor((x - lo) * 2^40 / Phi)) in FP64, and
 *     z = min(q + 2^40 - s_c, 2^41 - 1) for the integer shift s_c in
 *     [0, 2^40] (sigma = s * Phi / 2^40, Sec. 2 random shift).  The cell at
 *     depth k is z >> (41 - k); children are ordered by the bit vector of the
 *     halving, dimension 0 most significant; points in one deepest cell are
 *     ordered by point id.  This order is the quadtree "rank".
 *   - masses are integers summing to exactly 2^24 per distribution
 *     (largest-remainder rounding, ties to the smaller rank).
 *   - inside a tree node, leftover demands are matched in north-west-corner
 *     order (mu-items in rank order against nu-items in rank order); the
 *     paper allows any order.  A point carried by both distributions is
 *     matched with itself first (distance 0).
 *   - the ground metric is Euclidean.
 */
#ifndef FLOWTREE_H
#define FLOWTREE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FT_OK = 0,
    FT_EINVAL = -1,        /* bad argument or malformed input data          */
    FT_ENOMEM = -2,        /* device allocation failed (handle creation)    */
    FT_ECUDA = -3,         /* a CUDA runtime call failed                    */
    FT_ETIMEOUT = -4,      /* a bounded device-side wait gave up            */
    FT_EOVERFLOW = -5,     /* a device-side capacity was exceeded           */
    FT_EUNSUPPORTED = -6,  /* valid input outside the compiled limits       */
    FT_EWORKSPACE = -7,    /* workspace NULL or smaller than required       */
    FT_ETOOBIG = -8        /* batch needs more than the fixed static scratch */
} ft_status;

typedef struct ft_tree ft_tree;   /* quadtree over the ground points          */
typedef struct ft_docs ft_docs;   /* a set of distributions on the tree       */
typedef struct ft_flows ft_flows; /* saved tree flows of a batch of pairs     */

/* Compile-time limits of the library. */
#define FT_MAX_LEVELS 14          /* L <= 14                                  */
#define FT_MAX_SUPPORT 16383      /* distinct points per distribution (a merged
                                     pair's positions then fit 15 bits)        */
#define FT_MASS_ONE 16777216      /* 2^24: total mass of every distribution   */

/* Human-readable name of a status code (static string). */
const char* ft_status_string(ft_status s);

/* ------------------------------------------------------------------------
 * Quadtree (Sec. 2, "Generic Quadtree").
 *
 * points_dev : float32 [n_points][dim], row-major, the ground set X (also
 *              the "vocabulary" table priced by the Flowtree estimate).
 * levels     : L, 1 <= L <= FT_MAX_LEVELS.
 * shift_host : dim integers in [0, 2^40], the random shift; or NULL to draw
 *              them from splitmix64(seed): s_c = splitmix64 output c (c-th
 *              call on the state seed) modulo (2^40 + 1).
 * n_points   : 1 <= n_points < 2^24.
 * Synchronous.  On success *out owns the tree's device memory.
 * ------------------------------------------------------------------------ */
ft_status ft_build_quadtree(const float* points_dev, int64_t n_points, int32_t dim, int32_t levels,
                            const uint64_t* shift_host, uint64_t seed, void* stream, ft_tree** out);
void ft_tree_free(ft_tree* t);

typedef struct {
    int64_t n_points;
    int32_t dim;
    int32_t levels;
    int32_t phi_log2;      /* Phi = 2^phi_log2                                */
    int32_t rmq_levels;    /* rows of the LCA range-minimum table             */
} ft_tree_info;
ft_status ft_tree_get_info(const ft_tree* t, ft_tree_info* info);

/* Copy the tree's order out (synchronous):
 *   rank_of_point[n], point_of_rank[n] (uint32), lcp[n-1] (uint8): depth of
 *   the lowest common ancestor of the points at ranks r and r+1,
 *   shift[dim] (uint64).  Any pointer may be NULL. */
ft_status ft_tree_export(const ft_tree* t, uint32_t* rank_of_point_host, uint32_t* point_of_rank_host,
                         uint8_t* lcp_host, uint64_t* shift_host);

/* Read and clear the tree's device status word (synchronous on stream).
 * Returns FT_OK, or the first error recorded by a kernel since the last
 * read. */
ft_status ft_tree_status(const ft_tree* t, void* stream);

/* ------------------------------------------------------------------------
 * Distributions (Sec. 5 datasets: a document is a distribution over its
 * terms; an image over its pixels, mass proportional to intensity).
 *
 * CSR input, all on the device: row_ptr_dev int64 [n_docs+1] (row_ptr[0]=0,
 * non-decreasing), word_dev int32 [nnz] (ground-point ids), weight_dev
 * float32 [nnz] (finite, >= 0).  Duplicate word ids are merged (weights
 * summed in CSR order); zero weights are dropped; every document needs a
 * positive total.  Masses: W = FP64 sum of the weights in CSR order,
 * m_i = floor(w_i / W * 2^24), the remaining units go one each to the
 * largest fractional parts (ties: smaller rank); items left at 0 are dropped.
 * Also builds each document's sparse quadtree embedding (Sec. 2, l1
 * embedding of tree W1) and the set's inverted index over it (for every
 * tree node, the documents whose embedding holds it, ascending, with their
 * masses: 12 B per embedding entry) for ft_quadtree_scan.
 * Synchronous.  FT_EINVAL for malformed CSR or weights; FT_EUNSUPPORTED for
 * a document with more than FT_MAX_SUPPORT distinct points.
 * ------------------------------------------------------------------------ */
ft_status ft_embed_docs(const ft_tree* t, const int64_t* row_ptr_dev, const int32_t* word_dev,
                        const float* weight_dev, int64_t n_docs, void* stream, ft_docs** out);
void ft_docs_free(ft_docs* d);

typedef struct {
    int64_t n_docs;
    int64_t n_items;       /* total support items                             */
    int32_t max_support;   /* largest support of one document                 */
    int64_t n_embed;       /* total sparse-embedding entries                  */
} ft_docs_info;
ft_status ft_docs_get_info(const ft_docs* d, ft_docs_info* info);

/* Copy supports out (synchronous): sup_ptr[n_docs+1] (int64),
 * sup_point[n_items] (uint32 ground-point id), sup_mass[n_items] (uint32),
 * items of a document sorted by quadtree rank.  Any pointer may be NULL. */
ft_status ft_docs_export(const ft_docs* d, int64_t* sup_ptr_host, uint32_t* sup_point_host,
                         uint32_t* sup_mass_host);

/* ------------------------------------------------------------------------
 * Flowtree estimate, batched (Sec. 3; greedy flow of App. A.1).
 *
 * For pair i, cost_out_dev[i] = sum over tree-flow pairs (x, y) of
 * f(x, y) / 2^24 * ||vocab[x] - vocab[y]||_2: exact integer flows, FP32
 * distances, per-lane Neumaier-compensated FP32 sums added across the warp
 * (within 1e-5 relative of the FP64 definition), FP32 output.
 * Pair i is (document pair_a_dev[i] of a, document pair_b_dev[i] of b).  If
 * both pair arrays are NULL the batch is the cross product: pair
 * i = qa * nb + jb for qa < na(a), jb < nb(b), and n_pairs must equal
 * na * nb.
 * vocab_dev  : float32 [n_points][dim] (normally the tree's own points).
 * flows_out  : NULL, or a handle from ft_flows_create for the same pairs;
 *              then every tree-flow pair is saved for ft_flowtree_backward.
 * workspace  : >= ft_flowtree_batch_workspace_size() bytes of device memory.
 * One persistent launch; pairs are taken longest-first from a device work
 * queue; pairs too long for on-chip staging use the workspace.  No host
 * synchronisation, no allocation: capturable in a CUDA graph.
 * ------------------------------------------------------------------------ */
size_t ft_flowtree_batch_workspace_size(const ft_tree* t, const ft_docs* a, const ft_docs* b, int64_t n_pairs);
ft_status ft_flowtree_batch(const ft_tree* t, const float* vocab_dev, const ft_docs* a, const ft_docs* b,
                            const int32_t* pair_a_dev, const int32_t* pair_b_dev, int64_t n_pairs,
                            float* cost_out_dev, ft_flows* flows_out, void* workspace, size_t ws_bytes,
                            void* stream);

/* Allocation-free variant of ft_flowtree_batch (the paper has no
 * counterpart; this is a deployment convenience).  For callers that cannot
 * allocate device memory at all -- a host whose device memory is held by its
 * own pooled allocator with nothing exposed to plug-ins, or a latency-bound
 * loop where cudaMalloc's implicit device synchronisation is not allowed --
 * and so cannot provide ft_flowtree_batch's workspace.  Same inputs and outputs
 * (no saved flows); the workspace comes from a fixed device array of
 * FT_STATIC_SCRATCH_BYTES compiled into the library, held by every GPU that
 * loads it until the library is unloaded.  Calls no cudaMalloc/cudaFree.
 *   - Limit: a batch whose launch needs more workspace than
 *     FT_STATIC_SCRATCH_BYTES is rejected with FT_ETOOBIG before any launch.
 *     The need is that of the launch this call makes: an explicit pair list
 *     needs about 13 bytes per pair for its longest-first order (up to about
 *     1.2 million pairs); a cross product needs only the work-queue counter,
 *     whatever its size, unless the FT_ALGO_WARP form has to spill pairs
 *     longer than its on-chip staging to per-warp overflow space.  Planning
 *     errors (FT_EUNSUPPORTED for a configuration the device cannot run) are
 *     returned as ft_flowtree_batch would return them.
 *   - The first call on a device (with that device current) looks up the
 *     array's device address (cudaGetSymbolAddress) on that call only.
 *     The address is cached per device ordinal for the life of the process:
 *     it does not survive cudaDeviceReset (or any other teardown of the
 *     device's primary context), after which this entry point must not be
 *     called again in the same process.
 *   - Every call shares the array, which keeps the previous call's contents
 *     (what must start at zero is cleared by each call): calls that overlap on
 *     the GPU race and give undefined results; serialise them on one stream. */
#define FT_STATIC_SCRATCH_BYTES (16u << 20)
ft_status ft_flowtree_batch_static(const ft_tree* t, const float* vocab_dev, const ft_docs* a, const ft_docs* b,
                                   const int32_t* pair_a_dev, const int32_t* pair_b_dev, int64_t n_pairs,
                                   float* cost_out_dev, void* stream);

/* The plain form: the same computation with one kernel launch per pair
 * (one warp), in pair order.  Used as the per-pair baseline. */
ft_status ft_flowtree_plain(const ft_tree* t, const float* vocab_dev, const ft_docs* a, const ft_docs* b,
                            const int32_t* pair_a_dev, const int32_t* pair_b_dev, int64_t n_pairs,
                            float* cost_out_dev, void* workspace, size_t ws_bytes, void* stream);

/* Launch configuration of ft_flowtree_batch.  0 = default for every field.
 *   algo          : FT_ALGO_AUTO, FT_ALGO_WARP (a warp per pair, level by
 *                   level over the merged supports staged in shared memory,
 *                   compacted after every depth), FT_ALGO_THREAD (a thread
 *                   per pair, one sweep with a stack of open tree nodes, its
 *                   per-position state as bit arrays in shared memory;
 *                   dim <= 8 only) or FT_ALGO_BLOCKED (a warp per pair, each
 *                   lane owning a contiguous block of merged items in shared
 *                   memory; pairs longer than the warp's staging are listed
 *                   and then computed by a second launch with a CTA of 8
 *                   warps per pair, up to 7,936 merged items).  AUTO =
 *                   BLOCKED when the device can hold its buffers for the
 *                   batch's longest pair, else WARP; ft_flowtree_autotune
 *                   picks among all three.
 *   warps_per_cta : warps per CTA (1..8).
 *   stage_items   : merged support items each warp stages on chip (WARP;
 *                   BLOCKED: the warp's staging, rounded up to 32 x an odd
 *                   number; 0 = 416 items, or less when every pair is
 *                   shorter).
 *   stage_tables  : 1 = copy the vocabulary and the LCA table into shared
 *                   memory per CTA when they fit (at most 32 KiB); 0 = read
 *                   them through L1 (the default: one cached copy per SM
 *                   leaves more shared memory for resident warps).
 *   deep_loads    : WARP with dim > 8 (pricing by 8-lane groups): 1 = the
 *                   build of the kernel that may use up to 255 registers per
 *                   thread, so that a warp's pricing rounds keep more row
 *                   loads in flight at the cost of resident warps: for
 *                   batches too small to fill the GPU, whose time is the
 *                   longest pairs' latency; 0 = the occupancy build (the
 *                   default).  Ignored by the other forms and for dim <= 8.
 *                   Both builds compute the same values bit for bit.
 * ft_flowtree_autotune times a few configurations on the given pairs (with
 * CUDA events on `stream`) and installs the fastest for this tree. */
#define FT_ALGO_AUTO 0
#define FT_ALGO_WARP 1
#define FT_ALGO_THREAD 2
#define FT_ALGO_BLOCKED 3
typedef struct {
    int32_t warps_per_cta;
    int32_t stage_items;
    int32_t algo;
    int32_t stage_tables;
    int32_t deep_loads;
} ft_flowtree_config;
ft_status ft_flowtree_set_config(ft_tree* t, const ft_flowtree_config* cfg);
ft_status ft_flowtree_get_config(const ft_tree* t, ft_flowtree_config* cfg);
ft_status ft_flowtree_autotune(ft_tree* t, const float* vocab_dev, const ft_docs* a, const ft_docs* b,
                               const int32_t* pair_a_dev, const int32_t* pair_b_dev, int64_t n_pairs,
                               float* cost_scratch_dev, void* workspace, size_t ws_bytes, void* stream,
                               ft_flowtree_config* chosen);

/* ------------------------------------------------------------------------
 * Saved flows (for the adjoint).  Slots: pair i owns
 * [slot_ptr[i], slot_ptr[i+1]) with slot_ptr[i+1]-slot_ptr[i] =
 * s_a + s_b (the greedy makes at most s_a + s_b - 1 pairs, App. A.1).
 * Synchronous creation (allocates).  Export is synchronous:
 * slot_ptr[n_pairs+1] int64, count[n_pairs] int32, item_a/item_b/flow
 * [capacity] uint32 (indices into the two supports), depth[capacity]
 * uint8 (node depth of the match, L+1 = same point).
 * ------------------------------------------------------------------------ */
ft_status ft_flows_create(const ft_tree* t, const ft_docs* a, const ft_docs* b, const int32_t* pair_a_dev,
                          const int32_t* pair_b_dev, int64_t n_pairs, void* stream, ft_flows** out);
void ft_flows_free(ft_flows* f);
ft_status ft_flows_capacity(const ft_flows* f, int64_t* n_pairs, int64_t* capacity);
ft_status ft_flows_export(const ft_flows* f, int64_t* slot_ptr_host, int32_t* count_host, uint32_t* item_a_host,
                          uint32_t* item_b_host, uint32_t* flow_host, uint8_t* depth_host);

/* Rebindable saved flows, for a training loop whose pairs change every step:
 * ft_flows_create_capacity allocates (once, without synchronising) room for
 * any max_pairs pairs of the document sets a and b, i.e. max_pairs *
 * (a's longest support + b's longest support) slots; ft_flows_bind then
 * points the flows at a pair list (pair_a_dev/pair_b_dev, n_pairs <=
 * max_pairs, copied on `stream`; both NULL = the a x b cross product, which
 * must then have at most max_pairs pairs) with no allocation and no host
 * synchronisation: the slot offsets are computed on the device.  The bound
 * flows go to ft_flowtree_batch (with the same pairs) and to
 * ft_flowtree_backward exactly like those of ft_flows_create; the adjoint's
 * work grows with the capacity, not only with the bound pairs.  a and b
 * must outlive the flows.  Pair indices out of range flag FT_EINVAL in the
 * tree's status word (ft_tree_status). */
ft_status ft_flows_create_capacity(const ft_tree* t, const ft_docs* a, const ft_docs* b, int64_t max_pairs,
                                   ft_flows** out);
ft_status ft_flows_bind(ft_flows* f, const int32_t* pair_a_dev, const int32_t* pair_b_dev, int64_t n_pairs,
                        void* stream);

/* ------------------------------------------------------------------------
 * Adjoint of the Flowtree estimate for the frozen flow (derived from the
 * pricing sum of Sec. 3; the paper does not differentiate):
 *   grad_vocab[x] += sum_i g_i sum_{pairs (x,y)} f/2^24 (x - y)/||x - y||
 *   grad_vocab[y] -= the same,
 * with g_i = grad_cost_dev[i]; pairs at distance 0 contribute nothing.
 * grad_vocab_dev float32 [n_points][dim] is accumulated into (not zeroed).
 * Deterministic: contributions are sorted by point and reduced in a fixed
 * order (no floating-point atomics).
 * ------------------------------------------------------------------------ */
size_t ft_flowtree_backward_workspace_size(const ft_tree* t, const ft_flows* flows);
ft_status ft_flowtree_backward(const ft_tree* t, const ft_docs* a, const ft_docs* b, const ft_flows* flows,
                               const float* vocab_dev, const float* grad_cost_dev, float* grad_vocab_dev,
                               void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Quadtree W1 prefilter (Sec. 2 closed form) + top-k select.
 *
 * For every query q and database document j:
 *   L1(q, j) = sum_{k=1..L+1} 2^(L+1-k) sum_{v at depth k} |mu_q(v) - mu_j(v)|
 * in units of u * 2^-24 (u = 2 Phi / 2^(L+1)), exact int64.
 * cand_ids_out_dev int32 [nq][k1]: the k1 smallest per query, ascending by
 * (L1, document id).  cand_l1_out_dev int64 [nq][k1] or NULL.
 * l1_all_out_dev (ft_quadtree_l1_dense) int64 [nq][n_db].
 * k1 <= min(n_db, 4096).
 * ------------------------------------------------------------------------ */
size_t ft_quadtree_scan_workspace_size(const ft_tree* t, const ft_docs* queries, const ft_docs* db, int32_t k1);
ft_status ft_quadtree_scan(const ft_tree* t, const ft_docs* queries, const ft_docs* db, int32_t k1,
                           void* workspace, size_t ws_bytes, int32_t* cand_ids_out_dev,
                           int64_t* cand_l1_out_dev, void* stream);
ft_status ft_quadtree_l1_dense(const ft_tree* t, const ft_docs* queries, const ft_docs* db,
                               int64_t* l1_all_out_dev, void* stream);

/* Work of the scan, for measurement: the number of (query node, database
 * document) matches the scan visits, i.e. the sum over the queries and the
 * nodes of their embeddings of the number of database documents holding
 * that node.  Each visit reads one 8-byte posting.  Synchronous; writes the
 * count to *matches_out_host. */
ft_status ft_quadtree_scan_matches(const ft_tree* t, const ft_docs* queries, const ft_docs* db,
                                   int64_t* matches_out_host);

/* ------------------------------------------------------------------------
 * k-nearest-neighbour pipeline (Sec. 5.2): quadtree scan -> top-k1 ->
 * batched Flowtree on the nq*k1 candidates -> top-k per query.
 * ids_out_dev int32 [nq][k], dist_out_dev float32 [nq][k], ascending by
 * (Flowtree value, document id).  k <= k1.  Allocation-free and
 * synchronisation-free: capturable in a CUDA graph (see the graph calls).
 * ------------------------------------------------------------------------ */
size_t ft_knn_workspace_size(const ft_tree* t, const ft_docs* db, const ft_docs* queries, int32_t k1, int32_t k);
ft_status ft_knn(const ft_tree* t, const float* vocab_dev, const ft_docs* db, const ft_docs* queries, int32_t k1,
                 int32_t k, void* workspace, size_t ws_bytes, int32_t* ids_out_dev, float* dist_out_dev,
                 void* stream);

/* ------------------------------------------------------------------------
 * Exact W1 (Eq. 1) of document pairs: the re-ranking stage of the Sec. 5.2
 * pipelines (the paper runs a network-simplex code on the CPU).
 *
 * For pair i, the min-cost transportation between the supports of
 * a[pair_a_dev[i]] and b[pair_b_dev[i]] (their 2^24 fixed-point masses,
 * equal totals) with arc cost ||x - y||_2 over the rows of vocab_dev
 * float32 [n_points][dim] (the tree's ground set and dimension):
 *   cost_out_dev[i] = sum f(x, y) ||x - y|| / 2^24.
 * Solved per pair by one warp with successive shortest paths and node
 * potentials (Dijkstra over the dense bipartite graph); the flow is exact
 * integers, costs and potentials are FP32, so the value is optimal up to the
 * FP32 rounding of the costs.  Time about (s_a + s_b)^3 / 32 warp steps per
 * pair: meant for the few candidates that reach the last stage.
 * a and b must share one tree.  pair arrays int32 [n_pairs] on the device
 * (an index out of range flags FT_EINVAL in the status word and yields NaN).
 * A pair that does not converge within 8 (s_a + s_b) + 64 augmentations
 * (not expected) flags FT_ETIMEOUT and yields NaN.  Workspace per resident
 * warp: 8 B x max_support(a) x max_support(b).  Allocation-free.
 * ------------------------------------------------------------------------ */
size_t ft_exact_w1_workspace_size(const ft_docs* a, const ft_docs* b, int64_t n_pairs);
ft_status ft_exact_w1_batch(const float* vocab_dev, const ft_docs* a, const ft_docs* b, const int32_t* pair_a_dev,
                            const int32_t* pair_b_dev, int64_t n_pairs, float* cost_out_dev, void* workspace,
                            size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Mean-distance prefilter (the "Mean" method of Sec. 5): for every query q
 * and database document d, ||sum_i mu_q(i) x_i - sum_j mu_d(j) y_j||_2, the
 * distance between the mass-weighted centroids over the rows of vocab_dev
 * float32 [n_points][dim] (a lower bound on W1).  cand_ids_out_dev int32
 * [nq][k1] / cand_dist_out_dev float32 [nq][k1]: the k1 smallest per query,
 * ascending by (distance, document id).  FP32 throughout (the library's own
 * tiled kernel: centroid cross products with the distance epilogue
 * sqrt(|c_q|^2 + |c_d|^2 - 2 c_q . c_d) fused, then a radix select over each
 * query's distance row).  k1 <= min(n_db, 4096); at most 65535 * 128
 * queries per call.  Allocation-free: the centroids and the [nq][n_db]
 * distance matrix live in the workspace.
 * ------------------------------------------------------------------------ */
size_t ft_mean_scan_workspace_size(const ft_docs* queries, const ft_docs* db, int32_t k1);
ft_status ft_mean_scan(const float* vocab_dev, const ft_docs* queries, const ft_docs* db, int32_t k1,
                       void* workspace, size_t ws_bytes, int32_t* cand_ids_out_dev, float* cand_dist_out_dev,
                       void* stream);

/* ------------------------------------------------------------------------
 * Three-stage nearest-neighbour pipeline (Sec. 5.2; Flowtree as the
 * intermediate stage of Sec. 5.3's tuned pipelines): quadtree scan ->
 * top-k1 -> batched Flowtree -> top-k2 -> exact W1 -> top-k per query.
 * ids_out_dev int32 [nq][k], dist_out_dev float32 [nq][k] (exact W1),
 * ascending by (W1, document id).  k <= k2 <= k1.  Allocation-free and
 * synchronisation-free: capturable in a CUDA graph.
 * ------------------------------------------------------------------------ */
size_t ft_knn_exact_workspace_size(const ft_tree* t, const ft_docs* db, const ft_docs* queries, int32_t k1,
                                   int32_t k2, int32_t k);
ft_status ft_knn_exact(const ft_tree* t, const float* vocab_dev, const ft_docs* db, const ft_docs* queries,
                       int32_t k1, int32_t k2, int32_t k, void* workspace, size_t ws_bytes, int32_t* ids_out_dev,
                       float* dist_out_dev, void* stream);

/* ------------------------------------------------------------------------
 * Per-row top-k of FP32 values (final selection, Sec. 5.2): for each of
 * n_rows rows of values_dev [n_rows][n_cols] (row-major, non-negative
 * values such as Flowtree costs), the k smallest ascending by (value,
 * column), written to ids_out_dev / vals_out_dev [n_rows][k].  NaN sorts
 * last.  k <= min(n_cols, 4096).  Allocation-free.
 * ------------------------------------------------------------------------ */
size_t ft_topk_f32_workspace_size(int64_t n_rows, int64_t n_cols);
ft_status ft_topk_f32(const float* values_dev, int64_t n_rows, int64_t n_cols, int32_t k, void* workspace,
                      size_t ws_bytes, int32_t* ids_out_dev, float* vals_out_dev, void* stream);

/* ------------------------------------------------------------------------
 * Read-bandwidth probe (measurement utility, not part of the method): the
 * measured peak that the row-gathering kernels' L2 roofline divides by.
 * Every SM reads buf_dev[0 .. bytes) `passes` times with independent
 * 16-byte loads that bypass L1; a buffer that fits in L2 (after one warm
 * pass) measures L2 read bandwidth, a larger one HBM.  The XOR of all
 * loaded 32-bit words (passes even: 0) is XOR-ed into *sink_dev, so the
 * loads cannot be elided.  buf_dev 16-byte aligned, bytes a multiple of
 * 16 (>= 16), passes >= 1, else FT_EINVAL.  Asynchronous on stream; the
 * caller times it with events.
 * ------------------------------------------------------------------------ */
ft_status ft_read_probe(const void* buf_dev, size_t bytes, int32_t passes, uint32_t* sink_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FLOWTREE_H */
