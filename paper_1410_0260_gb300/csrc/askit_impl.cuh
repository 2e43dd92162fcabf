// Internal declarations of the GB300 ASKIT library: the tree object, error
// plumbing, and the canonical FP64 arithmetic that makes the setup stages
// (kNN, tree, skeletons) reproducible bit for bit on any IEEE machine.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <string>
#include <vector>

#include "askit.h"

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
void askit_set_error(const char *fmt, ...);

#define ASK_CUDA(call)                                                                 \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            askit_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,                 \
                            cudaGetErrorString(e_));                                   \
            return e_ == cudaErrorMemoryAllocation ? ASKIT_ERR_OOM : ASKIT_ERR_CUDA;   \
        }                                                                              \
    } while (0)

#define ASK_TRY(call)                                \
    do {                                             \
        askit_status s_ = (call);                    \
        if (s_ != ASKIT_OK) return s_;               \
    } while (0)

#define ASK_LAUNCH()                                 \
    do {                                             \
        ASK_CUDA(cudaGetLastError());                \
    } while (0)

// Sticky device status codes (written by kernels with bounded waits).
enum { ASK_DEV_OK = 0, ASK_DEV_TIMEOUT = 1, ASK_DEV_BAD_ITEM = 2 };

// Rows of each skeleton block and of the target/source arrays are padded to a
// multiple of this, so that tensor-core tiles never straddle two blocks.
constexpr int ASK_ROW_PAD = 32;
// Targets per evaluation item (one tensor-core M tile).
constexpr int ASK_TILE_M = 128;
// Source rows per sub-block (one tensor-core N tile); leaves and skeletons
// longer than this are split into consecutive sub-blocks.
constexpr int ASK_BLK_N = 128;
// Items per segment of a sub-block's items (schedule of the K-chunked kernel's
// paired items).
constexpr int ASK_SEG_ITEMS = 8;
// Columns of the tensor-core operand arrays (d <= TC_K).
constexpr int TC_K = 64;
// Default and largest entries of one in-sample work-list batch (entry
// offsets inside a batch are int32).
constexpr int64_t ASK_BATCH_ENTRIES = (int64_t)1 << 28;
constexpr int64_t ASK_BATCH_ENTRIES_MAX = (int64_t)1 << 30;

// ---------------------------------------------------------------------------
// Device memory owned by a tree: every allocation is recorded and freed by
// askit_destroy.
// ---------------------------------------------------------------------------
struct DevArena {
    std::vector<void *> ptrs;
    size_t bytes = 0;
    // stream-ordered mode (per-call temporaries): cudaMallocAsync/cudaFreeAsync
    // on `stream`, so freeing does not synchronize the device
    bool async = false;
    cudaStream_t stream = nullptr;
    template <class T>
    askit_status alloc(T **p, size_t count) {
        *p = nullptr;
        if (count == 0) count = 1;
        void *q = nullptr;
        cudaError_t e = async ? cudaMallocAsync(&q, count * sizeof(T), stream) : cudaMalloc(&q, count * sizeof(T));
        if (e != cudaSuccess) {
            askit_set_error("cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? ASKIT_ERR_OOM : ASKIT_ERR_CUDA;
        }
        ptrs.push_back(q);
        bytes += count * sizeof(T);
        *p = static_cast<T *>(q);
        return ASKIT_OK;
    }
    void release(void *p) {
        for (auto &q : ptrs)
            if (q == p) { cudaFree(q); q = nullptr; }
    }
    void free_all() {
        for (void *q : ptrs)
            if (q) {
                if (async) cudaFreeAsync(q, stream);
                else cudaFree(q);
            }
        ptrs.clear();
        bytes = 0;
    }
};

// One evaluation work item: one source sub-block (up to ASK_BLK_N rows of a
// leaf's points, evaluated directly, or of a node's skeleton) against up to
// ASK_TILE_M targets that all need it.  Its targets are entries
// e0 .. e0 + cnt - 1 of the work lists' sorted entry array.
struct __align__(16) EvalItem {
    int32_t row0;    // first source row (in Xt for leaves, in the skeleton pool else)
    int32_t nrows;   // valid source rows; bit 31 set = skeleton (far-field) block
    int32_t e0;      // first entry
    int32_t cnt;     // targets (entries) of this item
    int32_t cidx;    // sub-block index (its center in the centered operand arrays)
    int32_t pad_[3];
};

// Target rows of one evaluation in the global-centered FP16x3 form: hi / lo
// [rows, TC_K] FP16 of (x - xbar) g_sigma and the norm blocks x [rows, 16].
struct QuerySplit {
    const uint16_t *hi = nullptr, *lo = nullptr, *x = nullptr;
    int64_t rows = 0;
};

// Work lists of one set of targets (in-sample, or one out-of-sample batch).
struct WorkLists {
    int64_t T = 0, n_entries = 0, n_items = 0, n_blocks = 0;
    int64_t *off = nullptr;          // [T + 1] entries of target q: emission slots off[q] .. off[q+1)
    int32_t *slot_of_emit = nullptr; // [n_entries] sorted position of each emitted entry
    int32_t *tgt = nullptr;          // [n_entries] target slot of each sorted entry
    EvalItem *items = nullptr;       // [n_items], grouped by sub-block
    int32_t *block_off = nullptr;    // [n_blocks + 1] items of each sub-block
    int32_t *block_order = nullptr;  // [n_blocks] heaviest first
    // persistent-kernel schedule: sub-blocks dealt to n_ctas CTAs, heaviest
    // first, each to the CTA with the least work so far
    int n_ctas = 0;
    int32_t *cta_off = nullptr;      // [n_ctas + 1] the schedule in use (one of the two below)
    int32_t *cta_blocks = nullptr;   // [n_blocks]
    // 0: longest first (LPT), 1: tree-order ranges, 2: LPT over sub-block
    // pairs (the leader of each pair; followers are processed with it)
    int32_t *sched_off[3] = {nullptr, nullptr, nullptr};
    int32_t *sched_blocks[3] = {nullptr, nullptr, nullptr};
    int n_ctas_sched[3] = {0, 0, 0};
    int32_t *partner = nullptr;      // [n_blocks] the paired follower of a leader block, else -1
    int64_t n_pairs = 0;
    // segments: every sub-block's items cut into runs of at most
    // ASK_SEG_ITEMS (a follower at its leader's cuts), the leaders' segments
    // dealt block by block, heaviest first, to the least-loaded CTA (the
    // K-chunked kernel's paired items: the CTAs work on few blocks at a time)
    int64_t n_seg = 0;
    int32_t *seg_off = nullptr;      // [n_seg + 1] items of each segment
    int32_t *seg_partner = nullptr;  // [n_seg] the follower's segment, else -1
    int32_t *seg_sched_off = nullptr;   // [n_ctas + 1]
    int32_t *seg_sched = nullptr;       // [leader segments]
    int64_t pairs_alg = 0, pairs_cmp = 0, near_tot = 0, far_tot = 0;
};

// Weights of one evaluation context: W in tree order, the skeleton weights
// of the upward pass, and the per-entry partial sums of Evaluate.  A tree
// has a default context; askit_weights_create adds independent ones, so
// several weight sets can be evaluated concurrently on different streams.
struct WeightCtx {
    int r = 0, r_cap = 0;
    float *Wt = nullptr;       // [N_pad, r] weights in tree order
    float *Ws = nullptr;       // [rows of the skeleton pool, r] skeleton weights
    float *partial = nullptr;  // [in-sample entries, r_cap]
    float4 *colv = nullptr;    // [n_sub, 128] per-sub-block column data (16-bit tensor-core path)
    float *colw = nullptr;     // [n_sub, 128 * 16 + 16] per-sub-block weights (r > 1)
    int64_t ent_cap = 0;       // entries the partial sums hold
    bool ready = false;
    DevArena arena;
};

struct askit_tree_s;
struct askit_weights_s {
    askit_tree_s *t = nullptr;
    WeightCtx ctx;
};

// A captured set_weights + evaluate step with its own weight context.
struct askit_graph_s {
    askit_tree_s *t = nullptr;
    WeightCtx ctx;
    cudaGraphExec_t exec = nullptr;
    int64_t n_nodes = 0;
};

struct askit_tree_s {
    askit_params prm;
    int64_t N = 0;
    int d = 0, d_pad = 0, L = 0, kappa = 0, rp_leaf = 0, ell_max = 0;
    int64_t n_nodes = 0;
    DevArena arena;

    // caller-order data
    float *X = nullptr;        // [N, d]
    float *hsrc = nullptr;     // [N]
    int32_t *knn = nullptr;    // [N, kappa]
    double *knnd = nullptr;    // [N, kappa]

    // tree
    int32_t *perm = nullptr;   // [N] tree position -> point id
    int32_t *pos = nullptr;    // [N] point id -> tree position
    int32_t *leafof = nullptr; // [N] point id -> leaf heap index
    std::vector<int64_t> h_start, h_size;
    int32_t *nstart = nullptr, *nsize = nullptr;  // [n_nodes]

    // node neighbor lists and sampled targets ([n_nodes, ell_max])
    int32_t *nl_cnt = nullptr, *nl_ids = nullptr;
    double *nl_key = nullptr;
    int32_t *trows = nullptr;

    // skeletons, heap order pools
    std::vector<int32_t> h_s, h_ncol;
    std::vector<int64_t> h_skoff, h_pivoff, h_poff, h_spool;
    int64_t skel_total = 0, piv_total = 0, p_total = 0, spool_rows = 0;
    int32_t *skel_ids = nullptr;  // [skel_total]
    int32_t *piv = nullptr;       // [piv_total]
    double *P64 = nullptr;        // [p_total]
    float *P32 = nullptr;         // [p_total]
    int64_t *d_skoff = nullptr, *d_pivoff = nullptr, *d_poff = nullptr, *d_spool = nullptr;
    int32_t *d_s = nullptr, *d_ncol = nullptr;

    // evaluation operands
    int64_t N_pad = 0;
    float *Xt = nullptr;       // [N_pad, d_pad] tree order, zero padded
    float *Xs = nullptr;       // [spool_rows, d_pad] skeleton coordinate pool
    float *nrm_t = nullptr, *nrm_s = nullptr;   // squared norms
    float *sc_t = nullptr, *sc_s = nullptr;     // c * log2(e) / h_j^2 per source row
    WeightCtx dw;              // default weight context (askit_set_weights)
    int precision = ASKIT_PREC_TF32X3;

    // in-sample work lists, one per batch of consecutive target slots
    // [wl_t0[b], wl_t0[b + 1]); the partial sums are sized for the largest
    std::vector<WorkLists> wl;
    std::vector<int64_t> wl_t0;
    int64_t wl_entries = 0, wl_entries_max = 0;

    // tensor-core operands: every source sub-block centered on its own mean,
    // split into hi + lo parts (TF32 and BF16), kw columns (TC_K, or d_pad
    // for wide rows, whose 16-bit splits are stored as planes of 8-column K
    // groups, [kw / 8][rows][8]), and the squared norms of the centered rows
    int64_t n_sub = 0;
    int32_t *leaf_cbase = nullptr; // [2^L] first sub-block of each leaf
    int32_t *node_cbase = nullptr; // [n_nodes] first sub-block of each skeleton
    float *cent = nullptr;         // [n_sub, kw]
    float *Xt_hi = nullptr, *Xt_lo = nullptr, *Xs_hi = nullptr, *Xs_lo = nullptr;   // TF32 split
    uint16_t *Xt_bhi = nullptr, *Xt_blo = nullptr, *Xs_bhi = nullptr, *Xs_blo = nullptr; // BF16 split
    uint16_t *Xt_hhi = nullptr, *Xt_hlo = nullptr, *Xs_hhi = nullptr, *Xs_hlo = nullptr; // FP16 split (prescaled)
    float f16_scale = 1.f;         // power of 2 keeping centered coordinates within FP16 range
    float *nrmc_t = nullptr, *nrmc_s = nullptr;
    int64_t srows = 0;             // rows of the skeleton-pool arrays

    // global-centered FP16x3 operands (d <= TC_K, eval_g16.cu): every point
    // centered on the data mean g_xbar; targets (x - xbar) g_sigma and
    // sources (y - xbar) 2 sc_j / g_sigma split into FP16 hi + lo; the norm
    // blocks of targets [rows, 16] and of every source sub-block (scales
    // g_tau, g_kappa); n = |x - xbar|^2.  g_rho = max_j sc_j * max_i n_i
    // decides the automatic choice (g_ok)
    uint16_t *Xg_hi = nullptr, *Xg_lo = nullptr, *Xg_x = nullptr;   // tree points as targets
    uint16_t *Xb_hi = nullptr, *Xb_lo = nullptr;                    // tree points as sources
    uint16_t *Sb_hi = nullptr, *Sb_lo = nullptr;                    // skeleton pool as sources
    uint16_t *g_bx = nullptr;                                       // [n_sub, 128 x 16]
    float *ng_t = nullptr, *ng_s = nullptr;
    float *g_xbar = nullptr;       // [TC_K] device
    float g_sigma = 1.f, g_tau = 1.f, g_kappa = 1.f;
    double g_rho = 0.0;
    bool g_ok = false;
    int fp16_centering = 0;        // 0 automatic (global when g_ok), 1 per sub-block, 2 global
    void *g16 = nullptr;           // tensor maps of the global-centered kernel

    int *d_status = nullptr;       // sticky kernel status
    int *d_ticket = nullptr;       // persistent-kernel work counter
    void *tc = nullptr;            // tensor-core kernel state (tensor maps)
    void *tcw = nullptr;           // the same for the wide (d > TC_K) kernel
    void *tc16 = nullptr;          // the same for the 16-bit narrow kernel
    int64_t *sb_row0 = nullptr;    // [n_sub] first row of each sub-block (Xt rows, then Xs rows)
    int32_t *sb_nr = nullptr;      // [n_sub] rows of each sub-block
    int64_t n_leaf_sub = 0;        // sub-blocks of leaves (the rest are skeleton sub-blocks)
    std::vector<int64_t> h_sub_pos; // [n_sub] tree position of each sub-block's node (schedule order)
    std::vector<int64_t> h_sub_node; // [n_sub] heap index of each sub-block's node
    // launch configuration of the evaluation kernels (askit_autotune)
    int tune_sched = 0;            // block-to-CTA schedule: 0 LPT, 1 tree-order ranges
    int tune_stages = 3;           // gathered target-row stages of the FP16x3 kernel (2 or 3)
    int tune_runs = 1;             // 8-row tiled loads for runs of consecutive targets
    int tune_pairs = 0;            // FP16x3: items over two sub-blocks of a node (256 columns)
    int spin_limit = 0;            // polls of the FP16x3 kernel's bounded waits (0: default)
    // refinements of the pruning (askit_set_pruning): skeletons only for nodes
    // at most far_height levels above the leaves (-1: all), and the kernel cut
    // of the adaptive kappa_i (0: all kappa neighbors)
    int far_height = -1;
    double kappa_cut = 0.0;
    int kw = TC_K;                 // row width of the pre-split operands and centers
    // wall time of the setup stages (askit_info.setup_ms)
    double setup_ms[7] = {0, 0, 0, 0, 0, 0, 0};
    std::chrono::steady_clock::time_point stage_t0;
    // CUDA events around each launch of the evaluation kernel while timing
    // is on (askit_kernel_timing): begin/end pairs, reused across sessions
    struct KTimer {
        bool on = false;
        std::vector<cudaEvent_t> ev;
        size_t used = 0;
    } kt;
};

// Records the begin (end = false) or end event of one evaluation-kernel
// launch on stream s while the tree's kernel timer is on; a no-op otherwise
// and while s is being captured into a graph.
askit_status ktimer_mark(askit_tree t, cudaStream_t s, bool end);

// ---------------------------------------------------------------------------
// Canonical FP64 arithmetic (device).  Every operation is an explicitly
// rounded IEEE operation, so no multiply-add is ever fused and results are
// identical to any sequential IEEE-754 binary64 evaluation in the same order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double c_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double c_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double c_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double c_div(double a, double b) { return __ddiv_rn(a, b); }

// Squared distance, coordinates ascending: sum (x_k - y_k)^2.
__device__ __forceinline__ double c_dist2(const float *x, const float *y, int d) {
    double acc = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = c_sub((double)x[k], (double)y[k]);
        acc = c_add(acc, c_mul(t, t));
    }
    return acc;
}

// exp(a) for the ID's kernel matrices: Cody-Waite reduction a = n ln2 + r
// with ln2 split into a 32-significant-bit head and its tail, the degree-13
// Taylor polynomial of e^r in Horner form, and an exact scaling by 2^n
// (n >= -1010 keeps the result normal).  Arguments below -700 give 0.
__device__ __forceinline__ double c_exp(double a) {
    if (a < -700.0) return 0.0;
    if (a > 700.0) return __longlong_as_double(0x7ff0000000000000LL);
    const double inv_ln2 = 0x1.71547652b82fep+0;
    const double ln2_head = 0x1.62e42ff000000p-1;
    const double ln2_tail = -0x1.718432a1b0e26p-35;
    double n = rint(c_mul(a, inv_ln2));
    double r = c_sub(c_sub(a, c_mul(n, ln2_head)), c_mul(n, ln2_tail));
    // 1/k! for k = 13 down to 0
    const double coef[14] = {0x1.6124613a86d09p-33, 0x1.1eed8eff8d898p-29, 0x1.ae64567f544e4p-26,
                             0x1.27e4fb7789f5cp-22, 0x1.71de3a556c734p-19, 0x1.a01a01a01a01ap-16,
                             0x1.a01a01a01a01ap-13, 0x1.6c16c16c16c17p-10, 0x1.1111111111111p-7,
                             0x1.5555555555555p-5,  0x1.5555555555555p-3,  0x1.0000000000000p-1,
                             0x1.0000000000000p+0,  0x1.0000000000000p+0};
    double p = coef[0];
#pragma unroll
    for (int k = 1; k < 14; ++k) p = c_add(c_mul(p, r), coef[k]);
    long long e = (long long)n + 1023;
    return c_mul(p, __longlong_as_double(e << 52));
}

// Philox4x64-10 (Salmon et al., SC'11): 10 rounds of the two 64x64->128
// multiplications with key bumps between rounds.
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) { k0 += W0; k1 += W1; }
        uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

// Word n of the stream keyed (k0, k1) under counter prefix c0: block n/4, lane n%4.
__device__ __forceinline__ uint64_t philox_word(uint64_t k0, uint64_t k1, uint64_t c0, uint64_t n) {
    uint64_t c[4] = {c0, n >> 2, 0, 0};
    philox4x64_10(c, k0, k1);
    return c[n & 3];
}

// Depth of heap node a (root 1 has depth 0).
__host__ __device__ __forceinline__ int heap_depth(int64_t a) {
    int t = 0;
    while (((int64_t)2 << t) <= a) ++t;
    return t;
}

// ---------------------------------------------------------------------------
// Stage entry points (one translation unit each)
// ---------------------------------------------------------------------------
// setup_sort.cu: segmented sorts (CUB) used by the tree and node-list stages.
askit_status seg_sort_f64_i32(const double *kin, double *kout, const int32_t *vin, int32_t *vout,
                              int64_t n, int nseg, const int32_t *beg, const int32_t *end,
                              void *tmp, size_t *tmp_bytes, cudaStream_t s);
askit_status seg_sort_i32_f64(const int32_t *kin, int32_t *kout, const double *vin, double *vout,
                              int64_t n, int nseg, const int32_t *beg, const int32_t *end,
                              void *tmp, size_t *tmp_bytes, cudaStream_t s);
askit_status seg_sort_i32(const int32_t *kin, int32_t *kout, int64_t n, int nseg,
                          const int32_t *beg, const int32_t *end, void *tmp, size_t *tmp_bytes,
                          cudaStream_t s);
askit_status sort_u64_i32(const uint64_t *kin, uint64_t *kout, const int32_t *vin, int32_t *vout,
                          int64_t n, void *tmp, size_t *tmp_bytes, cudaStream_t s);
askit_status sort_u64_i64(const uint64_t *kin, uint64_t *kout, const int64_t *vin, int64_t *vout,
                          int64_t n, void *tmp, size_t *tmp_bytes, cudaStream_t s);
askit_status scan_i64(const int64_t *in, int64_t *out, int64_t n, void *tmp, size_t *tmp_bytes,
                      cudaStream_t s);

// setup_tree.cu
int tree_depth(int64_t N, int64_t leaf);
void tree_ranges(int64_t N, int L, std::vector<int64_t> &start, std::vector<int64_t> &size);
askit_status build_tree_gpu(const float *X, int64_t N, int d, int L, int kind, uint64_t seed,
                            int iter, int32_t *order, cudaStream_t s);
// self (optional, [Q]): the point id each query Y row is, excluded from its list
askit_status knn_exact_gpu(const float *X, int64_t N, int d, int kappa, const float *Y, int64_t Q,
                           int32_t *ids, double *dist, cudaStream_t s, const int32_t *self = nullptr);
askit_status knn_rp_gpu(const float *X, int64_t N, int d, int kappa, int iters, int64_t rp_leaf,
                        uint64_t seed, int32_t *ids, double *dist, cudaStream_t s);
askit_status knn_dist_gpu(const float *X, int64_t N, int d, int kappa, const int32_t *ids,
                          double *dist, cudaStream_t s);

// setup_skel.cu
askit_status build_node_lists(askit_tree t, cudaStream_t s);
askit_status build_samples(askit_tree t, cudaStream_t s);
askit_status skeletonize(askit_tree t, cudaStream_t s);

// eval_lists.cu
askit_status build_eval_operands(askit_tree t, cudaStream_t s);
askit_status build_tc_operands(askit_tree t, cudaStream_t s);
// Prune sets of a set of targets: rows of `stride` sorted leaf indices
// padded with INT_MAX; target q uses row set_row[q] (leaf-grouped lists, one
// row per leaf) or, with set_row == nullptr, row q.  cudaMalloc'd.
struct PruneSets {
    int32_t *sets = nullptr;
    int stride = 0;
    int32_t *set_row = nullptr;
};
void free_prune_sets(PruneSets &ps);
askit_status build_insample_lists(askit_tree t, const PruneSets &ps, cudaStream_t s);
void use_schedule(askit_tree t);
askit_status build_work_lists(askit_tree t, const int32_t *sets, int stride, const int32_t *set_row, int64_t T,
                              WorkLists &w, DevArena &arena, cudaStream_t s);
askit_status reduce_partials(const WorkLists &w, const float *partial, int r, const int32_t *out_rows,
                             float *U, int64_t ldu, cudaStream_t s);
askit_status insample_prune_sets(askit_tree t, PruneSets &ps, cudaStream_t s);
askit_status oos_prune_sets(askit_tree t, const int32_t *knn, const double *dist, int64_t T, int stride,
                            int32_t *sets, cudaStream_t s);
// every array of w back to the arena
void free_work_lists(WorkLists &w, DevArena &arena);

// weights.cu
askit_status weights_reserve(askit_tree t, WeightCtx &c, int r, cudaStream_t s);
askit_status upward_weights(askit_tree t, WeightCtx &c, const float *W, int r, int64_t ldw, cudaStream_t s);

// eval_simt.cu / eval_tc.cu: partial[e * r + z] for every entry e of w
askit_status eval_simt(askit_tree t, const WeightCtx &c, const float *Xq, int64_t ldq, const WorkLists &w,
                       float *partial, cudaStream_t s);
askit_status eval_tc(askit_tree t, const WeightCtx &c, int precision, const float *Xq, int64_t ldq,
                     int64_t q_rows, const QuerySplit *qs, const WorkLists &w, float *partial, cudaStream_t s);
void eval_tc_free(askit_tree t);
askit_status eval_tc_wide(askit_tree t, const WeightCtx &c, int precision, const float *Xq, int64_t ldq,
                          int64_t q_rows, const WorkLists &w, float *partial, cudaStream_t s);
void eval_tc_wide_free(askit_tree t);
askit_status eval_tc16(askit_tree t, const WeightCtx &c, int precision, const float *Xq, int64_t ldq, int64_t q_rows,
                       const WorkLists &w, float *partial, cudaStream_t s);
void eval_tc16_free(askit_tree t);
// eval_g16.cu: the global-centered FP16x3 kernel (targets pre-split in q)
askit_status eval_g16(askit_tree t, const WeightCtx &c, const QuerySplit &q, const WorkLists &w, float *partial,
                      cudaStream_t s);
void eval_g16_free(askit_tree t);
askit_status build_g16_operands(askit_tree t, cudaStream_t s);
// target rows X [rows, ldx] (d columns) in the global-centered form of tree t;
// *overflow (if given) is set when a value leaves the FP16-safe range
askit_status g16_split_rows(const float *X, int64_t ldx, int d, int64_t rows, const askit_tree_s *t, uint16_t *hi,
                            uint16_t *lo, uint16_t *nx, int *overflow, cudaStream_t s);
// whether FP16x3 evaluations of this tree take the global-centered kernel
inline bool use_g16(const askit_tree_s *t) {
    return t->Xg_hi && (t->fp16_centering == 2 || (t->fp16_centering == 0 && t->g_ok));
}
askit_status knn_shortlist_tc16(askit_tree t, const float *Yp, int64_t T, const float *U, int *cnt, int32_t *cand,
                                int cap, float eta, cudaStream_t s);
// exact kNN of out-of-sample points Y [T, d] against the tree's points:
// tensor-core shortlist + canonical FP64 re-rank where the operands exist,
// else the tiled exhaustive search; ids / dist [T, kappa] as knn_exact_gpu
askit_status knn_oos(askit_tree t, const float *Y, int64_t T, int kappa, int32_t *ids, double *dist, cudaStream_t s);
