/*
 * askit.h -- C ABI of the GB300 ASKIT evaluation library (libaskit.so).
 *
 * ASKIT (March, Xiao & Biros, "ASKIT: Approximate Skeletonization
 * Kernel-Independent Treecode in High Dimensions") approximates the kernel
 * sums of eq. (1.1),
 *
 *     u_i = sum_j K(x_i, x_j) w_j,   K(x, y) = exp(-c ||x - y||^2 / h_y^2),
 *
 * (the Gaussian of Section 4; c = 1 in the paper, c = 1/2 gives the usual
 * exp(-r^2 / 2h^2)) by a binary tree, the kNN graph (pruning rule eq. (2.5))
 * and sampled interpolative decompositions of every node (Section 2.1,
 * Algorithm 3).  Algorithm 5 splits the method into a setup (tree, kNN,
 * node neighbor lists, skeletonization) and Evaluate (Algorithm 4), which is
 * the per-weight-vector cost; this library runs both on one GPU.
 *
 * Conventions
 *  - Every pointer argument named *_dev is a device pointer owned by the
 *    caller; the library reads or writes it on `stream` and never frees it.
 *    *_host pointers are host memory owned by the caller.
 *  - Matrices are row-major with a leading dimension (ld*) in elements.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *  - Calls are stream-ordered.  askit_setup, askit_get_* and askit_sync
 *    block the host; askit_set_weights, askit_evaluate and
 *    askit_evaluate_targets only enqueue work.
 *  - Errors are returned as askit_status, never by aborting; the message of
 *    the last failure on the calling thread is askit_last_error().  A kernel
 *    that gives up a bounded wait sets a sticky status that askit_sync
 *    reports as ASKIT_ERR_TIMEOUT.
 *  - A tree is not thread-safe: calls on one tree must not race.
 */
#ifndef ASKIT_H
#define ASKIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct askit_tree_s *askit_tree;

typedef enum {
    ASKIT_OK = 0,
    ASKIT_ERR_INVALID_ARG = 1,
    ASKIT_ERR_OOM = 2,
    ASKIT_ERR_CUDA = 3,
    ASKIT_ERR_TIMEOUT = 4,
    ASKIT_ERR_NOT_READY = 5,
    ASKIT_ERR_UNSUPPORTED = 6
} askit_status;

/* Distance-contraction precision of Evaluate. */
enum {
    ASKIT_PREC_SIMT_FP32 = 0, /* plain FP32 difference form on CUDA cores */
    ASKIT_PREC_TF32X3 = 1,    /* tcgen05 tensor cores, 3xTF32 split, FP32 accumulate */
    ASKIT_PREC_BF16X3 = 2,    /* tcgen05 tensor cores, BF16x3 split, FP32 accumulate */
    ASKIT_PREC_FP16X3 = 3     /* tcgen05 tensor cores, FP16x3 split (power-of-2 prescaled), FP32 accumulate */
};

/* Bandwidth of the Gaussian (Section 4: constant h, or h_j per source). */
enum {
    ASKIT_BW_CONSTANT = 0, /* h_j = h */
    ASKIT_BW_ARRAY = 1,    /* h_j from the caller's array */
    ASKIT_BW_KNN = 2       /* h_j = distance from x_j to its bw_k-th nearest neighbor */
};

typedef struct {
    int32_t leaf_size;   /* m: points per leaf (Section 3); >= 2 */
    int32_t kappa;       /* kappa: nearest neighbors per point, self excluded; 1..32 */
    int32_t knn_mode;    /* 0 exact kNN, 1 random-projection trees (Section 2.2) */
    int32_t rp_iters;    /* number of random-projection trees (knn_mode 1) */
    int32_t rp_leaf;     /* points per RP leaf; 0 = max(2 kappa + 2, m) */
    int32_t s_max;       /* largest skeleton (Section 3, s) */
    int32_t s_min;       /* smallest skeleton (adaptive rank floor) */
    int32_t ell_extra;   /* sampled rows ell = s_max + ell_extra (paper: 20) */
    int32_t prune;       /* 1: neighbor pruning eq. (2.5) per target; 0: every leaf
                            direct; 2: leaf-grouped lists -- every target of a leaf
                            is pruned with the union of {p} U N_p over the leaf's
                            points p, so the targets of a leaf share one Near and
                            one Far list (the overlap Section 3 notes for the
                            targets of one leaf; out-of-sample targets keep N_y) */
    int32_t bw_mode;     /* ASKIT_BW_* */
    int32_t bw_k;        /* neighbor rank for ASKIT_BW_KNN (1..kappa) */
    int32_t precision;   /* ASKIT_PREC_* used by askit_evaluate */
    double id_tol;       /* rank cut: first k with |R_kk| <= id_tol |R_00| */
    double kernel_scale; /* c in exp(-c r^2 / h^2) */
    double h;            /* constant bandwidth (ASKIT_BW_CONSTANT) */
    uint64_t seed;       /* Philox key for RP directions and row sampling */
    int64_t batch_entries; /* in-sample work lists are built and evaluated in
                              batches of consecutive targets (tree order) of at
                              most this many (target, sub-block) entries, which
                              bounds the build's sort buffers and the partial
                              sums; 0 = 2^28, at most 2^30 */
} askit_params;

/* Fill `p` with defaults (m = 128, kappa = 16, exact kNN, s_max = 64,
 * ell_extra = 20, prune = 1, constant h = 1, c = 1/2, id_tol = 1e-6,
 * TF32x3 evaluation, seed = 1, batch_entries = 0). */
void askit_default_params(askit_params *p);

/*
 * Setup: Algorithm 5 up to Evaluate -- kNN (Section 2.2, exact or RP
 * trees), the median-split binary tree (Section 2.2), node neighbor lists
 * (Algorithm 2), sampled targets (eq. (2.4)), skeletons and interpolation
 * matrices by FP64 pivoted QR (Section 2.1, Algorithm 3), and the
 * evaluation work lists of every target tile (pruning rule eq. (2.5)).
 *
 *   X_dev   [N, d] FP32 points (row stride ldx >= d), read during the call only.
 *   h_dev   [N] FP32 per-point bandwidth for ASKIT_BW_ARRAY, else NULL.
 *   knn_dev optional [N, kappa] int32 caller-given neighbor ids (the paper's
 *           N(X) argument of Algorithm 5, self excluded), or NULL to compute.
 *   out     receives the tree handle (library-owned; askit_destroy frees it).
 * Errors: INVALID_ARG for N < 1, d < 1, m < 2, kappa outside 1..min(32, N-1),
 * s_max < 1, non-positive h or id_tol < 0; OOM when device memory runs out;
 * UNSUPPORTED for N >= 2^31, leaf_size or s_max above 2048 (16 sub-blocks
 * of 128 rows) or a tree deeper than 25 levels.  Blocks until the setup is
 * complete.
 */
askit_status askit_setup(const float *X_dev, int64_t N, int32_t d, int64_t ldx,
                         const float *h_dev, const int32_t *knn_dev,
                         const askit_params *p, void *stream, askit_tree *out);

/*
 * New weight vectors: stores W in tree order and runs the upward pass of
 * skeleton weights w~_a = w(S_a) + P_a w(R) (Section 2.1, Algorithm 3),
 * level by level from the leaves up.
 *   W_dev [N, r] FP32 (row stride ldw >= r), in the caller's point order;
 *   read on `stream` before the call's work completes.  1 <= r <= 64.
 */
askit_status askit_set_weights(askit_tree t, const float *W_dev, int32_t r, int64_t ldw,
                               void *stream);

/*
 * Evaluate (Algorithm 4) at every point: U_dev [N, r] FP32 (row stride
 * ldu >= r) receives u_i in the caller's point order.  Near-field leaves
 * are summed directly, pruned nodes through their skeletons; the work runs
 * as one persistent launch over all (target tile, source block) items of
 * each target batch (askit_params.batch_entries; one batch unless the
 * entries exceed it), then a fixed-order reduction of the partial sums.
 * Requires askit_set_weights first (NOT_READY otherwise).
 */
askit_status askit_evaluate(askit_tree t, float *U_dev, int64_t ldu, void *stream);

/*
 * Evaluate at out-of-sample targets Y (the paper takes targets = sources;
 * here the prune set of y is its exact kappa nearest sources, eq. (2.5)
 * with {i} replaced by nothing).  Y_dev [T, d] FP32 (stride ldy),
 * U_dev [T, r] FP32 (stride ldu).  Allocates per-call work lists and
 * blocks the host until they are built.
 */
askit_status askit_evaluate_targets(askit_tree t, const float *Y_dev, int64_t T, int64_t ldy,
                                    float *U_dev, int64_t ldu, void *stream);

/*
 * End-to-end call on host memory: copies W_host [N, r] (stride ldw) to the
 * device, runs askit_set_weights and askit_evaluate, copies u back into
 * U_host [N, r] (stride ldu) and waits for completion.
 */
askit_status askit_evaluate_host(askit_tree t, const float *W_host, int32_t r, int64_t ldw,
                                 float *U_host, int64_t ldu, void *stream);

/*
 * Exact kNN of new points against the tree's points (the prune set of an
 * out-of-sample target, Algorithm 4 with N_y in place of N_i): for each row
 * of Y_dev [T, d] (stride ldy), the kappa (<= 32, the tree's kappa) nearest
 * points by (squared distance, id), ties by id, distances in canonical FP64
 * from the FP32 coordinates -- the same lists the exhaustive search gives.
 *   ids_dev  [T, kappa] int32 point ids (caller order); dist_dev [T, kappa]
 *   double squared distances.  Blocks until done.
 * For d <= 64 a tensor-core FP16x3 shortlist (every point within a bound of
 * each query's k-th distance, with a margin five times the arithmetic's error)
 * is re-ranked in FP64; queries whose shortlist overflows take the exhaustive
 * search.
 */
askit_status askit_knn_targets(askit_tree t, const float *Y_dev, int64_t T, int64_t ldy, int32_t *ids_dev,
                               double *dist_dev, void *stream);

/*
 * Exact kNN of some of the tree's own points (Section 4 measures the hit rate
 * hr of approximate neighbor lists against an exhaustive search): for each id
 * in ids_dev [Q] (caller order, 0 .. N-1), the tree's kappa nearest other
 * points by (squared distance, id) in canonical FP64 from the FP32
 * coordinates, self excluded -- the lists of the setup's exact kNN
 * (knn_mode 0) for those points.  nbr_dev [Q, kappa] int32, dist_dev
 * [Q, kappa] double.  INVALID_ARG for an id out of range.  Blocks until done.
 */
askit_status askit_knn_points(askit_tree t, const int32_t *ids_dev, int64_t Q, int32_t *nbr_dev,
                              double *dist_dev, void *stream);

/*
 * Evaluate with one part of Algorithm 4 only: part 1 the near field (the
 * direct sums over the leaves of Near(i)), part 2 the far field (the
 * skeleton sums over Far(i)), part 0 both (askit_evaluate).  The near field
 * alone gives the error eps_kappa the paper reports beside eps (Table 4).
 * U_dev [N, r] as askit_evaluate; uses the tree's default weights.
 */
askit_status askit_evaluate_part(askit_tree t, int32_t part, float *U_dev, int64_t ldu, void *stream);

/*
 * Pruning statistics of Section 3's Table 1 for the points X_dev [N, d]
 * (stride ldx) as targets: the number of tree nodes the downward pass visits
 * (Evaluate calls, pruned nodes included) with leaves of at most leaf_size
 * points, under neighbor pruning (eq. (2.5) with the exact kappa nearest
 * neighbors, kappa <= 256) into visited_knn_dev [N] and under distance
 * pruning (a node is pruned when ||x - c|| > rscale R, c its centroid and R
 * the largest distance from c to its points; rscale = 1 as printed) into
 * visited_dist_dev [N] (int64, caller order).  The tree has 2^(L+1) - 1
 * nodes, L the least depth whose nodes hold at most leaf_size points.
 * Decisions in canonical FP64 (reproducible).  N <= 2^22, d <= 4096.
 * Allocates its own scratch; blocks until done.
 */
askit_status askit_prune_stats(const float *X_dev, int64_t N, int32_t d, int64_t ldx, int32_t leaf_size,
                               int32_t kappa, double rscale, int64_t *visited_knn_dev,
                               int64_t *visited_dist_dev, void *stream);

/*
 * Direct sum of eq. (1.1) at selected points, without approximation: for
 * each target id, the sum over all N points of K(x_i, x_j) w_j with the
 * tree's points, bandwidths and current weights (plain FP32, difference
 * form).  The yardstick of ASKIT's error (Section 4 measures the relative
 * error against direct evaluation on sampled points).
 *   tgt_dev [T] int32 point ids (caller order); U_dev [T, r] (stride ldu).
 * Cost O(T N d); requires askit_set_weights first.
 */
askit_status askit_direct(askit_tree t, const int32_t *tgt_dev, int64_t T, float *U_dev, int64_t ldu,
                          void *stream);

/*
 * Weight contexts.  askit_set_weights/askit_evaluate use the tree's default
 * weights; a context holds its own weight vectors, skeleton weights (the
 * upward pass of Section 2.1) and Evaluate scratch, so that several weight
 * sets can be evaluated concurrently on different streams while the tree
 * structures are shared read-only (a serving loop batching requests).  A
 * context is tied to its tree and must be destroyed before it.  Calls on one
 * context must not overlap on the GPU.
 */
typedef struct askit_weights_s *askit_weights;
askit_status askit_weights_create(askit_tree t, askit_weights *out);
/* upward pass for W_dev [N, r] (stride ldw, caller order), 1 <= r <= 64 */
askit_status askit_weights_set(askit_weights w, const float *W_dev, int32_t r, int64_t ldw, void *stream);
/* Evaluate at every point with the context's weights: U_dev [N, r] */
askit_status askit_weights_evaluate(askit_weights w, float *U_dev, int64_t ldu, void *stream);
/* Evaluate at out-of-sample targets Y_dev [T, d] with the context's weights */
askit_status askit_weights_evaluate_targets(askit_weights w, const float *Y_dev, int64_t T, int64_t ldy,
                                            float *U_dev, int64_t ldu, void *stream);
askit_status askit_weights_destroy(askit_weights w);

/*
 * A captured evaluation step.  askit_graph_create records, as one CUDA graph,
 * the upward pass of skeleton weights for W_dev (Section 2.1, Algorithm 3)
 * followed by Evaluate at every point (Algorithm 4) into U_dev; each
 * askit_graph_launch replays it with a single launch on `stream`.
 *   W_dev [N, r] (stride ldw, caller order, 1 <= r <= 64) and U_dev [N, r]
 *   (stride ldu) are caller-owned and bound at creation: every replay reads
 *   the current contents of W_dev and overwrites U_dev.  Both must stay
 *   allocated while the graph exists.
 * The graph owns a weight context of its own (the tree's default weights are
 * not touched) and uses the tree's precision at creation time.  Creation runs
 * one step uncaptured on `stream` (allocations and operand preparation happen
 * there), waits for it, then captures a second step on a private stream in
 * thread-local capture mode; it must not be called while `stream` is itself
 * being captured.
 * Replays of one graph must not overlap on the GPU.  Destroy the graph before
 * its tree.
 */
typedef struct askit_graph_s *askit_graph;
askit_status askit_graph_create(askit_tree t, const float *W_dev, int32_t r, int64_t ldw, float *U_dev,
                                int64_t ldu, void *stream, askit_graph *out);
askit_status askit_graph_launch(askit_graph g, void *stream);
askit_status askit_graph_destroy(askit_graph g);

/*
 * Autotuner of the evaluation kernels' launch configuration.  Times every
 * candidate configuration of the persistent Evaluate kernel for the tree's
 * current precision on its own work lists and default weights (set them
 * first), keeps the fastest for later evaluations of this tree, and reports
 * each candidate.  Candidates:
 *   schedule    0: sub-blocks dealt heaviest first to the least-loaded CTA;
 *               1: sub-blocks taken in tree order, each to the least-loaded
 *                  CTA (the CTAs advance through the tree together, so the
 *                  sub-blocks in flight share targets: L2 reuse);
 *   stages      target-row stages of the FP16x3 kernels (per sub-block
 *               centering: 2 or 3, 2 with paired items; global centering:
 *               3 or 4);
 *   tiled_runs  1: runs of 8 consecutive target rows arrive in one tiled
 *               copy (per-sub-block FP16x3 kernel), 0: every row by
 *               tile::gather4;
 *   pairs       1: the FP16x3 kernels take sub-blocks 2k and 2k+1 of a node
 *               (same targets) in one 256-column item (schedule 2: the
 *               leaders dealt longest first), r <= 4; so does the K-chunked
 *               kernel for d > 64 (FP16x3 and BF16x3, any r <= 16), which
 *               then copies and splits each target row once for both.
 * Only the schedule (and, for d > 64, pairs) varies for the other tensor-core
 * kernels; the plain FP32 kernel has one configuration.  Schedules, stages and tiled runs change no
 * result bit (every work item is computed the same way; partials are reduced
 * in a fixed order); paired items sum both sub-blocks' columns in one
 * accumulator, which changes the FP32 summation order only.  `reps` timed evaluations per candidate after one warm-up; at most
 * `max_out` entries are written to `out`, the count to `n_out`.  Blocks.
 */
typedef struct {
    int32_t schedule, stages, tiled_runs, pairs, chosen;
    double ms;   /* mean Evaluate time of the candidate */
} askit_tune_entry;
askit_status askit_autotune(askit_tree t, int32_t reps, void *stream, askit_tune_entry *out, int32_t max_out,
                            int32_t *n_out);
/* Set the launch configuration directly (schedule 0|1, stages 2..4,
 * tiled_runs 0|1, pairs 0|1; pairs uses its own schedule; each kernel takes
 * the nearest stage count it has).  Host call; applies to later evaluations
 * of the tree. */
askit_status askit_set_launch(askit_tree t, int32_t schedule, int32_t stages, int32_t tiled_runs, int32_t pairs);

/*
 * Device time of the evaluation kernel itself (Algorithm 4's work: the
 * persistent kernel of the tree's precision, without the per-Evaluate column
 * setup and the partial-sum reduction).  enable = 1 starts a timing session:
 * every later launch of that kernel for this tree (askit_evaluate,
 * askit_evaluate_targets, the weight-context calls; one launch per target
 * batch) is bracketed by CUDA events on its own stream; launches captured
 * into a graph are not timed.  enable = 0 ends the session, waits for the
 * recorded events and returns the summed kernel time in `ms` and the number
 * of timed launches in `launches` (both required then).  Host call.
 */
askit_status askit_kernel_timing(askit_tree t, int32_t enable, double *ms, int64_t *launches);

/*
 * Device bytes a request needs, for admission by memory footprint.
 *   kind 0: a weight context for r vectors (n ignored);
 *   kind 1: an out-of-sample batch of n targets with r weight vectors
 *           (work lists estimated from the in-sample entries per target, x2).
 */
askit_status askit_footprint(askit_tree t, int32_t kind, int64_t n, int32_t r, size_t *bytes);

/*
 * Refinements of the pruning that Section 3 proposes against the error's
 * growth with the node size (after eq. (3.5)); both rebuild the tree's
 * in-sample work lists:
 *   far_height >= 0: level restriction -- skeletons are used only for nodes
 *     at most far_height levels above the leaves; a higher node that eq. (2.5)
 *     prunes is replaced by its descendants at that height (-1: off).
 *   kappa_cut > 0: adaptive kappa_i -- the prune set of point i keeps its
 *     neighbors up to the last rank z whose kernel value exceeds e^-kappa_cut,
 *     kappa_i = 1 + max{z : c D(i, N_i[z]) / h^2 < kappa_cut} (0 if none),
 *     decided in FP64; out-of-sample targets likewise (0: all kappa).
 * Blocks until the lists are rebuilt (waits for the device first).  Skeleton
 * weights do not depend on the lists and stay valid; a weight context (the
 * tree's own included) whose partial-sum buffer is smaller than the new
 * lists returns NOT_READY from its evaluations until its weights are set
 * again.  Graphs captured before must be destroyed.
 */
askit_status askit_set_pruning(askit_tree t, int32_t far_height, double kappa_cut, void *stream);

/* Precision of subsequent askit_evaluate calls (ASKIT_PREC_*). */
askit_status askit_set_precision(askit_tree t, int32_t precision);

/*
 * Target centering of the FP16x3 kernels for d <= 64 (an implementation
 * choice below the paper's level; the result changes only within rounding):
 *   0 automatic (default): mode 2 while askit_info.fp16_rho <= 512, else 1;
 *   1 every item's target rows are centered on the source sub-block's mean
 *     and split on the chip (the smallest rounding error);
 *   2 every point is centered once on the data mean and pre-split in HBM, so
 *     target rows reach the tensor cores without conversion (the fastest;
 *     relative error of u about 1e-5 against about 1e-6 for mode 1, both
 *     within the split-product tolerance 1e-4).
 * Out-of-sample batches with a target outside the FP16-safe range of mode 2
 * (beyond about 7 times the data's extent from its mean) take mode 1.
 * Host call; applies to later evaluations.
 */
askit_status askit_set_fp16_centering(askit_tree t, int32_t mode);

/* Sizes and work counts (host call). */
typedef struct {
    int64_t N;
    int32_t d, d_pad, L, kappa, r;
    int64_t n_nodes;          /* heap slots, 2^(L+1) */
    int64_t skel_total;       /* sum of skeleton sizes over non-root nodes */
    int64_t skel_rows_padded; /* rows of the skeleton coordinate pool */
    int64_t n_blocks;         /* source sub-blocks (<= 128 rows of a leaf or a skeleton) */
    int64_t n_items;          /* work items: a sub-block against <= 128 targets needing it */
    int64_t n_entries;        /* (target, sub-block) pairs */
    int64_t pairs_algorithmic;/* sum over targets of near + far source points */
    int64_t pairs_computed;   /* 128 x 128 target-source slots the items cover */
    int64_t near_total, far_total; /* sum over targets of |Near(i)| and |Far(i)| */
    int64_t device_bytes;     /* library-owned device memory */
    int64_t n_batches;        /* in-sample target batches (askit_params.batch_entries) */
    double setup_ms[7];       /* askit_setup's wall time by stage: kNN, tree, node lists
                                 (Algorithm 2), sampled rows (eq. 2.4), skeletons and
                                 interpolation matrices (Algorithm 3), evaluation
                                 operands, work lists */
    int32_t fp16_centering;   /* FP16x3 kernel askit_evaluate takes (d <= 64): 1 targets
                                 centered per source sub-block on the chip, 2 all points
                                 pre-split around the data mean (askit_set_fp16_centering) */
    int32_t pad_;
    double fp16_rho;          /* max_j sc_j * max_i |x_i - mean|^2, sc = c log2(e) / h_j^2:
                                 the global form's exponent error is a few 2^-24 rho; the
                                 automatic choice takes it while rho <= 512 */
} askit_info;
askit_status askit_get_info(askit_tree t, askit_info *info);

/* Structures for inspection and bit-exact checks (host call, blocks).
 * `which` and the host buffer's layout:
 *   ASKIT_STRUCT_PERM      int32 [N]          leaf order -> point id
 *   ASKIT_STRUCT_KNN       int32 [N, kappa]   neighbor ids, sorted by (D, id)
 *   ASKIT_STRUCT_KNN_DIST  double [N, kappa]  FP64 squared distances
 *   ASKIT_STRUCT_SKEL_S    int32 [n_nodes]    skeleton size per heap node
 *   ASKIT_STRUCT_SKEL_IDS  int32 [skel_total] skeleton point ids, nodes in heap order
 *   ASKIT_STRUCT_NL_CNT    int32 [n_nodes]    node neighbor-list length
 *   ASKIT_STRUCT_NL_IDS    int32 [n_nodes, ell_max] node neighbor lists (padded with -1)
 *   ASKIT_STRUCT_TROWS     int32 [n_nodes, ell_max] sampled target rows (padded with -1)
 *   ASKIT_STRUCT_HSRC      float [N]          bandwidth of each point
 *   ASKIT_STRUCT_P         double [sum s (c - s)] interpolation matrices, heap order
 *   ASKIT_STRUCT_NCOL      int32 [n_nodes]    columns c of each node's ID
 *   ASKIT_STRUCT_WSKEL     float [skel_total, r] skeleton weights, heap order
 * `bytes` must equal the buffer's size; INVALID_ARG otherwise. */
enum {
    ASKIT_STRUCT_PERM = 0, ASKIT_STRUCT_KNN = 1, ASKIT_STRUCT_KNN_DIST = 2,
    ASKIT_STRUCT_SKEL_S = 3, ASKIT_STRUCT_SKEL_IDS = 4, ASKIT_STRUCT_NL_CNT = 5,
    ASKIT_STRUCT_NL_IDS = 6, ASKIT_STRUCT_TROWS = 7, ASKIT_STRUCT_HSRC = 8,
    ASKIT_STRUCT_P = 9, ASKIT_STRUCT_NCOL = 10, ASKIT_STRUCT_WSKEL = 11
};
askit_status askit_get_structure(askit_tree t, int32_t which, void *host, size_t bytes);

/* Waits for the tree's work on `stream` and reports sticky kernel errors
 * (TIMEOUT: a kernel gave up a bounded wait and its results are invalid).  A
 * reported status is cleared, so the tree serves later calls. */
askit_status askit_sync(askit_tree t, void *stream);

/*
 * Poll limit of the bounded mbarrier waits in the FP16x3 evaluation kernel
 * (every wait of a producer/consumer role; each poll is one try_wait, which
 * suspends the thread for a short time before giving up).  0 restores the
 * default of 2^24 polls, far beyond any legitimate wait.  A small limit makes
 * the waits give up: the kernel then records a sticky timeout (askit_sync
 * returns TIMEOUT), every role leaves its loop, the copies and MMAs in
 * flight are waited for, TMEM is freed and the kernel returns, so the
 * context stays usable.  A debugging and test aid (no counterpart in the
 * paper).  Host call; applies to later evaluations of the tree.
 */
askit_status askit_set_wait_limit(askit_tree t, int32_t polls);

/* Frees the tree and everything it owns (waits for its work first). */
askit_status askit_destroy(askit_tree t);

const char *askit_status_string(askit_status s);
const char *askit_last_error(void);

/*
 * Exact kNN without allocating device memory.  The paper has no counterpart:
 * this is a library service for callers that cannot call cudaMalloc -- for
 * instance a serving process that reserves its device memory once, up front,
 * for the resident tree and its request buffers and must not grow afterwards,
 * or a latency-critical caller that cannot afford cudaMalloc's implicit
 * device synchronization.
 *
 * Same result as the exact kNN of askit_setup (knn_mode 0): for each query
 * the kappa smallest (D, id) over the N points, D the FP64 squared distance
 * summed in coordinate order, ties by the smaller id.
 *   X_dev   [N, d] FP32 points, rows contiguous (stride d).
 *   Y_dev   [Q, d] FP32 queries (stride d), or NULL: the queries are the N
 *           points themselves (Q must equal N) and each excludes itself.
 *   ids_dev [Q, kappa] int32 and dist_dev [Q, kappa] double receive the
 *           neighbors, nearest first.  All buffers are caller-owned.
 * Limits: Q <= 8192 per call (INVALID_ARG beyond), 1 <= kappa <= 32,
 * d <= 1536, N < 2^31 - 1024 (ids are int32; UNSUPPORTED beyond).  Scratch: a fixed 3 MiB device array inside the library,
 * resident on every GPU that loads it until the process exits.  The first
 * call on a device looks up that array's device address (so make the first
 * call before any stream capture); every call shares the array, so calls
 * that overlap on the GPU race and must be serialized by the caller.
 * Enqueues on `stream` and returns without waiting.
 */
askit_status askit_knn_noalloc(const float *X_dev, int64_t N, int32_t d, const float *Y_dev, int64_t Q,
                               int32_t kappa, int32_t *ids_dev, double *dist_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* ASKIT_H */
