// C ABI of the GB300 ASKIT library: validation, the setup pipeline of
// Algorithm 5 (kNN, tree, node lists, samples, skeletons, work lists), the
// per-weight-vector upward pass and Evaluate, and structure export.
#include <float.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <string>

#include "askit_impl.cuh"

static thread_local std::string g_err;

void askit_set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

askit_status evaluate_targets_ctx(askit_tree t, const WeightCtx &c, const float *Y_dev, int64_t T, int64_t ldy,
                                  float *U_dev, int64_t ldu, cudaStream_t s);

namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__global__ void fill_f32(float *a, int64_t n, float v) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < n) a[q] = v;
}

__global__ void h_from_knn(const double *knnd, int64_t N, int kappa, int k, float *h) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < N) h[j] = (float)__dsqrt_rn(knnd[j * kappa + (k - 1)]);
}

__global__ void leafof_kernel(const int32_t *perm, const int32_t *nstart, const int32_t *nsize,
                              int64_t a0, int32_t *leafof) {
    int64_t a = a0 + blockIdx.x;
    for (int q = threadIdx.x; q < nsize[a]; q += blockDim.x) leafof[perm[nstart[a] + q]] = (int32_t)a;
}

// Caller-given neighbor ids must lie in [0, N) and exclude the point itself.
__global__ void check_knn_kernel(const int32_t *knn, int64_t N, int kappa, int *bad) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * kappa) return;
    int32_t j = knn[e];
    if (j < 0 || j >= N || j == e / kappa) atomicExch(bad, 1);
}

__global__ void pos_kernel(const int32_t *perm, int64_t N, int32_t *pos) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < N) pos[perm[q]] = (int32_t)q;
}

// Order out-of-sample queries by the tree position of their nearest source
// (so a tile's targets share near and far blocks): key (pos << 32) | q.
__global__ void oos_keys_kernel(const int32_t *knn, int kappa, const int32_t *pos, int64_t T,
                                uint64_t *keys, int32_t *vals) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= T) return;
    keys[q] = ((uint64_t)pos[knn[q * kappa]] << 32) | (uint64_t)q;
    vals[q] = (int32_t)q;
}

template <class V>
__global__ void gather_knn_kernel(const V *knn, int kappa, const int32_t *order, int64_t T, V *out) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= T * kappa) return;
    int64_t q = e / kappa;
    out[e] = knn[(int64_t)order[q] * kappa + (e % kappa)];
}

__global__ void gather_y_kernel(const float *Y, int64_t ldy, int d, int d_pad, const int32_t *order,
                                int64_t T, int64_t T_pad, float *out, float *nrm) {
    int64_t row = blockIdx.x;
    if (row >= T_pad) return;
    int64_t q = row < T ? order[row] : -1;
    for (int k = threadIdx.x; k < d_pad; k += blockDim.x)
        out[row * d_pad + k] = (q >= 0 && k < d) ? Y[q * ldy + k] : 0.f;
    if (threadIdx.x == 0) {
        double acc = 0.0;
        if (q >= 0)
            for (int k = 0; k < d; ++k) acc += (double)Y[q * ldy + k] * Y[q * ldy + k];
        nrm[row] = (float)acc;
    }
}

// Rows X[ids[q]] of the caller-order points; an id out of range sets *bad
// and gives a zero row.
__global__ void gather_points_kernel(const float *X, int64_t N, int d, const int32_t *ids, int64_t Q, float *Y,
                                     int32_t *bad) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= Q * d) return;
    const int64_t q = e / d;
    const int32_t i = ids[q];
    const bool ok = i >= 0 && i < N;
    if (!ok && e % d == 0) *bad = 1;
    Y[e] = ok ? X[(int64_t)i * d + e % d] : 0.f;
}

std::mutex g_kt_mu;

askit_status validate(const askit_params *p, int64_t N, int32_t d, int64_t ldx, const float *h_dev) {
    if (!p) { askit_set_error("params is NULL"); return ASKIT_ERR_INVALID_ARG; }
    if (N < 1 || d < 1 || ldx < d) { askit_set_error("need N >= 1, d >= 1, ldx >= d"); return ASKIT_ERR_INVALID_ARG; }
    if (N >= ((int64_t)1 << 31) - 1024) { askit_set_error("N must be below 2^31"); return ASKIT_ERR_UNSUPPORTED; }
    if (p->leaf_size < 2) { askit_set_error("leaf_size must be >= 2"); return ASKIT_ERR_INVALID_ARG; }
    if (p->kappa < 1 || p->kappa > 32 || p->kappa > N - 1) {
        askit_set_error("kappa must be in 1..min(32, N-1)");
        return ASKIT_ERR_INVALID_ARG;
    }
    if (p->s_max < 1 || p->s_min < 0 || p->ell_extra < 0) { askit_set_error("need s_max >= 1, s_min >= 0, ell_extra >= 0"); return ASKIT_ERR_INVALID_ARG; }
    // a source block (a leaf's points or a skeleton) is cut into at most 16
    // sub-blocks of ASK_BLK_N rows (the work lists keep the sub-block index in
    // 4 bits), and a node's heap index must fit the lists' 27-bit node field
    if (p->leaf_size > 16 * ASK_BLK_N || p->s_max > 16 * ASK_BLK_N) {
        askit_set_error("leaf_size and s_max must be at most %d", 16 * ASK_BLK_N);
        return ASKIT_ERR_UNSUPPORTED;
    }
    if (tree_depth(N, p->leaf_size) > 25) {
        askit_set_error("the tree would have more than 2^25 leaves; raise leaf_size");
        return ASKIT_ERR_UNSUPPORTED;
    }
    if (!(p->id_tol >= 0.0) || !(p->kernel_scale > 0.0)) { askit_set_error("need id_tol >= 0 and kernel_scale > 0"); return ASKIT_ERR_INVALID_ARG; }
    if (p->bw_mode == ASKIT_BW_CONSTANT && !(p->h > 0.0)) { askit_set_error("h must be > 0"); return ASKIT_ERR_INVALID_ARG; }
    if (p->bw_mode == ASKIT_BW_ARRAY && !h_dev) { askit_set_error("ASKIT_BW_ARRAY needs h_dev"); return ASKIT_ERR_INVALID_ARG; }
    if (p->bw_mode == ASKIT_BW_KNN && (p->bw_k < 1 || p->bw_k > p->kappa)) { askit_set_error("bw_k must be in 1..kappa"); return ASKIT_ERR_INVALID_ARG; }
    if (p->bw_mode < 0 || p->bw_mode > 2) { askit_set_error("bad bw_mode"); return ASKIT_ERR_INVALID_ARG; }
    if (p->knn_mode < 0 || p->knn_mode > 1) { askit_set_error("bad knn_mode"); return ASKIT_ERR_INVALID_ARG; }
    if (p->knn_mode == 1 && p->rp_iters < 1) { askit_set_error("rp_iters must be >= 1"); return ASKIT_ERR_INVALID_ARG; }
    if (p->precision < 0 || p->precision > 3) { askit_set_error("bad precision"); return ASKIT_ERR_INVALID_ARG; }
    if (p->prune < 0 || p->prune > 2) { askit_set_error("prune must be 0, 1 or 2"); return ASKIT_ERR_INVALID_ARG; }
    if (p->batch_entries != 0 && (p->batch_entries < 4096 || p->batch_entries > ASK_BATCH_ENTRIES_MAX)) {
        askit_set_error("batch_entries must be 0 or in 4096..2^30");
        return ASKIT_ERR_INVALID_ARG;
    }
    return ASKIT_OK;
}

// Wall time of setup stage k (host clock, the stream drained at each mark).
askit_status stage_mark(askit_tree t, int k, cudaStream_t s) {
    ASK_CUDA(cudaStreamSynchronize(s));
    const auto now = std::chrono::steady_clock::now();
    t->setup_ms[k] = std::chrono::duration<double, std::milli>(now - t->stage_t0).count();
    t->stage_t0 = now;
    return ASKIT_OK;
}

askit_status setup_impl(askit_tree t, const float *X_dev, int64_t ldx, const float *h_dev,
                        const int32_t *knn_dev, cudaStream_t s) {
    t->stage_t0 = std::chrono::steady_clock::now();
    const int64_t N = t->N;
    const int d = t->d, kappa = t->kappa;
    ASK_TRY(t->arena.alloc(&t->X, (size_t)N * d));
    ASK_CUDA(cudaMemcpy2DAsync(t->X, sizeof(float) * d, X_dev, sizeof(float) * ldx, sizeof(float) * d, N,
                               cudaMemcpyDeviceToDevice, s));
    // nearest neighbors (Section 2.2)
    ASK_TRY(t->arena.alloc(&t->knn, (size_t)N * kappa));
    ASK_TRY(t->arena.alloc(&t->knnd, (size_t)N * kappa));
    if (knn_dev) {
        ASK_CUDA(cudaMemcpyAsync(t->knn, knn_dev, sizeof(int32_t) * N * kappa, cudaMemcpyDeviceToDevice, s));
        int *bad = nullptr, hbad = 0;
        ASK_TRY(t->arena.alloc(&bad, 1));
        ASK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
        check_knn_kernel<<<nblk(N * kappa, 256), 256, 0, s>>>(t->knn, N, kappa, bad);
        ASK_LAUNCH();
        ASK_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        ASK_CUDA(cudaStreamSynchronize(s));
        t->arena.release(bad);
        if (hbad) { askit_set_error("knn_dev holds an id outside [0, N) or the point itself"); return ASKIT_ERR_INVALID_ARG; }
        ASK_TRY(knn_dist_gpu(t->X, N, d, kappa, t->knn, t->knnd, s));
    } else if (t->prm.knn_mode == 0) {
        ASK_TRY(knn_exact_gpu(t->X, N, d, kappa, nullptr, N, t->knn, t->knnd, s));
    } else {
        ASK_TRY(knn_rp_gpu(t->X, N, d, kappa, t->prm.rp_iters, t->rp_leaf, t->prm.seed, t->knn, t->knnd, s));
    }
    ASK_TRY(stage_mark(t, 0, s));
    // bandwidth of every source point (Section 4)
    ASK_TRY(t->arena.alloc(&t->hsrc, N));
    if (t->prm.bw_mode == ASKIT_BW_CONSTANT) {
        fill_f32<<<nblk(N, 256), 256, 0, s>>>(t->hsrc, N, (float)t->prm.h);
    } else if (t->prm.bw_mode == ASKIT_BW_ARRAY) {
        ASK_CUDA(cudaMemcpyAsync(t->hsrc, h_dev, sizeof(float) * N, cudaMemcpyDeviceToDevice, s));
    } else {
        h_from_knn<<<nblk(N, 256), 256, 0, s>>>(t->knnd, N, kappa, t->prm.bw_k, t->hsrc);
    }
    ASK_LAUNCH();
    // the ASKIT tree (Section 2.2)
    t->L = tree_depth(N, t->prm.leaf_size);
    t->n_nodes = (int64_t)2 << t->L;
    tree_ranges(N, t->L, t->h_start, t->h_size);
    ASK_TRY(t->arena.alloc(&t->perm, N));
    ASK_TRY(t->arena.alloc(&t->pos, N));
    ASK_TRY(t->arena.alloc(&t->leafof, N));
    ASK_TRY(build_tree_gpu(t->X, N, d, t->L, 0, 0, 0, t->perm, s));
    {
        std::vector<int32_t> hs(t->n_nodes), hz(t->n_nodes);
        for (int64_t a = 0; a < t->n_nodes; ++a) { hs[a] = (int32_t)t->h_start[a]; hz[a] = (int32_t)t->h_size[a]; }
        ASK_TRY(t->arena.alloc(&t->nstart, t->n_nodes));
        ASK_TRY(t->arena.alloc(&t->nsize, t->n_nodes));
        ASK_CUDA(cudaMemcpyAsync(t->nstart, hs.data(), sizeof(int32_t) * t->n_nodes, cudaMemcpyHostToDevice, s));
        ASK_CUDA(cudaMemcpyAsync(t->nsize, hz.data(), sizeof(int32_t) * t->n_nodes, cudaMemcpyHostToDevice, s));
        int64_t a0 = (int64_t)1 << t->L;
        leafof_kernel<<<(unsigned)a0, 128, 0, s>>>(t->perm, t->nstart, t->nsize, a0, t->leafof);
        pos_kernel<<<nblk(N, 256), 256, 0, s>>>(t->perm, N, t->pos);
        ASK_LAUNCH();
        ASK_CUDA(cudaStreamSynchronize(s));
    }
    ASK_TRY(stage_mark(t, 1, s));
    // node neighbor lists, sampled targets, skeletons (Algorithms 2, 3)
    const int64_t nn = t->n_nodes;
    t->ell_max = t->prm.s_max + t->prm.ell_extra;
    ASK_TRY(t->arena.alloc(&t->nl_cnt, nn));
    ASK_TRY(t->arena.alloc(&t->nl_ids, (size_t)nn * t->ell_max));
    ASK_TRY(t->arena.alloc(&t->nl_key, (size_t)nn * t->ell_max));
    ASK_TRY(t->arena.alloc(&t->trows, (size_t)nn * t->ell_max));
    ASK_TRY(t->arena.alloc(&t->d_s, nn));
    ASK_TRY(t->arena.alloc(&t->d_ncol, nn));
    ASK_CUDA(cudaMemsetAsync(t->nl_cnt, 0, sizeof(int32_t) * nn, s));
    ASK_CUDA(cudaMemsetAsync(t->nl_ids, 0xff, sizeof(int32_t) * nn * t->ell_max, s));
    ASK_CUDA(cudaMemsetAsync(t->trows, 0xff, sizeof(int32_t) * nn * t->ell_max, s));
    ASK_CUDA(cudaMemsetAsync(t->d_ncol, 0, sizeof(int32_t) * nn, s));
    ASK_TRY(build_node_lists(t, s));
    ASK_TRY(stage_mark(t, 2, s));
    ASK_TRY(build_samples(t, s));
    ASK_TRY(stage_mark(t, 3, s));
    ASK_TRY(skeletonize(t, s));
    ASK_TRY(stage_mark(t, 4, s));
    if (t->L == 0) {
        // a single leaf: no skeletons, empty pools
        t->h_skoff.assign(nn + 1, 0); t->h_pivoff.assign(nn + 1, 0);
        t->h_poff.assign(nn + 1, 0); t->h_spool.assign(nn + 1, 0);
        ASK_TRY(t->arena.alloc(&t->skel_ids, 1)); ASK_TRY(t->arena.alloc(&t->piv, 1));
        ASK_TRY(t->arena.alloc(&t->P64, 1)); ASK_TRY(t->arena.alloc(&t->P32, 1));
        ASK_TRY(t->arena.alloc(&t->d_poff, nn + 1)); ASK_TRY(t->arena.alloc(&t->d_skoff, nn + 1));
        ASK_TRY(t->arena.alloc(&t->d_pivoff, nn + 1)); ASK_TRY(t->arena.alloc(&t->d_spool, nn + 1));
        ASK_CUDA(cudaMemsetAsync(t->d_poff, 0, sizeof(int64_t) * (nn + 1), s));
        ASK_CUDA(cudaMemsetAsync(t->d_skoff, 0, sizeof(int64_t) * (nn + 1), s));
        ASK_CUDA(cudaMemsetAsync(t->d_pivoff, 0, sizeof(int64_t) * (nn + 1), s));
        ASK_CUDA(cudaMemsetAsync(t->d_spool, 0, sizeof(int64_t) * (nn + 1), s));
        ASK_CUDA(cudaMemsetAsync(t->d_s, 0, sizeof(int32_t) * nn, s));
    }
    // evaluation operands and the in-sample work lists (eq. (2.5), Algorithm 4)
    ASK_TRY(build_eval_operands(t, s));
    ASK_TRY(build_tc_operands(t, s));
    ASK_TRY(stage_mark(t, 5, s));
    {
        PruneSets ps;
        askit_status rc = insample_prune_sets(t, ps, s);
        if (rc == ASKIT_OK) rc = build_insample_lists(t, ps, s);
        free_prune_sets(ps);
        ASK_TRY(rc);
    }
    ASK_TRY(stage_mark(t, 6, s));
    ASK_TRY(t->arena.alloc(&t->d_status, 4));
    ASK_TRY(t->arena.alloc(&t->d_ticket, 4));
    ASK_CUDA(cudaMemsetAsync(t->d_status, 0, sizeof(int) * 4, s));
    ASK_CUDA(cudaMemsetAsync(t->d_ticket, 0, sizeof(int) * 4, s));
    ASK_CUDA(cudaStreamSynchronize(s));
    return ASKIT_OK;
}

}  // namespace

askit_status ktimer_mark(askit_tree t, cudaStream_t s, bool end) {
    std::lock_guard<std::mutex> lock(g_kt_mu);
    if (!t->kt.on) return ASKIT_OK;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    ASK_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return ASKIT_OK;
    if (!end) {
        while (t->kt.ev.size() < t->kt.used + 2) {
            cudaEvent_t e = nullptr;
            ASK_CUDA(cudaEventCreate(&e));
            t->kt.ev.push_back(e);
        }
        ASK_CUDA(cudaEventRecord(t->kt.ev[t->kt.used], s));
    } else {
        ASK_CUDA(cudaEventRecord(t->kt.ev[t->kt.used + 1], s));
        t->kt.used += 2;
    }
    return ASKIT_OK;
}

namespace {

// Evaluate over one set of work lists: every (target, sub-block) entry's
// partial sum, then each target's entries summed in their fixed order.
// Partial sums of the items of the excluded field set to zero: part 1 keeps
// the near field (leaf blocks), part 2 the far field (skeleton blocks).
__global__ void keep_part_kernel(const EvalItem *items, int part, int r, float *partial) {
    const EvalItem it = items[blockIdx.x];
    const bool far = it.nrows < 0;
    if ((part == 1) != far) return;                      // kept
    for (int e = threadIdx.x; e < it.cnt * r; e += blockDim.x) partial[(int64_t)it.e0 * r + e] = 0.f;
}

askit_status run_eval(askit_tree t, const WeightCtx &c, int precision, const float *Xq, int64_t ldq,
                      int64_t q_rows, const QuerySplit *qs, const WorkLists &w, float *partial,
                      const int32_t *out_rows, float *U, int64_t ldu, cudaStream_t s, int part = 0) {
    if (precision == ASKIT_PREC_SIMT_FP32)
        ASK_TRY(eval_simt(t, c, Xq, ldq, w, partial, s));
    else
        ASK_TRY(eval_tc(t, c, precision, Xq, ldq, q_rows, qs, w, partial, s));
    if (part != 0 && w.n_items > 0) {
        keep_part_kernel<<<(unsigned)w.n_items, 128, 0, s>>>(w.items, part, c.r, partial);
        ASK_LAUNCH();
    }
    return reduce_partials(w, partial, c.r, out_rows, U, ldu, s);
}

askit_status set_weights_ctx(askit_tree t, WeightCtx &c, const float *W_dev, int32_t r, int64_t ldw,
                             cudaStream_t s) {
    if (!W_dev) { askit_set_error("W_dev must be non-NULL"); return ASKIT_ERR_INVALID_ARG; }
    if (r < 1 || r > 64 || ldw < r) { askit_set_error("need 1 <= r <= 64 and ldw >= r"); return ASKIT_ERR_INVALID_ARG; }
    return upward_weights(t, c, W_dev, r, ldw, s);
}

askit_status evaluate_ctx(askit_tree t, const WeightCtx &c, float *U_dev, int64_t ldu, cudaStream_t s,
                          int part = 0) {
    if (!U_dev) { askit_set_error("U_dev must be non-NULL"); return ASKIT_ERR_INVALID_ARG; }
    if (!c.ready) { askit_set_error("no weights set"); return ASKIT_ERR_NOT_READY; }
    if (ldu < c.r) { askit_set_error("ldu < r"); return ASKIT_ERR_INVALID_ARG; }
    if (c.ent_cap < t->wl_entries_max) {
        askit_set_error("the work lists grew (askit_set_pruning): set this context's weights again");
        return ASKIT_ERR_NOT_READY;
    }
    // batch b covers target slots [t0, t1): its target rows start at row t0
    // of Xt and its results go to the points perm[t0 .. t1)
    for (size_t b = 0; b < t->wl.size(); ++b) {
        const int64_t t0 = t->wl_t0[b];
        QuerySplit q;   // the same target rows in the global-centered FP16x3 form
        if (t->Xg_hi) {
            q.hi = t->Xg_hi + t0 * TC_K;
            q.lo = t->Xg_lo + t0 * TC_K;
            q.x = t->Xg_x + t0 * 16;
            q.rows = t->N_pad - t0;
        }
        ASK_TRY(run_eval(t, c, t->precision, t->Xt + t0 * t->d_pad, t->d_pad, t->N_pad - t0, t->Xg_hi ? &q : nullptr,
                         t->wl[b], c.partial, t->perm + t0, U_dev, ldu, s, part));
    }
    return ASKIT_OK;
}

}  // namespace

extern "C" {

void askit_default_params(askit_params *p) {
    if (!p) return;
    p->leaf_size = 128;
    p->kappa = 16;
    p->knn_mode = 0;
    p->rp_iters = 4;
    p->rp_leaf = 0;
    p->s_max = 64;
    p->s_min = 1;
    p->ell_extra = 20;
    p->prune = 1;
    p->bw_mode = ASKIT_BW_CONSTANT;
    p->bw_k = 16;
    p->precision = ASKIT_PREC_TF32X3;
    p->id_tol = 1e-6;
    p->kernel_scale = 0.5;
    p->h = 1.0;
    p->seed = 1;
    p->batch_entries = 0;
}

const char *askit_status_string(askit_status s) {
    switch (s) {
        case ASKIT_OK: return "ok";
        case ASKIT_ERR_INVALID_ARG: return "invalid argument";
        case ASKIT_ERR_OOM: return "out of device memory";
        case ASKIT_ERR_CUDA: return "CUDA error";
        case ASKIT_ERR_TIMEOUT: return "device wait timed out";
        case ASKIT_ERR_NOT_READY: return "not ready";
        case ASKIT_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *askit_last_error(void) { return g_err.c_str(); }

askit_status askit_setup(const float *X_dev, int64_t N, int32_t d, int64_t ldx, const float *h_dev,
                         const int32_t *knn_dev, const askit_params *p, void *stream, askit_tree *out) {
    if (!out || !X_dev) { askit_set_error("X_dev and out must be non-NULL"); return ASKIT_ERR_INVALID_ARG; }
    *out = nullptr;
    ASK_TRY(validate(p, N, d, ldx, h_dev));
    askit_tree t = new askit_tree_s();
    t->prm = *p;
    t->N = N;
    t->d = d;
    t->d_pad = (d + 31) / 32 * 32;
    t->kappa = p->kappa;
    t->rp_leaf = p->rp_leaf > 0 ? p->rp_leaf : std::max(2 * p->kappa + 2, p->leaf_size);
    if (t->prm.knn_mode == 1 && t->rp_leaf < 2 * p->kappa + 2) {
        delete t;
        askit_set_error("rp_leaf must be >= 2 kappa + 2");
        return ASKIT_ERR_INVALID_ARG;
    }
    t->precision = p->precision;
    if (!p->prune && (N << tree_depth(N, p->leaf_size)) > ((int64_t)1 << 28)) {
        delete t;
        askit_set_error("prune = 0 lists every leaf for every target; N x leaves must stay below 2^28");
        return ASKIT_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    askit_status rc = setup_impl(t, X_dev, ldx, h_dev, knn_dev, s);
    if (rc != ASKIT_OK) {
        cudaStreamSynchronize(s);
        eval_tc_free(t);
        t->arena.free_all();
        delete t;
        return rc;
    }
    *out = t;
    return ASKIT_OK;
}

askit_status askit_set_weights(askit_tree t, const float *W_dev, int32_t r, int64_t ldw, void *stream) {
    if (!t) { askit_set_error("tree is NULL"); return ASKIT_ERR_INVALID_ARG; }
    return set_weights_ctx(t, t->dw, W_dev, r, ldw, (cudaStream_t)stream);
}

askit_status askit_set_precision(askit_tree t, int32_t precision) {
    if (!t || precision < 0 || precision > 3) { askit_set_error("bad tree or precision"); return ASKIT_ERR_INVALID_ARG; }
    t->precision = precision;
    return ASKIT_OK;
}

askit_status askit_evaluate(askit_tree t, float *U_dev, int64_t ldu, void *stream) {
    if (!t) { askit_set_error("tree is NULL"); return ASKIT_ERR_INVALID_ARG; }
    return evaluate_ctx(t, t->dw, U_dev, ldu, (cudaStream_t)stream);
}

askit_status askit_evaluate_targets(askit_tree t, const float *Y_dev, int64_t T, int64_t ldy, float *U_dev,
                                    int64_t ldu, void *stream) {
    if (!t) { askit_set_error("tree is NULL"); return ASKIT_ERR_INVALID_ARG; }
    return evaluate_targets_ctx(t, t->dw, Y_dev, T, ldy, U_dev, ldu, (cudaStream_t)stream);
}

}  // extern "C"

askit_status evaluate_targets_ctx(askit_tree t, const WeightCtx &c, const float *Y_dev, int64_t T, int64_t ldy,
                                  float *U_dev, int64_t ldu, cudaStream_t s) {
    if (!Y_dev || !U_dev) { askit_set_error("Y_dev and U_dev must be non-NULL"); return ASKIT_ERR_INVALID_ARG; }
    if (!c.ready) { askit_set_error("no weights set"); return ASKIT_ERR_NOT_READY; }
    if (T < 1 || ldy < t->d || ldu < c.r) { askit_set_error("need T >= 1, ldy >= d, ldu >= r"); return ASKIT_ERR_INVALID_ARG; }
    const int kappa = t->kappa, d = t->d;
    // per-call temporaries are stream-ordered: releasing them does not
    // synchronize the device, so concurrent calls on other streams overlap
    DevArena tmp;
    tmp.async = true;
    tmp.stream = s;
    float *Yc = nullptr, *Yt = nullptr, *nrm = nullptr;
    int32_t *ids = nullptr, *ids_s = nullptr, *order = nullptr, *vals = nullptr, *sets = nullptr;
    double *dist = nullptr, *dist_s = nullptr;
    uint64_t *keys = nullptr, *keys_s = nullptr;
    void *cub = nullptr;
    size_t cb = 0;
    WorkLists w;
    float *partial = nullptr;
    uint16_t *yg_hi = nullptr, *yg_lo = nullptr, *yg_x = nullptr;
    int *yg_flag = nullptr;
    QuerySplit qs;
    int64_t T_pad = (T + ASK_TILE_M - 1) / ASK_TILE_M * ASK_TILE_M;
    askit_status rc = ASKIT_OK;
#define OTRY(x) do { rc = (x); if (rc != ASKIT_OK) goto out; } while (0)
    OTRY(tmp.alloc(&Yc, (size_t)T * d));
    if (cudaMemcpy2DAsync(Yc, sizeof(float) * d, Y_dev, sizeof(float) * ldy, sizeof(float) * d, T,
                          cudaMemcpyDeviceToDevice, s) != cudaSuccess) { askit_set_error("copy Y"); rc = ASKIT_ERR_CUDA; goto out; }
    OTRY(tmp.alloc(&ids, (size_t)T * kappa));
    OTRY(tmp.alloc(&dist, (size_t)T * kappa));
    OTRY(knn_oos(t, Yc, T, kappa, ids, dist, s));
    OTRY(tmp.alloc(&keys, T)); OTRY(tmp.alloc(&keys_s, T));
    OTRY(tmp.alloc(&vals, T)); OTRY(tmp.alloc(&order, T));
    oos_keys_kernel<<<nblk(T, 256), 256, 0, s>>>(ids, kappa, t->pos, T, keys, vals);
    OTRY(sort_u64_i32(nullptr, nullptr, nullptr, nullptr, T, nullptr, &cb, s));
    OTRY(tmp.alloc((char **)&cub, cb));
    OTRY(sort_u64_i32(keys, keys_s, vals, order, T, cub, &cb, s));
    OTRY(tmp.alloc(&ids_s, (size_t)T * kappa));
    OTRY(tmp.alloc(&dist_s, (size_t)T * kappa));
    gather_knn_kernel<<<nblk(T * kappa, 256), 256, 0, s>>>(ids, kappa, order, T, ids_s);
    gather_knn_kernel<<<nblk(T * kappa, 256), 256, 0, s>>>(dist, kappa, order, T, dist_s);
    OTRY(tmp.alloc(&Yt, (size_t)T_pad * t->d_pad));
    OTRY(tmp.alloc(&nrm, T_pad));
    gather_y_kernel<<<(unsigned)T_pad, 128, 0, s>>>(Yc, d, d, t->d_pad, order, T, T_pad, Yt, nrm);
    OTRY(tmp.alloc(&sets, (size_t)T * kappa));
    OTRY(oos_prune_sets(t, ids_s, dist_s, T, kappa, sets, s));
    OTRY(build_work_lists(t, sets, kappa, nullptr, T, w, tmp, s));
    OTRY(tmp.alloc(&partial, (size_t)w.n_entries * c.r));
    if (t->precision == ASKIT_PREC_FP16X3 && t->d <= TC_K && use_g16(t)) {
        // the targets in the global-centered FP16x3 form; a batch reaching
        // outside the FP16-safe range (far from the data) takes the
        // per-sub-block centered kernel instead
        OTRY(tmp.alloc(&yg_hi, (size_t)T_pad * TC_K));
        OTRY(tmp.alloc(&yg_lo, (size_t)T_pad * TC_K));
        OTRY(tmp.alloc(&yg_x, (size_t)T_pad * 16));
        OTRY(tmp.alloc(&yg_flag, 1));
        if (cudaMemsetAsync(yg_flag, 0, sizeof(int), s) != cudaSuccess) { askit_set_error("flag"); rc = ASKIT_ERR_CUDA; goto out; }
        OTRY(g16_split_rows(Yt, t->d_pad, d, T_pad, t, yg_hi, yg_lo, yg_x, yg_flag, s));
        int flag = 0;
        if (cudaMemcpyAsync(&flag, yg_flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { askit_set_error("range flag"); rc = ASKIT_ERR_CUDA; goto out; }
        if (!flag) {
            qs.hi = yg_hi;
            qs.lo = yg_lo;
            qs.x = yg_x;
            qs.rows = T_pad;
        }
    }
    OTRY(run_eval(t, c, t->precision, Yt, t->d_pad, T_pad, qs.hi ? &qs : nullptr, w, partial, order, U_dev, ldu, s));
    if (cudaStreamSynchronize(s) != cudaSuccess) { askit_set_error("out-of-sample evaluate: %s", cudaGetErrorString(cudaGetLastError())); rc = ASKIT_ERR_CUDA; }
out:
#undef OTRY
    tmp.free_all();
    cudaStreamSynchronize(s);
    return rc;
}

extern "C" {

askit_status askit_evaluate_host(askit_tree t, const float *W_host, int32_t r, int64_t ldw, float *U_host,
                                 int64_t ldu, void *stream) {
    if (!t || !W_host || !U_host) { askit_set_error("tree, W_host and U_host must be non-NULL"); return ASKIT_ERR_INVALID_ARG; }
    if (r < 1 || r > 64 || ldw < r || ldu < r) { askit_set_error("need 1 <= r <= 64, ldw >= r, ldu >= r"); return ASKIT_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    static thread_local DevArena io;
    static thread_local float *dW = nullptr, *dU = nullptr;
    static thread_local size_t cap = 0;
    size_t need = (size_t)t->N * r;
    if (need > cap) {
        io.free_all();
        ASK_TRY(io.alloc(&dW, need));
        ASK_TRY(io.alloc(&dU, need));
        cap = need;
    }
    ASK_CUDA(cudaMemcpy2DAsync(dW, sizeof(float) * r, W_host, sizeof(float) * ldw, sizeof(float) * r, t->N,
                               cudaMemcpyHostToDevice, s));
    ASK_TRY(askit_set_weights(t, dW, r, r, stream));
    ASK_TRY(askit_evaluate(t, dU, r, stream));
    ASK_CUDA(cudaMemcpy2DAsync(U_host, sizeof(float) * ldu, dU, sizeof(float) * r, sizeof(float) * r, t->N,
                               cudaMemcpyDeviceToHost, s));
    ASK_CUDA(cudaStreamSynchronize(s));
    return askit_sync(t, stream);
}

askit_status askit_get_info(askit_tree t, askit_info *info) {
    if (!t || !info) { askit_set_error("tree and info must be non-NULL"); return ASKIT_ERR_INVALID_ARG; }
    info->N = t->N;
    info->d = t->d;
    info->d_pad = t->d_pad;
    info->L = t->L;
    info->kappa = t->kappa;
    info->r = t->dw.r;
    info->n_nodes = t->n_nodes;
    info->skel_total = t->skel_total;
    info->skel_rows_padded = t->spool_rows;
    info->n_blocks = info->n_items = info->n_entries = 0;
    info->pairs_algorithmic = info->pairs_computed = info->near_total = info->far_total = 0;
    for (const WorkLists &w : t->wl) {
        info->n_blocks += w.n_blocks;
        info->n_items += w.n_items;
        info->n_entries += w.n_entries;
        info->pairs_algorithmic += w.pairs_alg;
        info->pairs_computed += w.pairs_cmp;
        info->near_total += w.near_tot;
        info->far_total += w.far_tot;
    }
    info->device_bytes = (int64_t)t->arena.bytes;
    info->n_batches = (int64_t)t->wl.size();
    info->fp16_centering = use_g16(t) ? 2 : 1;
    info->pad_ = 0;
    info->fp16_rho = t->g_rho;
    for (int k = 0; k < 7; ++k) info->setup_ms[k] = t->setup_ms[k];
    return ASKIT_OK;
}

askit_status askit_get_structure(askit_tree t, int32_t which, void *host, size_t bytes) {
    if (!t || !host) { askit_set_error("tree and host must be non-NULL"); return ASKIT_ERR_INVALID_ARG; }
    const int64_t N = t->N, nn = t->n_nodes;
    const void *src = nullptr;
    size_t want = 0;
    std::vector<int32_t> tmp;
    switch (which) {
        case ASKIT_STRUCT_PERM: src = t->perm; want = sizeof(int32_t) * N; break;
        case ASKIT_STRUCT_KNN: src = t->knn; want = sizeof(int32_t) * N * t->kappa; break;
        case ASKIT_STRUCT_KNN_DIST: src = t->knnd; want = sizeof(double) * N * t->kappa; break;
        case ASKIT_STRUCT_SKEL_S:
            tmp.assign(t->h_s.begin(), t->h_s.end());
            tmp.resize(nn, 0);
            want = sizeof(int32_t) * nn;
            if (bytes != want) break;
            memcpy(host, tmp.data(), want);
            return ASKIT_OK;
        case ASKIT_STRUCT_NCOL:
            tmp.assign(t->h_ncol.begin(), t->h_ncol.end());
            tmp.resize(nn, 0);
            want = sizeof(int32_t) * nn;
            if (bytes != want) break;
            memcpy(host, tmp.data(), want);
            return ASKIT_OK;
        case ASKIT_STRUCT_SKEL_IDS: src = t->skel_ids; want = sizeof(int32_t) * t->skel_total; break;
        case ASKIT_STRUCT_NL_CNT: src = t->nl_cnt; want = sizeof(int32_t) * nn; break;
        case ASKIT_STRUCT_NL_IDS: src = t->nl_ids; want = sizeof(int32_t) * nn * t->ell_max; break;
        case ASKIT_STRUCT_TROWS: src = t->trows; want = sizeof(int32_t) * nn * t->ell_max; break;
        case ASKIT_STRUCT_HSRC: src = t->hsrc; want = sizeof(float) * N; break;
        case ASKIT_STRUCT_P: src = t->P64; want = sizeof(double) * t->p_total; break;
        case ASKIT_STRUCT_WSKEL: {
            const WeightCtx &c = t->dw;
            if (!c.ready) { askit_set_error("no weights set"); return ASKIT_ERR_NOT_READY; }
            want = sizeof(float) * t->skel_total * c.r;
            if (bytes != want) break;
            float *h = (float *)host;
            for (int64_t a = 2; a < nn; ++a) {
                if (!t->h_s[a]) continue;
                ASK_CUDA(cudaMemcpy(h + t->h_skoff[a] * c.r, c.Ws + t->h_spool[a] * c.r,
                                    sizeof(float) * t->h_s[a] * c.r, cudaMemcpyDeviceToHost));
            }
            return ASKIT_OK;
        }
        default: askit_set_error("unknown structure %d", which); return ASKIT_ERR_INVALID_ARG;
    }
    if (bytes != want) {
        askit_set_error("structure %d needs %zu bytes, got %zu", which, want, bytes);
        return ASKIT_ERR_INVALID_ARG;
    }
    if (want) ASK_CUDA(cudaMemcpy(host, src, want, cudaMemcpyDeviceToHost));
    return ASKIT_OK;
}

askit_status askit_sync(askit_tree t, void *stream) {
    if (!t) { askit_set_error("tree is NULL"); return ASKIT_ERR_INVALID_ARG; }
    ASK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int st = 0;
    ASK_CUDA(cudaMemcpy(&st, t->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st == ASK_DEV_OK) return ASKIT_OK;
    // reported once: cleared so that the tree serves later calls
    ASK_CUDA(cudaMemset(t->d_status, 0, sizeof(int)));
    if (st == ASK_DEV_TIMEOUT) { askit_set_error("a kernel gave up a bounded wait"); return ASKIT_ERR_TIMEOUT; }
    askit_set_error("kernel status %d", st);
    return ASKIT_ERR_CUDA;
}

askit_status askit_kernel_timing(askit_tree t, int32_t enable, double *ms, int64_t *launches) {
    if (!t || (!enable && (!ms || !launches))) {
        askit_set_error("need a tree, and ms and launches to stop timing");
        return ASKIT_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_kt_mu);
    if (enable) {
        t->kt.on = true;
        t->kt.used = 0;
        return ASKIT_OK;
    }
    t->kt.on = false;
    double tot = 0.0;
    for (size_t k = 0; k + 1 < t->kt.used; k += 2) {
        ASK_CUDA(cudaEventSynchronize(t->kt.ev[k + 1]));
        float x = 0.f;
        ASK_CUDA(cudaEventElapsedTime(&x, t->kt.ev[k], t->kt.ev[k + 1]));
        tot += x;
    }
    *ms = tot;
    *launches = (int64_t)(t->kt.used / 2);
    t->kt.used = 0;
    return ASKIT_OK;
}

askit_status askit_destroy(askit_tree t) {
    if (!t) return ASKIT_OK;
    cudaDeviceSynchronize();
    for (cudaEvent_t e : t->kt.ev) cudaEventDestroy(e);
    eval_tc_free(t);
    t->dw.arena.free_all();
    t->arena.free_all();
    delete t;
    return ASKIT_OK;
}

askit_status askit_weights_create(askit_tree t, askit_weights *out) {
    if (!t || !out) { askit_set_error("tree and out must be non-NULL"); return ASKIT_ERR_INVALID_ARG; }
    askit_weights w = new askit_weights_s();
    w->t = t;
    *out = w;
    return ASKIT_OK;
}

askit_status askit_weights_set(askit_weights w, const float *W_dev, int32_t r, int64_t ldw, void *stream) {
    if (!w) { askit_set_error("weights handle is NULL"); return ASKIT_ERR_INVALID_ARG; }
    return set_weights_ctx(w->t, w->ctx, W_dev, r, ldw, (cudaStream_t)stream);
}

askit_status askit_weights_evaluate(askit_weights w, float *U_dev, int64_t ldu, void *stream) {
    if (!w) { askit_set_error("weights handle is NULL"); return ASKIT_ERR_INVALID_ARG; }
    return evaluate_ctx(w->t, w->ctx, U_dev, ldu, (cudaStream_t)stream);
}

askit_status askit_weights_evaluate_targets(askit_weights w, const float *Y_dev, int64_t T, int64_t ldy,
                                            float *U_dev, int64_t ldu, void *stream) {
    if (!w) { askit_set_error("weights handle is NULL"); return ASKIT_ERR_INVALID_ARG; }
    return evaluate_targets_ctx(w->t, w->ctx, Y_dev, T, ldy, U_dev, ldu, (cudaStream_t)stream);
}

askit_status askit_weights_destroy(askit_weights w) {
    if (!w) return ASKIT_OK;
    cudaDeviceSynchronize();
    w->ctx.arena.free_all();
    delete w;
    return ASKIT_OK;
}

askit_status askit_knn_targets(askit_tree t, const float *Y_dev, int64_t T, int64_t ldy, int32_t *ids_dev,
                               double *dist_dev, void *stream) {
    if (!t || !Y_dev || !ids_dev || !dist_dev || T < 1 || ldy < t->d) {
        askit_set_error("need a tree, T >= 1, ldy >= d and the three buffers");
        return ASKIT_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int d = t->d;
    float *Yc = nullptr;
    ASK_CUDA(cudaMallocAsync(&Yc, sizeof(float) * (size_t)T * d, s));
    askit_status rc = ASKIT_OK;
    if (cudaMemcpy2DAsync(Yc, sizeof(float) * d, Y_dev, sizeof(float) * ldy, sizeof(float) * d, T,
                          cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        askit_set_error("copy Y");
        rc = ASKIT_ERR_CUDA;
    }
    if (rc == ASKIT_OK) rc = knn_oos(t, Yc, T, t->kappa, ids_dev, dist_dev, s);
    cudaFreeAsync(Yc, s);
    cudaStreamSynchronize(s);
    return rc;
}

askit_status askit_knn_points(askit_tree t, const int32_t *ids_dev, int64_t Q, int32_t *nbr_dev, double *dist_dev,
                              void *stream) {
    if (!t || !ids_dev || !nbr_dev || !dist_dev || Q < 1) {
        askit_set_error("need a tree, Q >= 1 and the three buffers");
        return ASKIT_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int d = t->d;
    float *Y = nullptr;
    int32_t *bad = nullptr;
    ASK_CUDA(cudaMallocAsync(&Y, sizeof(float) * (size_t)Q * d, s));
    askit_status rc = ASKIT_OK;
    if (cudaMallocAsync(&bad, sizeof(int32_t), s) != cudaSuccess || cudaMemsetAsync(bad, 0, sizeof(int32_t), s) != cudaSuccess) {
        askit_set_error("allocation");
        rc = ASKIT_ERR_OOM;
    }
    if (rc == ASKIT_OK) {
        gather_points_kernel<<<nblk(Q * d, 256), 256, 0, s>>>(t->X, t->N, d, ids_dev, Q, Y, bad);
        int hbad = 0;
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            askit_set_error("gather points");
            rc = ASKIT_ERR_CUDA;
        } else if (hbad) {
            askit_set_error("a point id is outside 0 .. N-1");
            rc = ASKIT_ERR_INVALID_ARG;
        }
    }
    if (rc == ASKIT_OK) rc = knn_exact_gpu(t->X, t->N, d, t->kappa, Y, Q, nbr_dev, dist_dev, s, ids_dev);
    cudaFreeAsync(Y, s);
    if (bad) cudaFreeAsync(bad, s);
    cudaStreamSynchronize(s);
    return rc;
}

askit_status askit_evaluate_part(askit_tree t, int32_t part, float *U_dev, int64_t ldu, void *stream) {
    if (!t || part < 0 || part > 2) { askit_set_error("need a tree and part 0, 1 or 2"); return ASKIT_ERR_INVALID_ARG; }
    return evaluate_ctx(t, t->dw, U_dev, ldu, (cudaStream_t)stream, part);
}

askit_status askit_set_launch(askit_tree t, int32_t schedule, int32_t stages, int32_t tiled_runs, int32_t pairs) {
    if (!t || schedule < 0 || schedule > 1 || stages < 2 || stages > 4 || tiled_runs < 0 || tiled_runs > 1 ||
        pairs < 0 || pairs > 1) {
        askit_set_error("need schedule 0|1, stages 2..4, tiled_runs 0|1, pairs 0|1");
        return ASKIT_ERR_INVALID_ARG;
    }
    t->tune_sched = pairs ? 0 : schedule;
    t->tune_stages = stages;
    t->tune_runs = tiled_runs;
    t->tune_pairs = pairs;
    use_schedule(t);
    return ASKIT_OK;
}

askit_status askit_set_pruning(askit_tree t, int32_t far_height, double kappa_cut, void *stream) {
    if (!t || far_height < -1 || !(kappa_cut >= 0.0) || kappa_cut > 1e300) {
        askit_set_error("need a tree, far_height >= -1 and a finite kappa_cut >= 0");
        return ASKIT_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    ASK_CUDA(cudaStreamSynchronize(s));
    ASK_CUDA(cudaDeviceSynchronize());       // no evaluation may still read the old lists
    for (WorkLists &w : t->wl) free_work_lists(w, t->arena);
    t->far_height = far_height;
    t->kappa_cut = kappa_cut;
    PruneSets ps;
    askit_status rc = insample_prune_sets(t, ps, s);
    if (rc == ASKIT_OK) rc = build_insample_lists(t, ps, s);
    free_prune_sets(ps);
    ASK_TRY(rc);
    use_schedule(t);
    ASK_CUDA(cudaStreamSynchronize(s));
    return ASKIT_OK;
}

askit_status askit_set_fp16_centering(askit_tree t, int32_t mode) {
    if (!t || mode < 0 || mode > 2) { askit_set_error("need a tree and mode 0, 1 or 2"); return ASKIT_ERR_INVALID_ARG; }
    t->fp16_centering = mode;
    return ASKIT_OK;
}

askit_status askit_set_wait_limit(askit_tree t, int32_t polls) {
    if (!t || polls < 0) { askit_set_error("need a tree and polls >= 0"); return ASKIT_ERR_INVALID_ARG; }
    t->spin_limit = polls;
    return ASKIT_OK;
}

askit_status askit_autotune(askit_tree t, int32_t reps, void *stream, askit_tune_entry *out, int32_t max_out,
                            int32_t *n_out) {
    if (!t || !n_out || (max_out > 0 && !out) || reps < 1) {
        askit_set_error("need a tree, reps >= 1, n_out and room for the entries");
        return ASKIT_ERR_INVALID_ARG;
    }
    if (!t->dw.ready) { askit_set_error("set weights before autotuning"); return ASKIT_ERR_NOT_READY; }
    cudaStream_t s = (cudaStream_t)stream;
    struct Cand { int sched, stages, runs, pairs; double ms; };
    std::vector<Cand> cand;
    const bool tc = t->precision != ASKIT_PREC_SIMT_FP32;
    const bool fp16 = t->precision == ASKIT_PREC_FP16X3 && t->d <= TC_K;
    // the global-centered kernel has 3 or 4 target-row stages and copies its
    // rows without TMA (no tiled runs); the per-sub-block kernel 2 or 3 stages
    // (two with paired items) and tiled runs on or off
    const bool g16 = fp16 && use_g16(t);
    const int st_lo = fp16 ? (g16 ? 3 : 2) : t->tune_stages;
    const int st_hi = fp16 ? (g16 ? 4 : 3) : t->tune_stages;
    const int ru_lo = fp16 && !g16 ? 0 : t->tune_runs, ru_hi = fp16 && !g16 ? 1 : t->tune_runs;
    for (int sc = 0; sc < (tc ? 2 : 1); ++sc)
        for (int st = st_lo; st <= st_hi; ++st)
            for (int ru = ru_lo; ru <= ru_hi; ++ru)
                cand.push_back({sc, st, ru, 0, 0.0});
    // paired 256-column items (FP16x3, r <= 4): their own schedule
    int64_t n_pairs = 0;
    for (const WorkLists &w : t->wl) n_pairs += w.n_pairs;
    if (fp16 && t->dw.r <= 4 && n_pairs > 0)
        for (int st = g16 ? st_lo : 2; st <= (g16 ? st_hi : 2); ++st)
            for (int ru = ru_lo; ru <= ru_hi; ++ru) cand.push_back({2, st, ru, 1, 0.0});
    // the K-chunked kernel (d > TC_K, 16-bit splits) pairs at any r; its
    // stages and runs are fixed
    const bool wide = t->d > TC_K && (t->precision == ASKIT_PREC_FP16X3 || t->precision == ASKIT_PREC_BF16X3);
    if (wide && n_pairs > 0) cand.push_back({2, t->tune_stages, t->tune_runs, 1, 0.0});
    float *U = nullptr;
    ASK_CUDA(cudaMallocAsync(&U, sizeof(float) * (size_t)t->N * std::max(1, t->dw.r), s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    askit_status rc = ASKIT_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        askit_set_error("events");
        rc = ASKIT_ERR_CUDA;
    }
    auto apply = [&](const Cand &c) {
        t->tune_sched = c.pairs ? 0 : c.sched;
        t->tune_stages = c.stages;
        t->tune_runs = c.runs;
        t->tune_pairs = c.pairs;
        use_schedule(t);
    };
    for (size_t k = 0; k < cand.size() && rc == ASKIT_OK; ++k) {
        apply(cand[k]);
        rc = evaluate_ctx(t, t->dw, U, std::max(1, t->dw.r), s);                 // warm-up
        if (rc == ASKIT_OK && cudaEventRecord(e0, s) != cudaSuccess) rc = ASKIT_ERR_CUDA;
        for (int q = 0; q < reps && rc == ASKIT_OK; ++q) rc = evaluate_ctx(t, t->dw, U, std::max(1, t->dw.r), s);
        if (rc == ASKIT_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)) {
            askit_set_error("autotune timing: %s", cudaGetErrorString(cudaGetLastError()));
            rc = ASKIT_ERR_CUDA;
        }
        float ms = 0.f;
        if (rc == ASKIT_OK) cudaEventElapsedTime(&ms, e0, e1);
        cand[k].ms = ms / reps;
    }
    size_t best = 0;
    for (size_t k = 1; k < cand.size(); ++k)
        if (cand[k].ms < cand[best].ms) best = k;
    if (!cand.empty()) apply(cand[best]);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(U, s);
    cudaStreamSynchronize(s);
    if (rc != ASKIT_OK) return rc;
    *n_out = (int32_t)std::min<size_t>(cand.size(), (size_t)std::max(0, max_out));
    for (int32_t k = 0; k < *n_out; ++k)
        out[k] = {cand[k].sched, cand[k].stages, cand[k].runs, cand[k].pairs, (int32_t)((size_t)k == best), cand[k].ms};
    return ASKIT_OK;
}

askit_status askit_graph_create(askit_tree t, const float *W_dev, int32_t r, int64_t ldw, float *U_dev,
                                int64_t ldu, void *stream, askit_graph *out) {
    if (!t || !out || !U_dev) { askit_set_error("tree, U_dev and out must be non-NULL"); return ASKIT_ERR_INVALID_ARG; }
    *out = nullptr;
    if (ldu < r) { askit_set_error("ldu < r"); return ASKIT_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    ASK_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) {
        askit_set_error("askit_graph_create must not run inside a stream capture");
        return ASKIT_ERR_INVALID_ARG;
    }
    askit_graph g = new askit_graph_s();
    g->t = t;
    askit_status rc = ASKIT_OK;
    cudaGraph_t graph = nullptr;
    // uncaptured step: grows the context's buffers, builds operand state
    rc = set_weights_ctx(t, g->ctx, W_dev, r, ldw, s);
    if (rc == ASKIT_OK) rc = evaluate_ctx(t, g->ctx, U_dev, ldu, s);
    if (rc == ASKIT_OK && cudaStreamSynchronize(s) != cudaSuccess) {
        askit_set_error("graph warm-up step: %s", cudaGetErrorString(cudaGetLastError()));
        rc = ASKIT_ERR_CUDA;
    }
    // capture on a private stream: the caller's may be the legacy default
    // stream, which cannot be captured
    cudaStream_t cs = nullptr;
    if (rc == ASKIT_OK && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        askit_set_error("capture stream: %s", cudaGetErrorString(cudaGetLastError()));
        rc = ASKIT_ERR_CUDA;
    }
    if (rc == ASKIT_OK) {
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            askit_set_error("begin capture: %s", cudaGetErrorString(cudaGetLastError()));
            rc = ASKIT_ERR_CUDA;
        } else {
            rc = set_weights_ctx(t, g->ctx, W_dev, r, ldw, cs);
            if (rc == ASKIT_OK) rc = evaluate_ctx(t, g->ctx, U_dev, ldu, cs);
            cudaError_t e = cudaStreamEndCapture(cs, &graph);      // always end the capture
            if (rc == ASKIT_OK && e != cudaSuccess) {
                askit_set_error("end capture: %s", cudaGetErrorString(e));
                rc = ASKIT_ERR_CUDA;
            }
        }
    }
    if (cs) cudaStreamDestroy(cs);
    if (rc == ASKIT_OK && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
        askit_set_error("graph instantiate: %s", cudaGetErrorString(cudaGetLastError()));
        rc = ASKIT_ERR_CUDA;
    }
    if (graph) {
        size_t nn = 0;
        if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess) g->n_nodes = (int64_t)nn;
        cudaGraphDestroy(graph);
    }
    if (rc != ASKIT_OK) {
        cudaGetLastError();
        askit_graph_destroy(g);
        return rc;
    }
    *out = g;
    return ASKIT_OK;
}

askit_status askit_graph_launch(askit_graph g, void *stream) {
    if (!g || !g->exec) { askit_set_error("graph is NULL"); return ASKIT_ERR_INVALID_ARG; }
    ASK_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return ASKIT_OK;
}

askit_status askit_graph_destroy(askit_graph g) {
    if (!g) return ASKIT_OK;
    cudaDeviceSynchronize();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    g->ctx.arena.free_all();
    delete g;
    return ASKIT_OK;
}

askit_status askit_footprint(askit_tree t, int32_t kind, int64_t n, int32_t r, size_t *bytes) {
    if (!t || !bytes || r < 1 || n < 0 || (kind != 0 && kind != 1)) {
        askit_set_error("need a tree, kind 0 or 1, n >= 0, r >= 1 and bytes");
        return ASKIT_ERR_INVALID_ARG;
    }
    const int64_t srows = std::max<int64_t>(t->spool_rows, 1) + 256;
    const double per_target = (double)t->wl_entries / std::max<int64_t>(1, t->N);
    size_t b = 0;
    if (kind == 0) {
        // a weight context: W in tree order, skeleton weights, partials
        b = sizeof(float) * ((size_t)t->N_pad * r + (size_t)srows * r + (size_t)t->wl_entries_max * r);
        // the 16-bit tensor-core kernels' per-sub-block column data and weights
        if (t->n_sub > 0 && t->d <= TC_K)
            b += sizeof(float4) * (size_t)t->n_sub * 128 + (r > 1 ? sizeof(float) * (size_t)t->n_sub * (128 * 16 + 16) : 0);
    } else {
        // an out-of-sample batch of n targets: queries, kNN, prune sets and
        // work lists (entries estimated from the in-sample rate, doubled)
        const double ent = 2.0 * per_target * n + 1024;
        // kNN shortlist: candidates (1024 a query), seed lists, padded rows, and
        // the dense work items (every leaf sub-block against each 128 queries)
        const double knn = (double)n * (1024 * 4 + 32 * 12 + (size_t)t->d_pad * 4 + 32) +
                           (double)t->n_leaf_sub * ((n + 127) / 128) * sizeof(EvalItem);
        b = (size_t)(n * ((size_t)t->d * 4 + (size_t)t->d_pad * 4 + (size_t)t->kappa * (4 + 8 + 4 + 4) + 64) +
                     ent * (8 * 4 + 4 + 4 * r + 32 / 128.0) + knn + (1 << 20));
    }
    *bytes = b;
    return ASKIT_OK;
}

}  // extern "C"
