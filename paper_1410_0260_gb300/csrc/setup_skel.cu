// Skeletonization on the GPU (Sections 2.1-2.2, Algorithms 2 and 3).
//
//  * Node neighbor lists (Algorithm 2): a leaf collects its points' kNN
//    entries outside the leaf, an internal node its children's lists minus
//    its own points; each id keeps its smallest recorded distance, the list
//    is ordered by (distance, id) and truncated to ell = s_max + ell_extra.
//  * Sampled targets (eq. (2.4)): the list, then uniform draws without
//    replacement outside the node and the list (Philox stream of the node).
//  * ID (Section 2.1): FP64 kernel block K(T_a, C_a), Householder QR with
//    column pivoting on recomputed trailing norms, rank by |R_kk| <= tol
//    |R_00| within [s_min, s_max], P = R11^{-1} R12 by back substitution.
// Every FP64 operation is explicitly rounded and sequenced so the lists,
// pivots and skeletons reproduce bit for bit on any IEEE machine.
#include <float.h>
#include <limits.h>

#include <algorithm>

#include "askit_impl.cuh"

namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__device__ __forceinline__ bool in_subtree(int32_t leaf, int64_t a, int L, int depth_a) {
    return ((int64_t)leaf >> (L - depth_a)) == a;
}

// Leaf-level candidates: entry (q, z) of tree position q is the z-th
// neighbor of point perm[q]; neighbors inside the point's own leaf are
// removed (id INT_MAX, key DBL_MAX).
__global__ void leaf_cand_kernel(const int32_t *perm, const int32_t *leafof, const int32_t *knn,
                                 const double *knnd, int64_t N, int kappa, int32_t *cj, double *ck) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * kappa) return;
    int64_t q = e / kappa;
    int z = (int)(e % kappa);
    int32_t i = perm[q];
    int32_t j = knn[(int64_t)i * kappa + z];
    if (leafof[j] == leafof[i]) {
        cj[e] = INT_MAX;
        ck[e] = DBL_MAX;
    } else {
        cj[e] = j;
        ck[e] = knnd[(int64_t)i * kappa + z];
    }
}

// Internal-level candidates: node a = a0 + g takes both children's lists,
// removing ids inside a.  Slots [g * 2 ell, (g + 1) * 2 ell).
__global__ void inner_cand_kernel(int64_t a0, int ngroups, int ell, int L, int depth,
                                  const int32_t *leafof, const int32_t *nl_cnt, const int32_t *nl_ids,
                                  const double *nl_key, int32_t *cj, double *ck) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)ngroups * 2 * ell) return;
    int64_t g = e / (2 * ell);
    int slot = (int)(e % (2 * ell));
    int64_t a = a0 + g;
    int64_t ch = 2 * a + (slot >= ell);
    int q = slot % ell;
    int32_t j = INT_MAX;
    double k = DBL_MAX;
    if (q < nl_cnt[ch]) {
        int32_t jj = nl_ids[ch * ell + q];
        if (!in_subtree(leafof[jj], a, L, depth)) {
            j = jj;
            k = nl_key[ch * ell + q];
        }
    }
    cj[e] = j;
    ck[e] = k;
}

// After a stable sort by id: the first entry of each id group carries the
// group's smallest key; the rest are removed.  Counts survivors per segment.
__global__ void dedupe_kernel(const int32_t *sj, const double *sk, int32_t *oj, double *ok,
                              const int32_t *seg_of, const int32_t *seg_beg, int64_t n,
                              int32_t *seg_cnt) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    int32_t j = sj[e];
    int g = seg_of[e];
    bool first = (j != INT_MAX) && (e == seg_beg[g] || sj[e - 1] != j);
    if (!first) {
        oj[e] = INT_MAX;
        ok[e] = DBL_MAX;
        return;
    }
    double m = sk[e];
    int64_t end = n;
    for (int64_t f = e + 1; f < end && sj[f] == j && seg_of[f] == g; ++f) m = fmin(m, sk[f]);
    oj[e] = j;
    ok[e] = m;
    atomicAdd(seg_cnt + g, 1);
}

__global__ void seg_of_kernel(const int32_t *beg, const int32_t *end, int nseg, int32_t *seg_of) {
    int g = blockIdx.x;
    if (g >= nseg) return;
    for (int64_t e = beg[g] + threadIdx.x; e < end[g]; e += blockDim.x) seg_of[e] = g;
}

__global__ void nl_write_kernel(int64_t a0, int nseg, const int32_t *beg, const int32_t *sj,
                                const double *sk, const int32_t *cnt, int ell, int32_t *nl_cnt,
                                int32_t *nl_ids, double *nl_key) {
    int g = blockIdx.x;
    if (g >= nseg) return;
    int64_t a = a0 + g;
    int c = min(cnt[g], ell);
    if (threadIdx.x == 0) nl_cnt[a] = c;
    for (int q = threadIdx.x; q < ell; q += blockDim.x) {
        nl_ids[a * ell + q] = q < c ? sj[beg[g] + q] : -1;
        nl_key[a * ell + q] = q < c ? sk[beg[g] + q] : 0.0;
    }
}

// Sampled targets of node a (one thread per node): T_a = the first
// min(|N_a|, ell_a) list entries, then draw n gives j = floor(u N / 2^32)
// with u the top 32 bits of Philox word n keyed (seed, 0), counter (a, n/4);
// rejected inside a, in the list or already drawn.
__global__ void sample_kernel(int64_t n_nodes, int64_t N, int L, int ell, const int32_t *nsize,
                              const int32_t *leafof, const int32_t *nl_cnt, const int32_t *nl_ids,
                              uint64_t seed, int32_t *trows) {
    int64_t a = 2 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n_nodes) return;
    int depth = heap_depth(a);
    int64_t ell_a = (N - nsize[a] < ell) ? N - nsize[a] : ell;
    int32_t *rows = trows + a * ell;
    int nr = min(nl_cnt[a], (int)ell_a);
    for (int q = 0; q < nr; ++q) rows[q] = nl_ids[a * ell + q];
    for (uint64_t draw = 0; nr < ell_a; ++draw) {
        uint64_t w = philox_word(seed, 0, (uint64_t)a, draw);
        int32_t j = (int32_t)(((w >> 32) * (uint64_t)N) >> 32);
        if (in_subtree(leafof[j], a, L, depth)) continue;
        bool seen = false;
        for (int q = 0; q < nr && !seen; ++q) seen = (rows[q] == j);
        if (seen) continue;
        rows[nr++] = j;
    }
    for (int q = nr; q < ell; ++q) rows[q] = -1;
}

// Columns of each node of a level: leaf points in tree order (ascending id)
// or the children's skeletons (left then right, pivot order).
__global__ void cols_kernel(int64_t a0, int nseg, bool leaf_level, const int32_t *perm,
                            const int32_t *nstart, const int32_t *nsize, const int32_t *skel_fixed,
                            const int32_t *s, int s_max, int cmax, int32_t *cols) {
    int g = blockIdx.x;
    if (g >= nseg) return;
    int64_t a = a0 + g;
    int32_t *out = cols + (int64_t)g * cmax;
    if (leaf_level) {
        for (int q = threadIdx.x; q < nsize[a]; q += blockDim.x) out[q] = perm[nstart[a] + q];
    } else {
        int sl = s[2 * a], sr = s[2 * a + 1];
        for (int q = threadIdx.x; q < sl + sr; q += blockDim.x)
            out[q] = q < sl ? skel_fixed[(2 * a) * s_max + q] : skel_fixed[(2 * a + 1) * s_max + (q - sl)];
    }
}

// K(T_a, C_a) with the canonical exp: entry (i, q) = exp(-(c D) / h_q^2).
__global__ void fill_kernel(const float *X, int d, const float *hsrc, double kscale, int64_t a0,
                            const int32_t *batch_nodes, const int64_t *woff, const int32_t *ncol,
                            const int32_t *ellv, const int32_t *trows, int ell, const int32_t *cols,
                            int cmax, double *work) {
    int g = blockIdx.y;
    int64_t a = batch_nodes[g];
    int c = ncol[a], rows = ellv[a];
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)rows * c) return;
    int i = (int)(e / c), q = (int)(e % c);
    int32_t ri = trows[a * ell + i];
    int32_t cq = cols[(a - a0) * cmax + q];
    double D = c_dist2(X + (int64_t)ri * d, X + (int64_t)cq * d, d);
    double h = (double)hsrc[cq];
    double arg = c_div(c_mul(kscale, D), c_mul(h, h));
    work[woff[g] + e] = c_exp(-arg);
}

// Column-pivoted Householder QR of one node's block and the interpolation
// matrix P = R11^{-1} R12 (one CTA per node).  At step k the pivot is the
// column with the largest trailing squared norm (recomputed; ties to the
// smallest position), |R_kk| is its norm, the reflector is H = I - tau v v^T
// with v_k = 1 and beta = -sign(alpha) ||x||.
constexpr int QR_THREADS = 256;
__global__ void __launch_bounds__(QR_THREADS) cpqr_kernel(
    const int32_t *batch_nodes, const int64_t *woff, const int64_t *poff_ws, const int32_t *ncol,
    const int32_t *ellv, double tol, int s_min, int s_max, double *work, int32_t *piv_fixed,
    int cmax, int32_t *s_out) {
    extern __shared__ double sh[];           // v[rows]
    __shared__ double red_v[QR_THREADS / 32];
    __shared__ int red_j[QR_THREADS / 32];
    __shared__ double s_best;
    __shared__ int s_p;
    int g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int64_t a = batch_nodes[g];
    int cols = ncol[a], rows = ellv[a];
    double *A = work + woff[g];
    double *P = work + poff_ws[g];
    int32_t *piv = piv_fixed + a * cmax;
    double *v = sh;
    int s_hi = min(min(s_max, cols), rows);
    int s_lo = min(min(s_min, cols), s_hi);
    for (int j = tid; j < cols; j += QR_THREADS) piv[j] = j;
    __syncthreads();
    double r00 = 0.0;
    int s = s_hi;
    for (int k = 0; k < s_hi; ++k) {
        double best = -1.0;
        int bj = INT_MAX;
        for (int j = k + tid; j < cols; j += QR_THREADS) {
            double acc = 0.0;
            for (int i = k; i < rows; ++i) {
                double x = A[(int64_t)i * cols + j];
                acc = c_add(acc, c_mul(x, x));
            }
            if (acc > best) { best = acc; bj = j; }   // j increases: ties keep the smaller
        }
        for (int o = 16; o > 0; o >>= 1) {
            double ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (ob > best || (ob == best && oj < bj)) { best = ob; bj = oj; }
        }
        if (lane == 0) { red_v[wid] = best; red_j[wid] = bj; }
        __syncthreads();
        if (tid == 0) {
            double b = red_v[0];
            int p = red_j[0];
            for (int w = 1; w < QR_THREADS / 32; ++w)
                if (red_v[w] > b || (red_v[w] == b && red_j[w] < p)) { b = red_v[w]; p = red_j[w]; }
            s_best = b;
            s_p = p;
        }
        __syncthreads();
        double nrm = __dsqrt_rn(s_best);
        int p = s_p;
        if (k == 0) r00 = nrm;
        if (nrm == 0.0 || (k >= s_lo && nrm <= c_mul(tol, r00))) { s = k; break; }
        if (p != k) {
            for (int i = tid; i < rows; i += QR_THREADS) {
                double t = A[(int64_t)i * cols + k];
                A[(int64_t)i * cols + k] = A[(int64_t)i * cols + p];
                A[(int64_t)i * cols + p] = t;
            }
            if (tid == 0) { int t = piv[k]; piv[k] = piv[p]; piv[p] = t; }
        }
        __syncthreads();
        double alpha = A[(int64_t)k * cols + k];
        double beta = (alpha >= 0.0) ? -nrm : nrm;
        double tau = c_div(c_sub(beta, alpha), beta);
        double scal = c_sub(alpha, beta);
        __syncthreads();
        for (int i = k + 1 + tid; i < rows; i += QR_THREADS) {
            v[i] = c_div(A[(int64_t)i * cols + k], scal);
            A[(int64_t)i * cols + k] = 0.0;
        }
        if (tid == 0) { v[k] = 1.0; A[(int64_t)k * cols + k] = beta; }
        __syncthreads();
        for (int j = k + 1 + tid; j < cols; j += QR_THREADS) {
            double dot = 0.0;
            for (int i = k; i < rows; ++i) dot = c_add(dot, c_mul(v[i], A[(int64_t)i * cols + j]));
            double tdot = c_mul(tau, dot);
            for (int i = k; i < rows; ++i)
                A[(int64_t)i * cols + j] = c_sub(A[(int64_t)i * cols + j], c_mul(tdot, v[i]));
        }
        __syncthreads();
    }
    int nr = cols - s;
    for (int j = tid; j < nr; j += QR_THREADS) {
        for (int i = s - 1; i >= 0; --i) {
            double acc = A[(int64_t)i * cols + (s + j)];
            for (int t = i + 1; t < s; ++t) acc = c_sub(acc, c_mul(A[(int64_t)i * cols + t], P[(int64_t)t * nr + j]));
            P[(int64_t)i * nr + j] = c_div(acc, A[(int64_t)i * cols + i]);
        }
    }
    if (tid == 0) s_out[a] = s;
}

// Skeleton ids of the batch's nodes (first s pivots) and P into the level pool.
__global__ void skel_out_kernel(const int32_t *batch_nodes, int64_t a0, const int64_t *poff_ws,
                                const int64_t *poff_lvl, const int32_t *s, const int32_t *ncol,
                                const int32_t *cols, int cmax, const int32_t *piv_fixed, int s_max,
                                const double *work, int32_t *skel_fixed, double *P64, float *P32) {
    int g = blockIdx.x;
    int64_t a = batch_nodes[g];
    int sa = s[a], c = ncol[a];
    for (int q = threadIdx.x; q < sa; q += blockDim.x)
        skel_fixed[a * s_max + q] = cols[(a - a0) * cmax + piv_fixed[a * cmax + q]];
    int64_t np = (int64_t)sa * (c - sa);
    for (int64_t e = threadIdx.x; e < np; e += blockDim.x) {
        double x = work[poff_ws[g] + e];
        P64[poff_lvl[g] + e] = x;
        P32[poff_lvl[g] + e] = (float)x;
    }
}

// Segmented dedupe + (key, id) sort + truncation shared by all levels.
askit_status dedupe_sort_truncate(int64_t a0, int nseg, const std::vector<int32_t> &hbeg,
                                  const std::vector<int32_t> &hend, int32_t *cj, double *ck,
                                  int64_t n, int ell, askit_tree t, cudaStream_t s) {
    int32_t *beg = nullptr, *end = nullptr, *seg_of = nullptr, *cnt = nullptr, *tj = nullptr;
    double *tk = nullptr;
    void *tmp = nullptr;
    askit_status rc = ASKIT_OK;
    size_t b1 = 0, b2 = 0;
    cudaError_t e = cudaSuccess;
#define DCHK(x) do { e = (x); if (e != cudaSuccess) goto fail; } while (0)
    DCHK(cudaMalloc(&beg, sizeof(int32_t) * nseg));
    DCHK(cudaMalloc(&end, sizeof(int32_t) * nseg));
    DCHK(cudaMalloc(&cnt, sizeof(int32_t) * nseg));
    DCHK(cudaMalloc(&seg_of, sizeof(int32_t) * (n ? n : 1)));
    DCHK(cudaMalloc(&tj, sizeof(int32_t) * (n ? n : 1)));
    DCHK(cudaMalloc(&tk, sizeof(double) * (n ? n : 1)));
    DCHK(cudaMemcpyAsync(beg, hbeg.data(), sizeof(int32_t) * nseg, cudaMemcpyHostToDevice, s));
    DCHK(cudaMemcpyAsync(end, hend.data(), sizeof(int32_t) * nseg, cudaMemcpyHostToDevice, s));
    DCHK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * nseg, s));
    if ((rc = seg_sort_i32_f64(nullptr, nullptr, nullptr, nullptr, n, nseg, nullptr, nullptr, nullptr, &b1, s)) != ASKIT_OK) goto out;
    if ((rc = seg_sort_f64_i32(nullptr, nullptr, nullptr, nullptr, n, nseg, nullptr, nullptr, nullptr, &b2, s)) != ASKIT_OK) goto out;
    b1 = std::max(b1, b2);
    DCHK(cudaMalloc(&tmp, b1));
    seg_of_kernel<<<nseg, 256, 0, s>>>(beg, end, nseg, seg_of);
    // by id (stable): each id's entries become contiguous
    if ((rc = seg_sort_i32_f64(cj, tj, ck, tk, n, nseg, beg, end, tmp, &b1, s)) != ASKIT_OK) goto out;
    dedupe_kernel<<<nblk(n, 256), 256, 0, s>>>(tj, tk, cj, ck, seg_of, beg, n, cnt);
    DCHK(cudaGetLastError());
    // by key (stable over ascending ids): (key, id) order, removed entries last
    if ((rc = seg_sort_f64_i32(ck, tk, cj, tj, n, nseg, beg, end, tmp, &b1, s)) != ASKIT_OK) goto out;
    nl_write_kernel<<<nseg, 256, 0, s>>>(a0, nseg, beg, tj, tk, cnt, ell, t->nl_cnt, t->nl_ids, t->nl_key);
    DCHK(cudaGetLastError());
    DCHK(cudaStreamSynchronize(s));
    goto out;
fail:
    askit_set_error("node lists: %s", cudaGetErrorString(e));
    rc = e == cudaErrorMemoryAllocation ? ASKIT_ERR_OOM : ASKIT_ERR_CUDA;
out:
#undef DCHK
    cudaStreamSynchronize(s);
    cudaFree(beg); cudaFree(end); cudaFree(cnt); cudaFree(seg_of); cudaFree(tj); cudaFree(tk); cudaFree(tmp);
    return rc;
}

}  // namespace

askit_status build_node_lists(askit_tree t, cudaStream_t s) {
    const int L = t->L, ell = t->ell_max, kappa = t->kappa;
    const int64_t N = t->N;
    if (L == 0) return ASKIT_OK;
    // leaves
    {
        int64_t n = N * kappa;
        int32_t *cj = nullptr;
        double *ck = nullptr;
        ASK_CUDA(cudaMalloc(&cj, sizeof(int32_t) * n));
        ASK_CUDA(cudaMalloc(&ck, sizeof(double) * n));
        leaf_cand_kernel<<<nblk(n, 256), 256, 0, s>>>(t->perm, t->leafof, t->knn, t->knnd, N, kappa, cj, ck);
        int64_t a0 = (int64_t)1 << L;
        int nseg = (int)a0;
        std::vector<int32_t> hb(nseg), he(nseg);
        for (int g = 0; g < nseg; ++g) {
            hb[g] = (int32_t)(t->h_start[a0 + g] * kappa);
            he[g] = (int32_t)((t->h_start[a0 + g] + t->h_size[a0 + g]) * kappa);
        }
        askit_status rc = dedupe_sort_truncate(a0, nseg, hb, he, cj, ck, n, ell, t, s);
        cudaFree(cj);
        cudaFree(ck);
        ASK_TRY(rc);
    }
    // internal levels, bottom-up
    for (int depth = L - 1; depth >= 1; --depth) {
        int64_t a0 = (int64_t)1 << depth;
        int nseg = (int)a0;
        int64_t n = (int64_t)nseg * 2 * ell;
        int32_t *cj = nullptr;
        double *ck = nullptr;
        ASK_CUDA(cudaMalloc(&cj, sizeof(int32_t) * n));
        ASK_CUDA(cudaMalloc(&ck, sizeof(double) * n));
        inner_cand_kernel<<<nblk(n, 256), 256, 0, s>>>(a0, nseg, ell, L, depth, t->leafof, t->nl_cnt,
                                                      t->nl_ids, t->nl_key, cj, ck);
        std::vector<int32_t> hb(nseg), he(nseg);
        for (int g = 0; g < nseg; ++g) {
            hb[g] = (int32_t)((int64_t)g * 2 * ell);
            he[g] = (int32_t)((int64_t)(g + 1) * 2 * ell);
        }
        askit_status rc = dedupe_sort_truncate(a0, nseg, hb, he, cj, ck, n, ell, t, s);
        cudaFree(cj);
        cudaFree(ck);
        ASK_TRY(rc);
    }
    return ASKIT_OK;
}

askit_status build_samples(askit_tree t, cudaStream_t s) {
    if (t->L == 0) return ASKIT_OK;
    int64_t n = t->n_nodes - 2;
    sample_kernel<<<nblk(n, 64), 64, 0, s>>>(t->n_nodes, t->N, t->L, t->ell_max, t->nsize, t->leafof,
                                            t->nl_cnt, t->nl_ids, t->prm.seed, t->trows);
    ASK_LAUNCH();
    ASK_CUDA(cudaStreamSynchronize(s));
    return ASKIT_OK;
}

// Bottom-up skeletonization, one tree level at a time, in batches of nodes
// whose FP64 blocks fit a workspace budget.
askit_status skeletonize(askit_tree t, cudaStream_t s) {
    const int L = t->L, ell = t->ell_max, d = t->d;
    const int s_max = t->prm.s_max;
    const int64_t N = t->N, nn = t->n_nodes;
    t->h_s.assign(nn, 0);
    t->h_ncol.assign(nn, 0);
    if (L == 0) return ASKIT_OK;
    const int cmax = (int)std::max<int64_t>(t->h_size[(int64_t)1 << L], 2 * (int64_t)s_max);
    std::vector<int32_t> h_ell(nn, 0);
    for (int64_t a = 2; a < nn; ++a) h_ell[a] = (int32_t)std::min<int64_t>(ell, N - t->h_size[a]);
    int32_t *d_ell = nullptr, *skel_fixed = nullptr, *piv_fixed = nullptr;
    ASK_TRY(t->arena.alloc(&d_ell, nn));
    ASK_TRY(t->arena.alloc(&skel_fixed, (size_t)nn * s_max));
    ASK_TRY(t->arena.alloc(&piv_fixed, (size_t)nn * cmax));
    ASK_CUDA(cudaMemcpyAsync(d_ell, h_ell.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice, s));
    ASK_CUDA(cudaMemsetAsync(t->d_s, 0, sizeof(int32_t) * nn, s));

    std::vector<double *> lvl_P64(L + 1, nullptr);
    std::vector<float *> lvl_P32(L + 1, nullptr);
    std::vector<int64_t> lvl_ptot(L + 1, 0);
    std::vector<int64_t> node_poff(nn, 0);   // offset within its level pool
    const size_t budget = (size_t)6 << 30;   // FP64 workspace per batch

    for (int depth = L; depth >= 1; --depth) {
        int64_t a0 = (int64_t)1 << depth, a1 = (int64_t)2 << depth;
        for (int64_t a = a0; a < a1; ++a)
            t->h_ncol[a] = depth == L ? (int32_t)t->h_size[a] : t->h_s[2 * a] + t->h_s[2 * a + 1];
        ASK_CUDA(cudaMemcpyAsync(t->d_ncol + a0, t->h_ncol.data() + a0, sizeof(int32_t) * (a1 - a0),
                                 cudaMemcpyHostToDevice, s));
        int32_t *cols = nullptr;
        ASK_CUDA(cudaMalloc(&cols, sizeof(int32_t) * (a1 - a0) * cmax));
        cols_kernel<<<(unsigned)(a1 - a0), 128, 0, s>>>(a0, (int)(a1 - a0), depth == L, t->perm, t->nstart,
                                                       t->nsize, skel_fixed, t->d_s, s_max, cmax, cols);
        ASK_LAUNCH();
        // level pool for P (sizes known only after the QR of each batch)
        std::vector<double *> batch_P64;
        std::vector<float *> batch_P32;
            std::vector<int64_t> batch_tot;
        int64_t a = a0;
        int64_t lvl_run = 0;   // offset of the current batch inside the level pool
        while (a < a1) {
            // pick a batch
            std::vector<int32_t> nodes;
            std::vector<int64_t> woff, pws;
            size_t used = 0;
            while (a < a1) {
                int64_t c = t->h_ncol[a], r = h_ell[a];
                int64_t sh = std::min<int64_t>(std::min<int64_t>(s_max, c), r);
                size_t need = (size_t)(r * c + sh * c + 2) * sizeof(double);
                if (!nodes.empty() && used + need > budget) break;
                nodes.push_back((int32_t)a);
                woff.push_back((int64_t)(used / sizeof(double)));
                pws.push_back((int64_t)(used / sizeof(double)) + r * c);
                used += need;
                ++a;
            }
            int nb = (int)nodes.size();
            double *work = nullptr;
            int32_t *d_nodes = nullptr;
            int64_t *d_woff = nullptr, *d_pws = nullptr, *d_plvl = nullptr;
            ASK_CUDA(cudaMalloc(&work, used ? used : 8));
            ASK_CUDA(cudaMalloc(&d_nodes, sizeof(int32_t) * nb));
            ASK_CUDA(cudaMalloc(&d_woff, sizeof(int64_t) * nb));
            ASK_CUDA(cudaMalloc(&d_pws, sizeof(int64_t) * nb));
            ASK_CUDA(cudaMalloc(&d_plvl, sizeof(int64_t) * nb));
            ASK_CUDA(cudaMemcpyAsync(d_nodes, nodes.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s));
            ASK_CUDA(cudaMemcpyAsync(d_woff, woff.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, s));
            ASK_CUDA(cudaMemcpyAsync(d_pws, pws.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, s));
            int64_t maxent = 0;
            for (int g = 0; g < nb; ++g) maxent = std::max<int64_t>(maxent, (int64_t)h_ell[nodes[g]] * t->h_ncol[nodes[g]]);
            if (maxent > 0) {
                fill_kernel<<<dim3(nblk(maxent, 256), nb), 256, 0, s>>>(
                    t->X, d, t->hsrc, t->prm.kernel_scale, a0, d_nodes, d_woff, t->d_ncol, d_ell, t->trows,
                    ell, cols, cmax, work);
                ASK_LAUNCH();
            }
            int maxrows = 0;
            for (int g = 0; g < nb; ++g) maxrows = std::max(maxrows, h_ell[nodes[g]]);
            cpqr_kernel<<<nb, QR_THREADS, sizeof(double) * (maxrows + 1), s>>>(
                d_nodes, d_woff, d_pws, t->d_ncol, d_ell, t->prm.id_tol, t->prm.s_min, s_max, work,
                piv_fixed, cmax, t->d_s);
            ASK_LAUNCH();
            ASK_CUDA(cudaMemcpyAsync(t->h_s.data() + nodes[0], t->d_s + nodes[0], sizeof(int32_t) * nb,
                                     cudaMemcpyDeviceToHost, s));
            ASK_CUDA(cudaStreamSynchronize(s));
            std::vector<int64_t> plvl(nb);
            int64_t tot = 0;
            for (int g = 0; g < nb; ++g) {
                int64_t nd = nodes[g];
                plvl[g] = tot;
                node_poff[nd] = lvl_run + tot;
                tot += (int64_t)t->h_s[nd] * (t->h_ncol[nd] - t->h_s[nd]);
            }
            double *P64 = nullptr;
            float *P32 = nullptr;
            ASK_CUDA(cudaMalloc(&P64, sizeof(double) * (tot ? tot : 1)));
            ASK_CUDA(cudaMalloc(&P32, sizeof(float) * (tot ? tot : 1)));
            ASK_CUDA(cudaMemcpyAsync(d_plvl, plvl.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, s));
            skel_out_kernel<<<nb, 256, 0, s>>>(d_nodes, a0, d_pws, d_plvl, t->d_s, t->d_ncol, cols, cmax,
                                              piv_fixed, s_max, work, skel_fixed, P64, P32);
            ASK_LAUNCH();
            ASK_CUDA(cudaStreamSynchronize(s));
            cudaFree(work); cudaFree(d_nodes); cudaFree(d_woff); cudaFree(d_pws); cudaFree(d_plvl);
            batch_P64.push_back(P64);
            batch_P32.push_back(P32);
            batch_tot.push_back(tot);
            lvl_run += tot;
        }
        cudaFree(cols);
        // concatenate the level's batches
        int64_t ltot = 0;
        for (auto x : batch_tot) ltot += x;
        ASK_CUDA(cudaMalloc(&lvl_P64[depth], sizeof(double) * (ltot ? ltot : 1)));
        ASK_CUDA(cudaMalloc(&lvl_P32[depth], sizeof(float) * (ltot ? ltot : 1)));
        int64_t off = 0;
        for (size_t b = 0; b < batch_tot.size(); ++b) {
            ASK_CUDA(cudaMemcpyAsync(lvl_P64[depth] + off, batch_P64[b], sizeof(double) * batch_tot[b], cudaMemcpyDeviceToDevice, s));
            ASK_CUDA(cudaMemcpyAsync(lvl_P32[depth] + off, batch_P32[b], sizeof(float) * batch_tot[b], cudaMemcpyDeviceToDevice, s));
            off += batch_tot[b];
        }
        ASK_CUDA(cudaStreamSynchronize(s));
        for (size_t b = 0; b < batch_P64.size(); ++b) { cudaFree(batch_P64[b]); cudaFree(batch_P32[b]); }
        lvl_ptot[depth] = ltot;
    }

    // heap-order pools: level 1 first
    t->h_poff.assign(nn + 1, 0);
    t->h_skoff.assign(nn + 1, 0);
    t->h_pivoff.assign(nn + 1, 0);
    t->h_spool.assign(nn + 1, 0);
    int64_t ptot = 0;
    std::vector<int64_t> lvl_base(L + 1, 0);
    for (int depth = 1; depth <= L; ++depth) { lvl_base[depth] = ptot; ptot += lvl_ptot[depth]; }
    for (int64_t a = 2; a < nn; ++a) t->h_poff[a] = lvl_base[heap_depth(a)] + node_poff[a];
    t->h_poff[nn] = ptot;
    t->p_total = ptot;
    ASK_TRY(t->arena.alloc(&t->P64, ptot));
    ASK_TRY(t->arena.alloc(&t->P32, ptot));
    for (int depth = 1; depth <= L; ++depth) {
        if (lvl_ptot[depth]) {
            ASK_CUDA(cudaMemcpyAsync(t->P64 + lvl_base[depth], lvl_P64[depth], sizeof(double) * lvl_ptot[depth], cudaMemcpyDeviceToDevice, s));
            ASK_CUDA(cudaMemcpyAsync(t->P32 + lvl_base[depth], lvl_P32[depth], sizeof(float) * lvl_ptot[depth], cudaMemcpyDeviceToDevice, s));
        }
    }
    int64_t sk = 0, pv = 0, sp = 0;
    for (int64_t a = 0; a < nn; ++a) {
        t->h_skoff[a] = sk;
        t->h_pivoff[a] = pv;
        t->h_spool[a] = sp;
        if (a >= 2) {
            sk += t->h_s[a];
            pv += t->h_ncol[a];
            sp += (t->h_s[a] + ASK_ROW_PAD - 1) / ASK_ROW_PAD * ASK_ROW_PAD;
        }
    }
    t->h_skoff[nn] = sk; t->h_pivoff[nn] = pv; t->h_spool[nn] = sp;
    t->skel_total = sk; t->piv_total = pv; t->spool_rows = sp;
    ASK_TRY(t->arena.alloc(&t->skel_ids, sk));
    ASK_TRY(t->arena.alloc(&t->piv, pv));
    for (int64_t a = 2; a < nn; ++a) {
        if (t->h_s[a])
            ASK_CUDA(cudaMemcpyAsync(t->skel_ids + t->h_skoff[a], skel_fixed + a * s_max, sizeof(int32_t) * t->h_s[a], cudaMemcpyDeviceToDevice, s));
        if (t->h_ncol[a])
            ASK_CUDA(cudaMemcpyAsync(t->piv + t->h_pivoff[a], piv_fixed + a * cmax, sizeof(int32_t) * t->h_ncol[a], cudaMemcpyDeviceToDevice, s));
    }
    ASK_TRY(t->arena.alloc(&t->d_poff, nn + 1));
    ASK_TRY(t->arena.alloc(&t->d_skoff, nn + 1));
    ASK_TRY(t->arena.alloc(&t->d_pivoff, nn + 1));
    ASK_TRY(t->arena.alloc(&t->d_spool, nn + 1));
    ASK_CUDA(cudaMemcpyAsync(t->d_poff, t->h_poff.data(), sizeof(int64_t) * (nn + 1), cudaMemcpyHostToDevice, s));
    ASK_CUDA(cudaMemcpyAsync(t->d_skoff, t->h_skoff.data(), sizeof(int64_t) * (nn + 1), cudaMemcpyHostToDevice, s));
    ASK_CUDA(cudaMemcpyAsync(t->d_pivoff, t->h_pivoff.data(), sizeof(int64_t) * (nn + 1), cudaMemcpyHostToDevice, s));
    ASK_CUDA(cudaMemcpyAsync(t->d_spool, t->h_spool.data(), sizeof(int64_t) * (nn + 1), cudaMemcpyHostToDevice, s));
    ASK_CUDA(cudaStreamSynchronize(s));
    for (int depth = 1; depth <= L; ++depth) { cudaFree(lvl_P64[depth]); cudaFree(lvl_P32[depth]); }
    t->arena.release(skel_fixed);
    t->arena.release(piv_fixed);
    t->arena.release(d_ell);
    return ASKIT_OK;
}
