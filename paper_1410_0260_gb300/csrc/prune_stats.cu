// Pruning statistics of Section 3's Table 1: for every point as a target,
// the number of tree nodes the downward pass visits (Evaluate calls, pruned
// nodes included) under
//   neighbor pruning, eq. (2.5): a node is pruned unless it holds the target
//     or one of its kappa nearest neighbors (exact kNN);
//   distance pruning: a node with centroid c and radius R (the largest
//     distance from c to its points) is pruned when ||x - c|| > rscale R
//     (rscale = 1 is the rule as printed; the paper notes that R has to be
//     scaled in practice).
// The root is never pruned.  The tree is the evaluation tree of the setup
// (median splits between the farthest pair, leaves of at most m points).
// Every decision is made in canonical FP64 (each operation rounded, no
// contraction, coordinates ascending), so the counts are reproducible on any
// IEEE machine: centroids are the mean of the node's points summed in leaf
// order, and distances are compared squared, D(x, c) > rscale^2 R^2.
//
// The neighbor lists here may hold up to 256 neighbors (the experiment uses
// kappa = 128): the exact search computes every FP64 distance of a batch of
// queries (64 x 64 tiles, shared-memory staging of 32 coordinates at a time)
// and sorts each query's row by (distance, id) with a stable segmented sort.
#include <cfloat>
#include <climits>

#include "askit_impl.cuh"

namespace {

inline unsigned nb(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

constexpr int PS_T = 64;          // queries and candidates per distance tile
constexpr int PS_K = 32;          // coordinates staged at a time

// FP64 squared distances of queries [q0, q0 + nq) against all N points:
// block (cx, qy) computes the 64 x 64 tile of candidates [64 cx, ...) and
// queries [q0 + 64 qy, ...); thread (tx, ty) the 4 x 4 pairs (ty + 16 i,
// tx + 16 j).  Sums run over the coordinates in ascending order.
__global__ void __launch_bounds__(256) ps_dist_kernel(const float *X, int64_t N, int d, int64_t q0, int64_t nq,
                                                      double *D, int32_t *J) {
    __shared__ float qs[PS_K][PS_T + 1], cs[PS_K][PS_T + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t cbase = (int64_t)blockIdx.x * PS_T, qbase = (int64_t)blockIdx.y * PS_T;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < d; k0 += PS_K) {
        __syncthreads();
        for (int e = threadIdx.x; e < PS_T * PS_K; e += 256) {
            const int r = e / PS_K, kk = e % PS_K;
            const int64_t q = qbase + r, c = cbase + r;
            qs[kk][r] = (q < nq && k0 + kk < d) ? X[(q0 + q) * d + k0 + kk] : 0.f;
            cs[kk][r] = (c < N && k0 + kk < d) ? X[c * d + k0 + kk] : 0.f;
        }
        __syncthreads();
        const int kn = d - k0 < PS_K ? d - k0 : PS_K;
        for (int kk = 0; kk < kn; ++kk) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const double xq = (double)qs[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const double t = c_sub(xq, (double)cs[kk][tx + 16 * j]);
                    acc[i][j] = c_add(acc[i][j], c_mul(t, t));
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t q = qbase + ty + 16 * i;
        if (q >= nq) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t c = cbase + tx + 16 * j;
            if (c >= N) continue;
            D[q * N + c] = acc[i][j];
            J[q * N + c] = (int32_t)c;
        }
    }
}

__global__ void ps_segments_kernel(int64_t nq, int64_t N, int32_t *beg, int32_t *end) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nq) return;
    beg[q] = (int32_t)(q * N);
    end[q] = (int32_t)((q + 1) * N);
}

// The first kappa entries of each sorted row other than the query itself.
__global__ void ps_take_kernel(const double *Ds, const int32_t *Js, int64_t q0, int64_t nq, int64_t N, int kappa,
                               int32_t *ids, double *dist) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const int64_t self = q0 + q;
    int n = 0;
    for (int64_t e = 0; e < N && n < kappa; ++e) {
        const int32_t j = Js[q * N + e];
        if (j == self) continue;
        ids[self * kappa + n] = j;
        dist[self * kappa + n] = Ds[q * N + e];
        ++n;
    }
}

// Leaf (heap index) of every point.
__global__ void ps_leafof_kernel(const int32_t *perm, const int32_t *nstart, const int32_t *nsize, int64_t a0,
                                 int32_t *leaf) {
    const int64_t a = a0 + blockIdx.x;
    for (int q = threadIdx.x; q < nsize[a]; q += blockDim.x) leaf[perm[nstart[a] + q]] = (int32_t)a;
}

// Centroid (mean in leaf order) and squared radius of every node; block a,
// threads over coordinates, then over the node's points.
__global__ void ps_centroid_kernel(const float *X, int d, const int32_t *perm, const int32_t *nstart,
                                   const int32_t *nsize, double *cent, double *r2) {
    extern __shared__ double red[];
    const int64_t a = 1 + blockIdx.x;
    const int n = nsize[a], s0 = nstart[a];
    double *c = cent + a * d;
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        double acc = 0.0;
        for (int q = 0; q < n; ++q) acc = c_add(acc, (double)X[(int64_t)perm[s0 + q] * d + k]);
        c[k] = n > 0 ? c_div(acc, (double)n) : 0.0;
    }
    __syncthreads();
    double mx = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const float *x = X + (int64_t)perm[s0 + q] * d;
        double acc = 0.0;
        for (int k = 0; k < d; ++k) {
            const double t = c_sub(c[k], (double)x[k]);
            acc = c_add(acc, c_mul(t, t));
        }
        mx = acc > mx ? acc : mx;
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] = red[threadIdx.x] > red[threadIdx.x + o] ? red[threadIdx.x] : red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) r2[a] = red[0];
}

constexpr int PS_MAXSET = 257;    // the target's leaf and up to 256 neighbors' leaves

// Visits of one target under both rules.  Neighbor pruning: the nodes kept
// (U: ancestors of the prune set's leaves) plus the pruned children of kept
// nodes, counted level by level from the sorted leaves.  Distance pruning: a
// depth-first walk with an explicit stack.
__global__ void ps_visit_kernel(const float *X, int64_t N, int d, int L, int kappa, const int32_t *leaf,
                                const int32_t *ids, const double *cent, const double *r2, double rs2,
                                int64_t *vk, int64_t *vd) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int32_t set[PS_MAXSET];
    int n = 0;
    for (int z = -1; z < kappa; ++z) {
        const int32_t lf = leaf[z < 0 ? i : ids[i * kappa + z]];
        int p = n;
        bool dup = false;
        for (int u = 0; u < n; ++u) dup |= set[u] == lf;
        if (dup) continue;
        while (p > 0 && set[p - 1] > lf) { set[p] = set[p - 1]; --p; }
        set[p] = lf;
        ++n;
    }
    // the root, and both children of every kept node above the leaves:
    // 1 + 2 (|U_0| + ... + |U_{L-1}|), U_t the distinct prefixes at depth t
    int64_t visits = 1;
    for (int depth = 0; depth < L; ++depth) {
        const int sh = L - depth;
        int32_t prev = -1;
        for (int u = 0; u < n; ++u) {
            const int32_t b = set[u] >> sh;
            if (b != prev) visits += 2;
            prev = b;
        }
    }
    vk[i] = visits;
    // distance pruning
    const float *x = X + i * d;
    int32_t stack[64];
    int sp = 0;
    int64_t v = 1;
    if (L > 0) { stack[sp++] = 3; stack[sp++] = 2; }
    while (sp > 0) {
        const int32_t a = stack[--sp];
        ++v;
        const double *c = cent + (int64_t)a * d;
        double acc = 0.0;
        for (int k = 0; k < d; ++k) {
            const double t = c_sub(c[k], (double)x[k]);
            acc = c_add(acc, c_mul(t, t));
        }
        if (acc > c_mul(rs2, r2[a])) continue;            // pruned
        if (a >= ((int32_t)1 << L)) continue;              // a leaf
        stack[sp++] = 2 * a + 1;
        stack[sp++] = 2 * a;
    }
    vd[i] = v;
}

}  // namespace

extern "C" askit_status askit_prune_stats(const float *X_dev, int64_t N, int32_t d, int64_t ldx, int32_t leaf_size,
                                          int32_t kappa, double rscale, int64_t *visited_knn_dev,
                                          int64_t *visited_dist_dev, void *stream) {
    if (!X_dev || !visited_knn_dev || !visited_dist_dev || N < 2 || d < 1 || ldx < d || leaf_size < 2 || kappa < 1 ||
        kappa > 256 || kappa > N - 1 || !(rscale >= 0.0)) {
        askit_set_error("need N >= 2, d >= 1, ldx >= d, leaf_size >= 2, 1 <= kappa <= min(256, N - 1), rscale >= 0");
        return ASKIT_ERR_INVALID_ARG;
    }
    if (N > ((int64_t)1 << 22) || d > 4096) {
        askit_set_error("askit_prune_stats handles N <= 2^22 and d <= 4096");
        return ASKIT_ERR_UNSUPPORTED;
    }
    const int L = tree_depth(N, leaf_size);
    if (L > 20) { askit_set_error("tree deeper than 20 levels"); return ASKIT_ERR_UNSUPPORTED; }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nn = (int64_t)2 << L;
    // query batch: nq x N FP64 distances and ids, twice (sort double buffer)
    const int64_t nq_max = std::max<int64_t>(1, std::min<int64_t>(N, ((int64_t)1 << 26) / N));
    DevArena ar;
    float *X = nullptr;
    int32_t *perm = nullptr, *nstart = nullptr, *nsize = nullptr, *leaf = nullptr, *ids = nullptr;
    int32_t *J = nullptr, *Js = nullptr, *beg = nullptr, *end = nullptr;
    double *dist = nullptr, *D = nullptr, *Ds = nullptr, *cent = nullptr, *r2 = nullptr;
    void *tmp = nullptr;
    size_t tb = 0;
    askit_status rc = ASKIT_OK;
    std::vector<int64_t> st, sz;
    std::vector<int32_t> hs, hz;
#define PSTRY(x) do { rc = (x); if (rc != ASKIT_OK) goto out; } while (0)
#define PSCHK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { askit_set_error("prune stats: %s", cudaGetErrorString(e_)); rc = e_ == cudaErrorMemoryAllocation ? ASKIT_ERR_OOM : ASKIT_ERR_CUDA; goto out; } } while (0)
    PSTRY(ar.alloc(&X, (size_t)N * d));
    PSCHK(cudaMemcpy2DAsync(X, sizeof(float) * d, X_dev, sizeof(float) * ldx, sizeof(float) * d, N,
                            cudaMemcpyDeviceToDevice, s));
    PSTRY(ar.alloc(&perm, N));
    PSTRY(build_tree_gpu(X, N, d, L, 0, 0, 0, perm, s));
    tree_ranges(N, L, st, sz);
    hs.resize(nn);
    hz.resize(nn);
    for (int64_t a = 0; a < nn; ++a) {
        hs[a] = (int32_t)st[a];
        hz[a] = (int32_t)sz[a];
    }
    PSTRY(ar.alloc(&nstart, nn));
    PSTRY(ar.alloc(&nsize, nn));
    PSCHK(cudaMemcpyAsync(nstart, hs.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice, s));
    PSCHK(cudaMemcpyAsync(nsize, hz.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice, s));
    PSTRY(ar.alloc(&leaf, N));
    ps_leafof_kernel<<<(unsigned)((int64_t)1 << L), 128, 0, s>>>(perm, nstart, nsize, (int64_t)1 << L, leaf);
    PSCHK(cudaGetLastError());
    // exact kNN by batches of queries
    PSTRY(ar.alloc(&ids, (size_t)N * kappa));
    PSTRY(ar.alloc(&dist, (size_t)N * kappa));
    PSTRY(ar.alloc(&D, (size_t)nq_max * N));
    PSTRY(ar.alloc(&Ds, (size_t)nq_max * N));
    PSTRY(ar.alloc(&J, (size_t)nq_max * N));
    PSTRY(ar.alloc(&Js, (size_t)nq_max * N));
    PSTRY(ar.alloc(&beg, nq_max));
    PSTRY(ar.alloc(&end, nq_max));
    PSTRY(seg_sort_f64_i32(nullptr, nullptr, nullptr, nullptr, nq_max * N, (int)nq_max, beg, end, nullptr, &tb, s));
    PSTRY(ar.alloc((char **)&tmp, tb));
    for (int64_t q0 = 0; q0 < N; q0 += nq_max) {
        const int64_t nq = std::min<int64_t>(nq_max, N - q0);
        ps_dist_kernel<<<dim3(nb(N, PS_T), nb(nq, PS_T)), 256, 0, s>>>(X, N, d, q0, nq, D, J);
        ps_segments_kernel<<<nb(nq, 128), 128, 0, s>>>(nq, N, beg, end);
        PSCHK(cudaGetLastError());
        size_t tb2 = tb;
        PSTRY(seg_sort_f64_i32(D, Ds, J, Js, nq * N, (int)nq, beg, end, tmp, &tb2, s));
        ps_take_kernel<<<nb(nq, 128), 128, 0, s>>>(Ds, Js, q0, nq, N, kappa, ids, dist);
        PSCHK(cudaGetLastError());
    }
    // node centroids and radii, then the visits
    PSTRY(ar.alloc(&cent, (size_t)nn * d));
    PSTRY(ar.alloc(&r2, nn));
    ps_centroid_kernel<<<(unsigned)(nn - 1), 128, 128 * sizeof(double), s>>>(X, d, perm, nstart, nsize, cent, r2);
    PSCHK(cudaGetLastError());
    ps_visit_kernel<<<nb(N, 128), 128, 0, s>>>(X, N, d, L, kappa, leaf, ids, cent, r2, rscale * rscale,
                                             visited_knn_dev, visited_dist_dev);
    PSCHK(cudaGetLastError());
    PSCHK(cudaStreamSynchronize(s));
out:
#undef PSTRY
#undef PSCHK
    cudaStreamSynchronize(s);
    ar.free_all();
    return rc;
}
