// Tree build and nearest-neighbor search on the GPU (Section 2.2).
//
// Both the ASKIT tree and the random-projection (RP) trees of the kNN search
// are built level by level: every node of a level computes its projection
// key per point, the level's nodes are sorted segment-wise by (key, id), the
// lower ceil(n/2) points form the left child, and each child is re-sorted by
// id.  All leaves sit at one depth L, the least depth at which no node holds
// more than the leaf size.  Distances and projections are FP64 sums in
// ascending coordinate order with no fused multiply-add, so the trees and
// neighbor lists are bit-exact functions of the input.
#include <float.h>
#include <limits.h>

#include <mutex>

#include "askit_impl.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ bool kv_less(double da, int ia, double db, int ib) {
    return da < db || (da == db && ia < ib);
}

// Squared distance with an FP64 first operand (the node center).
__device__ __forceinline__ double c_dist2_df(const double *x, const float *y, int d) {
    double acc = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = c_sub(x[k], (double)y[k]);
        acc = c_add(acc, c_mul(t, t));
    }
    return acc;
}

// Segment (node) of each position at one tree level, by binary search over
// the level's node starts.
__global__ void seg_of_pos_kernel(const int32_t *lvl_start, int nseg, int64_t N, int32_t *seg) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= N) return;
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (lvl_start[mid] <= q) lo = mid; else hi = mid - 1;
    }
    seg[q] = lo;
}

// Node centers: FP64 mean, points summed in the node's (ascending id) order.
__global__ void center_kernel(const float *X, int d, const int32_t *order, const int32_t *lvl_start,
                              const int32_t *lvl_size, double *xc) {
    int node = blockIdx.x;
    int k = blockIdx.y * blockDim.x + threadIdx.x;
    if (k >= d) return;
    int64_t b = lvl_start[node], n = lvl_size[node];
    double acc = 0.0;
    for (int64_t q = 0; q < n; ++q) acc = c_add(acc, (double)X[(int64_t)order[b + q] * d + k]);
    xc[(int64_t)node * d + k] = c_div(acc, (double)n);
}

// Farthest point from a per-node reference: max D, ties to the smallest id.
// Pass 1 raises best_bits to the largest D (non-negative doubles order like
// their bit patterns); pass 2 lowers best_id among the points attaining it.
template <bool FROM_CENTER>
__global__ void far_pass1(const float *X, int d, const int32_t *order, const int32_t *seg, int64_t N,
                          const double *xc, const int32_t *ref_id, double *Dq,
                          unsigned long long *best_bits) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= N) return;
    int node = seg[q];
    const float *xj = X + (int64_t)order[q] * d;
    double D = FROM_CENTER ? c_dist2_df(xc + (int64_t)node * d, xj, d)
                           : c_dist2(X + (int64_t)ref_id[node] * d, xj, d);
    Dq[q] = D;
    atomicMax(best_bits + node, (unsigned long long)__double_as_longlong(D));
}

__global__ void far_pass2(const int32_t *order, const int32_t *seg, int64_t N, const double *Dq,
                          const unsigned long long *best_bits, int32_t *best_id) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= N) return;
    int node = seg[q];
    if ((unsigned long long)__double_as_longlong(Dq[q]) == best_bits[node]) atomicMin(best_id + node, order[q]);
}

// Projection on the line (x_l, x_r) with origin x_l.
__global__ void proj_line_kernel(const float *X, int d, const int32_t *order, const int32_t *seg,
                                 int64_t N, const int32_t *xl, const int32_t *xr, double *p) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= N) return;
    int node = seg[q];
    const float *xj = X + (int64_t)order[q] * d;
    const float *a = X + (int64_t)xl[node] * d;
    const float *b = X + (int64_t)xr[node] * d;
    double acc = 0.0;
    for (int k = 0; k < d; ++k) {
        double u = c_sub((double)xj[k], (double)a[k]);
        double v = c_sub((double)b[k], (double)a[k]);
        acc = c_add(acc, c_mul(u, v));
    }
    p[q] = acc;
}

// Projection on a Rademacher direction: bit k%64 of Philox word k/64 keyed
// (seed, iter + 1) with counter (node, word/4) set means -1.
__global__ void proj_rp_kernel(const float *X, int d, const int32_t *order, const int32_t *seg,
                               int64_t N, int64_t node0, uint64_t seed, int iter, double *p) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= N) return;
    int64_t node = node0 + seg[q];
    const float *xj = X + (int64_t)order[q] * d;
    double acc = 0.0;
    uint64_t w = 0;
    for (int k = 0; k < d; ++k) {
        if ((k & 63) == 0) w = philox_word(seed, (uint64_t)iter + 1, (uint64_t)node, (uint64_t)(k >> 6));
        double v = ((w >> (k & 63)) & 1) ? -1.0 : 1.0;
        acc = c_add(acc, c_mul(v, (double)xj[k]));
    }
    p[q] = acc;
}

__global__ void iota_kernel(int32_t *a, int64_t n) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < n) a[q] = (int32_t)q;
}

template <class T>
__global__ void fill_kernel(T *a, int64_t n, T v) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < n) a[q] = v;
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// ---------------------------------------------------------------------------
// Warp-level best-32 list: lane l holds the l-th smallest (D, id) so far.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_sort32(double &d, int &i, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            double od = __shfl_xor_sync(FULL, d, j);
            int oi = __shfl_xor_sync(FULL, i, j);
            bool keep_min = (((lane & j) == 0) == ((lane & k) == 0));
            bool sw = keep_min ? kv_less(od, oi, d, i) : kv_less(d, i, od, oi);
            if (sw) { d = od; i = oi; }
        }
    }
}

// Merge sorted candidates (cd, ci) into the sorted list (ld, li), keeping the
// 32 smallest: half-cleaner against the reversed candidates, then a bitonic merge.
__device__ __forceinline__ void warp_merge32(double &ld, int &li, double cd, int ci, int lane) {
    double rd = __shfl_sync(FULL, cd, 31 - lane);
    int ri = __shfl_sync(FULL, ci, 31 - lane);
    if (kv_less(rd, ri, ld, li)) { ld = rd; li = ri; }
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        double od = __shfl_xor_sync(FULL, ld, j);
        int oi = __shfl_xor_sync(FULL, li, j);
        bool lower = (lane & j) == 0;
        bool sw = lower ? kv_less(od, oi, ld, li) : kv_less(ld, li, od, oi);
        if (sw) { ld = od; li = oi; }
    }
}

// Offer one batch of candidates (one per lane) to the list.  `dedup` drops
// candidates whose id is already listed (RP iterations revisit pairs).
__device__ __forceinline__ void warp_offer(double &ld, int &li, double cd, int ci, int kappa,
                                           bool dedup, int lane) {
    double wd = __shfl_sync(FULL, ld, kappa - 1);
    int wi = __shfl_sync(FULL, li, kappa - 1);
    bool useful = kv_less(cd, ci, wd, wi);
    if (!__ballot_sync(FULL, useful)) return;
    if (dedup) {
        bool dup = false;
#pragma unroll 8
        for (int l = 0; l < 32; ++l) dup |= (__shfl_sync(FULL, li, l) == ci);
        if (dup) useful = false;
    }
    if (!useful) { cd = DBL_MAX; ci = INT_MAX; }
    warp_sort32(cd, ci, lane);
    warp_merge32(ld, li, cd, ci, lane);
}

// Exhaustive search of a candidate range for a set of queries; one warp per
// query.  Candidates are rows cand[c0 .. c1) of X (ids), queries are ids
// (self excluded) or rows of Y (qid < 0 marks out-of-sample).
// The list of each query lives in (bd, bi)[q * 32 + lane].
__global__ void knn_block_kernel(const float *X, int d, const int32_t *cand, const int32_t *cbeg,
                                 const int32_t *cend, const int32_t *qids, const float *Y,
                                 int64_t nq_total, const int32_t *qbeg, const int32_t *qend,
                                 double *bd, int *bi, int kappa, bool dedup) {
    extern __shared__ float sq[];   // one query row per warp
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int seg = blockIdx.x;
    int64_t c0 = cbeg[seg], c1 = cend[seg];
    float *myq = sq + (int64_t)warp * d;
    for (int64_t q = qbeg[seg] + warp; q < qend[seg]; q += nw) {
        int self = qids ? qids[q] : -1;
        const float *xq = qids ? X + (int64_t)self * d : Y + q * d;
        for (int k = lane; k < d; k += 32) myq[k] = xq[k];
        __syncwarp();
        int64_t slot = (qids ? (int64_t)self : q) * 32 + lane;
        double ld = bd[slot];
        int li = bi[slot];
        // FP32 pre-filter: the FP32 difference-form sum of d squares is within a
        // factor (1 +- gam) of the exact value, gam = (d + 2) 2^-24 (plus slack),
        // so a candidate whose FP32 distance exceeds the current kappa-th FP64
        // distance by that factor cannot enter the list and needs no FP64 work.
        const float gam = (float)(d + 2) * 5.9604645e-8f * 1.25f + 1e-6f;
        for (int64_t cb = c0; cb < c1; cb += 32) {
            double cd = DBL_MAX;
            int ci = INT_MAX;
            int j = -1;
            float d32 = 3.4e38f;
            if (cb + lane < c1) {
                j = cand ? cand[cb + lane] : (int)(cb + lane);
                if (j != self) {
                    const float *xj = X + (int64_t)j * d;
                    float a = 0.f;
                    for (int k = 0; k < d; ++k) {
                        const float t = myq[k] - xj[k];
                        a = fmaf(t, t, a);
                    }
                    d32 = a;
                } else {
                    j = -1;
                }
            }
            const double kth = __shfl_sync(FULL, ld, kappa - 1);
            const bool need = j >= 0 && (!(d32 < 3.0e38f) || (double)d32 * (1.0 - (double)gam) <= kth);
            if (!__ballot_sync(FULL, need)) continue;
            if (need) {
                const float *xj = X + (int64_t)j * d;
                double acc = 0.0;
                for (int k = 0; k < d; ++k) {
                    double t = c_sub((double)myq[k], (double)xj[k]);
                    acc = c_add(acc, c_mul(t, t));
                }
                cd = acc;
                ci = j;
            }
            warp_offer(ld, li, cd, ci, kappa, dedup, lane);
        }
        bd[slot] = ld;
        bi[slot] = li;
        __syncwarp();
    }
}

// Tiled exhaustive search: block (qb, sp) takes queries [64 qb, 64 qb + 64)
// against the candidate split [c0, c1).  FP32 squared distances of 64 x 128
// tiles (difference form, k ascending, one FMA per coordinate: the same
// rounding bound as the per-warp search) go to shared memory; warp w then
// filters the rows of its 8 queries against their current kappa-th FP64
// distance and recomputes the survivors in canonical FP64.  Each split
// writes its own best-32 lists; knn_merge_kernel merges the splits.
constexpr int KT_Q = 64, KT_C = 128, KT_K = 32;

__global__ void __launch_bounds__(256) knn_tiled_kernel(const float *X, int64_t N, int d, const float *Y,
                                                         int64_t Q, int64_t split_len, int kappa, double *bd,
                                                         int *bi, const int32_t *self) {
    // the distance tile reuses the chunk buffers (the selection ends before
    // the next tile's first chunk is loaded)
    __shared__ float sbuf[KT_Q * (KT_C + 1)];
    float (*qs)[KT_Q + 1] = reinterpret_cast<float (*)[KT_Q + 1]>(sbuf);
    float (*cs)[KT_C + 1] = reinterpret_cast<float (*)[KT_C + 1]>(sbuf + KT_K * (KT_Q + 1));
    float (*dt)[KT_C + 1] = reinterpret_cast<float (*)[KT_C + 1]>(sbuf);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t q0 = (int64_t)blockIdx.x * KT_Q;
    const int64_t c0 = (int64_t)blockIdx.y * split_len;
    const int64_t c1 = c0 + split_len < N ? c0 + split_len : N;
    const float gam = (float)(d + 2) * 5.9604645e-8f * 1.25f + 1e-6f;
    double ld[8];
    int li[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) { ld[u] = DBL_MAX; li[u] = INT_MAX; }
    for (int64_t cb = c0; cb < c1; cb += KT_C) {
        float acc[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
        for (int k0 = 0; k0 < d; k0 += KT_K) {
            __syncthreads();
            // query chunk [64 x 32] and candidate chunk [128 x 32], transposed, zeros outside
            for (int e = tid; e < KT_Q * KT_K; e += 256) {
                const int qq = e / KT_K, kk = e % KT_K;
                const int64_t q = q0 + qq;
                float v = 0.f;
                if (q < Q && k0 + kk < d) v = Y ? Y[q * d + k0 + kk] : X[q * d + k0 + kk];
                qs[kk][qq] = v;
            }
            for (int e = tid; e < KT_C * KT_K; e += 256) {
                const int cc = e / KT_K, kk = e % KT_K;
                const int64_t j = cb + cc;
                cs[kk][cc] = (j < c1 && k0 + kk < d) ? X[j * d + k0 + kk] : 0.f;
            }
            __syncthreads();
            const int kn = d - k0 < KT_K ? d - k0 : KT_K;
            for (int kk = 0; kk < kn; ++kk) {
                float qv[4], cv[8];
#pragma unroll
                for (int i = 0; i < 4; ++i) qv[i] = qs[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 8; ++j) cv[j] = cs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float t = qv[i] - cv[j];
                        acc[i][j] = fmaf(t, t, acc[i][j]);
                    }
            }
        }
        __syncthreads();     // every thread is done with the chunk buffers
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) dt[ty + 16 * i][tx + 16 * j] = acc[i][j];
        __syncthreads();
        // selection: warp w owns queries 8w .. 8w+7 of the tile
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int qq = 8 * warp + u;
            const int64_t q = q0 + qq;
            if (q >= Q) continue;                         // warp-uniform
            const float *xq = Y ? Y + q * d : X + q * d;
            for (int rr = 0; rr < KT_C / 32; ++rr) {
                const int64_t j = cb + rr * 32 + lane;
                // queries Y exclude no point unless `self` names the point each
                // query is (the tree's own points as queries)
                const bool valid = j < c1 && (self ? j != self[q] : (Y || j != q));
                const float d32 = dt[qq][rr * 32 + lane];
                const double kth = __shfl_sync(FULL, ld[u], kappa - 1);
                const bool need = valid && (double)d32 * (1.0 - (double)gam) <= kth;
                if (!__ballot_sync(FULL, need)) continue;
                double cd = DBL_MAX;
                int ci = INT_MAX;
                if (need) {
                    const float *xj = X + j * d;
                    double a = 0.0;
                    for (int k = 0; k < d; ++k) {
                        const double t = c_sub((double)xq[k], (double)xj[k]);
                        a = c_add(a, c_mul(t, t));
                    }
                    cd = a;
                    ci = (int)j;
                }
                warp_offer(ld[u], li[u], cd, ci, kappa, false, lane);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int64_t q = q0 + 8 * warp + u;
        if (q < Q) {
            const int64_t o = ((int64_t)blockIdx.y * Q + q) * 32 + lane;
            bd[o] = ld[u];
            bi[o] = li[u];
        }
    }
}

// Merge the splits' best-32 lists of each query (one warp per query) and
// write the kappa nearest.
__global__ void knn_merge_kernel(const double *bd, const int *bi, int64_t Q, int nsplit, int kappa,
                                 int32_t *ids, double *dist) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (q >= Q) return;                                   // warp-uniform
    double ld = DBL_MAX;
    int li = INT_MAX;
    for (int sp = 0; sp < nsplit; ++sp) {
        const int64_t o = ((int64_t)sp * Q + q) * 32 + lane;
        warp_offer(ld, li, bd[o], bi[o], kappa, false, lane);
    }
    if (lane < kappa) {
        ids[q * kappa + lane] = li;
        dist[q * kappa + lane] = ld;
    }
}

__global__ void knn_extract_kernel(const double *bd, const int *bi, int64_t Q, int kappa,
                                   int32_t *ids, double *dist) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= Q * kappa) return;
    int64_t q = t / kappa;
    int z = (int)(t % kappa);
    ids[t] = bi[q * 32 + z];
    dist[t] = bd[q * 32 + z];
}

__global__ void knn_dist_kernel(const float *X, int64_t N, int d, int kappa, const int32_t *ids,
                                double *dist) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= N * kappa) return;
    int64_t i = t / kappa;
    dist[t] = c_dist2(X + i * d, X + (int64_t)ids[t] * d, d);
}

// Scratch shared by one tree build.
struct TreeScratch {
    int32_t *seg = nullptr, *tmp_ids = nullptr, *bid = nullptr, *xl = nullptr;
    double *keys = nullptr, *keys_out = nullptr, *xc = nullptr, *Dq = nullptr;
    unsigned long long *bbits = nullptr;
    int32_t *lvl_start = nullptr, *lvl_end = nullptr, *lvl_size = nullptr;
    void *cub = nullptr;
    size_t cub_bytes = 0;
};

void free_scratch(TreeScratch &s) {
    cudaFree(s.seg); cudaFree(s.tmp_ids); cudaFree(s.bid); cudaFree(s.xl); cudaFree(s.keys);
    cudaFree(s.keys_out); cudaFree(s.xc); cudaFree(s.Dq); cudaFree(s.bbits); cudaFree(s.lvl_start);
    cudaFree(s.lvl_end); cudaFree(s.lvl_size); cudaFree(s.cub);
}

}  // namespace

int tree_depth(int64_t N, int64_t leaf) {
    int L = 0;
    while (((N + ((int64_t)1 << L) - 1) >> L) > leaf) ++L;
    return L;
}

void tree_ranges(int64_t N, int L, std::vector<int64_t> &start, std::vector<int64_t> &size) {
    int64_t nn = (int64_t)2 << L;
    start.assign(nn, 0);
    size.assign(nn, 0);
    size[1] = N;
    for (int64_t a = 1; a < ((int64_t)1 << L); ++a) {
        start[2 * a] = start[a];
        size[2 * a] = (size[a] + 1) / 2;
        start[2 * a + 1] = start[a] + (size[a] + 1) / 2;
        size[2 * a + 1] = size[a] / 2;
    }
}

// kind 0: ASKIT split (center, two farthest-point scans, line projection);
// kind 1: RP split (Rademacher direction of (seed, iter, node)).
askit_status build_tree_gpu(const float *X, int64_t N, int d, int L, int kind, uint64_t seed,
                            int iter, int32_t *order, cudaStream_t s) {
    std::vector<int64_t> st, sz;
    tree_ranges(N, L, st, sz);
    int64_t nn = (int64_t)2 << L;
    std::vector<int32_t> hs(nn), he(nn), hz(nn);
    for (int64_t a = 0; a < nn; ++a) {
        hs[a] = (int32_t)st[a];
        he[a] = (int32_t)(st[a] + sz[a]);
        hz[a] = (int32_t)sz[a];
    }
    TreeScratch sc;
    askit_status rc = ASKIT_OK;
    auto fail = [&](cudaError_t e, const char *what) {
        askit_set_error("tree build: %s: %s", what, cudaGetErrorString(e));
        rc = e == cudaErrorMemoryAllocation ? ASKIT_ERR_OOM : ASKIT_ERR_CUDA;
    };
#define TCHK(x, what) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { fail(e_, what); goto done; } } while (0)
    {
        int64_t half = (int64_t)1 << (L > 0 ? L - 1 : 0);
        TCHK(cudaMalloc(&sc.seg, sizeof(int32_t) * N), "alloc");
        TCHK(cudaMalloc(&sc.tmp_ids, sizeof(int32_t) * N), "alloc");
        TCHK(cudaMalloc(&sc.keys, sizeof(double) * N), "alloc");
        TCHK(cudaMalloc(&sc.keys_out, sizeof(double) * N), "alloc");
        TCHK(cudaMalloc(&sc.Dq, sizeof(double) * N), "alloc");
        TCHK(cudaMalloc(&sc.bid, sizeof(int32_t) * half), "alloc");
        TCHK(cudaMalloc(&sc.xl, sizeof(int32_t) * half), "alloc");
        TCHK(cudaMalloc(&sc.bbits, sizeof(unsigned long long) * half), "alloc");
        TCHK(cudaMalloc(&sc.xc, sizeof(double) * half * d), "alloc");
        TCHK(cudaMalloc(&sc.lvl_start, sizeof(int32_t) * nn), "alloc");
        TCHK(cudaMalloc(&sc.lvl_end, sizeof(int32_t) * nn), "alloc");
        TCHK(cudaMalloc(&sc.lvl_size, sizeof(int32_t) * nn), "alloc");
        TCHK(cudaMemcpyAsync(sc.lvl_start, hs.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice, s), "copy");
        TCHK(cudaMemcpyAsync(sc.lvl_end, he.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice, s), "copy");
        TCHK(cudaMemcpyAsync(sc.lvl_size, hz.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice, s), "copy");
        // scratch for the largest segmented sort (all N keys, up to 2^L segments)
        size_t b1 = 0, b2 = 0;
        if ((rc = seg_sort_f64_i32(nullptr, nullptr, nullptr, nullptr, N, (int)half, nullptr, nullptr, nullptr, &b1, s)) != ASKIT_OK) goto done;
        if ((rc = seg_sort_i32(nullptr, nullptr, N, (int)(2 * half), nullptr, nullptr, nullptr, &b2, s)) != ASKIT_OK) goto done;
        sc.cub_bytes = b1 > b2 ? b1 : b2;
        TCHK(cudaMalloc(&sc.cub, sc.cub_bytes), "alloc");

        iota_kernel<<<nblk(N, 256), 256, 0, s>>>(order, N);
        for (int t = 0; t < L; ++t) {
            int64_t a0 = (int64_t)1 << t;
            int nseg = (int)a0;
            const int32_t *ls = sc.lvl_start + a0, *le = sc.lvl_end + a0, *lz = sc.lvl_size + a0;
            seg_of_pos_kernel<<<nblk(N, 256), 256, 0, s>>>(ls, nseg, N, sc.seg);
            if (kind == 0) {
                center_kernel<<<dim3(nseg, (d + 63) / 64), 64, 0, s>>>(X, d, order, ls, lz, sc.xc);
                // x_l: farthest from the center
                fill_kernel<unsigned long long><<<nblk(nseg, 256), 256, 0, s>>>(sc.bbits, nseg, 0ull);
                fill_kernel<int32_t><<<nblk(nseg, 256), 256, 0, s>>>(sc.bid, nseg, INT_MAX);
                far_pass1<true><<<nblk(N, 256), 256, 0, s>>>(X, d, order, sc.seg, N, sc.xc, nullptr, sc.Dq, sc.bbits);
                far_pass2<<<nblk(N, 256), 256, 0, s>>>(order, sc.seg, N, sc.Dq, sc.bbits, sc.bid);
                TCHK(cudaMemcpyAsync(sc.xl, sc.bid, sizeof(int32_t) * nseg, cudaMemcpyDeviceToDevice, s), "copy");
                // x_r: farthest from x_l
                fill_kernel<unsigned long long><<<nblk(nseg, 256), 256, 0, s>>>(sc.bbits, nseg, 0ull);
                fill_kernel<int32_t><<<nblk(nseg, 256), 256, 0, s>>>(sc.bid, nseg, INT_MAX);
                far_pass1<false><<<nblk(N, 256), 256, 0, s>>>(X, d, order, sc.seg, N, nullptr, sc.xl, sc.Dq, sc.bbits);
                far_pass2<<<nblk(N, 256), 256, 0, s>>>(order, sc.seg, N, sc.Dq, sc.bbits, sc.bid);
                proj_line_kernel<<<nblk(N, 256), 256, 0, s>>>(X, d, order, sc.seg, N, sc.xl, sc.bid, sc.keys);
            } else {
                proj_rp_kernel<<<nblk(N, 256), 256, 0, s>>>(X, d, order, sc.seg, N, a0, seed, iter, sc.keys);
            }
            TCHK(cudaGetLastError(), "projection kernels");
            // (key, id) order inside every node: stable sort of an id-ascending segment
            if ((rc = seg_sort_f64_i32(sc.keys, sc.keys_out, order, sc.tmp_ids, N, nseg, ls, le, sc.cub, &sc.cub_bytes, s)) != ASKIT_OK) goto done;
            // children back to ascending id
            if ((rc = seg_sort_i32(sc.tmp_ids, order, N, 2 * nseg, sc.lvl_start + 2 * a0, sc.lvl_end + 2 * a0, sc.cub, &sc.cub_bytes, s)) != ASKIT_OK) goto done;
        }
        TCHK(cudaStreamSynchronize(s), "sync");
    }
done:
#undef TCHK
    cudaStreamSynchronize(s);
    free_scratch(sc);
    return rc;
}

namespace {
askit_status knn_lists_init(int64_t Q, double **bd, int **bi, cudaStream_t s) {
    ASK_CUDA(cudaMallocAsync(bd, sizeof(double) * Q * 32, s));
    ASK_CUDA(cudaMallocAsync(bi, sizeof(int) * Q * 32, s));
    fill_kernel<double><<<nblk(Q * 32, 256), 256, 0, s>>>(*bd, Q * 32, DBL_MAX);
    fill_kernel<int><<<nblk(Q * 32, 256), 256, 0, s>>>(*bi, Q * 32, INT_MAX);
    ASK_LAUNCH();
    return ASKIT_OK;
}
}  // namespace

// Exact kNN: every point (Y == nullptr, self excluded) or every row of Y
// against all N points.  Query tiles of 64 x candidate splits, chosen so that
// about four blocks per SM have work; the splits' lists are merged.
askit_status knn_exact_gpu(const float *X, int64_t N, int d, int kappa, const float *Y, int64_t Q,
                           int32_t *ids, double *dist, cudaStream_t s, const int32_t *self) {
    const int64_t nqb = (Q + KT_Q - 1) / KT_Q;
    int64_t nsplit = (4 * 152 + nqb - 1) / nqb;
    nsplit = std::max<int64_t>(1, std::min<int64_t>(nsplit, N / (4 * KT_C)));
    nsplit = std::min<int64_t>(nsplit, 65535);
    int64_t split_len = (N + nsplit - 1) / nsplit;
    split_len = (split_len + KT_C - 1) / KT_C * KT_C;
    nsplit = (N + split_len - 1) / split_len;
    double *bd = nullptr;
    int *bi = nullptr;
    cudaError_t e = cudaMallocAsync(&bd, sizeof(double) * nsplit * Q * 32, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&bi, sizeof(int) * nsplit * Q * 32, s);
    if (e == cudaSuccess) {
        knn_tiled_kernel<<<dim3((unsigned)nqb, (unsigned)nsplit), 256, 0, s>>>(X, N, d, Y, Q, split_len, kappa, bd, bi,
                                                                               self);
        knn_merge_kernel<<<nblk(Q * 32, 256), 256, 0, s>>>(bd, bi, Q, (int)nsplit, kappa, ids, dist);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    askit_status rc = ASKIT_OK;
    if (e != cudaSuccess) {
        askit_set_error("exact kNN: %s", cudaGetErrorString(e));
        rc = ASKIT_ERR_CUDA;
    }
    if (bd) cudaFreeAsync(bd, s);
    if (bi) cudaFreeAsync(bi, s);
    return rc;
}

namespace {

// Out-of-sample kNN, step 1: the two leaves whose centers are nearest to each
// query (FP32; they only seed the search).  One warp per query, lanes over
// the leaves.
__global__ void knn_home_kernel(const float *Yp, int64_t T, int d_pad, const float *cent, const int32_t *leaf_cbase,
                                int64_t M, int32_t *home) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (q >= T) return;                                  // warp-uniform
    const float *y = Yp + q * d_pad;
    float b0 = 3.4e38f, b1 = 3.4e38f;
    int i0 = 0, i1 = 0;
    for (int64_t l = lane; l < M; l += 32) {
        const float *c = cent + (int64_t)leaf_cbase[l] * TC_K;
        float acc = 0.f;
        for (int k = 0; k < d_pad; ++k) {
            const float t = y[k] - c[k];
            acc = fmaf(t, t, acc);
        }
        if (acc < b0) { b1 = b0; i1 = i0; b0 = acc; i0 = (int)l; }
        else if (acc < b1) { b1 = acc; i1 = (int)l; }
    }
    for (int o = 16; o > 0; o >>= 1) {                   // merge the lanes' best two
        const float ob0 = __shfl_xor_sync(FULL, b0, o), ob1 = __shfl_xor_sync(FULL, b1, o);
        const int oi0 = __shfl_xor_sync(FULL, i0, o), oi1 = __shfl_xor_sync(FULL, i1, o);
        float n0, n1;
        int m0, m1;
        if (ob0 < b0) { n0 = ob0; m0 = oi0; n1 = b0 < ob1 ? b0 : ob1; m1 = b0 < ob1 ? i0 : oi1; }
        else { n0 = b0; m0 = i0; n1 = ob0 < b1 ? ob0 : b1; m1 = ob0 < b1 ? oi0 : i1; }
        b0 = n0; i0 = m0; b1 = n1; i1 = m1;
    }
    if (lane == 0) {
        home[2 * q] = i0;
        home[2 * q + 1] = M > 1 ? i1 : i0;
    }
}

// Step 2: the exact best-32 list of each query over the points of its two
// home leaves (canonical FP64), and U = its kappa-th distance rounded up to
// FP32: an upper bound of the query's true kappa-th distance.
__global__ void knn_seed_kernel(const float *X, int d, const float *Y, int64_t T, const int32_t *home, int64_t M,
                                const int32_t *nstart, const int32_t *nsize, const int32_t *perm, int kappa,
                                double *bd, int *bi, float *U) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (q >= T) return;                                  // warp-uniform
    const float *y = Y + q * d;
    double ld = DBL_MAX;
    int li = INT_MAX;
    for (int h = 0; h < 2; ++h) {
        const int l = home[2 * q + h];
        if (h == 1 && l == home[2 * q]) break;
        const int64_t a = M + l;
        const int p0 = nstart[a], np = nsize[a];
        for (int b = 0; b < np; b += 32) {
            double cd = DBL_MAX;
            int ci = INT_MAX;
            if (b + lane < np) {
                ci = perm[p0 + b + lane];
                cd = c_dist2(y, X + (int64_t)ci * d, d);
            }
            warp_offer(ld, li, cd, ci, kappa, false, lane);
        }
    }
    bd[q * 32 + lane] = ld;
    bi[q * 32 + lane] = li;
    const double kth = __shfl_sync(FULL, ld, kappa - 1);
    if (lane == 0) U[q] = kth < 3.0e38 ? __double2float_ru(kth) : 3.4e38f;
}

// Step 4: re-rank each query's shortlist (tree positions) in canonical FP64
// on top of its seed list; a query whose shortlist overflowed is queued for
// the exhaustive search.
__global__ void knn_rerank_kernel(const float *X, int d, const float *Y, int64_t T, const int32_t *perm,
                                  const int *cnt, const int32_t *cand, int cap, int kappa, double *bd, int *bi,
                                  int32_t *ids, double *dist, int *n_ovf, int32_t *ovf) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (q >= T) return;                                  // warp-uniform
    const int n = cnt[q];
    if (n > cap) {
        if (lane == 0) ovf[atomicAdd(n_ovf, 1)] = (int32_t)q;
        return;
    }
    const float *y = Y + q * d;
    double ld = bd[q * 32 + lane];
    int li = bi[q * 32 + lane];
    for (int b = 0; b < n; b += 32) {
        double cd = DBL_MAX;
        int ci = INT_MAX;
        if (b + lane < n) {
            ci = perm[cand[q * cap + b + lane]];
            cd = c_dist2(y, X + (int64_t)ci * d, d);
        }
        warp_offer(ld, li, cd, ci, kappa, true, lane);
    }
    if (lane < kappa) {
        ids[q * kappa + lane] = li;
        dist[q * kappa + lane] = ld;
    }
}

__global__ void knn_pad_rows_kernel(const float *Y, int64_t T, int d, int d_pad, float *Yp) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= T * d_pad) return;
    const int64_t q = e / d_pad;
    const int k = (int)(e % d_pad);
    Yp[e] = k < d ? Y[q * d + k] : 0.f;
}

__global__ void knn_gather_rows_kernel(const float *Y, int d, const int32_t *rows, int64_t n, float *out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * d) return;
    out[e] = Y[(int64_t)rows[e / d] * d + e % d];
}

__global__ void knn_scatter_kernel(const int32_t *ids_s, const double *dist_s, const int32_t *rows, int64_t n,
                                   int kappa, int32_t *ids, double *dist) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * kappa) return;
    const int64_t q = rows[e / kappa];
    ids[q * kappa + e % kappa] = ids_s[e];
    dist[q * kappa + e % kappa] = dist_s[e];
}

}  // namespace

askit_status knn_oos(askit_tree t, const float *Y, int64_t T, int kappa, int32_t *ids, double *dist, cudaStream_t s) {
    if (!t->Xt_hhi || t->d > TC_K || t->n_leaf_sub == 0 || kappa > 32)
        return knn_exact_gpu(t->X, t->N, t->d, kappa, Y, T, ids, dist, s);
    const int cap = 1024;
    const float eta = 1.52587890625e-05f;   // 2^-16: five times the FP16x3 distance error bound
    const int64_t M = (int64_t)1 << t->L;
    DevArena tmp;
    tmp.async = true;
    tmp.stream = s;
    float *Yp = nullptr, *U = nullptr;
    int32_t *home = nullptr, *cand = nullptr, *ovf = nullptr;
    int *cnt = nullptr, *bi = nullptr, *n_ovf = nullptr;
    double *bd = nullptr;
    int h_ovf = 0;
    askit_status rc = ASKIT_OK;
#define QTRY(x) do { rc = (x); if (rc != ASKIT_OK) goto out; } while (0)
    QTRY(tmp.alloc(&Yp, (size_t)T * t->d_pad));
    QTRY(tmp.alloc(&home, (size_t)T * 2));
    QTRY(tmp.alloc(&U, T));
    QTRY(tmp.alloc(&bd, (size_t)T * 32));
    QTRY(tmp.alloc(&bi, (size_t)T * 32));
    QTRY(tmp.alloc(&cnt, T));
    QTRY(tmp.alloc(&cand, (size_t)T * cap));
    QTRY(tmp.alloc(&ovf, T));
    QTRY(tmp.alloc(&n_ovf, 1));
    if (cudaMemsetAsync(cnt, 0, sizeof(int) * T, s) != cudaSuccess || cudaMemsetAsync(n_ovf, 0, sizeof(int), s) != cudaSuccess) {
        askit_set_error("kNN: memset");
        rc = ASKIT_ERR_CUDA;
        goto out;
    }
    knn_pad_rows_kernel<<<nblk(T * t->d_pad, 256), 256, 0, s>>>(Y, T, t->d, t->d_pad, Yp);
    knn_home_kernel<<<nblk(T * 32, 256), 256, 0, s>>>(Yp, T, t->d_pad, t->cent, t->leaf_cbase, M, home);
    knn_seed_kernel<<<nblk(T * 32, 256), 256, 0, s>>>(t->X, t->d, Y, T, home, M, t->nstart, t->nsize, t->perm, kappa,
                                                      bd, bi, U);
    if (cudaGetLastError() != cudaSuccess) { askit_set_error("kNN: seed launch"); rc = ASKIT_ERR_CUDA; goto out; }
    QTRY(knn_shortlist_tc16(t, Yp, T, U, cnt, cand, cap, eta, s));
    knn_rerank_kernel<<<nblk(T * 32, 256), 256, 0, s>>>(t->X, t->d, Y, T, t->perm, cnt, cand, cap, kappa, bd, bi, ids,
                                                        dist, n_ovf, ovf);
    if (cudaGetLastError() != cudaSuccess) { askit_set_error("kNN: re-rank launch"); rc = ASKIT_ERR_CUDA; goto out; }
    if (cudaMemcpyAsync(&h_ovf, n_ovf, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        askit_set_error("kNN: %s", cudaGetErrorString(cudaGetLastError()));
        rc = ASKIT_ERR_CUDA;
        goto out;
    }
    if (h_ovf > 0) {
        // queries whose shortlist overflowed: the exhaustive search
        float *Ys = nullptr;
        int32_t *ids_s = nullptr;
        double *dist_s = nullptr;
        QTRY(tmp.alloc(&Ys, (size_t)h_ovf * t->d));
        QTRY(tmp.alloc(&ids_s, (size_t)h_ovf * kappa));
        QTRY(tmp.alloc(&dist_s, (size_t)h_ovf * kappa));
        knn_gather_rows_kernel<<<nblk((int64_t)h_ovf * t->d, 256), 256, 0, s>>>(Y, t->d, ovf, h_ovf, Ys);
        QTRY(knn_exact_gpu(t->X, t->N, t->d, kappa, Ys, h_ovf, ids_s, dist_s, s));
        knn_scatter_kernel<<<nblk((int64_t)h_ovf * kappa, 256), 256, 0, s>>>(ids_s, dist_s, ovf, h_ovf, kappa, ids, dist);
        if (cudaGetLastError() != cudaSuccess) { askit_set_error("kNN: overflow launch"); rc = ASKIT_ERR_CUDA; goto out; }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        askit_set_error("kNN: %s", cudaGetErrorString(cudaGetLastError()));
        rc = ASKIT_ERR_CUDA;
    }
out:
#undef QTRY
    tmp.free_all();
    return rc;
}

// RP-tree kNN (Section 2.2): iters trees; in each, every point searches its
// leaf exhaustively and the best kappa candidates are kept across trees.
askit_status knn_rp_gpu(const float *X, int64_t N, int d, int kappa, int iters, int64_t rp_leaf,
                        uint64_t seed, int32_t *ids, double *dist, cudaStream_t s) {
    int L = tree_depth(N, rp_leaf);
    std::vector<int64_t> st, sz;
    tree_ranges(N, L, st, sz);
    int64_t nleaf = (int64_t)1 << L;
    std::vector<int32_t> h(2 * nleaf);
    for (int64_t a = 0; a < nleaf; ++a) {
        h[a] = (int32_t)st[nleaf + a];
        h[nleaf + a] = (int32_t)(st[nleaf + a] + sz[nleaf + a]);
    }
    double *bd = nullptr;
    int *bi = nullptr;
    int32_t *order = nullptr, *segs = nullptr;
    askit_status rc = knn_lists_init(N, &bd, &bi, s);
    cudaError_t e = cudaSuccess;
    if (rc == ASKIT_OK) {
        e = cudaMalloc(&order, sizeof(int32_t) * N);
        if (e == cudaSuccess) e = cudaMalloc(&segs, sizeof(int32_t) * 2 * nleaf);
        if (e == cudaSuccess) e = cudaMemcpyAsync(segs, h.data(), sizeof(int32_t) * 2 * nleaf, cudaMemcpyHostToDevice, s);
    }
    for (int it = 0; rc == ASKIT_OK && e == cudaSuccess && it < iters; ++it) {
        rc = build_tree_gpu(X, N, d, L, 1, seed, it, order, s);
        if (rc != ASKIT_OK) break;
        // queries of leaf b = its own points (ids in `order`), candidates = the same range
        knn_block_kernel<<<(unsigned)nleaf, 256, 8 * d * sizeof(float), s>>>(
            X, d, order, segs, segs + nleaf, order, nullptr, N, segs, segs + nleaf, bd, bi, kappa, true);
        e = cudaGetLastError();
    }
    if (rc == ASKIT_OK && e == cudaSuccess) {
        knn_extract_kernel<<<nblk(N * kappa, 256), 256, 0, s>>>(bd, bi, N, kappa, ids, dist);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (rc == ASKIT_OK && e != cudaSuccess) {
        askit_set_error("RP kNN: %s", cudaGetErrorString(e));
        rc = ASKIT_ERR_CUDA;
    }
    cudaFreeAsync(bd, s); cudaFreeAsync(bi, s); cudaFree(order); cudaFree(segs);
    return rc;
}

askit_status knn_dist_gpu(const float *X, int64_t N, int d, int kappa, const int32_t *ids,
                          double *dist, cudaStream_t s) {
    knn_dist_kernel<<<nblk(N * kappa, 256), 256, 0, s>>>(X, N, d, kappa, ids, dist);
    ASK_LAUNCH();
    return ASKIT_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free exact kNN (askit_knn_noalloc).
//
// The per-query best-32 lists live in this file-scope device array instead
// of memory from cudaMalloc: KNN_NOALLOC_MAX_Q queries x 32 slots x (8-byte
// distance + 4-byte id) = 3 MiB, held by every GPU that loads the library
// until the process exits.  Every call reuses it, so each call first resets
// the lists it uses, and calls that overlap on the GPU (on different
// streams, or from different threads) race on it.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t KNN_NOALLOC_MAX_Q = 8192;
constexpr int KNN_NOALLOC_QPB = 64;   // queries per block
static __device__ __align__(256) unsigned char g_knn_scratch[KNN_NOALLOC_MAX_Q * 32 * (sizeof(double) + sizeof(int))];

// Host-side address of g_knn_scratch on each device (the array's name is
// only a host stand-in; kernels must be given the device address).
std::mutex g_knn_scratch_mu;
void *g_knn_scratch_dev[64] = {nullptr};

askit_status knn_scratch_address(void **out) {
    int dev = 0;
    ASK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        askit_set_error("device ordinal %d out of range for the allocation-free kNN", dev);
        return ASKIT_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_knn_scratch_mu);
    if (!g_knn_scratch_dev[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_knn_scratch);
        if (e != cudaSuccess || !p) {
            askit_set_error("cudaGetSymbolAddress(knn scratch): %s", cudaGetErrorString(e));
            return ASKIT_ERR_CUDA;
        }
        g_knn_scratch_dev[dev] = p;
    }
    *out = g_knn_scratch_dev[dev];
    return ASKIT_OK;
}

// Exhaustive search of all N points for queries [64 b, 64 b + 64): one warp
// per query; Y == nullptr means the queries are the points themselves (self
// excluded).  Same FP64 distance and (D, id) order as the setup's kNN.
__global__ void knn_noalloc_kernel(const float *X, int64_t N, int d, const float *Y, int64_t Q, double *bd,
                                   int *bi, int kappa) {
    extern __shared__ float sq[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t q0 = (int64_t)blockIdx.x * KNN_NOALLOC_QPB;
    const int64_t q1 = q0 + KNN_NOALLOC_QPB < Q ? q0 + KNN_NOALLOC_QPB : Q;
    float *myq = sq + (int64_t)warp * d;
    for (int64_t q = q0 + warp; q < q1; q += nw) {
        const int64_t self = Y ? -1 : q;
        const float *xq = Y ? Y + q * d : X + q * d;
        for (int k = lane; k < d; k += 32) myq[k] = xq[k];
        __syncwarp();
        double ld = bd[q * 32 + lane];
        int li = bi[q * 32 + lane];
        for (int64_t cb = 0; cb < N; cb += 32) {
            double cd = DBL_MAX;
            int ci = INT_MAX;
            if (cb + lane < N && cb + lane != self) {
                const float *xj = X + (cb + lane) * d;
                double acc = 0.0;
                for (int k = 0; k < d; ++k) {
                    double t = c_sub((double)myq[k], (double)xj[k]);
                    acc = c_add(acc, c_mul(t, t));
                }
                cd = acc;
                ci = (int)(cb + lane);
            }
            warp_offer(ld, li, cd, ci, kappa, false, lane);
        }
        bd[q * 32 + lane] = ld;
        bi[q * 32 + lane] = li;
        __syncwarp();
    }
}

}  // namespace

extern "C" askit_status askit_knn_noalloc(const float *X_dev, int64_t N, int32_t d, const float *Y_dev, int64_t Q,
                                          int32_t kappa, int32_t *ids_dev, double *dist_dev, void *stream) {
    if (!X_dev || !ids_dev || !dist_dev) {
        askit_set_error("X_dev, ids_dev and dist_dev must be non-NULL");
        return ASKIT_ERR_INVALID_ARG;
    }
    if (N < 1 || d < 1 || Q < 1 || kappa < 1 || kappa > 32) {
        askit_set_error("need N >= 1, d >= 1, Q >= 1 and 1 <= kappa <= 32");
        return ASKIT_ERR_INVALID_ARG;
    }
    if (N >= ((int64_t)1 << 31) - 1024) {   // ids are int32 (the setup's bound)
        askit_set_error("askit_knn_noalloc handles N below 2^31 - 1024");
        return ASKIT_ERR_UNSUPPORTED;
    }
    if (Q > KNN_NOALLOC_MAX_Q) {
        askit_set_error("askit_knn_noalloc handles at most %lld queries per call (got %lld)",
                        (long long)KNN_NOALLOC_MAX_Q, (long long)Q);
        return ASKIT_ERR_INVALID_ARG;
    }
    if (!Y_dev && Q != N) {
        askit_set_error("with Y_dev == NULL the queries are the N points: Q must equal N");
        return ASKIT_ERR_INVALID_ARG;
    }
    if (kappa > (Y_dev ? N : N - 1)) {
        askit_set_error("kappa exceeds the number of candidate neighbors");
        return ASKIT_ERR_INVALID_ARG;
    }
    if ((size_t)8 * d * sizeof(float) > 48 * 1024) {
        askit_set_error("askit_knn_noalloc handles d <= %d", (int)(48 * 1024 / (8 * sizeof(float))));
        return ASKIT_ERR_UNSUPPORTED;
    }
    void *scratch = nullptr;
    ASK_TRY(knn_scratch_address(&scratch));
    double *bd = static_cast<double *>(scratch);
    int *bi = reinterpret_cast<int *>(bd + KNN_NOALLOC_MAX_Q * 32);
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's lists: reset the ones used here
    fill_kernel<double><<<nblk(Q * 32, 256), 256, 0, s>>>(bd, Q * 32, DBL_MAX);
    fill_kernel<int><<<nblk(Q * 32, 256), 256, 0, s>>>(bi, Q * 32, INT_MAX);
    knn_noalloc_kernel<<<(unsigned)((Q + KNN_NOALLOC_QPB - 1) / KNN_NOALLOC_QPB), 256, 8 * d * sizeof(float), s>>>(
        X_dev, N, d, Y_dev, Q, bd, bi, kappa);
    knn_extract_kernel<<<nblk(Q * kappa, 256), 256, 0, s>>>(bd, bi, Q, kappa, ids_dev, dist_dev);
    ASK_LAUNCH();
    return ASKIT_OK;
}
