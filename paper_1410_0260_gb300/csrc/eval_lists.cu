// Evaluation operands and work lists.
//
// Algorithm 4 visits, for target i, exactly the nodes of
//   U_i = union over j in {i} U N_i of the ancestors of leaf(j)
// (eq. (2.5): those nodes cannot be pruned).  The leaves of U_i are summed
// directly (Near(i)); every child of a node of U_i that is not itself in U_i
// is pruned and contributes through its skeleton (Far(i)).  The GPU forms
// every (target, source sub-block) pair of these sets -- an entry -- sorts
// the entries by (sub-block, target) and cuts each sub-block's run into work
// items of at most 128 targets (EvalItem: the sub-block's rows, the item's
// first entry and count), so every item is a dense tile of targets that all
// need the whole sub-block; one persistent kernel then runs all items and
// writes one partial sum per entry, reduced per target in a fixed order.
// Source sub-blocks are at most 128 contiguous rows: of a leaf's points in
// the tree-ordered coordinate array, or of a node's skeleton in the
// skeleton pool.
#include <limits.h>
#include <math.h>

#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "askit_impl.cuh"

namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Tree-ordered, zero-padded coordinates, squared norms (FP64 sum, rounded)
// and the per-source exponent scale c log2(e) / h_j^2.
__global__ void gather_rows_kernel(const float *X, int d, int d_pad, const int32_t *ids, int64_t n,
                                   int64_t n_rows, const float *hsrc, double kscale, float *out,
                                   float *nrm, float *sc) {
    int64_t row = blockIdx.x;
    if (row >= n_rows) return;
    int32_t id = row < n ? ids[row] : -1;
    for (int k = threadIdx.x; k < d_pad; k += blockDim.x)
        out[row * d_pad + k] = (id >= 0 && k < d) ? X[(int64_t)id * d + k] : 0.0f;
    if (threadIdx.x == 0) {
        double acc = 0.0;
        if (id >= 0)
            for (int k = 0; k < d; ++k) acc += (double)X[(int64_t)id * d + k] * X[(int64_t)id * d + k];
        nrm[row] = (float)acc;
        if (sc) {
            double h = id >= 0 ? (double)hsrc[id] : 1.0;
            sc[row] = id >= 0 ? (float)(kscale * 1.4426950408889634 / (h * h)) : 0.0f;
        }
    }
}

// Skeleton pool row ids: rows [spool[a], spool[a] + s_a) hold S_a, the
// padding up to a multiple of ASK_ROW_PAD is empty (-1).
__global__ void spool_ids_kernel(int64_t n_nodes, const int64_t *spool, const int64_t *skoff,
                                 const int32_t *s, const int32_t *skel_ids, int32_t *rows) {
    int64_t a = 2 + blockIdx.x;
    if (a >= n_nodes) return;
    int64_t r0 = spool[a], r1 = spool[a + 1];
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        int64_t q = r - r0;
        rows[r] = q < s[a] ? skel_ids[skoff[a] + q] : -1;
    }
}

// Adaptive kappa_i (the per-point selection Section 3 proposes from the
// distance to the neighbors): with a kernel cut a > 0, the neighbors kept in
// the prune set run up to the last rank whose kernel value exceeds e^-a,
// kappa_i = 1 + max{ z : c D_z / h_z^2 < a } (0 if none), h_z the
// neighbor's bandwidth, decided in canonical FP64 like the oracle; a <= 0
// keeps all kappa.
__device__ __forceinline__ int kappa_of(const double *dist, const int32_t *ids, int kappa, const float *hsrc,
                                        double kscale, double cut) {
    if (!(cut > 0.0)) return kappa;
    int ki = 0;
    for (int z = 0; z < kappa; ++z) {
        const double h = (double)hsrc[ids[z]];
        if (c_div(c_mul(kscale, dist[z]), c_mul(h, h)) < cut) ki = z + 1;
    }
    return ki;
}

// Prune set of each in-sample target (tree position q): the sorted distinct
// leaves of {i} U N_i (the first kappa_i neighbors), padded with INT_MAX to
// kappa + 1 entries.
__global__ void insample_sets_kernel(const int32_t *perm, const int32_t *leafof, const int32_t *knn,
                                     const double *knnd, const float *hsrc, double kscale, double cut,
                                     int64_t N, int kappa, int32_t *sets) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= N) return;
    int32_t i = perm[q];
    int32_t *o = sets + q * (kappa + 1);
    int n = 0;
    const int ki = kappa_of(knnd + (int64_t)i * kappa, knn + (int64_t)i * kappa, kappa, hsrc, kscale, cut);
    for (int z = -1; z < ki; ++z) {
        int32_t lf = leafof[z < 0 ? i : knn[(int64_t)i * kappa + z]];
        int p = n;
        bool dup = false;
        for (int u = 0; u < n; ++u) dup |= (o[u] == lf);
        if (dup) continue;
        while (p > 0 && o[p - 1] > lf) { o[p] = o[p - 1]; --p; }
        o[p] = lf;
        ++n;
    }
    for (int u = n; u < kappa + 1; ++u) o[u] = INT_MAX;
}

// Pruning switched off: every leaf is near for every target.
__global__ void all_leaves_sets_kernel(int64_t N, int L, int32_t *sets) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t M = (int64_t)1 << L;
    if (e >= N * M) return;
    sets[e] = (int32_t)(M + e % M);
}

// Leaf-grouped prune sets, step 1: for the point at tree position q, its
// own leaf and its neighbors' leaves, at q (kappa + 1) .. (q + 1)(kappa + 1);
// a leaf's points are consecutive positions, so each leaf owns one segment.
__global__ void leaf_keys_kernel(const int32_t *perm, const int32_t *leafof, const int32_t *knn, const double *knnd,
                                 const float *hsrc, double kscale, double cut, int64_t N, int kappa, int32_t *keys) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= N) return;
    const int32_t i = perm[q];
    int32_t *o = keys + q * (kappa + 1);
    o[0] = leafof[i];
    // neighbors past kappa_i repeat the own leaf (removed with the duplicates)
    const int ki = kappa_of(knnd + (int64_t)i * kappa, knn + (int64_t)i * kappa, kappa, hsrc, kscale, cut);
    for (int z = 0; z < kappa; ++z) o[z + 1] = z < ki ? leafof[knn[(int64_t)i * kappa + z]] : o[0];
}

// Step 2 (a warp per leaf, its segment sorted): count the distinct leaves
// (stride == 0), or write them to the leaf's row of `stride` entries padded
// with INT_MAX.
__global__ void leaf_unique_kernel(const int32_t *keys, const int32_t *beg, const int32_t *end, int stride,
                                   int32_t *rows, int32_t *cnt) {
    const int a = blockIdx.x, lane = threadIdx.x;
    const int32_t b0 = beg[a], b1 = end[a];
    int n = 0;
    for (int32_t base = b0; base < b1; base += 32) {
        const int32_t e = base + lane;
        const bool in = e < b1;
        const int32_t v = in ? keys[e] : 0;
        const bool first = in && (e == b0 || keys[e - 1] != v);
        const unsigned m = __ballot_sync(0xffffffffu, first);
        if (stride > 0 && first) rows[(int64_t)a * stride + n + __popc(m & ((1u << lane) - 1u))] = v;
        n += __popc(m);
    }
    if (stride > 0)
        for (int u = n + lane; u < stride; u += 32) rows[(int64_t)a * stride + u] = INT_MAX;
    else if (lane == 0)
        cnt[a] = n;
}

// Step 3: each target's row is its leaf's.
__global__ void leaf_row_kernel(const int32_t *perm, const int32_t *leafof, int64_t N, int32_t M, int32_t *row) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= N) return;
    row[q] = leafof[perm[q]] - M;
}

// Out-of-sample prune sets: distinct leaves of N_y (its first kappa_y
// neighbors; no self term).
__global__ void oos_sets_kernel(const int32_t *leafof, const int32_t *knn, const double *dist, const float *hsrc,
                                double kscale, double cut, int64_t T, int kappa, int stride, int32_t *sets) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= T) return;
    int32_t *o = sets + q * stride;
    int n = 0;
    const int ky = kappa_of(dist + q * kappa, knn + q * kappa, kappa, hsrc, kscale, cut);
    for (int z = 0; z < ky; ++z) {
        int32_t lf = leafof[knn[q * kappa + z]];
        int p = n;
        bool dup = false;
        for (int u = 0; u < n; ++u) dup |= (o[u] == lf);
        if (dup) continue;
        while (p > 0 && o[p - 1] > lf) { o[p] = o[p - 1]; --p; }
        o[p] = lf;
        ++n;
    }
    for (int u = n; u < stride; ++u) o[u] = INT_MAX;
}

// Near and Far sets of one target from its sorted prune leaves.  Near =
// the leaves; Far = for each depth, the sibling of every distinct ancestor
// at that depth when the sibling is not itself an ancestor of a near leaf.
// With a height limit fh >= 0 (skeletons only for nodes at most fh levels
// above the leaves, Section 3's level restriction), a higher Far node is
// replaced by its descendants fh levels above the leaves (none holds a near
// leaf).  emit(node, far) is called once per node of Near(i) and Far(i).
template <class F>
__device__ __forceinline__ void walk_lists(const int32_t *set, int stride, int L, int fh, F emit) {
    int n = 0;
    while (n < stride && set[n] != INT_MAX) ++n;
    for (int u = 0; u < n; ++u) emit(set[u], false);
    for (int depth = L; depth >= 1; --depth) {
        int sh = L - depth;
        for (int u = 0; u < n; ++u) {
            int32_t b = set[u] >> sh;
            if (u > 0 && (set[u - 1] >> sh) == b) continue;   // ancestor already handled
            int32_t sib = b ^ 1;
            // the set is sorted, so the leaves under sib form one run: find
            // the first leaf >= sib's first leaf
            const int32_t lo = sib << sh;
            int a = 0, z = n;
            while (a < z) {
                const int mid = (a + z) >> 1;
                if (set[mid] < lo) a = mid + 1; else z = mid;
            }
            const bool inU = a < n && (set[a] >> sh) == sib;
            if (inU) continue;
            if (fh >= 0 && sh > fh) {
                const int down = sh - fh;
                for (int32_t k = 0; k < ((int32_t)1 << down); ++k) emit((sib << down) + k, true);
            } else {
                emit(sib, true);
            }
        }
    }
}

// Source rows of a node's block: a leaf's points (near) or its skeleton (far).
__device__ __forceinline__ int block_rows(int32_t node, bool far, const int32_t *nsize, const int32_t *s) {
    return far ? s[node] : nsize[node];
}

// Entries are (target, source sub-block of <= ASK_BLK_N rows) pairs; the key
// of a sub-block is (node << 5) | (chunk << 1) | far.
__device__ __forceinline__ uint32_t sub_key(int32_t node, int chunk, bool far) {
    return ((uint32_t)node << 5) | ((uint32_t)chunk << 1) | (far ? 1u : 0u);
}

// Prune-set row of target q: its own row, or a shared one (leaf-grouped).
__device__ __forceinline__ const int32_t *set_of(const int32_t *sets, int stride, const int32_t *set_row, int64_t q) {
    return sets + (set_row ? (int64_t)set_row[q] : q) * stride;
}

__global__ void count_kernel(const int32_t *sets, int stride, const int32_t *set_row, int64_t T, int L, int fh,
                             const int32_t *nsize, const int32_t *s, int64_t *cnt, int64_t *nearc, int64_t *farc,
                             int64_t *pairs) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= T) return;
    int64_t c = 0, nf = 0, nn = 0, pr = 0;
    walk_lists(set_of(sets, stride, set_row, q), stride, L, fh, [&](int32_t node, bool far) {
        int rows = block_rows(node, far, nsize, s);
        c += (rows + ASK_BLK_N - 1) / ASK_BLK_N;
        pr += rows;
        if (far) ++nf; else ++nn;
    });
    cnt[q] = c;
    nearc[q] = nn;
    farc[q] = nf;
    pairs[q] = pr;
}

__global__ void emit_kernel(const int32_t *sets, int stride, const int32_t *set_row, int64_t T, int L, int fh,
                            const int32_t *nsize, const int32_t *s, const int64_t *off, uint64_t *keys,
                            int64_t *vals) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= T) return;
    int64_t o = off[q];
    walk_lists(set_of(sets, stride, set_row, q), stride, L, fh, [&](int32_t node, bool far) {
        int rows = block_rows(node, far, nsize, s);
        for (int ch = 0; ch * ASK_BLK_N < rows; ++ch) {
            keys[o] = ((uint64_t)sub_key(node, ch, far) << 32) | (uint64_t)q;
            vals[o] = o;
            ++o;
        }
    });
}

// After sorting by (sub-block, target): slot of every emitted entry, the
// target of every sorted entry, and the first entry of every sub-block.
__global__ void scatter_kernel(const uint64_t *keys, const int64_t *emit_of, int64_t n, int32_t *slot_of_emit,
                               int32_t *tgt, int64_t *bflag) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    slot_of_emit[emit_of[e]] = (int32_t)e;
    tgt[e] = (int32_t)(uint32_t)keys[e];
    bflag[e] = (e == 0 || (keys[e] >> 32) != (keys[e - 1] >> 32)) ? 1 : 0;
}

// Block index (inclusive scan of bflag minus one) and block starts.
__global__ void block_start_kernel(const int64_t *bflag, const int64_t *bidx_excl, int64_t n, int64_t *bstart) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    if (bflag[e]) bstart[bidx_excl[e]] = e;
}

__global__ void item_flag_kernel(const int64_t *bflag, const int64_t *bidx_excl, const int64_t *bstart, int64_t n,
                                 int64_t *iflag) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    int64_t b = bidx_excl[e] + bflag[e] - 1;
    iflag[e] = ((e - bstart[b]) % ASK_TILE_M) == 0 ? 1 : 0;
}

__global__ void build_items_kernel(const uint64_t *keys, const int64_t *bflag, const int64_t *bidx_excl,
                                   const int64_t *iflag, const int64_t *iidx_excl, int64_t n, int64_t nb,
                                   const int64_t *bstart, const int32_t *nstart, const int32_t *nsize,
                                   const int64_t *spool, const int32_t *s, const int32_t *leaf_cbase,
                                   const int32_t *node_cbase, int64_t leaf0, EvalItem *items, int32_t *block_off) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    int64_t b = bidx_excl[e] + bflag[e] - 1;
    if (bflag[e]) block_off[b] = (int32_t)iidx_excl[e];
    if (e == 0) block_off[nb] = (int32_t)(iidx_excl[n - 1] + iflag[n - 1]);
    if (!iflag[e]) return;
    uint32_t key = (uint32_t)(keys[e] >> 32);
    int32_t node = (int32_t)(key >> 5);
    int chunk = (int)((key >> 1) & 15);
    bool far = key & 1;
    int rows = far ? s[node] : nsize[node];
    int64_t bend = (b + 1 < nb) ? bstart[b + 1] : n;
    EvalItem x;
    x.row0 = (far ? (int32_t)spool[node] : nstart[node]) + chunk * ASK_BLK_N;
    x.nrows = min(ASK_BLK_N, rows - chunk * ASK_BLK_N) | (far ? (int32_t)0x80000000 : 0);
    x.e0 = (int32_t)e;
    x.cnt = (int32_t)((bend - e) < ASK_TILE_M ? (bend - e) : ASK_TILE_M);
    x.cidx = (far ? node_cbase[node] : leaf_cbase[node - leaf0]) + chunk;
    x.pad_[0] = x.pad_[1] = x.pad_[2] = 0;
    items[iidx_excl[e]] = x;
}

__global__ void reduce_partials_kernel(const float *partial, const int64_t *off, const int32_t *slot_of_emit,
                                       int64_t T, int r, const int32_t *out_rows, float *U, int64_t ldu) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= T * r) return;
    int64_t q = t / r;
    int z = (int)(t % r);
    float acc = 0.f;
    for (int64_t o = off[q]; o < off[q + 1]; ++o) acc += partial[(int64_t)slot_of_emit[o] * r + z];
    U[(int64_t)out_rows[q] * ldu + z] = acc;
}

}  // namespace

askit_status build_eval_operands(askit_tree t, cudaStream_t s) {
    const int64_t N = t->N;
    t->N_pad = (N + ASK_TILE_M - 1) / ASK_TILE_M * ASK_TILE_M + 256;
    ASK_TRY(t->arena.alloc(&t->Xt, (size_t)t->N_pad * t->d_pad));
    ASK_TRY(t->arena.alloc(&t->nrm_t, t->N_pad));
    ASK_TRY(t->arena.alloc(&t->sc_t, t->N_pad));
    gather_rows_kernel<<<(unsigned)t->N_pad, 128, 0, s>>>(t->X, t->d, t->d_pad, t->perm, N, t->N_pad, t->hsrc,
                                                         t->prm.kernel_scale, t->Xt, t->nrm_t, t->sc_t);
    ASK_LAUNCH();
    int64_t rows = std::max<int64_t>(t->spool_rows, 1) + 256;
    int32_t *ids = nullptr;
    ASK_TRY(t->arena.alloc(&ids, rows));
    ASK_CUDA(cudaMemsetAsync(ids, 0xff, sizeof(int32_t) * rows, s));
    if (t->n_nodes > 2)
        spool_ids_kernel<<<(unsigned)(t->n_nodes - 2), 128, 0, s>>>(t->n_nodes, t->d_spool, t->d_skoff, t->d_s,
                                                                   t->skel_ids, ids);
    ASK_LAUNCH();
    ASK_TRY(t->arena.alloc(&t->Xs, (size_t)rows * t->d_pad));
    ASK_TRY(t->arena.alloc(&t->nrm_s, rows));
    ASK_TRY(t->arena.alloc(&t->sc_s, rows));
    gather_rows_kernel<<<(unsigned)rows, 128, 0, s>>>(t->X, t->d, t->d_pad, ids, rows, rows, t->hsrc,
                                                     t->prm.kernel_scale, t->Xs, t->nrm_s, t->sc_s);
    ASK_LAUNCH();
    ASK_CUDA(cudaStreamSynchronize(s));
    t->arena.release(ids);
    return ASKIT_OK;
}

// One CTA per source sub-block: its center (FP64 mean of the rows of the
// sub-block's node, rounded), the centered rows split for the tensor cores -- TF32 (narrow
// rows only): hi = the FP32 value with the 13 low mantissa bits cleared,
// lo = x - hi; BF16: hi = bf16(x), lo = bf16(x - hi); FP16 likewise on the
// prescaled value -- and the squared norms of the centered rows.  Rows are
// kw wide (zeros past d); one warp per row, lanes across the columns.  Wide
// rows (kgplanes) store the 16-bit splits as planes of K groups,
// [kw / 8][rows_total][8], so that a K chunk of consecutive rows is a few
// contiguous runs (the wide kernel's TMA boxes).
__global__ void tc_prep_kernel(const float *X, int d_pad, int kw, bool kgplanes, const int64_t *sb_row0,
                               const int32_t *sb_nrows,
                               const int64_t *nd_row0, const int32_t *nd_nrows, int64_t rows_total, float f16_scale,
                               float *cent, float *Xhi, float *Xlo, uint16_t *Bhi, uint16_t *Blo, uint16_t *Hhi,
                               uint16_t *Hlo, float *nrmc) {
    extern __shared__ float c[];   // [kw]
    const int g = blockIdx.x;
    const int64_t r0 = sb_row0[g];
    const int nr = sb_nrows[g];
    // the center is the mean of the whole node (leaf or skeleton) the
    // sub-block belongs to, so that all sub-blocks of a node share it
    const int64_t n0 = nd_row0[g];
    const int nn = nd_nrows[g];
    for (int k = threadIdx.x; k < kw; k += blockDim.x) {
        double acc = 0.0;
        if (k < d_pad)
            for (int q = 0; q < nn; ++q) acc += (double)X[(n0 + q) * d_pad + k];
        c[k] = nn > 0 ? (float)(acc / nn) : 0.f;
        cent[(int64_t)g * kw + k] = c[k];
    }
    __syncthreads();
    // only the sub-block's own rows: the 128-row window of a short sub-block
    // overlaps the next one, whose rows its own CTA writes
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = warp; q < nr; q += nw) {
        const int64_t row = r0 + q;
        if (row >= rows_total) break;
        double nn = 0.0;
        for (int k = lane; k < kw; k += 32) {
            const float x = (k < d_pad) ? X[row * d_pad + k] - c[k] : 0.f;
            nn += (double)x * x;
            const int64_t o = kgplanes ? (((int64_t)(k >> 3) * rows_total + row) << 3) + (k & 7) : row * kw + k;
            if (Xhi) {
                const float hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
                Xhi[o] = hi;
                Xlo[o] = x - hi;
            }
            const __nv_bfloat16 bh = __float2bfloat16_rn(x);
            const __nv_bfloat16 bl = __float2bfloat16_rn(x - __bfloat162float(bh));
            Bhi[o] = __bfloat16_as_ushort(bh);
            Blo[o] = __bfloat16_as_ushort(bl);
            const float xs = x * f16_scale;
            const __half hh = __float2half_rn(xs);
            const __half hl = __float2half_rn(xs - __half2float(hh));
            Hhi[o] = __half_as_ushort(hh);
            Hlo[o] = __half_as_ushort(hl);
        }
        for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
        if (lane == 0) nrmc[row] = (float)nn;
    }
}

// Largest |x_k| over the data (bounds every centered coordinate by twice it).
__global__ void extent_kernel(const float *X, int64_t N, int d, float *ext) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float v = e < N * d ? fabsf(X[e]) : 0.f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(ext), __float_as_int(v));
}

askit_status build_tc_operands(askit_tree t, cudaStream_t s) {
    const int64_t nn = t->n_nodes, M = (int64_t)1 << t->L;
    std::vector<int32_t> lcb(M), ncb(nn, 0);
    std::vector<int64_t> r0;
    std::vector<int32_t> nr;
    std::vector<int64_t> node_r0;    // per sub-block: first row and rows of its node
    std::vector<int32_t> node_nr;    //   (every sub-block of a node shares the node's center)
    std::vector<int64_t> sub_node;   // per sub-block: heap index of its node
    for (int64_t l = 0; l < M; ++l) {
        lcb[l] = (int32_t)r0.size();
        int64_t a = M + l, sz = t->h_size[a];
        for (int64_t ch = 0; ch * ASK_BLK_N < sz; ++ch) {
            r0.push_back(t->h_start[a] + ch * ASK_BLK_N);
            nr.push_back((int32_t)std::min<int64_t>(ASK_BLK_N, sz - ch * ASK_BLK_N));
            node_r0.push_back(t->h_start[a]);
            node_nr.push_back((int32_t)sz);
            sub_node.push_back(a);
        }
    }
    int64_t n_leaf_sub = (int64_t)r0.size();
    for (int64_t a = 2; a < nn; ++a) {
        ncb[a] = (int32_t)(r0.size() - n_leaf_sub);
        int64_t sz = t->h_s[a];
        for (int64_t ch = 0; ch * ASK_BLK_N < sz; ++ch) {
            r0.push_back(t->h_spool[a] + ch * ASK_BLK_N);
            nr.push_back((int32_t)std::min<int64_t>(ASK_BLK_N, sz - ch * ASK_BLK_N));
            node_r0.push_back(t->h_spool[a]);
            node_nr.push_back((int32_t)sz);
            sub_node.push_back(a);
        }
    }
    for (int64_t a = 2; a < nn; ++a) ncb[a] += (int32_t)n_leaf_sub;
    t->n_sub = (int64_t)r0.size();
    // schedule order of the sub-blocks: the tree position of their node's
    // first point (leaf sub-blocks: their own first row), then their index
    t->h_sub_node = sub_node;
    t->h_sub_pos.assign(t->n_sub, 0);
    for (int64_t q = 0; q < n_leaf_sub; ++q) t->h_sub_pos[q] = r0[q];
    for (int64_t a = 2; a < nn; ++a)
        for (int64_t ch = 0; ch * ASK_BLK_N < t->h_s[a]; ++ch) t->h_sub_pos[ncb[a] + ch] = t->h_start[a];
    ASK_TRY(t->arena.alloc(&t->leaf_cbase, M));
    ASK_TRY(t->arena.alloc(&t->node_cbase, nn));
    ASK_CUDA(cudaMemcpyAsync(t->leaf_cbase, lcb.data(), sizeof(int32_t) * M, cudaMemcpyHostToDevice, s));
    ASK_CUDA(cudaMemcpyAsync(t->node_cbase, ncb.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice, s));
    // narrow rows (d <= TC_K) get TC_K columns and all three splits; wide
    // rows keep their d_pad columns (a multiple of 32, the K chunk of the
    // wide kernel) and get the 16-bit splits only
    const bool wide = t->d > TC_K;
    const int kw = wide ? t->d_pad : TC_K;
    if (kw > 8192) return ASKIT_OK;     // no tensor-core operands (plain FP32 path only)
    t->kw = kw;
    ASK_TRY(t->arena.alloc(&t->sb_row0, std::max<int64_t>(1, t->n_sub)));
    ASK_TRY(t->arena.alloc(&t->sb_nr, std::max<int64_t>(1, t->n_sub)));
    ASK_CUDA(cudaMemcpyAsync(t->sb_row0, r0.data(), sizeof(int64_t) * t->n_sub, cudaMemcpyHostToDevice, s));
    ASK_CUDA(cudaMemcpyAsync(t->sb_nr, nr.data(), sizeof(int32_t) * t->n_sub, cudaMemcpyHostToDevice, s));
    t->n_leaf_sub = n_leaf_sub;
    int64_t *d_r0 = t->sb_row0;
    int32_t *d_nr = t->sb_nr;
    int64_t *d_nd0 = nullptr;
    int32_t *d_ndn = nullptr;
    ASK_CUDA(cudaMallocAsync(&d_nd0, sizeof(int64_t) * std::max<int64_t>(1, t->n_sub), s));
    ASK_CUDA(cudaMallocAsync(&d_ndn, sizeof(int32_t) * std::max<int64_t>(1, t->n_sub), s));
    ASK_CUDA(cudaMemcpyAsync(d_nd0, node_r0.data(), sizeof(int64_t) * t->n_sub, cudaMemcpyHostToDevice, s));
    ASK_CUDA(cudaMemcpyAsync(d_ndn, node_nr.data(), sizeof(int32_t) * t->n_sub, cudaMemcpyHostToDevice, s));
    t->srows = std::max<int64_t>(t->spool_rows, 1) + 256;
    const size_t et = (size_t)t->N_pad * kw, es = (size_t)t->srows * kw;
    ASK_TRY(t->arena.alloc(&t->cent, (size_t)std::max<int64_t>(1, t->n_sub) * kw));
    if (!wide) {
        ASK_TRY(t->arena.alloc(&t->Xt_hi, et));
        ASK_TRY(t->arena.alloc(&t->Xt_lo, et));
        ASK_TRY(t->arena.alloc(&t->Xs_hi, es));
        ASK_TRY(t->arena.alloc(&t->Xs_lo, es));
        ASK_CUDA(cudaMemsetAsync(t->Xt_hi, 0, sizeof(float) * et, s));
        ASK_CUDA(cudaMemsetAsync(t->Xt_lo, 0, sizeof(float) * et, s));
        ASK_CUDA(cudaMemsetAsync(t->Xs_hi, 0, sizeof(float) * es, s));
        ASK_CUDA(cudaMemsetAsync(t->Xs_lo, 0, sizeof(float) * es, s));
    }
    uint16_t **h16[8] = {&t->Xt_bhi, &t->Xt_blo, &t->Xt_hhi, &t->Xt_hlo, &t->Xs_bhi, &t->Xs_blo, &t->Xs_hhi, &t->Xs_hlo};
    for (int i = 0; i < 8; ++i) {
        const size_t n = i < 4 ? et : es;
        ASK_TRY(t->arena.alloc(h16[i], n));
        ASK_CUDA(cudaMemsetAsync(*h16[i], 0, sizeof(uint16_t) * n, s));
    }
    ASK_TRY(t->arena.alloc(&t->nrmc_t, t->N_pad));
    ASK_TRY(t->arena.alloc(&t->nrmc_s, t->srows));
    ASK_CUDA(cudaMemsetAsync(t->nrmc_t, 0, sizeof(float) * t->N_pad, s));
    ASK_CUDA(cudaMemsetAsync(t->nrmc_s, 0, sizeof(float) * t->srows, s));
    // FP16 prescale: a power of 2 that maps the data's widest coordinate
    // range to at most 2^14, so centered values and their differences stay
    // far below the FP16 maximum (65504)
    {
        float *ext = nullptr;
        ASK_CUDA(cudaMalloc(&ext, sizeof(float)));
        ASK_CUDA(cudaMemsetAsync(ext, 0, sizeof(float), s));
        extent_kernel<<<(unsigned)((t->N * t->d + 255) / 256), 256, 0, s>>>(t->X, t->N, t->d, ext);
        float hext = 0.f;
        ASK_CUDA(cudaMemcpyAsync(&hext, ext, sizeof(float), cudaMemcpyDeviceToHost, s));
        ASK_CUDA(cudaStreamSynchronize(s));
        cudaFree(ext);
        int e = 0;
        if (hext > 0.f) frexpf(16384.f / (2.f * hext), &e);
        t->f16_scale = ldexpf(1.f, e - 1);
    }
    const size_t csm = sizeof(float) * kw;
    if (n_leaf_sub > 0)
        tc_prep_kernel<<<(unsigned)n_leaf_sub, 256, csm, s>>>(t->Xt, t->d_pad, kw, wide, d_r0, d_nr, d_nd0, d_ndn, t->N_pad,
                                                            t->f16_scale, t->cent, t->Xt_hi, t->Xt_lo, t->Xt_bhi,
                                                            t->Xt_blo, t->Xt_hhi, t->Xt_hlo, t->nrmc_t);
    if (t->n_sub > n_leaf_sub)
        tc_prep_kernel<<<(unsigned)(t->n_sub - n_leaf_sub), 256, csm, s>>>(
            t->Xs, t->d_pad, kw, wide, d_r0 + n_leaf_sub, d_nr + n_leaf_sub, d_nd0 + n_leaf_sub, d_ndn + n_leaf_sub,
            t->srows, t->f16_scale, t->cent + n_leaf_sub * kw, t->Xs_hi, t->Xs_lo, t->Xs_bhi, t->Xs_blo, t->Xs_hhi,
            t->Xs_hlo, t->nrmc_s);
    ASK_LAUNCH();
    cudaFreeAsync(d_nd0, s);
    cudaFreeAsync(d_ndn, s);
    ASK_CUDA(cudaStreamSynchronize(s));
    if (!wide) ASK_TRY(build_g16_operands(t, s));
    return ASKIT_OK;
}

void free_prune_sets(PruneSets &ps) {
    if (ps.sets) cudaFree(ps.sets);
    if (ps.set_row) cudaFree(ps.set_row);
    ps = PruneSets();
}

// Leaf-grouped prune sets: the sorted distinct leaves of {p} U N_p over the
// points p of each leaf (one row per leaf), and every target's row index.
askit_status leaf_prune_sets(askit_tree t, PruneSets &ps, cudaStream_t s) {
    const int64_t N = t->N, M = (int64_t)1 << t->L, k1 = t->kappa + 1;
    if (N * k1 >= ((int64_t)1 << 31)) {
        askit_set_error("leaf-grouped lists need N (kappa + 1) < 2^31");
        return ASKIT_ERR_UNSUPPORTED;
    }
    int32_t *keys = nullptr, *keys_s = nullptr, *beg = nullptr, *cnt = nullptr;
    void *tmp = nullptr;
    size_t tb = 0;
    askit_status rc = ASKIT_OK;
    std::vector<int32_t> hb(2 * M), hc(M);
    for (int64_t a = 0; a < M; ++a) {
        hb[a] = (int32_t)(t->h_start[M + a] * k1);
        hb[M + a] = (int32_t)((t->h_start[M + a] + t->h_size[M + a]) * k1);
    }
    int mx = 0;
#define PCHK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { askit_set_error("leaf prune sets: %s", cudaGetErrorString(e_)); rc = e_ == cudaErrorMemoryAllocation ? ASKIT_ERR_OOM : ASKIT_ERR_CUDA; goto out; } } while (0)
#define PTRY(x) do { rc = (x); if (rc != ASKIT_OK) goto out; } while (0)
    PCHK(cudaMalloc(&keys, sizeof(int32_t) * N * k1));
    PCHK(cudaMalloc(&keys_s, sizeof(int32_t) * N * k1));
    PCHK(cudaMalloc(&beg, sizeof(int32_t) * 2 * M));
    PCHK(cudaMalloc(&cnt, sizeof(int32_t) * M));
    PCHK(cudaMemcpyAsync(beg, hb.data(), sizeof(int32_t) * 2 * M, cudaMemcpyHostToDevice, s));
    leaf_keys_kernel<<<nblk(N, 128), 128, 0, s>>>(t->perm, t->leafof, t->knn, t->knnd, t->hsrc, t->prm.kernel_scale,
                                                  t->kappa_cut, N, t->kappa, keys);
    PCHK(cudaGetLastError());
    PTRY(seg_sort_i32(nullptr, nullptr, N * k1, (int)M, beg, beg + M, nullptr, &tb, s));
    PCHK(cudaMalloc(&tmp, tb));
    PTRY(seg_sort_i32(keys, keys_s, N * k1, (int)M, beg, beg + M, tmp, &tb, s));
    leaf_unique_kernel<<<(unsigned)M, 32, 0, s>>>(keys_s, beg, beg + M, 0, nullptr, cnt);
    PCHK(cudaGetLastError());
    PCHK(cudaMemcpyAsync(hc.data(), cnt, sizeof(int32_t) * M, cudaMemcpyDeviceToHost, s));
    PCHK(cudaStreamSynchronize(s));
    for (int64_t a = 0; a < M; ++a) mx = std::max(mx, hc[a]);
    ps.stride = std::max(mx, 1);
    PCHK(cudaMalloc(&ps.sets, sizeof(int32_t) * M * ps.stride));
    PCHK(cudaMalloc(&ps.set_row, sizeof(int32_t) * N));
    leaf_unique_kernel<<<(unsigned)M, 32, 0, s>>>(keys_s, beg, beg + M, ps.stride, ps.sets, cnt);
    leaf_row_kernel<<<nblk(N, 256), 256, 0, s>>>(t->perm, t->leafof, N, (int32_t)M, ps.set_row);
    PCHK(cudaGetLastError());
    PCHK(cudaStreamSynchronize(s));
out:
#undef PCHK
#undef PTRY
    for (void *q : {(void *)keys, (void *)keys_s, (void *)beg, (void *)cnt, tmp})
        if (q) cudaFree(q);
    if (rc != ASKIT_OK) free_prune_sets(ps);
    return rc;
}

askit_status insample_prune_sets(askit_tree t, PruneSets &ps, cudaStream_t s) {
    if (t->prm.prune == 2) return leaf_prune_sets(t, ps, s);
    // {i} U N_i as leaves; with pruning off, every leaf
    ps.stride = t->prm.prune ? t->kappa + 1 : (int)((int64_t)1 << t->L);
    ps.set_row = nullptr;
    ASK_CUDA(cudaMalloc(&ps.sets, sizeof(int32_t) * t->N * ps.stride));
    if (!t->prm.prune) {
        int64_t n = t->N << t->L;
        all_leaves_sets_kernel<<<nblk(n, 256), 256, 0, s>>>(t->N, t->L, ps.sets);
        ASK_LAUNCH();
        return ASKIT_OK;
    }
    insample_sets_kernel<<<nblk(t->N, 128), 128, 0, s>>>(t->perm, t->leafof, t->knn, t->knnd, t->hsrc,
                                                         t->prm.kernel_scale, t->kappa_cut, t->N, t->kappa, ps.sets);
    ASK_LAUNCH();
    return ASKIT_OK;
}

askit_status oos_prune_sets(askit_tree t, const int32_t *knn, const double *dist, int64_t T, int stride,
                            int32_t *sets, cudaStream_t s) {
    oos_sets_kernel<<<nblk(T, 128), 128, 0, s>>>(t->leafof, knn, dist, t->hsrc, t->prm.kernel_scale, t->kappa_cut, T,
                                                 t->kappa, stride, sets);
    ASK_LAUNCH();
    return ASKIT_OK;
}

// Work lists for T targets (slot order) with the given prune sets: every
// (target, source sub-block) pair becomes an entry; entries are sorted by
// (sub-block, target); each sub-block's entries are cut into items of up to
// ASK_TILE_M targets.  partial[e] receives the sub-block's contribution to
// the entry's target; reduce() then sums each target's entries in emission
// order (Near leaves ascending, then Far nodes from the deepest level up),
// which is fixed, so the result does not depend on scheduling.
askit_status build_work_lists(askit_tree t, const int32_t *sets, int stride, const int32_t *set_row, int64_t T,
                              WorkLists &wlst, DevArena &arena, cudaStream_t s) {
    int64_t *cnt = nullptr, *nearc = nullptr, *farc = nullptr, *pairs = nullptr, *vals = nullptr, *emit_of = nullptr;
    int64_t *bflag = nullptr, *bidx = nullptr, *bstart = nullptr, *iflag = nullptr, *iidx = nullptr;
    uint64_t *keys = nullptr, *keys_s = nullptr;
    void *tmp = nullptr;
    size_t tb = 0, tb2 = 0;
    askit_status rc = ASKIT_OK;
    cudaError_t e = cudaSuccess;
    int64_t total = 0, nb = 0, nit = 0;
    std::vector<int64_t> h_near(T), h_far(T), h_pairs(T);
    WorkLists &w = wlst;
    w.T = T;
#define WCHK(x) do { e = (x); if (e != cudaSuccess) goto fail; } while (0)
#define WTRY(x) do { rc = (x); if (rc != ASKIT_OK) goto out; } while (0)
    WCHK(cudaMallocAsync(&cnt, sizeof(int64_t) * (T + 1), s));
    WCHK(cudaMallocAsync(&nearc, sizeof(int64_t) * T, s));
    WCHK(cudaMallocAsync(&farc, sizeof(int64_t) * T, s));
    WCHK(cudaMallocAsync(&pairs, sizeof(int64_t) * T, s));
    WTRY(arena.alloc(&w.off, T + 1));
    WCHK(cudaMemsetAsync(cnt + T, 0, sizeof(int64_t), s));
    count_kernel<<<nblk(T, 128), 128, 0, s>>>(sets, stride, set_row, T, t->L, t->far_height, t->nsize, t->d_s, cnt,
                                              nearc, farc,
                                              pairs);
    WCHK(cudaGetLastError());
    WTRY(scan_i64(nullptr, nullptr, T + 1, nullptr, &tb, s));
    WCHK(cudaMallocAsync(&tmp, tb, s));
    WTRY(scan_i64(cnt, w.off, T + 1, tmp, &tb, s));
    WCHK(cudaMemcpyAsync(&total, w.off + T, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    WCHK(cudaMemcpyAsync(h_near.data(), nearc, sizeof(int64_t) * T, cudaMemcpyDeviceToHost, s));
    WCHK(cudaMemcpyAsync(h_far.data(), farc, sizeof(int64_t) * T, cudaMemcpyDeviceToHost, s));
    WCHK(cudaMemcpyAsync(h_pairs.data(), pairs, sizeof(int64_t) * T, cudaMemcpyDeviceToHost, s));
    WCHK(cudaStreamSynchronize(s));
    cudaFreeAsync(tmp, s);
    tmp = nullptr;
    w.n_entries = total;
    if (total >= ((int64_t)1 << 31)) {
        // entry offsets (work items, slots) are 32-bit
        askit_set_error("%lld (target, sub-block) entries in one work list; at most 2^31 - 1 (lower batch_entries)",
                        (long long)total);
        rc = ASKIT_ERR_UNSUPPORTED;
        goto out;
    }
    WCHK(cudaMallocAsync(&keys, sizeof(uint64_t) * total, s));
    WCHK(cudaMallocAsync(&keys_s, sizeof(uint64_t) * total, s));
    WCHK(cudaMallocAsync(&vals, sizeof(int64_t) * total, s));
    WCHK(cudaMallocAsync(&emit_of, sizeof(int64_t) * total, s));
    emit_kernel<<<nblk(T, 128), 128, 0, s>>>(sets, stride, set_row, T, t->L, t->far_height, t->nsize, t->d_s, w.off,
                                             keys, vals);
    WCHK(cudaGetLastError());
    WTRY(sort_u64_i64(nullptr, nullptr, nullptr, nullptr, total, nullptr, &tb, s));
    WTRY(scan_i64(nullptr, nullptr, total, nullptr, &tb2, s));
    tb = std::max(tb, tb2);
    WCHK(cudaMallocAsync(&tmp, tb, s));
    WTRY(sort_u64_i64(keys, keys_s, vals, emit_of, total, tmp, &tb, s));
    WTRY(arena.alloc(&w.slot_of_emit, total));
    WTRY(arena.alloc(&w.tgt, total));
    WCHK(cudaMallocAsync(&bflag, sizeof(int64_t) * total, s));
    WCHK(cudaMallocAsync(&bidx, sizeof(int64_t) * total, s));
    WCHK(cudaMallocAsync(&iflag, sizeof(int64_t) * total, s));
    WCHK(cudaMallocAsync(&iidx, sizeof(int64_t) * total, s));
    scatter_kernel<<<nblk(total, 256), 256, 0, s>>>(keys_s, emit_of, total, w.slot_of_emit, w.tgt, bflag);
    WCHK(cudaGetLastError());
    WTRY(scan_i64(bflag, bidx, total, tmp, &tb, s));
    {
        int64_t lastb = 0, lastf = 0;
        WCHK(cudaMemcpyAsync(&lastb, bidx + total - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        WCHK(cudaMemcpyAsync(&lastf, bflag + total - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        WCHK(cudaStreamSynchronize(s));
        nb = lastb + lastf;
    }
    WCHK(cudaMallocAsync(&bstart, sizeof(int64_t) * nb, s));
    block_start_kernel<<<nblk(total, 256), 256, 0, s>>>(bflag, bidx, total, bstart);
    item_flag_kernel<<<nblk(total, 256), 256, 0, s>>>(bflag, bidx, bstart, total, iflag);
    WCHK(cudaGetLastError());
    WTRY(scan_i64(iflag, iidx, total, tmp, &tb, s));
    {
        int64_t lasti = 0, lastf = 0;
        WCHK(cudaMemcpyAsync(&lasti, iidx + total - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        WCHK(cudaMemcpyAsync(&lastf, iflag + total - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        WCHK(cudaStreamSynchronize(s));
        nit = lasti + lastf;
    }
    WTRY(arena.alloc(&w.items, nit));
    WTRY(arena.alloc(&w.block_off, nb + 1));
    build_items_kernel<<<nblk(total, 256), 256, 0, s>>>(keys_s, bflag, bidx, iflag, iidx, total, nb, bstart, t->nstart,
                                                        t->nsize, t->d_spool, t->d_s, t->leaf_cbase, t->node_cbase,
                                                        (int64_t)1 << t->L, w.items, w.block_off);
    WCHK(cudaGetLastError());
    {
        std::vector<EvalItem> hi(nit);
        std::vector<int32_t> boff(nb + 1);
        WCHK(cudaMemcpyAsync(hi.data(), w.items, sizeof(EvalItem) * nit, cudaMemcpyDeviceToHost, s));
        WCHK(cudaMemcpyAsync(boff.data(), w.block_off, sizeof(int32_t) * (nb + 1), cudaMemcpyDeviceToHost, s));
        WCHK(cudaStreamSynchronize(s));
        std::vector<int64_t> cost(nb, 0);
        int64_t pc = 0;
        for (int64_t b = 0; b < nb; ++b)
            for (int32_t it = boff[b]; it < boff[b + 1]; ++it) {
                cost[b] += ASK_TILE_M * ASK_BLK_N;
                pc += (int64_t)ASK_TILE_M * ASK_BLK_N;
            }
        std::vector<int32_t> order(nb);
        for (int64_t b = 0; b < nb; ++b) order[b] = (int32_t)b;
        std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return cost[x] > cost[y]; });
        WTRY(arena.alloc(&w.block_order, nb));
        WCHK(cudaMemcpyAsync(w.block_order, order.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s));
        // Two schedules over one persistent CTA per SM (a sub-block costs its
        // items plus a fixed reload of its source tile); askit_autotune picks.
        //  0: LPT -- heaviest first, each to the least-loaded CTA;
        //  1: tree order -- sub-blocks taken in their node's tree order, each
        //     to the least-loaded CTA: the CTAs advance through the tree
        //     together, so the sub-blocks in flight at any time on all SMs
        //     share most of their targets (L2 reuse of target rows).
        int dev = 0, sms = 0;
        WCHK(cudaGetDevice(&dev));
        WCHK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int nc = (int)std::max<int64_t>(1, std::min<int64_t>(nb, sms));
        auto bcost = [&](int32_t b) { return (int64_t)(boff[b + 1] - boff[b]) * 4 + 3; };
        std::vector<int32_t> coff[3], cblk[3];
        {
            std::vector<std::vector<int32_t>> lists(nc);
            std::vector<std::pair<int64_t, int>> heap;   // (load, cta), min-heap
            for (int c = 0; c < nc; ++c) heap.push_back({0, c});
            auto cmp = [](const std::pair<int64_t, int> &x, const std::pair<int64_t, int> &y) {
                return x.first > y.first || (x.first == y.first && x.second > y.second);
            };
            std::make_heap(heap.begin(), heap.end(), cmp);
            for (int64_t q = 0; q < nb; ++q) {
                const int32_t bq = order[q];
                std::pop_heap(heap.begin(), heap.end(), cmp);
                auto top = heap.back();
                heap.pop_back();
                lists[top.second].push_back(bq);
                top.first += bcost(bq);
                heap.push_back(top);
                std::push_heap(heap.begin(), heap.end(), cmp);
            }
            coff[0].assign(nc + 1, 0);
            for (int c = 0; c < nc; ++c) {
                coff[0][c + 1] = coff[0][c] + (int32_t)lists[c].size();
                cblk[0].insert(cblk[0].end(), lists[c].begin(), lists[c].end());
            }
        }
        {
            std::vector<int64_t> bpos(nb, 0);
            for (int64_t b = 0; b < nb; ++b) {
                const int32_t cx = hi[boff[b]].cidx;
                bpos[b] = (cx >= 0 && cx < (int32_t)t->h_sub_pos.size()) ? t->h_sub_pos[cx] : 0;
            }
            std::vector<int32_t> tord(nb);
            for (int64_t b = 0; b < nb; ++b) tord[b] = (int32_t)b;
            std::stable_sort(tord.begin(), tord.end(), [&](int32_t x, int32_t y) { return bpos[x] < bpos[y]; });
            std::vector<std::vector<int32_t>> lists(nc);
            std::vector<std::pair<int64_t, int>> heap;   // (load, cta), min-heap
            for (int c = 0; c < nc; ++c) heap.push_back({0, c});
            auto cmp = [](const std::pair<int64_t, int> &x, const std::pair<int64_t, int> &y) {
                return x.first > y.first || (x.first == y.first && x.second > y.second);
            };
            std::make_heap(heap.begin(), heap.end(), cmp);
            for (int64_t q = 0; q < nb; ++q) {
                std::pop_heap(heap.begin(), heap.end(), cmp);
                auto top = heap.back();
                heap.pop_back();
                lists[top.second].push_back(tord[q]);
                top.first += bcost(tord[q]);
                heap.push_back(top);
                std::push_heap(heap.begin(), heap.end(), cmp);
            }
            coff[1].assign(nc + 1, 0);
            for (int c = 0; c < nc; ++c) {
                coff[1][c + 1] = coff[1][c] + (int32_t)lists[c].size();
                cblk[1].insert(cblk[1].end(), lists[c].begin(), lists[c].end());
            }
        }
        // Pairs: sub-blocks 2k and 2k+1 of one node need the same targets (a
        // target needing a node needs all its sub-blocks), so their items
        // match one to one; the FP16x3 kernel can take both in one 256-column
        // item.  The leader keeps its items, the follower's are skipped.
        std::vector<int32_t> partner(nb, -1);
        std::vector<char> follower(nb, 0);
        if (!t->h_sub_node.empty()) {
            std::vector<int32_t> blk_of_sub(t->h_sub_node.size(), -1);
            for (int64_t b = 0; b < nb; ++b) {
                const int32_t cx = hi[boff[b]].cidx;
                if (cx >= 0 && cx < (int32_t)blk_of_sub.size()) blk_of_sub[cx] = (int32_t)b;
            }
            for (int64_t b = 0; b < nb; ++b) {
                const int32_t cx = hi[boff[b]].cidx;
                if (cx < 0 || cx + 1 >= (int32_t)t->h_sub_node.size()) continue;
                const int64_t node = t->h_sub_node[cx];
                if (t->h_sub_node[cx + 1] != node) continue;
                int32_t first = cx;
                while (first > 0 && t->h_sub_node[first - 1] == node) --first;
                if ((cx - first) & 1) continue;           // odd position in its node
                const int32_t b2 = blk_of_sub[cx + 1];
                if (b2 < 0 || boff[b2 + 1] - boff[b2] != boff[b + 1] - boff[b]) continue;
                // a leader is never the last sub-block of its node, so it is
                // full and its follower's rows start 128 rows later
                bool same = (hi[boff[b]].nrows & 0x7fffffff) == ASK_BLK_N;
                for (int32_t k = 0; same && k < boff[b + 1] - boff[b]; ++k)
                    same = hi[boff[b] + k].cnt == hi[boff[b2] + k].cnt;
                if (!same) continue;
                partner[b] = b2;
                follower[b2] = 1;
            }
        }
        {
            std::vector<std::vector<int32_t>> lists(nc);
            std::vector<std::pair<int64_t, int>> heap;
            for (int c = 0; c < nc; ++c) heap.push_back({0, c});
            auto cmp = [](const std::pair<int64_t, int> &x, const std::pair<int64_t, int> &y) {
                return x.first > y.first || (x.first == y.first && x.second > y.second);
            };
            std::make_heap(heap.begin(), heap.end(), cmp);
            int64_t np = 0;
            for (int64_t q = 0; q < nb; ++q) {
                const int32_t bq = order[q];
                if (follower[bq]) continue;
                np += partner[bq] >= 0;
                std::pop_heap(heap.begin(), heap.end(), cmp);
                auto top = heap.back();
                heap.pop_back();
                lists[top.second].push_back(bq);
                top.first += bcost(bq) * (partner[bq] >= 0 ? 2 : 1);
                heap.push_back(top);
                std::push_heap(heap.begin(), heap.end(), cmp);
            }
            coff[2].assign(nc + 1, 0);
            for (int c = 0; c < nc; ++c) {
                coff[2][c + 1] = coff[2][c] + (int32_t)lists[c].size();
                cblk[2].insert(cblk[2].end(), lists[c].begin(), lists[c].end());
            }
            w.n_pairs = np;
        }
        {
            std::vector<int32_t> soff, sfirst(nb + 1, 0);
            for (int64_t b = 0; b < nb; ++b) {
                sfirst[b] = (int32_t)soff.size();
                for (int32_t i = boff[b]; i < boff[b + 1]; i += ASK_SEG_ITEMS) soff.push_back(i);
            }
            sfirst[nb] = (int32_t)soff.size();
            const int64_t nseg = (int64_t)soff.size();
            soff.push_back(boff[nb]);
            std::vector<int32_t> spart(std::max<int64_t>(1, nseg), -1);
            for (int64_t b = 0; b < nb; ++b)
                if (partner[b] >= 0)
                    for (int32_t k = 0; k < sfirst[b + 1] - sfirst[b]; ++k) spart[sfirst[b] + k] = sfirst[partner[b]] + k;
            std::vector<std::vector<int32_t>> lists(nc);
            std::vector<std::pair<int64_t, int>> heap;
            for (int c = 0; c < nc; ++c) heap.push_back({0, c});
            auto cmp = [](const std::pair<int64_t, int> &x, const std::pair<int64_t, int> &y) {
                return x.first > y.first || (x.first == y.first && x.second > y.second);
            };
            std::make_heap(heap.begin(), heap.end(), cmp);
            for (int64_t q = 0; q < nb; ++q) {
                const int32_t bq = order[q];
                if (follower[bq]) continue;
                for (int32_t sg = sfirst[bq]; sg < sfirst[bq + 1]; ++sg) {
                    std::pop_heap(heap.begin(), heap.end(), cmp);
                    auto top = heap.back();
                    heap.pop_back();
                    lists[top.second].push_back(sg);
                    top.first += ((int64_t)(soff[sg + 1] - soff[sg]) * 4 + 3) * (partner[bq] >= 0 ? 2 : 1);
                    heap.push_back(top);
                    std::push_heap(heap.begin(), heap.end(), cmp);
                }
            }
            std::vector<int32_t> so(nc + 1, 0), sl;
            for (int c = 0; c < nc; ++c) {
                so[c + 1] = so[c] + (int32_t)lists[c].size();
                sl.insert(sl.end(), lists[c].begin(), lists[c].end());
            }
            w.n_seg = nseg;
            WTRY(arena.alloc(&w.seg_off, nseg + 1));
            WTRY(arena.alloc(&w.seg_partner, std::max<int64_t>(1, nseg)));
            WTRY(arena.alloc(&w.seg_sched_off, nc + 1));
            WTRY(arena.alloc(&w.seg_sched, std::max<size_t>(1, sl.size())));
            WCHK(cudaMemcpyAsync(w.seg_off, soff.data(), sizeof(int32_t) * (nseg + 1), cudaMemcpyHostToDevice, s));
            WCHK(cudaMemcpyAsync(w.seg_partner, spart.data(), sizeof(int32_t) * spart.size(), cudaMemcpyHostToDevice, s));
            WCHK(cudaMemcpyAsync(w.seg_sched_off, so.data(), sizeof(int32_t) * (nc + 1), cudaMemcpyHostToDevice, s));
            if (!sl.empty())
                WCHK(cudaMemcpyAsync(w.seg_sched, sl.data(), sizeof(int32_t) * sl.size(), cudaMemcpyHostToDevice, s));
            // the host vectors must outlive the copies
            WCHK(cudaStreamSynchronize(s));
        }
        w.n_ctas = nc;
        for (int k = 0; k < 3; ++k) {
            WTRY(arena.alloc(&w.sched_off[k], nc + 1));
            WTRY(arena.alloc(&w.sched_blocks[k], std::max<int64_t>(1, nb)));
            WCHK(cudaMemcpyAsync(w.sched_off[k], coff[k].data(), sizeof(int32_t) * (nc + 1), cudaMemcpyHostToDevice, s));
            WCHK(cudaMemcpyAsync(w.sched_blocks[k], cblk[k].data(), sizeof(int32_t) * cblk[k].size(),
                                 cudaMemcpyHostToDevice, s));
            w.n_ctas_sched[k] = nc;
        }
        WTRY(arena.alloc(&w.partner, std::max<int64_t>(1, nb)));
        WCHK(cudaMemcpyAsync(w.partner, partner.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s));
        w.cta_off = w.sched_off[t->tune_sched & 1];
        w.cta_blocks = w.sched_blocks[t->tune_sched & 1];
        WCHK(cudaStreamSynchronize(s));
        int64_t sn = 0, sf = 0, pa = 0;
        for (int64_t q = 0; q < T; ++q) { sn += h_near[q]; sf += h_far[q]; pa += h_pairs[q]; }
        w.n_items = nit;
        w.n_blocks = nb;
        w.pairs_alg = pa;
        w.pairs_cmp = pc;
        w.near_tot = sn;
        w.far_tot = sf;
    }
    goto out;
fail:
    askit_set_error("work lists: %s", cudaGetErrorString(e));
    rc = e == cudaErrorMemoryAllocation ? ASKIT_ERR_OOM : ASKIT_ERR_CUDA;
out:
#undef WCHK
#undef WTRY
    cudaStreamSynchronize(s);
    for (void *q : {(void *)cnt, (void *)nearc, (void *)farc, (void *)pairs, (void *)vals, (void *)emit_of, (void *)bflag,
                    (void *)bidx, (void *)bstart, (void *)iflag, (void *)iidx, (void *)keys, (void *)keys_s, tmp})
        if (q) cudaFreeAsync(q, s);
    return rc;
}

// The in-sample work lists in batches of consecutive target slots: a count
// pass over all N targets, then cuts wherever the next target would take the
// running batch past the entry budget.  A sub-block's items and a pair's
// matching lists never straddle a cut (both are lists of targets), and every
// entry's partial sum is computed the same way in whichever batch holds it.
askit_status build_insample_lists(askit_tree t, const PruneSets &ps, cudaStream_t s) {
    const int64_t N = t->N;
    const int32_t *sets = ps.sets, *set_row = ps.set_row;
    const int stride = ps.stride;
    const int64_t budget = t->prm.batch_entries > 0 ? t->prm.batch_entries : ASK_BATCH_ENTRIES;
    std::vector<int64_t> h_cnt(N);
    {
        int64_t *buf = nullptr;
        ASK_CUDA(cudaMallocAsync(&buf, sizeof(int64_t) * 4 * N, s));
        count_kernel<<<nblk(N, 128), 128, 0, s>>>(sets, stride, set_row, N, t->L, t->far_height, t->nsize, t->d_s, buf,
                                                  buf + N, buf + 2 * N, buf + 3 * N);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_cnt.data(), buf, sizeof(int64_t) * N, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFreeAsync(buf, s);
        ASK_CUDA(e);
    }
    t->wl.clear();
    t->wl_t0.assign(1, 0);
    int64_t acc = 0;
    for (int64_t q = 0; q < N; ++q) {
        if (acc > 0 && acc + h_cnt[q] > budget) {
            t->wl_t0.push_back(q);
            acc = 0;
        }
        acc += h_cnt[q];
    }
    t->wl_t0.push_back(N);
    const size_t nb = t->wl_t0.size() - 1;
    t->wl.resize(nb);
    t->wl_entries = t->wl_entries_max = 0;
    for (size_t b = 0; b < nb; ++b) {
        const int64_t t0 = t->wl_t0[b], T = t->wl_t0[b + 1] - t0;
        // a batch's targets start at t0: shift the shared-row index, or the rows
        if (set_row)
            ASK_TRY(build_work_lists(t, sets, stride, set_row + t0, T, t->wl[b], t->arena, s));
        else
            ASK_TRY(build_work_lists(t, sets + t0 * stride, stride, nullptr, T, t->wl[b], t->arena, s));
        if (t->wl[b].n_entries >= ((int64_t)1 << 31)) {
            askit_set_error("a single target has more than 2^31 work entries");
            return ASKIT_ERR_UNSUPPORTED;
        }
        t->wl_entries += t->wl[b].n_entries;
        t->wl_entries_max = std::max(t->wl_entries_max, t->wl[b].n_entries);
    }
    return ASKIT_OK;
}

void free_work_lists(WorkLists &w, DevArena &arena) {
    void *ptrs[] = {w.off, w.slot_of_emit, w.tgt, w.items, w.block_off, w.block_order, w.sched_off[0],
                    w.sched_off[1], w.sched_off[2], w.sched_blocks[0], w.sched_blocks[1], w.sched_blocks[2],
                    w.partner, w.seg_off, w.seg_partner, w.seg_sched_off, w.seg_sched};
    for (void *p : ptrs)
        if (p) arena.release(p);
    w = WorkLists();
}

// The CTA schedule the kernels use: LPT or tree order (askit_set_launch);
// the paired schedule is taken by the FP16x3 kernel itself.
void use_schedule(askit_tree t) {
    for (WorkLists &w : t->wl) {
        w.cta_off = w.sched_off[t->tune_sched & 1];
        w.cta_blocks = w.sched_blocks[t->tune_sched & 1];
    }
}

askit_status reduce_partials(const WorkLists &w, const float *partial, int r, const int32_t *out_rows, float *U,
                             int64_t ldu, cudaStream_t s) {
    if (w.T == 0) return ASKIT_OK;
    reduce_partials_kernel<<<nblk(w.T * r, 256), 256, 0, s>>>(partial, w.off, w.slot_of_emit, w.T, r, out_rows, U, ldu);
    ASK_LAUNCH();
    return ASKIT_OK;
}
