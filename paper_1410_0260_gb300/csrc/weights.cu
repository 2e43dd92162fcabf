// Weights into tree order and the upward pass of skeleton weights
// (Section 2.1 and Algorithm 3): w~_a = v(S_a) + P_a v(R), where v is w on
// the leaf's points, or the concatenated skeleton weights [w~_l; w~_r] of
// the children; S and R are the first s and the remaining columns of the
// node's pivot order.  FP32, one kernel per tree level, leaves first.
#include <algorithm>

#include "askit_impl.cuh"

namespace {

__global__ void permute_in_kernel(const float *W, int64_t ldw, int r, const int32_t *perm, int64_t N,
                                  float *Wt) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * r) return;
    int64_t q = e / r;
    int z = (int)(e % r);
    Wt[e] = W[(int64_t)perm[q] * ldw + z];
}

// One block per node of the level; warps take rows q of w~_a; lanes split
// the unskeletonized columns u and reduce with shuffles.
template <int RC>
__global__ void upward_kernel(int64_t a0, bool leaf_level, int r, const int32_t *nstart,
                              const int32_t *s, const int32_t *ncol, const int64_t *pivoff,
                              const int32_t *piv, const int64_t *poff, const float *P32,
                              const int64_t *spool, const float *Wt, float *Ws) {
    int64_t a = a0 + blockIdx.x;
    int sa = s[a], c = ncol[a], nr = c - sa;
    if (sa == 0) return;
    const int32_t *pv = piv + pivoff[a];
    const float *P = P32 + poff[a];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int sl = leaf_level ? 0 : s[2 * a];
    const float *vl = leaf_level ? Wt + (int64_t)nstart[a] * r : Ws + spool[2 * a] * r;
    const float *vr = leaf_level ? nullptr : Ws + spool[2 * a + 1] * r;
    auto vrow = [&](int col) -> const float * {
        return (leaf_level || col < sl) ? vl + (int64_t)col * r : vr + (int64_t)(col - sl) * r;
    };
    float *out = Ws + spool[a] * r;
    for (int q = warp; q < sa; q += nw) {
        for (int z0 = 0; z0 < r; z0 += RC) {
            float acc[RC];
#pragma unroll
            for (int zz = 0; zz < RC; ++zz) acc[zz] = 0.f;
            for (int u = lane; u < nr; u += 32) {
                float p = P[(int64_t)q * nr + u];
                const float *vu = vrow(pv[sa + u]);
#pragma unroll
                for (int zz = 0; zz < RC; ++zz)
                    if (z0 + zz < r) acc[zz] = fmaf(p, vu[z0 + zz], acc[zz]);
            }
#pragma unroll
            for (int zz = 0; zz < RC; ++zz)
                for (int o = 16; o > 0; o >>= 1) acc[zz] += __shfl_xor_sync(0xffffffffu, acc[zz], o);
            if (lane == 0) {
                const float *vs = vrow(pv[q]);
#pragma unroll
                for (int zz = 0; zz < RC; ++zz)
                    if (z0 + zz < r) out[(int64_t)q * r + z0 + zz] = vs[z0 + zz] + acc[zz];
            }
        }
    }
}

}  // namespace

// Buffers of a weight context for r vectors (grow-only; the padding rows of
// Wt and Ws stay zero).
askit_status weights_reserve(askit_tree t, WeightCtx &c, int r, cudaStream_t s) {
    if (r <= c.r_cap) {
        c.r = r;
        return ASKIT_OK;
    }
    c.arena.free_all();
    c.Wt = c.Ws = c.partial = nullptr;
    const int64_t srows = std::max<int64_t>(t->spool_rows, 1) + 256;
    ASK_TRY(c.arena.alloc(&c.Wt, (size_t)t->N_pad * r));
    ASK_TRY(c.arena.alloc(&c.Ws, (size_t)srows * r));
    ASK_TRY(c.arena.alloc(&c.partial, (size_t)std::max<int64_t>(1, t->wl.n_entries) * r));
    ASK_CUDA(cudaMemsetAsync(c.Wt, 0, sizeof(float) * t->N_pad * r, s));
    ASK_CUDA(cudaMemsetAsync(c.Ws, 0, sizeof(float) * srows * r, s));
    c.r_cap = r;
    c.r = r;
    c.ready = true;
    return ASKIT_OK;
}

askit_status upward_weights(askit_tree t, WeightCtx &c, const float *W, int r, int64_t ldw, cudaStream_t s) {
    ASK_TRY(weights_reserve(t, c, r, s));
    int64_t N = t->N;
    // rows of Wt/Ws are r apart: with a smaller r than the capacity, rows past
    // the first r columns are not used, so a fresh layout per call is fine
    permute_in_kernel<<<(unsigned)((N * r + 255) / 256), 256, 0, s>>>(W, ldw, r, t->perm, N, c.Wt);
    ASK_LAUNCH();
    for (int depth = t->L; depth >= 1; --depth) {
        int64_t a0 = (int64_t)1 << depth;
        unsigned nb = (unsigned)a0;
        if (r == 1)
            upward_kernel<1><<<nb, 256, 0, s>>>(a0, depth == t->L, r, t->nstart, t->d_s, t->d_ncol, t->d_pivoff,
                                               t->piv, t->d_poff, t->P32, t->d_spool, c.Wt, c.Ws);
        else
            upward_kernel<8><<<nb, 256, 0, s>>>(a0, depth == t->L, r, t->nstart, t->d_s, t->d_ncol, t->d_pivoff,
                                               t->piv, t->d_poff, t->P32, t->d_spool, c.Wt, c.Ws);
        ASK_LAUNCH();
    }
    c.ready = true;
    return ASKIT_OK;
}
