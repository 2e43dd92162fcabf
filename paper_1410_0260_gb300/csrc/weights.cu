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

// Packed per-source-row column data of the tensor-core epilogue.
__global__ void pack_cols_kernel(const float *sc, const float *nrmc, const float *W, int r, int64_t rows,
                                 float4 *C) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= rows) return;
    const float s = sc[q];
    C[q] = make_float4(s, -s * nrmc[q], W[q * r], 0.f);
}

}  // namespace

askit_status upward_weights(askit_tree t, const float *W, int r, int64_t ldw, cudaStream_t s) {
    int64_t N = t->N;
    permute_in_kernel<<<(unsigned)((N * r + 255) / 256), 256, 0, s>>>(W, ldw, r, t->perm, N, t->Wt);
    ASK_LAUNCH();
    for (int depth = t->L; depth >= 1; --depth) {
        int64_t a0 = (int64_t)1 << depth;
        unsigned nb = (unsigned)a0;
        if (r == 1)
            upward_kernel<1><<<nb, 256, 0, s>>>(a0, depth == t->L, r, t->nstart, t->d_s, t->d_ncol, t->d_pivoff,
                                               t->piv, t->d_poff, t->P32, t->d_spool, t->Wt, t->Ws);
        else
            upward_kernel<8><<<nb, 256, 0, s>>>(a0, depth == t->L, r, t->nstart, t->d_s, t->d_ncol, t->d_pivoff,
                                               t->piv, t->d_poff, t->P32, t->d_spool, t->Wt, t->Ws);
        ASK_LAUNCH();
    }
    if (t->Ct) {
        pack_cols_kernel<<<(unsigned)((t->N_pad + 255) / 256), 256, 0, s>>>(t->sc_t, t->nrmc_t, t->Wt, r, t->N_pad, t->Ct);
        pack_cols_kernel<<<(unsigned)((t->srows + 255) / 256), 256, 0, s>>>(t->sc_s, t->nrmc_s, t->Ws, r, t->srows, t->Cs);
        ASK_LAUNCH();
    }
    return ASKIT_OK;
}
