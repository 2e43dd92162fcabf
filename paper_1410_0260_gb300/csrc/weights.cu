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

// Block (a, y) takes rows [rows y, rows y + rows) of node a's w~_a: 32 rows
// on the wide levels near the leaves, fewer (more blocks a node) on the
// levels near the root, whose few nodes would otherwise leave the GPU idle.
// A row's sum is formed the same way whatever the split.
// The rows v(R) the node's P multiplies (gathered through its pivot order)
// are staged in shared memory, in chunks of UP_KU rows and RC columns; warps
// then take rows q of w~_a, lanes split the columns u of P and reduce with
// shuffles (the same order for every split of the rows).
constexpr int UP_KU = 1024;

template <int RC>
__host__ __device__ constexpr int up_stride() { return RC == 1 ? 1 : RC + 4; }   // padded: conflict-free float4 reads

template <int RC>
__global__ void upward_kernel(int64_t a0, bool leaf_level, int r, int rows, const int32_t *nstart, const int32_t *s,
                              const int32_t *ncol, const int64_t *pivoff, const int32_t *piv, const int64_t *poff,
                              const float *P32, const int64_t *spool, const float *Wt, float *Ws) {
    extern __shared__ float vs[];
    constexpr int STR = up_stride<RC>();
    const int64_t a = a0 + blockIdx.x;
    const int sa = s[a], c = ncol[a], nr = c - sa;
    const int q0 = rows * blockIdx.y, q1 = min(sa, q0 + rows);
    if (q0 >= sa) return;                                 // block-uniform
    const int32_t *pv = piv + pivoff[a];
    const float *P = P32 + poff[a];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int sl = leaf_level ? 0 : s[2 * a];
    const float *vl = leaf_level ? Wt + (int64_t)nstart[a] * r : Ws + spool[2 * a] * r;
    const float *vr = leaf_level ? nullptr : Ws + spool[2 * a + 1] * r;
    auto vrow = [&](int col) -> const float * {
        return (leaf_level || col < sl) ? vl + (int64_t)col * r : vr + (int64_t)(col - sl) * r;
    };
    float *out = Ws + spool[a] * r;
    for (int z0 = 0; z0 < r; z0 += RC) {
        for (int u0 = 0; u0 < nr || u0 == 0; u0 += UP_KU) {
            const int ku = nr - u0 < UP_KU ? nr - u0 : UP_KU;
            __syncthreads();
            for (int e = threadIdx.x; e < ku * RC; e += blockDim.x) {
                const int uu = e / RC, z = e % RC;
                vs[uu * STR + z] = (z0 + z < r) ? vrow(pv[sa + u0 + uu])[z0 + z] : 0.f;
            }
            __syncthreads();
            for (int q = q0 + warp; q < q1; q += nw) {
                float acc[RC];
#pragma unroll
                for (int z = 0; z < RC; ++z) acc[z] = 0.f;
                for (int uu = lane; uu < ku; uu += 32) {
                    const float p = P[(int64_t)q * nr + u0 + uu];
                    if constexpr (RC == 1) {
                        acc[0] = fmaf(p, vs[uu], acc[0]);
                    } else {
#pragma unroll
                        for (int z4 = 0; z4 < RC / 4; ++z4) {
                            const float4 v = *reinterpret_cast<const float4 *>(vs + uu * STR + 4 * z4);
                            acc[4 * z4 + 0] = fmaf(p, v.x, acc[4 * z4 + 0]);
                            acc[4 * z4 + 1] = fmaf(p, v.y, acc[4 * z4 + 1]);
                            acc[4 * z4 + 2] = fmaf(p, v.z, acc[4 * z4 + 2]);
                            acc[4 * z4 + 3] = fmaf(p, v.w, acc[4 * z4 + 3]);
                        }
                    }
                }
#pragma unroll
                for (int z = 0; z < RC; ++z)
                    for (int o = 16; o > 0; o >>= 1) acc[z] += __shfl_xor_sync(0xffffffffu, acc[z], o);
                if (lane == 0) {
                    const float *vsk = vrow(pv[q]);
#pragma unroll
                    for (int z = 0; z < RC; ++z)
                        if (z0 + z < r) {
                            float *o = out + (int64_t)q * r + z0 + z;
                            *o = (u0 == 0 ? vsk[z0 + z] : *o) + acc[z];
                        }
                }
            }
            if (nr == 0) break;
        }
    }
}

template <int RC>
askit_status launch_upward(askit_tree t, WeightCtx &c, int depth, int r, cudaStream_t s) {
    const size_t smem = sizeof(float) * UP_KU * up_stride<RC>();
    // set once per kernel instance (thread-safe static initialisation)
    static const cudaError_t attr =
        cudaFuncSetAttribute(upward_kernel<RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ASK_CUDA(attr);
    const int64_t a0 = (int64_t)1 << depth;
    const int rows = a0 >= 512 ? 32 : (a0 >= 64 ? 8 : 2);     // rows of w~_a a block takes
    const unsigned ny = (unsigned)((std::max(1, t->prm.s_max) + rows - 1) / rows);
    const unsigned threads = 32u * (unsigned)std::min(8, rows);
    upward_kernel<RC><<<dim3((unsigned)a0, ny), threads, smem, s>>>(a0, depth == t->L, r, rows, t->nstart, t->d_s, t->d_ncol,
                                                                t->d_pivoff, t->piv, t->d_poff, t->P32, t->d_spool,
                                                                c.Wt, c.Ws);
    ASK_LAUNCH();
    return ASKIT_OK;
}

}  // namespace

// Buffers of a weight context for r vectors (grow-only in r and in the work
// lists' entries; the padding rows of Wt and Ws stay zero).
askit_status weights_reserve(askit_tree t, WeightCtx &c, int r, cudaStream_t s) {
    if (r <= c.r_cap && t->wl_entries_max <= c.ent_cap) {
        c.r = r;
        return ASKIT_OK;
    }
    const int r_req = r;
    r = std::max(r, c.r_cap);      // the capacity never shrinks
    c.arena.free_all();
    c.Wt = c.Ws = c.partial = nullptr;
    c.colv = nullptr;
    c.colw = nullptr;
    const int64_t srows = std::max<int64_t>(t->spool_rows, 1) + 256;
    ASK_TRY(c.arena.alloc(&c.Wt, (size_t)t->N_pad * r));
    ASK_TRY(c.arena.alloc(&c.Ws, (size_t)srows * r));
    ASK_TRY(c.arena.alloc(&c.partial, (size_t)std::max<int64_t>(1, t->wl_entries_max) * r));
    c.ent_cap = t->wl_entries_max;
    // per-sub-block column data of the 16-bit tensor-core kernel
    if (t->n_sub > 0 && t->d <= TC_K) {
        ASK_TRY(c.arena.alloc(&c.colv, (size_t)t->n_sub * 128));
        // [n_sub, 128, 16] floats, or (r > 4, the global-centered kernel's
        // weight MMA) split FP16 weights and 16 factors per sub-block
        if (r > 1) ASK_TRY(c.arena.alloc(&c.colw, (size_t)t->n_sub * (128 * 16 + 16)));
    }
    ASK_CUDA(cudaMemsetAsync(c.Wt, 0, sizeof(float) * t->N_pad * r, s));
    ASK_CUDA(cudaMemsetAsync(c.Ws, 0, sizeof(float) * srows * r, s));
    c.r_cap = r;
    c.r = r_req;
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
        if (r == 1)
            ASK_TRY(launch_upward<1>(t, c, depth, r, s));
        else if (r <= 4)
            ASK_TRY(launch_upward<4>(t, c, depth, r, s));
        else
            ASK_TRY(launch_upward<16>(t, c, depth, r, s));
    }
    c.ready = true;
    return ASKIT_OK;
}
