// Evaluate (Algorithm 4) on CUDA cores in plain FP32: the reference
// precision the split tensor-core paths are measured against.
//
// One block per source sub-block (a leaf's points, evaluated directly, or a
// node's skeleton, Algorithm 4 lines 1-2), looping over the sub-block's
// items; thread t of an item owns one target and adds
//     sum_j exp(-c ||x - y_j||^2 / h_j^2) w_j
// over the sub-block's rows, with the distance in difference form (no
// cancellation) and the exponent on exp2f.  The sum is the entry's partial.
#include "askit_impl.cuh"

namespace {

constexpr int CH = 32;    // source rows per staged chunk
constexpr int DK = 64;    // coordinates per staged slice

template <int RMAX>
__global__ void __launch_bounds__(ASK_TILE_M) eval_simt_kernel(
    const float *__restrict__ Xq, int64_t ldq, const EvalItem *__restrict__ items,
    const int32_t *__restrict__ block_off, const int32_t *__restrict__ block_order,
    const int32_t *__restrict__ tgt, float *__restrict__ partial, const float *__restrict__ Xt,
    const float *__restrict__ Xs, const float *__restrict__ sc_t, const float *__restrict__ sc_s,
    const float *__restrict__ Wt, const float *__restrict__ Ws, int d_pad, int r) {
    __shared__ float ys[CH][DK + 1];
    __shared__ float ysc[CH];
    __shared__ float yw[CH][RMAX];
    const int b = block_order[blockIdx.x];
    const int tid = threadIdx.x;
    for (int it = block_off[b]; it < block_off[b + 1]; ++it) {
        const EvalItem item = items[it];
        const bool far = item.nrows < 0;
        const int nrows = item.nrows & 0x7fffffff;
        const bool mine = tid < item.cnt;
        const float *xrow = Xq + (mine ? (int64_t)tgt[item.e0 + tid] : 0) * ldq;
        const float *Y = far ? Xs : Xt;
        const float *SC = far ? sc_s : sc_t;
        const float *WW = far ? Ws : Wt;
        float acc[RMAX];
#pragma unroll
        for (int z = 0; z < RMAX; ++z) acc[z] = 0.f;
        float xr[DK];
        for (int j0 = 0; j0 < nrows; j0 += CH) {
            const int nj = min(CH, nrows - j0);
            float D[CH];
#pragma unroll
            for (int j = 0; j < CH; ++j) D[j] = 0.f;
            for (int k0 = 0; k0 < d_pad; k0 += DK) {
                __syncthreads();
                for (int e = tid; e < CH * DK; e += ASK_TILE_M) {
                    int j = e / DK, k = e % DK;
                    ys[j][k] = (j < nj && k0 + k < d_pad) ? Y[(int64_t)(item.row0 + j0 + j) * d_pad + k0 + k] : 0.f;
                }
                if (k0 == 0) {
                    for (int e = tid; e < CH; e += ASK_TILE_M) ysc[e] = e < nj ? SC[item.row0 + j0 + e] : 0.f;
                    for (int e = tid; e < CH * RMAX; e += ASK_TILE_M) {
                        int j = e / RMAX, z = e % RMAX;
                        yw[j][z] = (j < nj && z < r) ? WW[(int64_t)(item.row0 + j0 + j) * r + z] : 0.f;
                    }
                }
                __syncthreads();
                if (mine) {
#pragma unroll
                    for (int k = 0; k < DK; ++k) xr[k] = k0 + k < d_pad ? xrow[k0 + k] : 0.f;
#pragma unroll
                    for (int j = 0; j < CH; ++j) {
                        float a = 0.f;
#pragma unroll
                        for (int k = 0; k < DK; ++k) {
                            float t = xr[k] - ys[j][k];
                            a = fmaf(t, t, a);
                        }
                        D[j] += a;
                    }
                }
            }
            if (mine) {
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    if (j < nj) {
                        float kv = exp2f(-ysc[j] * D[j]);
#pragma unroll
                        for (int z = 0; z < RMAX; ++z) acc[z] = fmaf(kv, yw[j][z], acc[z]);
                    }
                }
            }
        }
        if (mine) {
            float *p = partial + (int64_t)(item.e0 + tid) * r;
#pragma unroll
            for (int z = 0; z < RMAX; ++z)
                if (z < r) p[z] = acc[z];
        }
    }
}

}  // namespace

askit_status eval_simt(askit_tree t, const WeightCtx &c, const float *Xq, int64_t ldq, const WorkLists &w,
                       float *partial, cudaStream_t s) {
    if (w.n_blocks == 0) return ASKIT_OK;
    int r = c.r;
    ASK_TRY(ktimer_mark(t, s, false));
#define LAUNCH(R)                                                                                   \
    eval_simt_kernel<R><<<(unsigned)w.n_blocks, ASK_TILE_M, 0, s>>>(                                \
        Xq, ldq, w.items, w.block_off, w.block_order, w.tgt, partial, t->Xt, t->Xs, t->sc_t,        \
        t->sc_s, c.Wt, c.Ws, t->d_pad, r)
    if (r <= 1) LAUNCH(1);
    else if (r <= 4) LAUNCH(4);
    else if (r <= 16) LAUNCH(16);
    else LAUNCH(64);
#undef LAUNCH
    ASK_LAUNCH();
    return ktimer_mark(t, s, true);
}

// ---------------------------------------------------------------------------
// Direct sum of eq. (1.1) at selected points: every source point, no
// approximation (the yardstick of ASKIT's error, Section 4).  One block per
// target; threads stride over the sources in tree order and reduce in a
// fixed order.
// ---------------------------------------------------------------------------
namespace {
constexpr int DIRECT_THREADS = 256;
template <int RMAX>
__global__ void __launch_bounds__(DIRECT_THREADS) direct_kernel(const float *__restrict__ X, int d,
                                                               const int32_t *__restrict__ tgt,
                                                               const float *__restrict__ Xt, int d_pad, int64_t N,
                                                               const float *__restrict__ sc_t,
                                                               const float *__restrict__ Wt, int r, float *U,
                                                               int64_t ldu) {
    __shared__ float xs[1024];
    __shared__ float red[DIRECT_THREADS / 32][RMAX];
    const int q = blockIdx.x;
    const int64_t i = tgt[q];
    for (int k = threadIdx.x; k < d_pad; k += blockDim.x) xs[k] = k < d ? X[i * d + k] : 0.f;
    __syncthreads();
    float acc[RMAX];
#pragma unroll
    for (int z = 0; z < RMAX; ++z) acc[z] = 0.f;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
        const float *y = Xt + j * d_pad;
        float D = 0.f;
        for (int k = 0; k < d_pad; k += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(y + k);
            const float a = xs[k] - v.x, b = xs[k + 1] - v.y, c = xs[k + 2] - v.z, e = xs[k + 3] - v.w;
            D = fmaf(a, a, D); D = fmaf(b, b, D); D = fmaf(c, c, D); D = fmaf(e, e, D);
        }
        const float kv = exp2f(-sc_t[j] * D);
#pragma unroll
        for (int z = 0; z < RMAX; ++z)
            if (z < r) acc[z] = fmaf(kv, Wt[j * r + z], acc[z]);
    }
#pragma unroll
    for (int z = 0; z < RMAX; ++z) {
        float v = acc[z];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][z] = v;
    }
    __syncthreads();
    if (threadIdx.x < RMAX && threadIdx.x < r) {
        float v = 0.f;
        for (int w = 0; w < DIRECT_THREADS / 32; ++w) v += red[w][threadIdx.x];
        U[q * ldu + threadIdx.x] = v;
    }
}
}  // namespace

extern "C" askit_status askit_direct(askit_tree t, const int32_t *tgt_dev, int64_t T, float *U_dev, int64_t ldu,
                                     void *stream) {
    if (!t || !tgt_dev || !U_dev) { askit_set_error("tree, tgt_dev and U_dev must be non-NULL"); return ASKIT_ERR_INVALID_ARG; }
    if (!t->dw.ready) { askit_set_error("askit_set_weights has not been called"); return ASKIT_ERR_NOT_READY; }
    if (T < 1 || T > (1 << 30) || ldu < t->dw.r) { askit_set_error("need 1 <= T and ldu >= r"); return ASKIT_ERR_INVALID_ARG; }
    if (t->d_pad > 1024) { askit_set_error("askit_direct handles d <= 1024"); return ASKIT_ERR_UNSUPPORTED; }
    cudaStream_t s = (cudaStream_t)stream;
    const WeightCtx &c = t->dw;
    if (c.r <= 1)
        direct_kernel<1><<<(unsigned)T, DIRECT_THREADS, 0, s>>>(t->X, t->d, tgt_dev, t->Xt, t->d_pad, t->N, t->sc_t, c.Wt, c.r, U_dev, ldu);
    else if (c.r <= 16)
        direct_kernel<16><<<(unsigned)T, DIRECT_THREADS, 0, s>>>(t->X, t->d, tgt_dev, t->Xt, t->d_pad, t->N, t->sc_t, c.Wt, c.r, U_dev, ldu);
    else
        direct_kernel<64><<<(unsigned)T, DIRECT_THREADS, 0, s>>>(t->X, t->d, tgt_dev, t->Xt, t->d_pad, t->N, t->sc_t, c.Wt, c.r, U_dev, ldu);
    ASK_LAUNCH();
    return ASKIT_OK;
}
