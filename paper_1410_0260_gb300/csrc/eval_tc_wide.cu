// Evaluate (Algorithm 4) on the tcgen05 tensor cores for wide points
// (64 < d): the distance contraction runs over K = d in chunks of 64.
//
// Work items are the same as for the narrow kernel (one source sub-block of
// <= 128 rows against <= 128 targets that need it).  Here both sides are
// centered on the sub-block's mean c_B:
//
//     a = x - c_B (targets, split on chip),  b = y - c_B (sources, pre-split)
//     r^2 = |a|^2 + |b|^2 - 2 a.b
//
// a.b accumulates over the K chunks in TMEM: the hi*hi products in one FP32
// accumulator and the two cross products (hi*lo + lo*hi) in a second one, so
// that the small terms are not rounded against the large running sum.  The
// epilogue adds the two, forms exp2(-c log2(e) r^2 / h_j^2) on MUFU.EX2 and
// reduces against the weights.
//
// One CTA per SM, 448 threads:
//   warps 0-7  loaders: thread t handles half (t >> 7) of target row t & 127
//              of each K chunk: loads its 32 FP32 values straight from HBM
//              into registers one chunk ahead (the next item's row slot is
//              read one item ahead), subtracts c_B, accumulates |a|^2, splits
//              into FP16/BF16 hi + lo and stores both in the 128-byte
//              swizzled K-major layout; they also write the item's column
//              data (c log2(e) / h^2, |b|^2, w) for the epilogue;
//   warps 8-11 epilogue (TMEM lane quadrant = warp & 3);
//   warp 12    TMEM allocation; lane 0 issues the tcgen05.mma instructions;
//   warp 13    producer: TMA tiled load of the sub-block's hi and lo chunk
//              and a bulk copy of c_B's chunk (a TMA tile::gather4 of the
//              target rows cost about 75 issue cycles per four rows, several
//              times the chunk's MMA time).
// Two chunk stages in shared memory; two items' accumulators (main + cross)
// fill all 512 TMEM columns, so the MMAs of item i+1 overlap the epilogue
// of item i.  Every mbarrier wait is bounded: on timeout the kernel records
// ASK_DEV_TIMEOUT, every role leaves its loop, and TMEM is freed.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>

#include "askit_impl.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace tcx;

constexpr int W_THREADS = 448;
constexpr int W_ROWS = 128;
constexpr int W_KC = 64;                        // K elements per chunk (128 bytes of 16-bit)
constexpr int W_REGION = W_ROWS * 128;          // 128 rows x 128 bytes, swizzled (16 KB)
constexpr uint32_t W_TMEM_COLS = 512;           // [main acc 0, main acc 1, cross acc 0, cross acc 1]

template <int RC>
struct WSmem {
    // one chunk stage: A hi, A lo, B hi, B lo, c_B chunk
    static constexpr int A_HI = 0, A_LO = W_REGION, B_HI = 2 * W_REGION, B_LO = 3 * W_REGION;
    static constexpr int CENTC = 4 * W_REGION;
    static constexpr int STAGE = CENTC + 1024;   // c_B chunk (256 B), stage kept 1024-byte aligned
    // two buffers of a chunk's raw FP32 target rows [128 rows][64], copied by
    // the loaders themselves (lanes along a row)
    static constexpr int RAW0 = 2 * STAGE;
    static constexpr int RAW_BYTES = W_ROWS * W_KC * 4;
    static constexpr int ANORM = RAW0 + 2 * RAW_BYTES;   // float [2 acc][2 halves][128]
    static constexpr int COLV = ANORM + 2 * 2 * 128 * 4;   // float4 [2 acc][128]
    static constexpr int COLW = COLV + 2 * 128 * 16;       // float [2 acc][128][RC]
    static constexpr int BAR = COLW + 2 * 128 * RC * 4;    // 16 mbarriers
    static constexpr int MISC = BAR + 16 * 8;              // tmem address, abort flag
    static constexpr int BYTES = MISC + 16;
    static constexpr uint32_t TX = 2 * W_REGION + W_KC * 4;   // bytes landing per chunk
};

struct TcwArgs {
    const EvalItem *items;
    const int32_t *block_off;
    const int32_t *cta_off, *cta_blocks;
    const int32_t *tgt;       // entry -> target slot
    int nkc;                  // K chunks (kw / 64)
    int kw;                   // row width of the pre-split arrays and of the centers
    const float *cent;        // [n_sub, kw]
    const float *q;           // target rows [q_rows, ldq] FP32 (16-byte aligned)
    int64_t ldq;              // = d_pad: columns past it read as zero
    const float *sc_t, *sc_s; // c log2(e) / h^2 per source row
    const float *nrm_t, *nrm_s;   // |y - c_B|^2 per source row
    const float *Wt, *Ws;
    int r;
    float f16_scale, g_unscale;
    float *partial;
    int *status;
};

// GF(4) multiplication by a primitive element: x -> w x is a permutation of
// {0,1,2,3} and so is x -> w x ^ x (= w^2 x), which makes both the loaders'
// swizzled stores and their raw-row reads free of bank conflicts.
__device__ __forceinline__ int gf4_mulw(int x) { return (0x1320 >> (4 * x)) & 3; }

template <int P, int RC>
__global__ void __launch_bounds__(W_THREADS, 1)
eval_tcw_kernel(const __grid_constant__ CUtensorMap map_t_hi, const __grid_constant__ CUtensorMap map_t_lo,
                const __grid_constant__ CUtensorMap map_s_hi, const __grid_constant__ CUtensorMap map_s_lo,
                const TcwArgs args) {
    using S = WSmem<RC>;
    constexpr uint32_t FMT = P == ASKIT_PREC_BF16X3 ? 1u : 0u;
    constexpr uint32_t IDESC = make_idesc(FMT, W_ROWS, W_ROWS);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(sm);
    float *a_norm = reinterpret_cast<float *>(sm + S::ANORM);
    float4 *colv = reinterpret_cast<float4 *>(sm + S::COLV);
    float *colw = reinterpret_cast<float *>(sm + S::COLW);
    const uint32_t bar0 = sbase + S::BAR;
    auto BAR_A_FULL = [&](int s) { return bar0 + 8 * s; };          // loaders stored A of stage s (256)
    auto BAR_MMA_DONE = [&](int s) { return bar0 + 8 * (2 + s); };  // MMAs of stage s finished (commit)
    auto BAR_L_FULL = [&](int s) { return bar0 + 8 * (4 + s); };    // raw rows, B and c_B of stage s landed
    auto BAR_R_EMPTY = [&](int s) { return bar0 + 8 * (6 + s); };   // loaders done with raw/c_B of stage s (256)
    auto BAR_T_FULL = [&](int a) { return bar0 + 8 * (8 + a); };    // accumulators of item slot a complete
    auto BAR_T_EMPTY = [&](int a) { return bar0 + 8 * (10 + a); };  // epilogue drained slot a (128)
    auto BAR_RAW_FULL = [&](int b) { return bar0 + 8 * (12 + b); }; // raw rows of buffer b landed (256 copiers)
    auto BAR_RAW_FREE = [&](int b) { return bar0 + 8 * (14 + b); }; // buffer b split by every loader (256)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + S::MISC);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + S::MISC + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(BAR_A_FULL(s), 256);
            mbar_init(BAR_MMA_DONE(s), 1);
            mbar_init(BAR_L_FULL(s), 1);
            mbar_init(BAR_R_EMPTY(s), 256);
            mbar_init(BAR_T_FULL(s), 1);
            mbar_init(BAR_T_EMPTY(s), 128);
            mbar_init(BAR_RAW_FULL(s), 256);
            mbar_init(BAR_RAW_FREE(s), 256);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 12) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(W_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nkc = args.nkc;
    const int c_begin = args.cta_off[blockIdx.x], c_end = args.cta_off[blockIdx.x + 1];

    if (warp < 8) {
        // ------------------------------------------------------------ loaders
        // Copies: loader warp lw brings rows 16 lw .. 16 lw + 15 of the next
        // chunk into a raw buffer, two rows per instruction, 16 lanes along a
        // row's 256 bytes (so an instruction touches 4 cache lines, not 32),
        // zero-filled past ldq and for rows past the item's targets; each
        // thread's arrival on RAW_FULL fires when its copies have landed.
        // Split: thread (row, h) then centers, splits and stores its half of
        // row `row` of the chunk (conflict-free order of the 16-byte reads).
        const int row = tid & 127, h = tid >> 7;
        const int lw = tid >> 5, cpiece = lane & 15;
        int cs[8], ns[8];           // target slots of this lane's copy rows: current item, next item
        uint32_t cmask = 0, nmask = 0;
        auto copy_slots = [&](int ci, int it, int (&sl)[8], uint32_t &mask) {
            mask = 0;
            if (ci >= c_end) return;
            const EvalItem nx = args.items[it];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = 16 * lw + 2 * i + (lane >> 4);
                sl[i] = r < nx.cnt ? args.tgt[nx.e0 + r] : 0;
                if (r < nx.cnt) mask |= 1u << i;
            }
        };
        auto issue_copies = [&](const int (&sl)[8], uint32_t mask, int kc, int buf) {
            const uint32_t dst0 = sbase + S::RAW0 + buf * S::RAW_BYTES;
            const int64_t col = (int64_t)kc * W_KC + 4 * cpiece;
            const bool in_row = col < args.ldq;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = 16 * lw + 2 * i + (lane >> 4);
                const bool ok = in_row && ((mask >> i) & 1u);
                const float *src = ok ? args.q + (int64_t)sl[i] * args.ldq + col : args.q;
                cp_async16_zfill(dst0 + (uint32_t)(r * W_KC * 4 + cpiece * 16), src, ok ? 16u : 0u);
            }
            cp_async_mbar_arrive(BAR_RAW_FULL(buf));
        };
        // the item after (ci, it) in this CTA's order, or ci == c_end
        auto next_item = [&](int &ci, int &it) {
            ++it;
            while (ci < c_end && it >= args.block_off[args.cta_blocks[ci] + 1]) {
                if (++ci < c_end) it = args.block_off[args.cta_blocks[ci]];
            }
        };
        int g = 0, li = 0;
        if (c_begin < c_end) {
            copy_slots(c_begin, args.block_off[args.cta_blocks[c_begin]], cs, cmask);
            issue_copies(cs, cmask, 0, 0);          // chunk 0 into buffer 0
        }
        for (int ci = c_begin; ci < c_end && !*abort_flag; ++ci) {
            const int b = args.cta_blocks[ci];
            const int i0 = args.block_off[b], i1 = args.block_off[b + 1];
            const EvalItem first = args.items[i0];
            const bool far = first.nrows < 0;
            const int nrows = first.nrows & 0x7fffffff;
            const bool has_src = row < nrows;
            const int64_t srow = (int64_t)first.row0 + row;
            const float sc = has_src ? __ldg((far ? args.sc_s : args.sc_t) + srow) : 0.f;
            const float qn = has_src ? __ldg((far ? args.nrm_s : args.nrm_t) + srow) : 0.f;
            const float *wrow = (far ? args.Ws : args.Wt) + srow * args.r;
            for (int it = i0; it < i1; ++it, ++li) {
                const int a = li & 1;
                const int cnt = args.items[it].cnt;
                const bool has_tgt = row < cnt;
                // the next item's copy slots, one item ahead
                int nci = ci, nit = it;
                next_item(nci, nit);
                copy_slots(nci, nit, ns, nmask);
                const bool has_next = nci < c_end;
                if (!mbar_wait(BAR_T_EMPTY(a), ((li >> 1) & 1) ^ 1, abort_flag, args.status)) goto loader_done;
                // column data of source row `row` for this item's slot:
                // arg = g A + (C p + B) = -sc (p + q - 2 g / scale^2)
                if (h == 0) {
                    float *cp = reinterpret_cast<float *>(colv + a * 128 + 2 * (row >> 1));
                    const int o = row & 1;
                    cp[0 + o] = 2.f * args.g_unscale * sc;
                    cp[2 + o] = -sc * qn;
                    cp[4 + o] = -sc;
                    cp[6 + o] = has_src ? __ldg(wrow) : 0.f;
                } else if (RC > 1) {
#pragma unroll
                    for (int z = 0; z < RC; ++z)
                        colw[(a * 128 + row) * RC + z] = (has_src && z < args.r) ? __ldg(wrow + z) : 0.f;
                }
                float nn = 0.f;
                for (int kc = 0; kc < nkc; ++kc, ++g) {
                    const int s = g & 1;
                    const uint32_t par = (g >> 1) & 1;
                    // the next chunk's rows into the other raw buffer, once every
                    // loader has split the chunk it held (chunk g - 1)
                    const int nb = (g + 1) & 1;
                    if (kc + 1 < nkc || has_next) {
                        if (!mbar_wait(BAR_RAW_FREE(nb), (((g + 1) >> 1) & 1) ^ 1, abort_flag, args.status))
                            goto loader_done;
                        if (kc + 1 < nkc) issue_copies(cs, cmask, kc + 1, nb);
                        else issue_copies(ns, nmask, 0, nb);
                    }
                    if (!mbar_wait(BAR_MMA_DONE(s), par ^ 1, abort_flag, args.status)) goto loader_done;
                    if (!mbar_wait(BAR_L_FULL(s), par, abort_flag, args.status)) goto loader_done;
                    if (!mbar_wait(BAR_RAW_FULL(s), par, abort_flag, args.status)) goto loader_done;
                    uint8_t *st = sm + s * S::STAGE;
                    const float *raw = reinterpret_cast<const float *>(sm + S::RAW0 + s * S::RAW_BYTES) + row * W_KC;
                    const float *cen = reinterpret_cast<const float *>(st + S::CENTC);
                    const int flip = (row >> 2) & 1;
#pragma unroll
                    for (int j2 = 0; j2 < 4; ++j2) {
                        // swizzled 16-byte slot p of the row and the element chunk c16 it holds;
                        // c16 >> 2 == h, so the two halves of a row split the chunk
                        const int p = 4 * (h ^ flip) + (gf4_mulw(row & 3) ^ j2);
                        const int c16 = p ^ (row & 7);
                        const float4 x0 = *reinterpret_cast<const float4 *>(raw + 8 * c16 + 4 * flip);
                        const float4 x1 = *reinterpret_cast<const float4 *>(raw + 8 * c16 + 4 * (flip ^ 1));
                        const float4 m0 = *reinterpret_cast<const float4 *>(cen + 8 * c16 + 4 * flip);
                        const float4 m1 = *reinterpret_cast<const float4 *>(cen + 8 * c16 + 4 * (flip ^ 1));
                        const float4 xl = flip ? x1 : x0, xh = flip ? x0 : x1;   // elements 0-3, 4-7
                        const float4 ml = flip ? m1 : m0, mh = flip ? m0 : m1;
                        float v[8] = {xl.x - ml.x, xl.y - ml.y, xl.z - ml.z, xl.w - ml.w,
                                      xh.x - mh.x, xh.y - mh.y, xh.z - mh.z, xh.w - mh.w};
                        if (!has_tgt) {
#pragma unroll
                            for (int e = 0; e < 8; ++e) v[e] = 0.f;
                        }
#pragma unroll
                        for (int e = 0; e < 8; ++e) nn = fmaf(v[e], v[e], nn);
                        uint32_t hv[4], lv[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if constexpr (P == ASKIT_PREC_FP16X3) {
                                const float v0 = v[2 * e] * args.f16_scale, v1 = v[2 * e + 1] * args.f16_scale;
                                const __half2 hh = __floats2half2_rn(v0, v1);
                                const float2 hf = __half22float2(hh);
                                const __half2 ll = __floats2half2_rn(v0 - hf.x, v1 - hf.y);
                                hv[e] = *reinterpret_cast<const uint32_t *>(&hh);
                                lv[e] = *reinterpret_cast<const uint32_t *>(&ll);
                            } else {
                                const float v0 = v[2 * e], v1 = v[2 * e + 1];
                                const __nv_bfloat162 hh = __floats2bfloat162_rn(v0, v1);
                                const float2 hf = __bfloat1622float2(hh);
                                const __nv_bfloat162 ll = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
                                hv[e] = *reinterpret_cast<const uint32_t *>(&hh);
                                lv[e] = *reinterpret_cast<const uint32_t *>(&ll);
                            }
                        }
                        const int off = row * 128 + (p << 4);
                        *reinterpret_cast<uint4 *>(st + S::A_HI + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                        *reinterpret_cast<uint4 *>(st + S::A_LO + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
                    }
                    if (kc == nkc - 1) a_norm[(a * 2 + h) * 128 + row] = nn;
                    mbar_arrive(BAR_RAW_FREE(s));
                    // generic-proxy stores -> visible to the tensor core's async proxy
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_arrive(BAR_A_FULL(s));
                    mbar_arrive(BAR_R_EMPTY(s));
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) cs[i] = ns[i];
                cmask = nmask;
            }
        }
    loader_done:
        // no copy may land in shared memory after the CTA exits (also after
        // an abort)
        cp_async_wait<0>();
    } else if (warp < 12) {
        // ----------------------------------------------------------- epilogue
        const int row = tid - 256;
        const int q = warp & 3;
        int li = 0;
        for (int ci = c_begin; ci < c_end && !*abort_flag; ++ci) {
            const int b = args.cta_blocks[ci];
            for (int it = args.block_off[b]; it < args.block_off[b + 1]; ++it, ++li) {
                const int a = li & 1;
                const EvalItem item = args.items[it];
                const int nrows = item.nrows & 0x7fffffff;
                if (!mbar_wait(BAR_T_FULL(a), (li >> 1) & 1, abort_flag, args.status)) goto epi_done;
                tc_fence_after();
                float acc[RC];
#pragma unroll
                for (int z = 0; z < RC; ++z) acc[z] = 0.f;
                float2 acc2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                if (q * 32 < item.cnt) {
                    const float pt = a_norm[(a * 2) * 128 + row] + a_norm[(a * 2 + 1) * 128 + row];
                    const float2 pt2 = make_float2(pt, pt);
                    const float4 *cv4 = colv + a * 128;
                    const float *cwp = colw + a * 128 * RC;
                    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
                    for (int c = 0; c < 4 && c * 32 < nrows; ++c) {
                        float g[32], gx[32];
                        tmem_ld32(lane_base + (uint32_t)(a * 128 + c * 32), g);
                        tmem_ld32(lane_base + (uint32_t)(256 + a * 128 + c * 32), gx);
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) g[jj] += gx[jj];
                        if constexpr (RC == 1) {
#pragma unroll
                            for (int jj = 0; jj < 32; jj += 2) {
                                const float4 ab = cv4[c * 32 + jj];
                                const float4 cw = cv4[c * 32 + jj + 1];
                                const float2 inner = __ffma2_rn(make_float2(cw.x, cw.y), pt2, make_float2(ab.z, ab.w));
                                const float2 arg = __ffma2_rn(make_float2(g[jj], g[jj + 1]), make_float2(ab.x, ab.y), inner);
                                const float2 k = make_float2(ex2_approx(arg.x), ex2_approx(arg.y));
                                acc2[(jj >> 1) & 1] = __ffma2_rn(k, make_float2(cw.z, cw.w), acc2[(jj >> 1) & 1]);
                            }
                        } else {
#pragma unroll
                            for (int jj = 0; jj < 32; ++jj) {
                                const int j = c * 32 + jj;
                                const float4 ab = cv4[j & ~1];
                                const float4 cw = cv4[(j & ~1) + 1];
                                const bool o = j & 1;
                                const float A = o ? ab.y : ab.x, B = o ? ab.w : ab.z, Cc = o ? cw.y : cw.x;
                                const float k = ex2_approx(fmaf(g[jj], A, fmaf(Cc, pt, B)));
#pragma unroll
                                for (int z = 0; z < RC; ++z) acc[z] = fmaf(k, cwp[j * RC + z], acc[z]);
                            }
                        }
                    }
                    if constexpr (RC == 1) acc[0] = (acc2[0].x + acc2[0].y) + (acc2[1].x + acc2[1].y);
                }
                tc_fence_before();
                mbar_arrive(BAR_T_EMPTY(a));
                if (row < item.cnt) {
                    float *p = args.partial + (int64_t)(item.e0 + row) * args.r;
#pragma unroll
                    for (int z = 0; z < RC; ++z)
                        if (z < args.r) p[z] = acc[z];
                }
            }
        }
    epi_done:;
    } else if (warp == 13 && lane == 0) {
        // ------------------------------------------------------------ producer
        int g = 0, issued = 0;
        for (int ci = c_begin; ci < c_end && !*abort_flag; ++ci) {
            const int b = args.cta_blocks[ci];
            const int i0 = args.block_off[b], i1 = args.block_off[b + 1];
            const EvalItem first = args.items[i0];
            const bool far = first.nrows < 0;
            const CUtensorMap *mh = far ? &map_s_hi : &map_t_hi;
            const CUtensorMap *ml = far ? &map_s_lo : &map_t_lo;
            const float *cb = args.cent + (int64_t)first.cidx * args.kw;
            for (int it = i0; it < i1; ++it) {
                for (int kc = 0; kc < nkc; ++kc, ++g) {
                    const int s = g & 1;
                    const uint32_t par = ((g >> 1) & 1) ^ 1;
                    if (!mbar_wait(BAR_R_EMPTY(s), par, abort_flag, args.status)) goto prod_done;
                    if (!mbar_wait(BAR_MMA_DONE(s), par, abort_flag, args.status)) goto prod_done;
                    const uint32_t st = sbase + s * S::STAGE;
                    ++issued;
                    mbar_expect_tx(BAR_L_FULL(s), S::TX);
                    tma_load_2d(st + S::B_HI, mh, kc * W_KC, first.row0, BAR_L_FULL(s));
                    tma_load_2d(st + S::B_LO, ml, kc * W_KC, first.row0, BAR_L_FULL(s));
                    bulk_copy(st + S::CENTC, cb + kc * W_KC, W_KC * 4, BAR_L_FULL(s));
                }
            }
        }
    prod_done:
        // copies of the last two chunks may still be landing after an abort
        for (int gg = issued > 2 ? issued - 2 : 0; gg < issued; ++gg) mbar_drain(BAR_L_FULL(gg & 1), (gg >> 1) & 1);
    } else if (warp == 12 && lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        int g = 0, li = 0;
        for (int ci = c_begin; ci < c_end && !*abort_flag; ++ci) {
            const int b = args.cta_blocks[ci];
            for (int it = args.block_off[b]; it < args.block_off[b + 1]; ++it, ++li) {
                const int a = li & 1;
                const uint32_t d_main = tmem + (uint32_t)(a * 128), d_cross = tmem + (uint32_t)(256 + a * 128);
                for (int kc = 0; kc < nkc; ++kc, ++g) {
                    const int s = g & 1;
                    const uint32_t par = (g >> 1) & 1;
                    if (!mbar_wait(BAR_A_FULL(s), par, abort_flag, args.status)) goto mma_done;
                    if (!mbar_wait(BAR_L_FULL(s), par, abort_flag, args.status)) goto mma_done;
                    if (kc == 0 && !mbar_wait(BAR_T_EMPTY(a), ((li >> 1) & 1) ^ 1, abort_flag, args.status))
                        goto mma_done;
                    tc_fence_after();
                    const uint32_t st = sbase + s * S::STAGE;
                    const uint32_t a_hi = st + S::A_HI, a_lo = st + S::A_LO, b_hi = st + S::B_HI, b_lo = st + S::B_LO;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {   // K = 16 per MMA: 32 bytes into the 128-byte rows
                        const uint32_t off = (uint32_t)(k * 32);
                        tc_mma<P>(d_cross, sw128_desc(a_hi + off), sw128_desc(b_lo + off), IDESC, (kc | k) != 0);
                        tc_mma<P>(d_cross, sw128_desc(a_lo + off), sw128_desc(b_hi + off), IDESC, 1);
                        tc_mma<P>(d_main, sw128_desc(a_hi + off), sw128_desc(b_hi + off), IDESC, (kc | k) != 0);
                    }
                    tc_commit(BAR_MMA_DONE(s));
                    if (kc == nkc - 1) tc_commit(BAR_T_FULL(a));
                }
            }
        }
    mma_done:;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 12) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(W_TMEM_COLS) : "memory");
    }
}

// Tensor maps of the pre-split source arrays ([rows, kw] 16-bit; boxes of
// 64 x 128, 128-byte swizzle) for BF16 (index 0) and FP16 (index 1).
struct TcwState {
    CUtensorMap map[2][4];   // [t_hi, t_lo, s_hi, s_lo]
    bool ready[2] = {false, false};
    EncodeTiledFn encode = nullptr;
};

std::mutex g_tcw_mu;

askit_status tcw_state(askit_tree t, int pi, TcwState **out) {
    std::lock_guard<std::mutex> lock(g_tcw_mu);
    if (!t->tcw) t->tcw = new TcwState();
    TcwState *st = (TcwState *)t->tcw;
    if (!st->encode) ASK_TRY(encode_fn(&st->encode));
    if (!st->ready[pi]) {
        const CUtensorMapDataType ty = pi == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
        const void *arr[4] = {pi == 0 ? (void *)t->Xt_bhi : (void *)t->Xt_hhi,
                              pi == 0 ? (void *)t->Xt_blo : (void *)t->Xt_hlo,
                              pi == 0 ? (void *)t->Xs_bhi : (void *)t->Xs_hhi,
                              pi == 0 ? (void *)t->Xs_blo : (void *)t->Xs_hlo};
        for (int i = 0; i < 4; ++i)
            ASK_TRY(encode_2d(st->encode, &st->map[pi][i], ty, 2, arr[i], i < 2 ? t->N_pad : t->srows, t->kw, W_KC,
                              W_ROWS, CU_TENSOR_MAP_SWIZZLE_128B));
        st->ready[pi] = true;
    }
    *out = st;
    return ASKIT_OK;
}

template <int P, int RC>
askit_status launch_w(askit_tree t, TcwState *st, int pi, const TcwArgs &a, int grid, cudaStream_t s) {
    using S = WSmem<RC>;
    const size_t smem = S::BYTES + 1024;
    static bool attr_set = false;
    {
        std::lock_guard<std::mutex> lock(g_tcw_mu);
        if (!attr_set) {
            ASK_CUDA(cudaFuncSetAttribute(eval_tcw_kernel<P, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
            attr_set = true;
        }
    }
    ASK_TRY(ktimer_mark(t, s, false));
    eval_tcw_kernel<P, RC><<<(unsigned)grid, W_THREADS, smem, s>>>(st->map[pi][0], st->map[pi][1], st->map[pi][2],
                                                                   st->map[pi][3], a);
    ASK_LAUNCH();
    return ktimer_mark(t, s, true);
}

}  // namespace

askit_status eval_tc_wide(askit_tree t, const WeightCtx &c, int precision, const float *Xq, int64_t ldq,
                          int64_t q_rows, const WorkLists &w, float *partial, cudaStream_t s) {
    if (precision != ASKIT_PREC_BF16X3 && precision != ASKIT_PREC_FP16X3) {
        askit_set_error("for d > %d the tensor-core evaluation runs in BF16x3 or FP16x3", TC_K);
        return ASKIT_ERR_UNSUPPORTED;
    }
    if (c.r > 16) {
        askit_set_error("tensor-core evaluation covers r <= 16; use ASKIT_PREC_SIMT_FP32");
        return ASKIT_ERR_UNSUPPORTED;
    }
    if (w.n_blocks == 0) return ASKIT_OK;
    if (ldq != t->d_pad || !t->Xt_hhi) {
        askit_set_error("target rows must have d_pad columns and the wide operands must exist");
        return ASKIT_ERR_INVALID_ARG;
    }
    const int pi = precision == ASKIT_PREC_BF16X3 ? 0 : 1;
    TcwState *st = nullptr;
    ASK_TRY(tcw_state(t, pi, &st));
    if ((reinterpret_cast<uintptr_t>(Xq) & 15) != 0) {
        askit_set_error("target rows must be 16-byte aligned");
        return ASKIT_ERR_INVALID_ARG;
    }
    (void)q_rows;
    TcwArgs a;
    a.q = Xq;
    a.ldq = ldq;
    a.items = w.items;
    a.block_off = w.block_off;
    a.cta_off = w.cta_off;
    a.cta_blocks = w.cta_blocks;
    a.tgt = w.tgt;
    a.nkc = t->kw / W_KC;
    a.kw = t->kw;
    a.cent = t->cent;
    a.sc_t = t->sc_t;
    a.sc_s = t->sc_s;
    a.nrm_t = t->nrmc_t;
    a.nrm_s = t->nrmc_s;
    a.Wt = c.Wt;
    a.Ws = c.Ws;
    a.r = c.r;
    a.f16_scale = precision == ASKIT_PREC_FP16X3 ? t->f16_scale : 1.f;
    a.g_unscale = 1.f / (a.f16_scale * a.f16_scale);
    a.partial = partial;
    a.status = t->d_status;
    if (precision == ASKIT_PREC_BF16X3) {
        if (c.r == 1) return launch_w<ASKIT_PREC_BF16X3, 1>(t, st, pi, a, w.n_ctas, s);
        if (c.r <= 4) return launch_w<ASKIT_PREC_BF16X3, 4>(t, st, pi, a, w.n_ctas, s);
        return launch_w<ASKIT_PREC_BF16X3, 16>(t, st, pi, a, w.n_ctas, s);
    }
    if (c.r == 1) return launch_w<ASKIT_PREC_FP16X3, 1>(t, st, pi, a, w.n_ctas, s);
    if (c.r <= 4) return launch_w<ASKIT_PREC_FP16X3, 4>(t, st, pi, a, w.n_ctas, s);
    return launch_w<ASKIT_PREC_FP16X3, 16>(t, st, pi, a, w.n_ctas, s);
}

void eval_tc_wide_free(askit_tree t) {
    delete (TcwState *)t->tcw;
    t->tcw = nullptr;
}
