// Evaluate (Algorithm 4) on the tcgen05 tensor cores.
//
// Work item = one source sub-block (<= 128 rows of a leaf's points for the
// direct near field, or of a node's skeleton for the far field) against up
// to 128 targets that all need it (see eval_lists.cu).  For each item
//
//     G = A B^T             (tcgen05.mma, 128 x 128 x 64, FP32 accumulators in TMEM)
//     r^2 = (|a|^2 + 2 a.delta) + |y - c_T|^2 - 2 G
//     partial_t = sum_j exp2(-c log2(e) r^2 / h_j^2) w_j
//
// with a = x - c_T (targets centered on the item's first target c_T),
// b = y - c_B (sources centered on their sub-block's mean c_B, pre-split in
// HBM) and delta = c_T - c_B, an exact rewriting of |x - y|^2.  Every term
// is bounded by the spread of the item's targets or by |x - y| itself, so
// the FP32 rounding of the norm expansion stays at that scale even for the
// wide skeletons of high tree nodes.  The contraction is split in three
// products (hi*hi + hi*lo + lo*hi) of TF32 or BF16 parts with FP32
// accumulation.
//
// One CTA per SM, warp-specialized, 416 threads:
//   warps 0-7  loaders, two groups taking alternate items: thread t gathers
//              the item's target row t, centers and splits it, and stores it
//              in the 128-byte-swizzled K-major layout the tensor core reads
//              (stage = group); it also forms the row term of target t and
//              the column data of source row t;
//   warps 8-11 epilogue: tcgen05.ld of their 32 TMEM lanes (one row each),
//              exponent on MUFU.EX2, reduction against the weights;
//   warp 12    one thread issues the TMA loads of the sub-block (centered,
//              pre-split rows) and the tcgen05.mma instructions, and commits
//              them to mbarriers.
// Two TMEM accumulators (2 x 128 columns) let the MMAs of item i+1 run
// while the epilogue drains item i.  Every mbarrier wait is bounded: on
// timeout the kernel records ASK_DEV_TIMEOUT, all roles leave their loops,
// and TMEM is freed before the kernel returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "askit_impl.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace tcx;

constexpr int TC_THREADS = 448;
constexpr int TILE_ROWS = 128;                  // M = N = 128
constexpr int REGION = TILE_ROWS * 128;         // one 128-row x 128-byte swizzled region (16 KB)
constexpr uint32_t TMEM_COLS = 256;             // two 128-column FP32 accumulators

// Precision traits: element bytes, swizzle regions per operand (TC_K
// elements x element bytes / 128), MMA K steps, tcgen05 operand format.
template <int P> struct Prec;
template <> struct Prec<ASKIT_PREC_TF32X3> {
    static constexpr int EB = 4, NREG = 2, KSTEPS = 8;   // K = 8 per MMA
    static constexpr uint32_t FMT = 2;                   // TF32 in .kind::tf32
};
template <> struct Prec<ASKIT_PREC_BF16X3> {
    static constexpr int EB = 2, NREG = 1, KSTEPS = 4;   // K = 16 per MMA
    static constexpr uint32_t FMT = 1;                   // BF16 in .kind::f16
};

// Shared-memory plan (offsets from a 1024-byte aligned base).
template <int P>
struct Smem {
    // the 16-bit splits have room to stage raw rows: targets are then gathered
    // by TMA (tile::gather4) and the loaders work from shared memory only
    static constexpr bool GATHER = P != ASKIT_PREC_TF32X3;
    static constexpr int OPB = Prec<P>::NREG * REGION;    // one operand (hi or lo) of one tile
    static constexpr int B_HI = 0, B_LO = OPB;
    static constexpr int A0 = 2 * OPB;                     // stage s: hi at A0 + s*2*OPB, lo at + OPB
    static constexpr int TILES = 6 * OPB;
    static constexpr int RAWSTAGE = TILE_ROWS * TC_K * 4;  // one stage of gathered FP32 target rows
    static constexpr int RAW = TILES;                      // [2] stages (GATHER)
    static constexpr int RAWB = RAW + (GATHER ? 2 * RAWSTAGE : 0);        // raw FP32 source rows (GATHER)
    static constexpr int CENT = RAWB + (GATHER ? RAWSTAGE : 0);           // float [TC_K] c_B of the sub-block
    static constexpr int ANORM = CENT + TC_K * 4;                         // float [2][128] |a|^2 + 2 a.delta
    static constexpr int COLV = ANORM + 2 * 128 * 4;       // float4 [2][128]: per source pair {A, B}, {C, w} (see loader)
    static constexpr int RC_MAX = 16;
    static constexpr int COLW = COLV + 2 * 128 * 16;       // float [2][128][RC_MAX] weights (r > 1)
    static constexpr int BAR = COLW + 2 * 128 * RC_MAX * 4;   // 14 mbarriers
    static constexpr int MISC = BAR + 14 * 8;              // tmem address, abort flag
    static constexpr int BYTES = MISC + 16;
};

struct TcArgs {
    const EvalItem *items;
    const int32_t *block_off;
    const int32_t *cta_off, *cta_blocks;   // this CTA's sub-blocks: cta_blocks[cta_off[c] .. cta_off[c+1])
    const int32_t *tgt;       // entry -> target slot
    const float *Xq;          // target coordinates [*, ldq]
    int64_t ldq;
    int d_pad;
    const float *cent;        // [n_sub, TC_K]
    const float *sc_t, *sc_s; // c log2(e) / h^2 per source row
    const float *Xt, *Xs;     // raw source coordinates [*, d_pad] (column terms)
    const float *Wt, *Ws;
    int r;
    float f16_scale;          // prescale of the 16-bit operands (1: BF16 and TF32 are not prescaled)
    float g_unscale;          // 1 / f16_scale^2
    float *partial;
    int *status;
};

template <int P, int RC>
__global__ void __launch_bounds__(TC_THREADS, 1)
eval_tc_kernel(const __grid_constant__ CUtensorMap map_t_hi, const __grid_constant__ CUtensorMap map_t_lo,
               const __grid_constant__ CUtensorMap map_s_hi, const __grid_constant__ CUtensorMap map_s_lo,
               const __grid_constant__ CUtensorMap map_q, const __grid_constant__ CUtensorMap map_rt,
               const __grid_constant__ CUtensorMap map_rs, const TcArgs args) {
    using S = Smem<P>;
    constexpr int EB = Prec<P>::EB, NREG = Prec<P>::NREG, KSTEPS = Prec<P>::KSTEPS;
    constexpr uint32_t IDESC = make_idesc(Prec<P>::FMT, TILE_ROWS, TILE_ROWS);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(sm);
    float *a_norm = reinterpret_cast<float *>(sm + S::ANORM);
    float4 *colv = reinterpret_cast<float4 *>(sm + S::COLV);
    float *colw = reinterpret_cast<float *>(sm + S::COLW);
    const uint32_t bar0 = sbase + S::BAR;
    auto BAR_A_FULL = [&](int s) { return bar0 + 8 * s; };
    auto BAR_A_EMPTY = [&](int s) { return bar0 + 8 * (2 + s); };
    const uint32_t BAR_B_FULL = bar0 + 8 * 4, BAR_B_EMPTY = bar0 + 8 * 5;
    auto BAR_T_FULL = [&](int a) { return bar0 + 8 * (6 + a); };
    auto BAR_T_EMPTY = [&](int a) { return bar0 + 8 * (8 + a); };
    auto BAR_R_FULL = [&](int a) { return bar0 + 8 * (10 + a); };    // gathered target rows landed
    auto BAR_R_EMPTY = [&](int a) { return bar0 + 8 * (12 + a); };   // loader done with the raw stage
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + S::MISC);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + S::MISC + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        mbar_init(BAR_A_FULL(0), 128);
        mbar_init(BAR_A_FULL(1), 128);
        mbar_init(BAR_A_EMPTY(0), 1);
        mbar_init(BAR_A_EMPTY(1), 1);
        mbar_init(BAR_B_FULL, 1);
        mbar_init(BAR_B_EMPTY, 1);
        mbar_init(BAR_T_FULL(0), 1);
        mbar_init(BAR_T_FULL(1), 1);
        mbar_init(BAR_T_EMPTY(0), 128);
        mbar_init(BAR_T_EMPTY(1), 128);
        mbar_init(BAR_R_FULL(0), 1);
        mbar_init(BAR_R_FULL(1), 1);
        mbar_init(BAR_R_EMPTY(0), 128);
        mbar_init(BAR_R_EMPTY(1), 128);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 12) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < 8) {
        // ------------------------------------------------------------ loaders
        // two groups of four warps take alternate items (group g fills stage g);
        // thread t of a group owns target row t and source row t of its items
        const int grp = warp >> 2;
        const int t = tid & 127;
        const int nk4 = args.d_pad / 4;            // 16-byte chunks of a coordinate row
        int li = 0, lb = 0;
        for (int ci = args.cta_off[blockIdx.x]; ci < args.cta_off[blockIdx.x + 1] && !*abort_flag; ++ci) {
            const int b = args.cta_blocks[ci];
            const int i0 = args.block_off[b], i1 = args.block_off[b + 1];
            const int li_block_end = li + (i1 - i0);
            EvalItem item = args.items[i0];
            const bool far = item.nrows < 0;
            const int nrows = item.nrows & 0x7fffffff;
            const bool has_src = t < nrows;
            const int64_t srow = (int64_t)item.row0 + t;
            const float *ysrc = (far ? args.Xs : args.Xt) + srow * args.d_pad;
            const float *cB = args.cent + (int64_t)item.cidx * TC_K;
            // block-constant column data of source row t: c log2(e) / h^2 and w
            const float sc = has_src ? __ldg((far ? args.sc_s : args.sc_t) + srow) : 0.f;
            const float *wrow = (far ? args.Ws : args.Wt) + srow * args.r;
            const float w0 = has_src ? __ldg(wrow) : 0.f;
            bool waited_b = false;   // B_FULL of this block waited (gather path)
            // this group's first item of the block
            int it = i0 + (((li & 1) ^ grp) & 1);
            if (it < i1) item = args.items[it];
            int slot = (it < i1 && t < item.cnt) ? (S::GATHER ? 0 : args.tgt[item.e0 + t]) : -1;
            int first = (it < i1 && !S::GATHER) ? args.tgt[item.e0] : 0;
            li += ((li & 1) ^ grp) & 1;
            for (; it < i1; it += 2, li += 2) {
                const int s = li & 1;
                const uint32_t par = ((li >> 1) & 1) ^ 1;
                const int cnt = item.cnt;
                const float *xrow = args.Xq + (int64_t)(slot >= 0 ? slot : 0) * args.ldq;
                const float *xt0 = args.Xq + (int64_t)first * args.ldq;
                const bool has_tgt = slot >= 0;
                // prefetch this group's next item of the block (the gather path
                // needs only its size: the gather warp fetches the rows)
                if (it + 2 < i1) {
                    item = args.items[it + 2];
                    if constexpr (!S::GATHER) {
                        slot = t < item.cnt ? args.tgt[item.e0 + t] : -1;
                        first = args.tgt[item.e0];
                    } else {
                        slot = t < item.cnt ? 0 : -1;
                    }
                }
                if (!mbar_wait(BAR_A_EMPTY(s), par, abort_flag, args.status)) goto loader_done;
                if (!mbar_wait(BAR_T_EMPTY(s), par, abort_flag, args.status)) goto loader_done;
                uint8_t *ahi = sm + S::A0 + s * 2 * S::OPB;
                uint8_t *alo = ahi + S::OPB;
                float nn = 0.f, dd = 0.f, qq = 0.f;
                if constexpr (S::GATHER) {
                    // gathered target rows (stage s) and the sub-block's raw rows
                    if (!mbar_wait(BAR_R_FULL(s), (li >> 1) & 1, abort_flag, args.status)) goto loader_done;
                    if (!waited_b) {
                        if (!mbar_wait(BAR_B_FULL, lb & 1, abort_flag, args.status)) goto loader_done;
                        waited_b = true;
                    }
                    const float *raw = reinterpret_cast<const float *>(sm + S::RAW + s * S::RAWSTAGE);
                    const float *rawb = reinterpret_cast<const float *>(sm + S::RAWB);
                    const float *cBs = reinterpret_cast<const float *>(sm + S::CENT);
                    const int dp = args.d_pad;
                    // packed FP32x2 arithmetic: two coordinates per instruction
                    const float2 m1 = make_float2(-1.f, -1.f), z2 = make_float2(0.f, 0.f);
                    const float2 sc2 = make_float2(args.f16_scale, args.f16_scale);
                    float2 nn2 = z2, dd2 = z2, qq2 = z2;
#pragma unroll 4
                    for (int j = 0; j < TC_K / 4; ++j) {
                        // chunks in an order rotated by the row: conflict-free shared loads
                        const int k4 = (j + t) & (nk4 - 1);
                        float2 xa[2] = {z2, z2};
                        int kst = j;   // chunk to store (zeros past d_pad)
                        if (j < nk4) {
                            kst = k4;
                            const float4 tt = *reinterpret_cast<const float4 *>(raw + 4 * k4);   // c_T = row 0
                            const float4 bb = *reinterpret_cast<const float4 *>(cBs + 4 * k4);
                            const float4 xx = has_tgt ? *reinterpret_cast<const float4 *>(raw + t * dp + 4 * k4) : tt;
                            const float4 yy = has_src ? *reinterpret_cast<const float4 *>(rawb + t * dp + 4 * k4) : tt;
                            const float2 tv[2] = {make_float2(tt.x, tt.y), make_float2(tt.z, tt.w)};
                            const float2 bv[2] = {make_float2(bb.x, bb.y), make_float2(bb.z, bb.w)};
                            const float2 xv[2] = {make_float2(xx.x, xx.y), make_float2(xx.z, xx.w)};
                            const float2 yv[2] = {make_float2(yy.x, yy.y), make_float2(yy.z, yy.w)};
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                xa[e] = __ffma2_rn(tv[e], m1, xv[e]);                        // a = x - c_T
                                nn2 = __ffma2_rn(xa[e], xa[e], nn2);
                                dd2 = __ffma2_rn(xa[e], __ffma2_rn(bv[e], m1, tv[e]), dd2);   // a . delta
                                const float2 ya = __ffma2_rn(tv[e], m1, yv[e]);              // y - c_T
                                qq2 = __ffma2_rn(ya, ya, qq2);
                            }
                        }
                        // 4 elements = 8 bytes of the 128-byte row; packed 2-wide conversions
                        uint32_t hv[2], lv[2];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const float2 v = xa[e];
                            const __nv_bfloat162 h = __float22bfloat162_rn(v);
                            const __nv_bfloat162 l = __float22bfloat162_rn(__ffma2_rn(__bfloat1622float2(h), m1, v));
                            hv[e] = *reinterpret_cast<const uint32_t *>(&h);
                            lv[e] = *reinterpret_cast<const uint32_t *>(&l);
                        }
                        const int off = t * 128 + (((kst >> 1) ^ (t & 7)) << 4) + (kst & 1) * 8;
                        *reinterpret_cast<uint2 *>(ahi + off) = make_uint2(hv[0], hv[1]);
                        *reinterpret_cast<uint2 *>(alo + off) = make_uint2(lv[0], lv[1]);
                    }
                    nn = nn2.x + nn2.y;
                    dd = dd2.x + dd2.y;
                    qq = qq2.x + qq2.y;
                    if (!has_tgt) nn = dd = 0.f;
                } else {
                // two 4-column chunks per step: 32 contiguous bytes of a row
#pragma unroll 4
                for (int k8 = 0; k8 < TC_K / 8; ++k8) {
                    float xa[8], ya[8];
                    if (2 * k8 < nk4) {
                        const float4 x0 = has_tgt ? __ldg(reinterpret_cast<const float4 *>(xrow + 8 * k8)) : make_float4(0.f, 0.f, 0.f, 0.f);
                        const float4 x1 = has_tgt ? __ldg(reinterpret_cast<const float4 *>(xrow + 8 * k8 + 4)) : make_float4(0.f, 0.f, 0.f, 0.f);
                        const float4 t0 = __ldg(reinterpret_cast<const float4 *>(xt0 + 8 * k8));
                        const float4 t1 = __ldg(reinterpret_cast<const float4 *>(xt0 + 8 * k8 + 4));
                        const float4 b0 = *reinterpret_cast<const float4 *>(cB + 8 * k8);
                        const float4 b1 = *reinterpret_cast<const float4 *>(cB + 8 * k8 + 4);
                        const float4 y0 = has_src ? __ldg(reinterpret_cast<const float4 *>(ysrc + 8 * k8)) : t0;
                        const float4 y1 = has_src ? __ldg(reinterpret_cast<const float4 *>(ysrc + 8 * k8 + 4)) : t1;
                        const float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                        const float ts[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
                        const float bs[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
                        const float ys[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            xa[e] = has_tgt ? xs[e] - ts[e] : 0.f;       // a = x - c_T
                            nn = fmaf(xa[e], xa[e], nn);
                            dd = fmaf(xa[e], ts[e] - bs[e], dd);          // a . delta
                            ya[e] = ys[e] - ts[e];                        // y - c_T
                            qq = fmaf(ya[e], ya[e], qq);
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e) xa[e] = 0.f;
                    }
                    if constexpr (P == ASKIT_PREC_TF32X3) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int c4 = 2 * k8 + h, reg = c4 >> 3, chunk = c4 & 7;
                            float4 hi, lo;
                            hi.x = __uint_as_float(__float_as_uint(xa[4 * h + 0]) & 0xffffe000u);
                            hi.y = __uint_as_float(__float_as_uint(xa[4 * h + 1]) & 0xffffe000u);
                            hi.z = __uint_as_float(__float_as_uint(xa[4 * h + 2]) & 0xffffe000u);
                            hi.w = __uint_as_float(__float_as_uint(xa[4 * h + 3]) & 0xffffe000u);
                            lo.x = xa[4 * h + 0] - hi.x; lo.y = xa[4 * h + 1] - hi.y;
                            lo.z = xa[4 * h + 2] - hi.z; lo.w = xa[4 * h + 3] - hi.w;
                            const int off = reg * REGION + t * 128 + ((chunk ^ (t & 7)) << 4);
                            *reinterpret_cast<float4 *>(ahi + off) = hi;
                            *reinterpret_cast<float4 *>(alo + off) = lo;
                        }
                    } else {
                        // 8 elements = one 16-byte chunk of the 128-byte row
                        uint32_t hv[4], lv[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            float v0 = xa[2 * e], v1 = xa[2 * e + 1];
                            uint16_t h0, h1, l0, l1;
                            const __nv_bfloat16 a0 = __float2bfloat16_rn(v0), a1 = __float2bfloat16_rn(v1);
                            h0 = __bfloat16_as_ushort(a0); h1 = __bfloat16_as_ushort(a1);
                            l0 = __bfloat16_as_ushort(__float2bfloat16_rn(v0 - __bfloat162float(a0)));
                            l1 = __bfloat16_as_ushort(__float2bfloat16_rn(v1 - __bfloat162float(a1)));
                            hv[e] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                            lv[e] = (uint32_t)l0 | ((uint32_t)l1 << 16);
                        }
                        const int off = t * 128 + ((k8 ^ (t & 7)) << 4);
                        *reinterpret_cast<uint4 *>(ahi + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                        *reinterpret_cast<uint4 *>(alo + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
                    }
                }
                }
                (void)cnt;
                // row term |a|^2 + 2 a.delta; column data of source row t:
                // arg = g (2 u sc) + (-sc) p_t + (-sc q) = -sc (p_t + q - 2 u g)
                a_norm[s * 128 + t] = nn + 2.f * dd;
                {
                    // column pairs: [pair][0] = {A_j, A_j+1, B_j, B_j+1}, [pair][1] = {C_j, C_j+1, w_j, w_j+1}
                    float *cp = reinterpret_cast<float *>(colv + s * 128 + 2 * (t >> 1));
                    const int h = t & 1;
                    cp[0 + h] = 2.f * args.g_unscale * sc;
                    cp[2 + h] = -sc * qq;
                    cp[4 + h] = -sc;
                    cp[6 + h] = w0;
                }
                if (RC > 1) {
#pragma unroll
                    for (int z = 0; z < RC; ++z)
                        colw[(s * 128 + t) * RC + z] = (has_src && z < args.r) ? __ldg(wrow + z) : 0.f;
                }
                // generic-proxy stores -> visible to the tensor core's async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(BAR_A_FULL(s));
                if constexpr (S::GATHER) mbar_arrive(BAR_R_EMPTY(s));
            }
            // li now points past this block for this group; realign to the block end
            li = li_block_end;
            ++lb;
        }
    loader_done:;
    } else if (warp < 12) {
        // ----------------------------------------------------------- epilogue
        const int row = tid - 256;                 // TMEM lane = target row of the item
        const int q = warp & 3;                    // this warp's TMEM lane quadrant
        int li = 0;
        for (int ci = args.cta_off[blockIdx.x]; ci < args.cta_off[blockIdx.x + 1] && !*abort_flag; ++ci) {
            const int b = args.cta_blocks[ci];
            for (int it = args.block_off[b]; it < args.block_off[b + 1]; ++it, ++li) {
                const int a = li & 1;
                const uint32_t par = (li >> 1) & 1;
                const EvalItem item = args.items[it];
                const int nrows = item.nrows & 0x7fffffff;
                if (!mbar_wait(BAR_A_FULL(a), par, abort_flag, args.status)) goto epi_done;
                if (!mbar_wait(BAR_T_FULL(a), par, abort_flag, args.status)) goto epi_done;
                tc_fence_after();
                float acc[RC];
#pragma unroll
                for (int z = 0; z < RC; ++z) acc[z] = 0.f;
                float2 acc2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};   // RC == 1
                if (q * 32 < item.cnt) {   // warp-uniform: skip quadrants with no target
                    const float pt = a_norm[a * 128 + row];
                    const float2 pt2 = make_float2(pt, pt);
                    const float4 *cv4 = colv + a * 128;
                    const float *cwp = colw + a * 128 * RC;
                    // columns of 32 in pairs: both TMEM loads issued before one wait
                    auto cols = [&](int c, const uint32_t (&gr)[32]) {
                        float g[32];
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) g[jj] = __uint_as_float(gr[jj]);
                        if constexpr (RC == 1) {
                            // two columns per step with packed FP32x2 FMAs:
                            // arg = g A + (C p + B) = -sc (p + q - 2 u g); columns past
                            // nrows carry w = 0
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
                                const bool h = j & 1;
                                const float A = h ? ab.y : ab.x, B = h ? ab.w : ab.z, Cc = h ? cw.y : cw.x;
                                const float k = ex2_approx(fmaf(g[jj], A, fmaf(Cc, pt, B)));
#pragma unroll
                                for (int z = 0; z < RC; ++z) acc[z] = fmaf(k, cwp[j * RC + z], acc[z]);
                            }
                        }
                    };
                    const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * 128);
#pragma unroll 1
                    for (int c = 0; c < 4 && c * 32 < nrows; c += 2) {
                        uint32_t g0[32], g1[32];
                        const bool two = (c + 1) * 32 < nrows;      // warp-uniform
                        tmem_ld32_async(tbase + (uint32_t)(c * 32), g0);
                        if (two) tmem_ld32_async(tbase + (uint32_t)((c + 1) * 32), g1);
                        tmem_wait_pin(g0);
                        cols(c, g0);
                        if (two) {
                            reg_pin(g1);
                            cols(c + 1, g1);
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
    } else if (warp == 13) {
        // ---------------------------------------------- target-row gatherer (warp 13)
        if constexpr (S::GATHER) {
            const uint32_t bytes = (uint32_t)(TILE_ROWS * args.d_pad * 4);
            int li = 0, issued = 0;
            for (int ci = args.cta_off[blockIdx.x]; ci < args.cta_off[blockIdx.x + 1] && !*abort_flag; ++ci) {
                const int b = args.cta_blocks[ci];
                for (int it = args.block_off[b]; it < args.block_off[b + 1]; ++it, ++li) {
                    const int s = li & 1;
                    if (!mbar_wait(BAR_R_EMPTY(s), ((li >> 1) & 1) ^ 1, abort_flag, args.status)) goto gather_done;
                    const EvalItem item = args.items[it];
                    const int first = args.tgt[item.e0];
                    int r[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int row = 4 * lane + i;   // rows past cnt repeat the first target
                        r[i] = row < item.cnt ? args.tgt[item.e0 + row] : first;
                    }
                    ++issued;
                    if (lane == 0) mbar_expect_tx(BAR_R_FULL(s), bytes);
                    __syncwarp();
                    tma_gather4(sbase + S::RAW + s * S::RAWSTAGE + 4 * lane * args.d_pad * 4, &map_q, 0, r[0], r[1],
                                r[2], r[3], BAR_R_FULL(s));
                }
            }
        gather_done:
            // rows of the last two items may still be landing after an abort
            for (int gg = issued > 2 ? issued - 2 : 0; gg < issued; ++gg) mbar_drain(BAR_R_FULL(gg & 1), (gg >> 1) & 1);
        }
    } else if (warp == 12 && lane == 0) {
        // ------------------------------------------------- TMA + MMA issuer
        // hi + lo of one 128-row sub-block, and its raw FP32 rows (gather path)
        const uint32_t TX = 2 * NREG * REGION + (S::GATHER ? (uint32_t)(TILE_ROWS * args.d_pad * 4 + TC_K * 4) : 0u);
        int li = 0, lb = 0, b_issued = 0;
        for (int ci = args.cta_off[blockIdx.x]; ci < args.cta_off[blockIdx.x + 1] && !*abort_flag; ++ci, ++lb) {
            const int b = args.cta_blocks[ci];
            const EvalItem first = args.items[args.block_off[b]];
            const bool far = first.nrows < 0;
            if (!mbar_wait(BAR_B_EMPTY, (lb & 1) ^ 1, abort_flag, args.status)) goto mma_done;
            b_issued = lb + 1;
            mbar_expect_tx(BAR_B_FULL, TX);
            const CUtensorMap *mh = far ? &map_s_hi : &map_t_hi;
            const CUtensorMap *ml = far ? &map_s_lo : &map_t_lo;
#pragma unroll
            for (int g = 0; g < NREG; ++g) {
                const int x = g * (128 / EB);      // first element of swizzle region g
                tma_load_2d(sbase + S::B_HI + g * REGION, mh, x, first.row0, BAR_B_FULL);
                tma_load_2d(sbase + S::B_LO + g * REGION, ml, x, first.row0, BAR_B_FULL);
            }
            if constexpr (S::GATHER) {
                tma_load_2d(sbase + S::RAWB, far ? &map_rs : &map_rt, 0, first.row0, BAR_B_FULL);
                bulk_copy(sbase + S::CENT, args.cent + (int64_t)first.cidx * TC_K, TC_K * 4, BAR_B_FULL);
            }
            const int i0 = args.block_off[b], i1 = args.block_off[b + 1];
            for (int it = i0; it < i1; ++it, ++li) {
                const int s = li & 1;
                const uint32_t par = (li >> 1) & 1;
                if (!mbar_wait(BAR_A_FULL(s), par, abort_flag, args.status)) goto mma_done;
                if (it == i0 && !mbar_wait(BAR_B_FULL, lb & 1, abort_flag, args.status)) goto mma_done;
                if (!mbar_wait(BAR_T_EMPTY(s), par ^ 1, abort_flag, args.status)) goto mma_done;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(s * 128);
                const uint32_t a_hi = sbase + S::A0 + s * 2 * S::OPB, a_lo = a_hi + S::OPB;
                const uint32_t b_hi = sbase + S::B_HI, b_lo = sbase + S::B_LO;
                // The tensor core rounds each accumulation step to the running
                // sum's precision, so the small cross terms go in first (while the
                // accumulator is small) and the hi*hi products last.
#pragma unroll
                for (int k = 0; k < KSTEPS; ++k) {
                    // K step k: 32 bytes into swizzle region k / 4
                    const uint32_t off = (uint32_t)((k >> 2) * REGION + (k & 3) * 32);
                    tc_mma<P>(d_tmem, sw128_desc(a_hi + off), sw128_desc(b_lo + off), IDESC, k > 0);
                    tc_mma<P>(d_tmem, sw128_desc(a_lo + off), sw128_desc(b_hi + off), IDESC, 1);
                }
#pragma unroll
                for (int k = 0; k < KSTEPS; ++k) {
                    const uint32_t off = (uint32_t)((k >> 2) * REGION + (k & 3) * 32);
                    tc_mma<P>(d_tmem, sw128_desc(a_hi + off), sw128_desc(b_hi + off), IDESC, 1);
                }
                tc_commit(BAR_A_EMPTY(s));
                tc_commit(BAR_T_FULL(s));
                if (it == i1 - 1) tc_commit(BAR_B_EMPTY);
            }
        }
    mma_done:
        // the last sub-block's copies may still be landing after an abort
        if (b_issued > 0) mbar_drain(BAR_B_FULL, (b_issued - 1) & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 12) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Tensor maps of the four source operand arrays for one precision.
struct TcState {
    CUtensorMap map[2][4];   // [precision: 0 tf32, 1 bf16][t_hi, t_lo, s_hi, s_lo]
    bool ready[2] = {false, false};
    CUtensorMap raw_t, raw_s;   // raw FP32 source rows, 128-row boxes (gather path)
    bool raw_ready = false;
    void *encode = nullptr;     // cuTensorMapEncodeTiled
};

askit_status encode_map(EncodeTiledFn fn, CUtensorMap *m, void *base, int64_t rows, int ty) {
    const bool f32 = ty == 0;
    const int eb = f32 ? 4 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)TC_K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)TC_K * eb};
    cuuint32_t box[2] = {(cuuint32_t)(128 / eb), (cuuint32_t)TILE_ROWS};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, ty == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                       : ty == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        askit_set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return ASKIT_ERR_CUDA;
    }
    return ASKIT_OK;
}

// Unswizzled FP32 map over [rows, cols] with boxes of box_rows full rows
// (box_rows = 1 for tile::gather4).
askit_status encode_raw(EncodeTiledFn fn, CUtensorMap *m, const void *base, int64_t rows, int cols, int box_rows) {
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 4};
    cuuint32_t box[2] = {(cuuint32_t)cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        askit_set_error("cuTensorMapEncodeTiled (raw rows) failed (%d)", (int)r);
        return ASKIT_ERR_CUDA;
    }
    return ASKIT_OK;
}

std::mutex g_tc_mu;   // tensor-map state and launch attributes are built once, under a lock

askit_status tc_state(askit_tree t, int pi, TcState **out) {
    std::lock_guard<std::mutex> lock(g_tc_mu);
    if (!t->tc) t->tc = new TcState();
    TcState *st = (TcState *)t->tc;
    if (!st->encode) {
        void *fnp = nullptr;
        cudaDriverEntryPointQueryResult q;
        ASK_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fnp, 12000, cudaEnableDefault, &q));
        if (!fnp || q != cudaDriverEntryPointSuccess) {
            askit_set_error("cuTensorMapEncodeTiled not available");
            return ASKIT_ERR_CUDA;
        }
        st->encode = fnp;
    }
    EncodeTiledFn fn = (EncodeTiledFn)st->encode;
    if (!st->raw_ready) {
        ASK_TRY(encode_raw(fn, &st->raw_t, t->Xt, t->N_pad, t->d_pad, TILE_ROWS));
        ASK_TRY(encode_raw(fn, &st->raw_s, t->Xs, t->srows, t->d_pad, TILE_ROWS));
        st->raw_ready = true;
    }
    if (!st->ready[pi]) {
        const int ty = pi;   // 0 fp32 (tf32), 1 bf16
        void *th = pi == 0 ? (void *)t->Xt_hi : (void *)t->Xt_bhi;
        void *tl = pi == 0 ? (void *)t->Xt_lo : (void *)t->Xt_blo;
        void *sh = pi == 0 ? (void *)t->Xs_hi : (void *)t->Xs_bhi;
        void *sl = pi == 0 ? (void *)t->Xs_lo : (void *)t->Xs_blo;
        ASK_TRY(encode_map(fn, &st->map[pi][0], th, t->N_pad, ty));
        ASK_TRY(encode_map(fn, &st->map[pi][1], tl, t->N_pad, ty));
        ASK_TRY(encode_map(fn, &st->map[pi][2], sh, t->srows, ty));
        ASK_TRY(encode_map(fn, &st->map[pi][3], sl, t->srows, ty));
        st->ready[pi] = true;
    }
    *out = st;
    return ASKIT_OK;
}

template <int P, int RC>
askit_status launch(askit_tree t, TcState *st, const CUtensorMap &map_q, const TcArgs &a, int a_grid,
                    cudaStream_t s) {
    using S = Smem<P>;
    const int pi = P == ASKIT_PREC_TF32X3 ? 0 : 1;
    const size_t smem = S::BYTES + 1024;
    static bool attr_set = false;
    {
        std::lock_guard<std::mutex> lock(g_tc_mu);
        if (!attr_set) {
            ASK_CUDA(cudaFuncSetAttribute(eval_tc_kernel<P, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr_set = true;
        }
    }
    const unsigned grid = (unsigned)a_grid;
    ASK_TRY(ktimer_mark(t, s, false));
    eval_tc_kernel<P, RC><<<grid, TC_THREADS, smem, s>>>(st->map[pi][0], st->map[pi][1], st->map[pi][2],
                                                         st->map[pi][3], map_q, st->raw_t, st->raw_s, a);
    ASK_LAUNCH();
    return ktimer_mark(t, s, true);
}

}  // namespace

askit_status eval_tc(askit_tree t, const WeightCtx &c, int precision, const float *Xq, int64_t ldq,
                     int64_t q_rows, const QuerySplit *qs, const WorkLists &w, float *partial, cudaStream_t s) {
    if (t->d > TC_K) return eval_tc_wide(t, c, precision, Xq, ldq, q_rows, w, partial, s);
    // FP16x3 with pre-split, globally centered targets where that keeps FP32
    // grade (eval_g16.cu)
    if (precision == ASKIT_PREC_FP16X3 && qs && use_g16(t)) return eval_g16(t, c, *qs, w, partial, s);
    // FP16x3 centers both sides on the sub-block mean (eval_tc16.cu); BF16x3
    // keeps the per-item target centering below: its 8-bit significands leave
    // a residual of about 2^-17 of |a| |b| per product, so the smaller |a| of
    // the per-item center is what keeps it within the split-path tolerance
    if (precision == ASKIT_PREC_FP16X3) return eval_tc16(t, c, precision, Xq, ldq, q_rows, w, partial, s);
    if (precision != ASKIT_PREC_TF32X3 && precision != ASKIT_PREC_BF16X3) {
        askit_set_error("unknown tensor-core precision %d", precision);
        return ASKIT_ERR_INVALID_ARG;
    }
    if (c.r > Smem<ASKIT_PREC_TF32X3>::RC_MAX) {
        askit_set_error("tensor-core evaluation covers r <= %d; use ASKIT_PREC_SIMT_FP32", Smem<ASKIT_PREC_TF32X3>::RC_MAX);
        return ASKIT_ERR_UNSUPPORTED;
    }
    if (w.n_blocks == 0) return ASKIT_OK;
    if (ldq != t->d_pad) {
        askit_set_error("target rows must have d_pad columns");
        return ASKIT_ERR_INVALID_ARG;
    }
    TcState *st = nullptr;
    ASK_TRY(tc_state(t, precision == ASKIT_PREC_TF32X3 ? 0 : 1, &st));
    // gather map over this call's target rows (one box row per gathered row)
    CUtensorMap map_q;
    ASK_TRY(encode_raw((EncodeTiledFn)st->encode, &map_q, Xq, q_rows, t->d_pad, 1));
    TcArgs a;
    a.items = w.items;
    a.block_off = w.block_off;
    a.cta_off = w.cta_off;
    a.cta_blocks = w.cta_blocks;
    a.tgt = w.tgt;
    a.Xq = Xq;
    a.ldq = ldq;
    a.d_pad = t->d_pad;
    a.cent = t->cent;
    a.sc_t = t->sc_t;
    a.sc_s = t->sc_s;
    a.Xt = t->Xt;
    a.Xs = t->Xs;
    a.Wt = c.Wt;
    a.Ws = c.Ws;
    a.r = c.r;
    a.partial = partial;
    a.status = t->d_status;
    a.f16_scale = 1.f;
    a.g_unscale = 1.f / (a.f16_scale * a.f16_scale);
    if (precision == ASKIT_PREC_TF32X3) {
        if (c.r == 1) return launch<ASKIT_PREC_TF32X3, 1>(t, st, map_q, a, w.n_ctas, s);
        if (c.r <= 4) return launch<ASKIT_PREC_TF32X3, 4>(t, st, map_q, a, w.n_ctas, s);
        return launch<ASKIT_PREC_TF32X3, 16>(t, st, map_q, a, w.n_ctas, s);
    }
    if (precision == ASKIT_PREC_BF16X3) {
        if (c.r == 1) return launch<ASKIT_PREC_BF16X3, 1>(t, st, map_q, a, w.n_ctas, s);
        if (c.r <= 4) return launch<ASKIT_PREC_BF16X3, 4>(t, st, map_q, a, w.n_ctas, s);
        return launch<ASKIT_PREC_BF16X3, 16>(t, st, map_q, a, w.n_ctas, s);
    }
    askit_set_error("unknown tensor-core precision %d", precision);
    return ASKIT_ERR_INVALID_ARG;
}

void eval_tc_free(askit_tree t) {
    delete (TcState *)t->tc;
    t->tc = nullptr;
    eval_tc_wide_free(t);
    eval_tc16_free(t);
    eval_g16_free(t);
}
