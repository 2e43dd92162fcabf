// Evaluate (Algorithm 4) on the tcgen05 tensor cores with FP16x3 split
// operands, d <= 64 (the kernel is written for both 16-bit types; BF16x3 is
// served by eval_tc.cu's per-item centering, see there).
//
// Work item = one source sub-block (<= 128 rows of a leaf's points for the
// direct near field, or of a node's skeleton for the far field) against up
// to 128 targets that all need it (eval_lists.cu).  Both sides are centered
// on the sub-block's mean c_B:
//
//     a = x - c_B (targets, centered and split on chip)
//     b = y - c_B (sources, pre-split in HBM)
//     r^2 = |a|^2 + |b|^2 - 2 a.b,   G = a.b on the tensor cores
//     partial_t = sum_j exp2(-c log2(e) r^2 / h_j^2) w_j
//
// The products are split in three (hi*hi + hi*lo + lo*hi) with FP32
// accumulation, the small cross terms issued first.  A sub-block's column
// data (c log2(e) / h_j^2, |b_j|^2, w_j) does not depend on the targets: it
// is built once per Evaluate (tc16_cols_kernel) and bulk-copied with the
// sub-block, so the loaders only center and split target rows.
//
// One CTA per SM; r <= 4: 576 threads (r = 16: 448, numbers in brackets):
//   warps 0-7   two loader groups taking alternate items: each warp centers
//               and splits 32 target rows (gathered by the last warp), two
//               rows at a time, into the 128-byte swizzled K-major layout and
//               forms |a|^2 in a fixed order;
//   warps 8-15  two epilogue groups, each taking one half of every item's
//               columns [8-11: one group, all columns]: tcgen05.ld of their
//               32 TMEM lanes (one row each), exponent on MUFU.EX2, reduction
//               against the weights; the second half's sums reach the first
//               group through shared memory and are added last;
//   warp 16 [12] TMEM allocation; lane 0 loads each sub-block (TMA tiles of
//               the pre-split rows, bulk copies of its center and column
//               data) and issues the tcgen05.mma instructions;
//   warp 17 [13] TMA tile::gather4 of each item's target rows (8-row tiled
//               boxes for runs of consecutive rows), two or three stages.
// Four TMEM accumulators (4 x 128 columns) let the MMAs run up to three items
// ahead of the epilogue.  Every mbarrier wait is bounded: on timeout the
// kernel records ASK_DEV_TIMEOUT, all roles leave their loops, producers
// wait for their copies in flight, and TMEM is freed before the kernel
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>

#include "askit_impl.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace tcx;

constexpr int T16_ROWS = 128;
constexpr int T16_REGION = T16_ROWS * 128;     // 128 rows x 128 bytes (64 16-bit elements), swizzled
constexpr uint32_t T16_TMEM_COLS = 512;        // four 128-column FP32 accumulators

// NRAW: stages of gathered target rows (2 or 3); NB: sub-blocks per item
// (1, or 2 for the paired 256-column items of one node); NACC = 4 / NB
// TMEM accumulators of 128 NB columns.  Chosen by askit_autotune.
template <int RC, int NRAW, int NB>
struct S16 {
    static constexpr int NACC = 4 / NB;
    static constexpr int B_HI = 0, B_LO = NB * T16_REGION;    // NB x 128 rows each, contiguous
    static constexpr int A0 = 2 * NB * T16_REGION;            // stage s: hi at A0 + 2s REGION, lo + REGION
    static constexpr int RAW = A0 + 4 * T16_REGION;           // [NRAW] stages of 128 rows x d_pad floats
    static constexpr int RAWSTAGE = T16_ROWS * TC_K * 4;
    static constexpr int BLK = RAW + NRAW * RAWSTAGE;         // [2] per-item-block slots
    static constexpr int BLK_CENT = 0;                        // float [64] c_B
    static constexpr int BLK_COLV = 256;                      // float4 [128 NB] pair-interleaved column data
    static constexpr int BLK_COLW = BLK_COLV + NB * 128 * 16; // float [128 NB][RC] weights (RC > 1)
    static constexpr int COLW_BYTES = RC > 1 ? NB * 128 * RC * 4 : 0;
    static constexpr int BLKSLOT = BLK_COLW + COLW_BYTES;
    static constexpr int ANORM = BLK + 2 * BLKSLOT;           // float [NACC][128] |a|^2
    static constexpr bool EPI2 = RC <= 4;                     // two epilogue groups (column halves)
    static constexpr int THREADS = EPI2 ? 576 : 448;          // 2 loader groups, 1 or 2 epilogue groups, 2 warps
    static constexpr int XBUF = ANORM + 4 * 128 * 4;          // float [NACC][128][RC]: second half's sums
    static constexpr int BAR = XBUF + (EPI2 ? 4 * 128 * RC * 4 : 0);   // 32 mbarriers
    static constexpr int MISC = BAR + 32 * 8;                 // tmem address, abort flag
    static constexpr int BYTES = MISC + 16;
};

struct T16Args {
    const EvalItem *items;
    const int32_t *block_off;
    const int32_t *cta_off, *cta_blocks;
    const int32_t *tgt;       // entry -> target slot (row of Xq)
    int d_pad;
    const float *cent;        // [n_sub, TC_K]
    const float4 *colv;       // [n_sub, 128] pair-interleaved {A_j, A_j+1, B_j, B_j+1}, {C_j, C_j+1, w_j, w_j+1}
    const float *colw;        // [n_sub, 128, RC] (RC > 1)
    int r;
    float f16_scale;
    int runs;                 // 8-row tiled loads for runs of consecutive target rows
    float uni_a, uni_c;       // UNI: A = 2 sc / scale^2 and C = -sc
    // UNI == 2 (kNN shortlist): emit every source with D <= U_q (1 + eta) + eta (|a|^2 + |b|^2)
    const float *knn_u;       // [queries] upper bound of each query's kappa-th distance
    int *knn_cnt;             // [queries] candidates emitted
    int32_t *knn_cand;        // [queries, knn_cap] tree positions of the candidates
    int knn_cap;
    float knn_eta, knn_m2u;   // margin, and -2 / scale^2
    const int32_t *partner;   // [n_blocks] paired follower block, or -1 (NB == 2)
    float *partial;
    int *status;
    int spin;                 // polls of a bounded mbarrier wait before it gives up
};

// UNI == 1: one bandwidth for all sources (c log2(e) / h^2 = sc for every j):
// the column data is then {B_j, B_j+1, w_j, w_j+1} per pair (8 bytes a
// column), half of the general layout, and A = 2 sc / scale^2, C = -sc are
// scalars.  UNI == 2: the kernel is the exact kNN's tensor-core shortlist
// (queries against every source): the column data is {|b_j|^2 (1 - eta),
// the same for j+1, position_j, position_j+1}; no kernel sum is formed.
template <int P, int RC, int NRAW, int NB, int UNI>
__global__ void __launch_bounds__(S16<RC, NRAW, NB>::THREADS, 1)
eval_tc16_kernel(const __grid_constant__ CUtensorMap map_t_hi, const __grid_constant__ CUtensorMap map_t_lo,
                 const __grid_constant__ CUtensorMap map_s_hi, const __grid_constant__ CUtensorMap map_s_lo,
                 const __grid_constant__ CUtensorMap map_q, const __grid_constant__ CUtensorMap map_q8,
                 const T16Args args) {
    using S = S16<RC, NRAW, NB>;
    constexpr int NACC = S::NACC;
    // r <= 4: two epilogue groups (warps 8-11 and 12-15) take the two
    // halves of each item's columns, so two warps per SM sub-partition share
    // the exponentials; r = 16: one epilogue group (its weight sums leave no
    // room for the exchange buffer)
    constexpr bool EPI2 = S::EPI2;
    constexpr int NLG = 2;
    constexpr int EPI_W0 = 4 * NLG;
    constexpr int EPI_END = EPI2 ? 16 : 12;
    constexpr int W_MMA = EPI_END, W_GAT = EPI_END + 1;
    constexpr int NEPI = (EPI_END - EPI_W0) * 32;
    static_assert(!UNI || RC == 1, "the uniform-bandwidth and kNN layouts serve r = 1");
    constexpr uint32_t FMT = P == ASKIT_PREC_BF16X3 ? 1u : 0u;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(sm);
    float *a_norm = reinterpret_cast<float *>(sm + S::ANORM);
    const uint32_t bar0 = sbase + S::BAR;
    auto BAR_A_FULL = [&](int s) { return bar0 + 8 * s; };           // loader group stored A stage s (128)
    auto BAR_A_EMPTY = [&](int s) { return bar0 + 8 * (2 + s); };    // MMAs reading A stage s done (commit)
    auto BAR_R_FULL = [&](int s) { return bar0 + 8 * (4 + s); };     // target rows of raw stage s landed
    auto BAR_R_EMPTY = [&](int s) { return bar0 + 8 * (7 + s); };    // loaders done with raw stage s (128)
    const uint32_t BAR_B_FULL = bar0 + 8 * 10, BAR_B_EMPTY = bar0 + 8 * 11;
    auto BAR_BLK_FULL = [&](int s) { return bar0 + 8 * (12 + s); };  // center + column data of slot s landed
    auto BAR_BLK_EMPTY = [&](int s) { return bar0 + 8 * (14 + s); }; // epilogue done with slot s (128)
    auto BAR_T_FULL = [&](int a) { return bar0 + 8 * (16 + a); };    // accumulator a complete (commit)
    auto BAR_T_EMPTY = [&](int a) { return bar0 + 8 * (20 + a); };   // epilogue drained accumulator a (128)
    auto BAR_N_EMPTY = [&](int a) { return bar0 + 8 * (24 + a); };   // epilogue read |a|^2 slot a (NEPI)
    auto BAR_X_FULL = [&](int a) { return bar0 + 8 * (28 + a); };    // second epilogue half's sums of a (128)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + S::MISC);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + S::MISC + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(BAR_A_FULL(s), 128);
            mbar_init(BAR_A_EMPTY(s), 1);
            mbar_init(BAR_BLK_FULL(s), 1);
            mbar_init(BAR_BLK_EMPTY(s), NEPI);
        }
        for (int s = 0; s < NRAW; ++s) {
            mbar_init(BAR_R_FULL(s), 1);
            mbar_init(BAR_R_EMPTY(s), 128);
        }
        mbar_init(BAR_B_FULL, 1);
        mbar_init(BAR_B_EMPTY, 1);
        for (int a = 0; a < NACC; ++a) {
            mbar_init(BAR_T_FULL(a), 1);
            mbar_init(BAR_T_EMPTY(a), NEPI);
            mbar_init(BAR_N_EMPTY(a), NEPI);
            mbar_init(BAR_X_FULL(a), 128);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == W_MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(T16_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int c_begin = args.cta_off[blockIdx.x], c_end = args.cta_off[blockIdx.x + 1];

    if (warp < EPI_W0) {
        // ------------------------------------------------------------ loaders
        // A warp converts its 32 rows two at a time: lane (h, k) takes
        // 4-coordinate chunk k of row 2i + h, so each half-warp reads one
        // row's contiguous bytes (no bank conflicts) and writes the row's
        // whole 128-byte swizzled line.  |a|^2 is summed over the chunks by a
        // butterfly across the 16 lanes in a fixed order, so a row's value
        // does not depend on its position in the item.
        const int grp = warp >> 2, wl = warp & 3;
        const int hh = lane >> 4, kc = lane & 15;
        const int dp = args.d_pad, nk4 = dp / 4;
        const bool kin = kc < nk4;
        const float2 m1 = make_float2(-1.f, -1.f), z2 = make_float2(0.f, 0.f);
        const float2 sc2 = make_float2(args.f16_scale, args.f16_scale);
        const float inv_sc2 = 1.f / (args.f16_scale * args.f16_scale);   // a power of 2
        int li = 0, lb = 0;
        for (int ci = c_begin; ci < c_end && !*abort_flag; ++ci, ++lb) {
            const int b = args.cta_blocks[ci];
            const int i0 = args.block_off[b], i1 = args.block_off[b + 1];
            bool need_blk = true;
            float4 cc = make_float4(0.f, 0.f, 0.f, 0.f);   // this lane's chunk of c_B
            // this group's first item of the block: li and it advance together
            const int first = i0 + (NLG == 2 ? ((grp - li) & 1) : 0);
            int cnt_next = first < i1 ? args.items[first].cnt : 0;
            for (int it = i0; it < i1; ++it, ++li) {
                if (NLG == 2 && (li & 1) != grp) continue;
                const int cnt = cnt_next;
                if (it + NLG < i1) cnt_next = args.items[it + NLG].cnt;   // in flight while this item waits
                const int sa = li & 1, sr = li % NRAW, a4 = li % NACC;
                if (!mbar_wait(BAR_A_EMPTY(sa), ((li >> 1) & 1) ^ 1, abort_flag, args.status, args.spin)) goto loader_done;
                // the |a|^2 slot of this item's accumulator: free once the
                // epilogue of the item NACC back has read it (at its start)
                if (!mbar_wait(BAR_N_EMPTY(a4), ((li / NACC) & 1) ^ 1, abort_flag, args.status, args.spin)) goto loader_done;
                if (!mbar_wait(BAR_R_FULL(sr), (li / NRAW) & 1, abort_flag, args.status, args.spin)) goto loader_done;
                if (need_blk) {
                    if (!mbar_wait(BAR_BLK_FULL(lb & 1), (lb >> 1) & 1, abort_flag, args.status, args.spin)) goto loader_done;
                    need_blk = false;
                    if (kin)
                        cc = *reinterpret_cast<const float4 *>(sm + S::BLK + (lb & 1) * S::BLKSLOT + S::BLK_CENT +
                                                               16 * kc);
                    if constexpr (P == ASKIT_PREC_FP16X3) {
                        // -c_B * scale, exact (the scale is a power of 2): one fused
                        // operation then gives (x - c_B) * scale with a single rounding
                        cc = make_float4(-cc.x * args.f16_scale, -cc.y * args.f16_scale, -cc.z * args.f16_scale,
                                         -cc.w * args.f16_scale);
                    }
                }
                const float *raw = reinterpret_cast<const float *>(sm + S::RAW + sr * S::RAWSTAGE);
                uint8_t *ahi = sm + S::A0 + sa * 2 * T16_REGION;
                uint8_t *alo = ahi + T16_REGION;
                float part[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int row = 32 * wl + 2 * i + hh;
                    float2 xa[2] = {z2, z2};
                    if (kin && row < cnt) {
                        const float4 xx = *reinterpret_cast<const float4 *>(raw + row * dp + 4 * kc);
                        if constexpr (P == ASKIT_PREC_FP16X3) {   // scaled: v = (x - c_B) * scale
                            xa[0] = __ffma2_rn(make_float2(xx.x, xx.y), sc2, make_float2(cc.x, cc.y));
                            xa[1] = __ffma2_rn(make_float2(xx.z, xx.w), sc2, make_float2(cc.z, cc.w));
                        } else {
                            xa[0] = __ffma2_rn(make_float2(cc.x, cc.y), m1, make_float2(xx.x, xx.y));
                            xa[1] = __ffma2_rn(make_float2(cc.z, cc.w), m1, make_float2(xx.z, xx.w));
                        }
                    }
                    const float2 sq = __ffma2_rn(xa[1], xa[1], __fmul2_rn(xa[0], xa[0]));
                    part[i] = sq.x + sq.y;
                    uint32_t hv[2], lv[2];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        if constexpr (P == ASKIT_PREC_FP16X3) {
                            const float2 v = xa[e];
                            const __half2 h = __float22half2_rn(v);
                            const __half2 l = __float22half2_rn(__ffma2_rn(__half22float2(h), m1, v));
                            hv[e] = *reinterpret_cast<const uint32_t *>(&h);
                            lv[e] = *reinterpret_cast<const uint32_t *>(&l);
                        } else {
                            const __nv_bfloat162 h = __float22bfloat162_rn(xa[e]);
                            const __nv_bfloat162 l = __float22bfloat162_rn(__ffma2_rn(__bfloat1622float2(h), m1, xa[e]));
                            hv[e] = *reinterpret_cast<const uint32_t *>(&h);
                            lv[e] = *reinterpret_cast<const uint32_t *>(&l);
                        }
                    }
                    const int off = row * 128 + (((kc >> 1) ^ (row & 7)) << 4) + (kc & 1) * 8;
                    *reinterpret_cast<uint2 *>(ahi + off) = make_uint2(hv[0], hv[1]);
                    *reinterpret_cast<uint2 *>(alo + off) = make_uint2(lv[0], lv[1]);
                }
                // butterfly over the 16 chunk lanes: after the step with mask m
                // a lane keeps the rows whose index bit m matches its own, so
                // lane k ends with row 2k + h, each sum paired the same way
#pragma unroll
                for (int m = 8; m >= 1; m >>= 1) {
                    const bool up = kc & m;
#pragma unroll
                    for (int q = 0; q < m; ++q) {
                        const float send = up ? part[q] : part[q + m];
                        const float keep = up ? part[q + m] : part[q];
                        part[q] = keep + __shfl_xor_sync(0xffffffffu, send, m);
                    }
                }
                // FP16x3: the sums of the scaled rows, scaled back exactly
                a_norm[a4 * 128 + 32 * wl + 2 * kc + hh] = P == ASKIT_PREC_FP16X3 ? part[0] * inv_sc2 : part[0];
                // generic-proxy stores -> visible to the tensor core's async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(BAR_A_FULL(sa));
                mbar_arrive(BAR_R_EMPTY(sr));
            }
        }
    loader_done:;
    } else if (warp < EPI_END) {
        // ----------------------------------------------------------- epilogue
        const int q = warp & 3;                    // this warp's TMEM lane quadrant
        const int row = q * 32 + lane;             // TMEM lane = target row of the item
        const int eg = EPI2 ? (warp - EPI_W0) >> 2 : 0; // column half of this group
        int li = 0, lb = 0;
        for (int ci = c_begin; ci < c_end && !*abort_flag; ++ci, ++lb) {
            const int b = args.cta_blocks[ci];
            const int bs = lb & 1;
            if (!mbar_wait(BAR_BLK_FULL(bs), (lb >> 1) & 1, abort_flag, args.status, args.spin)) goto epi_done;
            const float4 *cv4 = reinterpret_cast<const float4 *>(sm + S::BLK + bs * S::BLKSLOT + S::BLK_COLV);
            const float *cwp = reinterpret_cast<const float *>(sm + S::BLK + bs * S::BLKSLOT + S::BLK_COLW);
            const int i0 = args.block_off[b], i1 = args.block_off[b + 1];
            // a paired follower's columns follow the leader's 128
            const int pb = NB == 2 ? args.partner[b] : -1;
            const int f0 = pb >= 0 ? args.block_off[pb] : 0;
            const int ncols_f = pb >= 0 ? (args.items[f0].nrows & 0x7fffffff) : 0;
            EvalItem nxt = args.items[i0];
            for (int it = i0; it < i1; ++it, ++li) {
                const int a4 = li % NACC;
                const EvalItem item = nxt;
                if (it + 1 < i1) nxt = args.items[it + 1];   // in flight while this item waits
                const int nrows = (item.nrows & 0x7fffffff) + ncols_f;
                const int e0f = pb >= 0 ? args.items[f0 + (it - i0)].e0 : 0;
                if (!mbar_wait(BAR_T_FULL(a4), (li / NACC) & 1, abort_flag, args.status, args.spin)) goto epi_done;
                tc_fence_after();
                const float pt = a_norm[a4 * 128 + row];   // NACC <= 4 slots
                mbar_arrive(BAR_N_EMPTY(a4));
                float acc[RC];
#pragma unroll
                for (int z = 0; z < RC; ++z) acc[z] = 0.f;
                float2 acc2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};   // RC == 1
                float2 accw[RC > 1 ? RC / 2 : 1];                                    // RC > 1
#pragma unroll
                for (int z = 0; z < (RC > 1 ? RC / 2 : 1); ++z) accw[z] = make_float2(0.f, 0.f);
                // kNN shortlist: this row's query and its bound (loaded before the wait)
                const int qs = UNI == 2 && row < item.cnt ? args.tgt[item.e0 + row] : -1;
                const float qu = qs >= 0 ? args.knn_u[qs] : 0.f;
                if (q * 32 < item.cnt) {   // warp-uniform: skip quadrants with no target
                    const float2 pt2 = make_float2(pt, pt);
                    // arg = g A + (C p + B) = -sc (p + q - 2 g / scale^2); columns past
                    // nrows carry A = B = C = w = 0
                    const float rth = qs >= 0 ? qu * (1.f + args.knn_eta) + args.knn_eta * pt : -INFINITY;
                    const float2 m2u2 = make_float2(args.knn_m2u, args.knn_m2u);
                    auto emit = [&](uint32_t pos) {
                        const int k = atomicAdd(args.knn_cnt + qs, 1);
                        if (k < args.knn_cap) args.knn_cand[(int64_t)qs * args.knn_cap + k] = (int32_t)pos;
                    };
                    auto cols = [&](int c, const uint32_t (&gr)[32]) {
                        if constexpr (UNI == 2) {
#pragma unroll
                            for (int jj = 0; jj < 32; jj += 2) {
                                const float4 bp = cv4[(c * 32 + jj) >> 1];   // {B'_j, B'_j+1, pos_j, pos_j+1}
                                const float2 inner = __fadd2_rn(pt2, make_float2(bp.x, bp.y));
                                const float2 dd = __ffma2_rn(make_float2(__uint_as_float(gr[jj]), __uint_as_float(gr[jj + 1])),
                                                             m2u2, inner);
                                if (dd.x <= rth) emit(__float_as_uint(bp.z));
                                if (dd.y <= rth) emit(__float_as_uint(bp.w));
                            }
                        } else if constexpr (RC == 1 && UNI == 1) {
                            const float2 a2 = make_float2(args.uni_a, args.uni_a);
                            const float2 c2 = make_float2(args.uni_c, args.uni_c);
#pragma unroll
                            for (int jj = 0; jj < 32; jj += 2) {
                                const float4 bw = cv4[(c * 32 + jj) >> 1];   // {B_j, B_j+1, w_j, w_j+1}
                                const float2 inner = __ffma2_rn(c2, pt2, make_float2(bw.x, bw.y));
                                const float2 arg = __ffma2_rn(make_float2(__uint_as_float(gr[jj]), __uint_as_float(gr[jj + 1])),
                                                              a2, inner);
                                const float2 k = make_float2(ex2_approx(arg.x), ex2_approx(arg.y));
                                acc2[(jj >> 1) & 1] = __ffma2_rn(k, make_float2(bw.z, bw.w), acc2[(jj >> 1) & 1]);
                            }
                        } else if constexpr (RC == 1) {
#pragma unroll
                            for (int jj = 0; jj < 32; jj += 2) {
                                const float4 ab = cv4[c * 32 + jj];
                                const float4 cw = cv4[c * 32 + jj + 1];
                                const float2 inner = __ffma2_rn(make_float2(cw.x, cw.y), pt2, make_float2(ab.z, ab.w));
                                const float2 arg = __ffma2_rn(make_float2(__uint_as_float(gr[jj]), __uint_as_float(gr[jj + 1])),
                                                              make_float2(ab.x, ab.y), inner);
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
                                const float k = ex2_approx(fmaf(__uint_as_float(gr[jj]), A, fmaf(Cc, pt, B)));
                                // the r weight sums as packed pairs: the same fused
                                // products in the same order, half the instructions
                                const float2 k2 = make_float2(k, k);
                                const float4 *w4 = reinterpret_cast<const float4 *>(cwp + j * RC);
#pragma unroll
                                for (int z = 0; z < RC / 4; ++z) {
                                    const float4 wv = w4[z];
                                    accw[2 * z] = __ffma2_rn(k2, make_float2(wv.x, wv.y), accw[2 * z]);
                                    accw[2 * z + 1] = __ffma2_rn(k2, make_float2(wv.z, wv.w), accw[2 * z + 1]);
                                }
                            }
                        }
                    };
                    const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a4 * 128 * NB);
                    // 32-column chunks; the TMEM load of chunk c + 1 is in flight
                    // while chunk c is computed (two register buffers).  With two
                    // groups, group g takes chunks [c_lo, c_hi) of its half.
                    const int nch = (nrows + 31) >> 5;
                    const int hch = EPI2 ? (nch + 1) >> 1 : nch;
                    const int c_lo = eg * hch, c_hi = min(nch, c_lo + hch);
                    if constexpr (RC >= 16) {
                        // r = 16: the weight sums give each chunk enough work to
                        // cover the load; one buffer leaves registers to them.  The
                        // two column halves are summed apart and then added, the
                        // order the two-group epilogue of r <= 4 uses, so a weight
                        // vector's result does not depend on how many others share
                        // its evaluation
                        const int hsplit = (nch + 1) >> 1;
                        float2 h0[RC / 2];
                        uint32_t ga[32];
#pragma unroll 1
                        for (int c = 0; c < nch; ++c) {
                            if (c == hsplit) {
#pragma unroll
                                for (int z = 0; z < RC / 2; ++z) {
                                    h0[z] = accw[z];
                                    accw[z] = make_float2(0.f, 0.f);
                                }
                            }
                            tmem_ld32_async(tbase + (uint32_t)(c * 32), ga);
                            tmem_wait_pin(ga);
                            cols(c, ga);
                        }
                        if (nch > hsplit) {
#pragma unroll
                            for (int z = 0; z < RC / 2; ++z) accw[z] = __fadd2_rn(h0[z], accw[z]);
                        } else {
#pragma unroll
                            for (int z = 0; z < RC / 2; ++z) accw[z] = __fadd2_rn(accw[z], make_float2(0.f, 0.f));
                        }
                    } else if (EPI2) {
                        // two warps per sub-partition: one buffer each, the other
                        // warp's work covers the load
                        uint32_t ga[32];
#pragma unroll 1
                        for (int c = c_lo; c < c_hi; ++c) {
                            tmem_ld32_async(tbase + (uint32_t)(c * 32), ga);
                            tmem_wait_pin(ga);
                            cols(c, ga);
                        }
                    } else if (c_lo < c_hi) {
                        uint32_t ga[32], gb[32];
                        tmem_ld32_async(tbase + (uint32_t)(c_lo * 32), ga);
                        tmem_wait_pin(ga);
#pragma unroll 1
                        for (int c = c_lo; c < c_hi; c += 2) {
                            const bool h1 = c + 1 < c_hi, h2 = c + 2 < c_hi;   // warp-uniform
                            if (h1) tmem_ld32_async(tbase + (uint32_t)((c + 1) * 32), gb);
                            cols(c, ga);
                            if (h1) {
                                tmem_wait_pin(gb);
                                if (h2) tmem_ld32_async(tbase + (uint32_t)((c + 2) * 32), ga);
                                cols(c + 1, gb);
                                if (h2) tmem_wait_pin(ga);
                            }
                        }
                    }
                    if constexpr (RC == 1) {
                        acc[0] = (acc2[0].x + acc2[0].y) + (acc2[1].x + acc2[1].y);
                    } else {
#pragma unroll
                        for (int z = 0; z < RC / 2; ++z) {
                            acc[2 * z] = accw[z].x;
                            acc[2 * z + 1] = accw[z].y;
                        }
                    }
                }
                tc_fence_before();
                if constexpr (EPI2) {
                    // the second half's sums go to the first group through shared
                    // memory; the first group releases the accumulator only after
                    // reading them, so the buffer is free when the slot is reused
                    float *xb = reinterpret_cast<float *>(sm + S::XBUF) + (a4 * 128 + row) * RC;
                    if (eg == 1) {
#pragma unroll
                        for (int z = 0; z < RC; ++z) xb[z] = acc[z];
                        mbar_arrive(BAR_X_FULL(a4));
                        mbar_arrive(BAR_T_EMPTY(a4));
                        continue;
                    }
                    if (!mbar_wait(BAR_X_FULL(a4), (li / NACC) & 1, abort_flag, args.status, args.spin)) goto epi_done;
#pragma unroll
                    for (int z = 0; z < RC; ++z) acc[z] += xb[z];
                }
                mbar_arrive(BAR_T_EMPTY(a4));
                if (UNI != 2 && row < item.cnt) {
                    float *p = args.partial + (int64_t)(item.e0 + row) * args.r;
#pragma unroll
                    for (int z = 0; z < RC; ++z)
                        if (z < args.r) p[z] = acc[z];
                    if (pb >= 0) {   // the follower's entry: its share is in the leader's sum
                        float *pf = args.partial + (int64_t)(e0f + row) * args.r;
#pragma unroll
                        for (int z = 0; z < RC; ++z)
                            if (z < args.r) pf[z] = 0.f;
                    }
                }
            }
            mbar_arrive(BAR_BLK_EMPTY(bs));
        }
    epi_done:;
    } else if (warp == W_GAT) {
        // ------------------------------------------------- target-row gatherer
        // The next item's descriptor and target slots are loaded while this
        // item waits for its stage, so the two dependent global loads are
        // off the critical path.
        const uint32_t bytes = (uint32_t)(T16_ROWS * args.d_pad * 4);
        int issued = 0;
        int ci = c_begin, it = 0;
        auto seek = [&](int &c, int &i) {   // first item at or after (c, i) in this CTA's order
            while (c < c_end && i >= args.block_off[args.cta_blocks[c] + 1]) {
                ++c;
                if (c < c_end) i = args.block_off[args.cta_blocks[c]];
            }
        };
        auto rows = [&](int i, int (&r)[4]) {
            const EvalItem item = args.items[i];
            const int first = args.tgt[item.e0];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int rw = 4 * lane + k;   // rows past cnt repeat the first target
                r[k] = rw < item.cnt ? args.tgt[item.e0 + rw] : first;
            }
        };
        if (ci < c_end) it = args.block_off[args.cta_blocks[ci]];
        seek(ci, it);
        int r[4] = {0, 0, 0, 0};
        if (ci < c_end) rows(it, r);
        for (int li = 0; ci < c_end && !*abort_flag; ++li) {
            int ci2 = ci, it2 = it + 1;
            seek(ci2, it2);
            int rn[4] = {0, 0, 0, 0};
            if (ci2 < c_end) rows(it2, rn);
            const int sr = li % NRAW;
            if (!mbar_wait(BAR_R_EMPTY(sr), ((li / NRAW) & 1) ^ 1, abort_flag, args.status, args.spin)) goto gather_done;
            ++issued;
            if (lane == 0) mbar_expect_tx(BAR_R_FULL(sr), bytes);
            __syncwarp();
            {
                // rows 8m .. 8m+7 (lanes 2m, 2m+1) that are 8 consecutive target
                // slots arrive in one tiled copy; the rest by tile::gather4
                const bool mine4 = r[1] == r[0] + 1 && r[2] == r[0] + 2 && r[3] == r[0] + 3;
                const int r0_hi = __shfl_down_sync(0xffffffffu, r[0], 1);
                const bool both4 = __shfl_down_sync(0xffffffffu, (int)mine4, 1) != 0;
                const bool run8_lo = (lane & 1) == 0 && mine4 && both4 && r0_hi == r[0] + 4;
                const bool run8 = args.runs && __shfl_sync(0xffffffffu, (int)run8_lo, lane & ~1) != 0;
                const uint32_t dst = sbase + S::RAW + sr * S::RAWSTAGE + 4 * lane * args.d_pad * 4;
                if (run8) {
                    if ((lane & 1) == 0) tma_load_2d(dst, &map_q8, 0, r[0], BAR_R_FULL(sr));
                } else {
                    tma_gather4(dst, &map_q, 0, r[0], r[1], r[2], r[3], BAR_R_FULL(sr));
                }
            }
            ci = ci2;
            it = it2;
#pragma unroll
            for (int k = 0; k < 4; ++k) r[k] = rn[k];
        }
    gather_done:
        // rows of the last stages may still be landing after an abort
        for (int gg = issued > NRAW ? issued - NRAW : 0; gg < issued; ++gg)
            mbar_drain(BAR_R_FULL(gg % NRAW), (gg / NRAW) & 1);
    } else if (warp == W_MMA && lane == 0) {
        // ------------------------------------- sub-block loads + MMA issuer
        int li = 0, lb = 0, b_issued = 0;
        int blk_last[2] = {-1, -1};   // last block whose column data went to slot 0 / 1
        int li_done = -1;             // last item whose MMAs were committed
        for (int ci = c_begin; ci < c_end && !*abort_flag; ++ci, ++lb) {
            const int b = args.cta_blocks[ci];
            const int i0 = args.block_off[b], i1 = args.block_off[b + 1];
            const EvalItem first = args.items[i0];
            const bool far = first.nrows < 0;
            const int bs = lb & 1;
            // a paired follower (NB == 2) is the next sub-block of the same
            // node: its rows, column data and weights follow the leader's
            const int pb = NB == 2 ? args.partner[b] : -1;
            const int nsb = pb >= 0 ? 2 : 1;
            const int ncols = (first.nrows & 0x7fffffff) + (pb >= 0 ? (args.items[args.block_off[pb]].nrows & 0x7fffffff) : 0);
            // N covers every 32-column chunk the epilogue reads, so no column it
            // reads holds a stale accumulator
            const uint32_t idesc = make_idesc(FMT, T16_ROWS, (ncols + 31) & ~31);
            if (!mbar_wait(BAR_B_EMPTY, (lb & 1) ^ 1, abort_flag, args.status, args.spin)) goto mma_done;
            if (!mbar_wait(BAR_BLK_EMPTY(bs), ((lb >> 1) & 1) ^ 1, abort_flag, args.status, args.spin)) goto mma_done;
            b_issued = lb + 1;
            blk_last[bs] = lb;
            mbar_expect_tx(BAR_B_FULL, (uint32_t)(2 * nsb * T16_REGION));
            for (int h = 0; h < nsb; ++h) {
                tma_load_2d(sbase + S::B_HI + h * T16_REGION, far ? &map_s_hi : &map_t_hi, 0, first.row0 + 128 * h,
                            BAR_B_FULL);
                tma_load_2d(sbase + S::B_LO + h * T16_REGION, far ? &map_s_lo : &map_t_lo, 0, first.row0 + 128 * h,
                            BAR_B_FULL);
            }
            const uint32_t slot = sbase + S::BLK + bs * S::BLKSLOT;
            const uint32_t colw_bytes = RC > 1 ? (uint32_t)(nsb * 128 * RC * 4) : 0u;
            constexpr int CV = UNI ? 64 : 128;   // float4 of column data per sub-block (UNI 1, 2: compact)
            mbar_expect_tx(BAR_BLK_FULL(bs), (uint32_t)(256 + nsb * CV * 16) + colw_bytes);
            bulk_copy(slot + S::BLK_CENT, args.cent + (int64_t)first.cidx * TC_K, TC_K * 4, BAR_BLK_FULL(bs));
            bulk_copy(slot + S::BLK_COLV, args.colv + (int64_t)first.cidx * CV, nsb * CV * 16, BAR_BLK_FULL(bs));
            if constexpr (RC > 1)
                bulk_copy(slot + S::BLK_COLW, args.colw + (int64_t)first.cidx * 128 * RC, colw_bytes, BAR_BLK_FULL(bs));
            for (int it = i0; it < i1; ++it, ++li) {
                const int sa = li & 1, a4 = li % NACC;
                if (!mbar_wait(BAR_A_FULL(sa), (li >> 1) & 1, abort_flag, args.status, args.spin)) goto mma_done;
                if (it == i0 && !mbar_wait(BAR_B_FULL, lb & 1, abort_flag, args.status, args.spin)) goto mma_done;
                if (!mbar_wait(BAR_T_EMPTY(a4), ((li / NACC) & 1) ^ 1, abort_flag, args.status, args.spin)) goto mma_done;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(a4 * 128 * NB);
                const uint32_t a_hi = sbase + S::A0 + sa * 2 * T16_REGION, a_lo = a_hi + T16_REGION;
                const uint32_t b_hi = sbase + S::B_HI, b_lo = sbase + S::B_LO;
                // the tensor core rounds each accumulation step to the running sum's
                // precision: the small cross terms first, the hi*hi products last
#pragma unroll
                for (int k = 0; k < 4; ++k) {   // K = 16 per MMA: 32 bytes into the 128-byte rows
                    const uint32_t off = (uint32_t)(k * 32);
                    tc_mma<P>(d_tmem, sw128_desc(a_hi + off), sw128_desc(b_lo + off), idesc, k > 0);
                    tc_mma<P>(d_tmem, sw128_desc(a_lo + off), sw128_desc(b_hi + off), idesc, 1);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t off = (uint32_t)(k * 32);
                    tc_mma<P>(d_tmem, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc, 1);
                }
                tc_commit(BAR_A_EMPTY(sa));
                tc_commit(BAR_T_FULL(a4));
                if (it == i1 - 1) tc_commit(BAR_B_EMPTY);
                li_done = li;
            }
        }
    mma_done:
        // after an abort: the last sub-block's tiles and the latest column
        // data of each slot may still be landing (earlier copies were
        // consumed before the slot was refilled), and MMAs may still be
        // writing TMEM -- wait for all of them before TMEM is freed and the
        // CTA exits (no-ops on the normal path, where all are complete)
        if (b_issued > 0) mbar_drain(BAR_B_FULL, (b_issued - 1) & 1);
        for (int k = 0; k < 2; ++k)
            if (blk_last[k] >= 0) mbar_drain(BAR_BLK_FULL(k), (blk_last[k] >> 1) & 1);
        if (li_done >= 0) mbar_drain(BAR_T_FULL(li_done % NACC), (li_done / NACC) & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == W_MMA) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T16_TMEM_COLS) : "memory");
    }
}

// Column data of every sub-block for one Evaluate: thread t of block b takes
// source row t of sub-block b.  colv pairs rows (2p, 2p+1):
// {A_2p, A_2p+1, B_2p, B_2p+1}, {C_2p, C_2p+1, w_2p, w_2p+1} with
// A = 2 sc / scale^2, B = -sc |b|^2, C = -sc (zeros past the sub-block's rows).
template <int RC, int UNI>
__global__ void tc16_cols_kernel(const int64_t *sb_row0, const int32_t *sb_nr, int64_t n_leaf_sub, const float *sc_t,
                                 const float *sc_s, const float *nrm_t, const float *nrm_s, const float *Wt,
                                 const float *Ws, int r, float g_unscale, float4 *colv, float *colw) {
    const int64_t b = blockIdx.x;
    const int t = threadIdx.x;
    const bool far = b >= n_leaf_sub;
    const int64_t row = sb_row0[b] + t;
    const bool valid = t < sb_nr[b];
    const float sc = valid ? (far ? sc_s : sc_t)[row] : 0.f;
    const float nrm = valid ? (far ? nrm_s : nrm_t)[row] : 0.f;
    const float *w = (far ? Ws : Wt) + row * r;
    const int o = t & 1;
    if (UNI) {   // {B_j, B_j+1, w_j, w_j+1}; B = -inf past the rows: exp2 gives 0 there
        float *cp = reinterpret_cast<float *>(colv + b * 64 + (t >> 1));
        cp[0 + o] = valid ? -sc * nrm : -INFINITY;
        cp[2 + o] = valid ? w[0] : 0.f;
        return;
    }
    float *cp = reinterpret_cast<float *>(colv + b * 128 + 2 * (t >> 1));
    cp[0 + o] = 2.f * g_unscale * sc;
    cp[2 + o] = -sc * nrm;
    cp[4 + o] = -sc;
    cp[6 + o] = valid ? w[0] : 0.f;
    if (RC > 1) {
#pragma unroll
        for (int z = 0; z < RC; ++z) colw[(b * 128 + t) * RC + z] = (valid && z < r) ? w[z] : 0.f;
    }
}

// Column data of the kNN shortlist (leaf sub-blocks only): {|b_j|^2 (1 - eta)
// or +inf past the rows, the same for j+1, tree position of row j, of j+1}.
__global__ void tc16_knn_cols_kernel(const int64_t *sb_row0, const int32_t *sb_nr, const float *nrm_t, float eta,
                                     float4 *colv) {
    const int64_t b = blockIdx.x;
    const int t = threadIdx.x;
    const int64_t row = sb_row0[b] + t;
    const bool valid = t < sb_nr[b];
    float *cp = reinterpret_cast<float *>(colv + b * 64 + (t >> 1));
    const int o = t & 1;
    cp[0 + o] = valid ? nrm_t[row] * (1.f - eta) : INFINITY;
    cp[2 + o] = __int_as_float(valid ? (int)row : 0);
}

// Dense work lists of the shortlist: every leaf sub-block b against every
// tile of 128 queries k (item b * n_qt + k); the queries are the identity.
__global__ void knn_items_kernel(const int64_t *sb_row0, const int32_t *sb_nr, int64_t n_sub, int n_qt, int64_t T,
                                 EvalItem *items, int32_t *block_off) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e <= n_sub) block_off[e] = (int32_t)(e * n_qt);
    if (e >= n_sub * n_qt) return;
    const int64_t b = e / n_qt, k = e % n_qt;
    EvalItem it;
    it.row0 = (int32_t)sb_row0[b];
    it.nrows = sb_nr[b];
    it.e0 = (int32_t)(k * 128);
    it.cnt = (int32_t)(T - k * 128 < 128 ? T - k * 128 : 128);
    it.cidx = (int32_t)b;
    it.pad_[0] = it.pad_[1] = it.pad_[2] = 0;
    items[e] = it;
}

__global__ void iota32_kernel(int32_t *a, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) a[e] = (int32_t)e;
}


// 64 x 128, 128-byte swizzle) for BF16 (index 0) and FP16 (index 1).
struct T16State {
    CUtensorMap map[2][4];   // [t_hi, t_lo, s_hi, s_lo]
    bool ready[2] = {false, false};
    EncodeTiledFn encode = nullptr;
};

std::mutex g_t16_mu;

askit_status t16_state(askit_tree t, int pi, T16State **out) {
    std::lock_guard<std::mutex> lock(g_t16_mu);
    if (!t->tc16) t->tc16 = new T16State();
    T16State *st = (T16State *)t->tc16;
    if (!st->encode) ASK_TRY(encode_fn(&st->encode));
    if (!st->ready[pi]) {
        const CUtensorMapDataType ty = pi == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
        const void *arr[4] = {pi == 0 ? (void *)t->Xt_bhi : (void *)t->Xt_hhi,
                              pi == 0 ? (void *)t->Xt_blo : (void *)t->Xt_hlo,
                              pi == 0 ? (void *)t->Xs_bhi : (void *)t->Xs_hhi,
                              pi == 0 ? (void *)t->Xs_blo : (void *)t->Xs_hlo};
        for (int i = 0; i < 4; ++i)
            ASK_TRY(encode_2d(st->encode, &st->map[pi][i], ty, 2, arr[i], i < 2 ? t->N_pad : t->srows, TC_K, 64,
                              T16_ROWS, CU_TENSOR_MAP_SWIZZLE_128B));
        st->ready[pi] = true;
    }
    *out = st;
    return ASKIT_OK;
}

template <int P, int RC, int NRAW, int NB, int UNI>
askit_status launch16(T16State *st, int pi, const CUtensorMap &map_q, const CUtensorMap &map_q8, const T16Args &a,
                      int grid, cudaStream_t s) {
    using S = S16<RC, NRAW, NB>;
    const size_t smem = S::BYTES + 1024;
    static_assert(S::BYTES + 1024 <= 232448, "shared-memory plan exceeds 227 KB");
    static const cudaError_t attr = cudaFuncSetAttribute(eval_tc16_kernel<P, RC, NRAW, NB, UNI>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ASK_CUDA(attr);
    eval_tc16_kernel<P, RC, NRAW, NB, UNI><<<(unsigned)grid, S::THREADS, smem, s>>>(
        st->map[pi][0], st->map[pi][1], st->map[pi][2], st->map[pi][3], map_q, map_q8, a);
    ASK_LAUNCH();
    return ASKIT_OK;
}

template <int P, int RC>
askit_status run16(askit_tree t, const WeightCtx &c, T16State *st, int pi, const CUtensorMap &map_q,
                   const CUtensorMap &map_q8, T16Args a, const WorkLists &w, cudaStream_t s) {
    const float g_unscale = 1.f / (a.f16_scale * a.f16_scale);
    // one bandwidth for every source: compact column data (r = 1)
    const bool uni = RC == 1 && t->prm.bw_mode == ASKIT_BW_CONSTANT;
    if (uni) {
        // the same rounding as the per-row values (h held in FP32)
        const double hf = (double)(float)t->prm.h;
        const float sc = (float)(t->prm.kernel_scale * 1.4426950408889634 / (hf * hf));
        a.uni_a = 2.f * g_unscale * sc;
        a.uni_c = -sc;
        tc16_cols_kernel<RC, 1><<<(unsigned)t->n_sub, 128, 0, s>>>(t->sb_row0, t->sb_nr, t->n_leaf_sub, t->sc_t,
                                                                   t->sc_s, t->nrmc_t, t->nrmc_s, c.Wt, c.Ws, c.r,
                                                                   g_unscale, c.colv, c.colw);
    } else {
        tc16_cols_kernel<RC, 0><<<(unsigned)t->n_sub, 128, 0, s>>>(t->sb_row0, t->sb_nr, t->n_leaf_sub, t->sc_t,
                                                                   t->sc_s, t->nrmc_t, t->nrmc_s, c.Wt, c.Ws, c.r,
                                                                   g_unscale, c.colv, c.colw);
    }
    ASK_LAUNCH();
    a.colv = c.colv;
    a.colw = c.colw;
    auto go = [&]() -> askit_status {
        if constexpr (RC == 1) {
            if (uni) {
                if (t->tune_pairs && w.sched_off[2]) {
                    a.cta_off = w.sched_off[2];
                    a.cta_blocks = w.sched_blocks[2];
                    a.partner = w.partner;
                    return launch16<P, RC, 2, 2, 1>(st, pi, map_q, map_q8, a, w.n_ctas, s);
                }
                if (t->tune_stages == 2) return launch16<P, RC, 2, 1, 1>(st, pi, map_q, map_q8, a, w.n_ctas, s);
                return launch16<P, RC, 3, 1, 1>(st, pi, map_q, map_q8, a, w.n_ctas, s);
            }
        }
        if constexpr (RC <= 4) {
            // paired 256-column items: two stages fit next to the 64 KB source tile
            if (t->tune_pairs && w.sched_off[2]) {
                a.cta_off = w.sched_off[2];
                a.cta_blocks = w.sched_blocks[2];
                a.partner = w.partner;
                return launch16<P, RC, 2, 2, 0>(st, pi, map_q, map_q8, a, w.n_ctas, s);
            }
        }
        if (t->tune_stages == 2) return launch16<P, RC, 2, 1, 0>(st, pi, map_q, map_q8, a, w.n_ctas, s);
        return launch16<P, RC, 3, 1, 0>(st, pi, map_q, map_q8, a, w.n_ctas, s);
    };
    ASK_TRY(ktimer_mark(t, s, false));
    ASK_TRY(go());
    return ktimer_mark(t, s, true);
}

template <int P>
askit_status dispatch16(askit_tree t, const WeightCtx &c, T16State *st, int pi, const CUtensorMap &map_q,
                        const CUtensorMap &map_q8, const T16Args &a, const WorkLists &w, cudaStream_t s) {
    if (c.r == 1) return run16<P, 1>(t, c, st, pi, map_q, map_q8, a, w, s);
    if (c.r <= 4) return run16<P, 4>(t, c, st, pi, map_q, map_q8, a, w, s);
    return run16<P, 16>(t, c, st, pi, map_q, map_q8, a, w, s);
}

}  // namespace

askit_status eval_tc16(askit_tree t, const WeightCtx &c, int precision, const float *Xq, int64_t ldq, int64_t q_rows,
                       const WorkLists &w, float *partial, cudaStream_t s) {
    if (c.r > 16) {
        askit_set_error("tensor-core evaluation covers r <= 16; use ASKIT_PREC_SIMT_FP32");
        return ASKIT_ERR_UNSUPPORTED;
    }
    if (w.n_blocks == 0) return ASKIT_OK;
    if (ldq != t->d_pad || !c.colv || (c.r > 1 && !c.colw)) {
        askit_set_error("target rows must have d_pad columns and the column buffers must exist");
        return ASKIT_ERR_INVALID_ARG;
    }
    const int pi = precision == ASKIT_PREC_BF16X3 ? 0 : 1;
    T16State *st = nullptr;
    ASK_TRY(t16_state(t, pi, &st));
    CUtensorMap map_q;   // one box row per gathered target row
    ASK_TRY(encode_2d(st->encode, &map_q, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, Xq, q_rows, t->d_pad, t->d_pad, 1,
                      CU_TENSOR_MAP_SWIZZLE_NONE));
    CUtensorMap map_q8;  // runs of 8 consecutive target rows: one tiled box
    ASK_TRY(encode_2d(st->encode, &map_q8, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, Xq, q_rows, t->d_pad, t->d_pad, 8,
                      CU_TENSOR_MAP_SWIZZLE_NONE));
    T16Args a;
    a.items = w.items;
    a.block_off = w.block_off;
    a.cta_off = w.cta_off;
    a.cta_blocks = w.cta_blocks;
    a.tgt = w.tgt;
    a.d_pad = t->d_pad;
    a.cent = t->cent;
    a.colv = nullptr;
    a.colw = nullptr;
    a.r = c.r;
    a.f16_scale = precision == ASKIT_PREC_FP16X3 ? t->f16_scale : 1.f;
    a.runs = t->tune_runs;
    a.partner = nullptr;
    a.uni_a = a.uni_c = 0.f;
    a.knn_u = nullptr;
    a.knn_cnt = nullptr;
    a.knn_cand = nullptr;
    a.knn_cap = 0;
    a.knn_eta = a.knn_m2u = 0.f;
    a.partial = partial;
    a.status = t->d_status;
    a.spin = t->spin_limit > 0 ? t->spin_limit : SPIN_LIMIT;
    if (precision != ASKIT_PREC_FP16X3) {
        askit_set_error("eval_tc16 runs FP16x3");
        return ASKIT_ERR_INVALID_ARG;
    }
    return dispatch16<ASKIT_PREC_FP16X3>(t, c, st, pi, map_q, map_q8, a, w, s);
}

// The exact kNN's tensor-core shortlist for T queries Yp [T, d_pad] (FP32):
// every tree position whose FP16x3 distance to query q is at most
// U[q] (1 + eta) + eta (|a|^2 + |b|^2) goes to cand[q, 0 .. cap) (cnt[q]
// counts them, also past cap).  Leaf sub-blocks only (every point once).
askit_status knn_shortlist_tc16(askit_tree t, const float *Yp, int64_t T, const float *U, int *cnt, int32_t *cand,
                                int cap, float eta, cudaStream_t s) {
    if (!t->Xt_hhi || t->d > TC_K || t->n_leaf_sub == 0) {
        askit_set_error("the tensor-core shortlist needs the FP16 operands (d <= %d)", TC_K);
        return ASKIT_ERR_UNSUPPORTED;
    }
    const int64_t nsub = t->n_leaf_sub;
    const int n_qt = (int)((T + 127) / 128);
    // pairs: sub-blocks 2k and 2k+1 of one leaf; the schedule deals leaders and
    // singles to the CTAs in tree order, contiguous ranges of equal cost
    std::vector<int32_t> partner(nsub, -1), blocks;
    std::vector<int64_t> cost;
    for (int64_t b = 0; b < nsub; ++b) {
        const int64_t node = t->h_sub_node[b];
        int64_t first = b;
        while (first > 0 && t->h_sub_node[first - 1] == node) --first;
        if ((b - first) & 1) continue;                            // a follower
        if (b + 1 < nsub && t->h_sub_node[b + 1] == node) partner[b] = (int32_t)(b + 1);
        blocks.push_back((int32_t)b);
        cost.push_back(partner[b] >= 0 ? 2 : 1);
    }
    int dev = 0, sms = 0;
    ASK_CUDA(cudaGetDevice(&dev));
    ASK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int nc = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)blocks.size(), sms));
    int64_t total = 0;
    for (int64_t c : cost) total += c;
    std::vector<int32_t> coff(nc + 1, 0);
    {
        int c = 0;
        int64_t acc = 0;
        for (size_t q = 0; q < blocks.size(); ++q) {
            acc += cost[q];
            ++coff[c + 1];
            if (c < nc - 1 && acc * nc >= (int64_t)(c + 1) * total) ++c;
        }
        for (int k = 0; k < nc; ++k) coff[k + 1] += coff[k];
    }
    DevArena tmp;
    tmp.async = true;
    tmp.stream = s;
    EvalItem *items = nullptr;
    int32_t *boff = nullptr, *tgt = nullptr, *d_coff = nullptr, *d_blk = nullptr, *d_part = nullptr;
    float4 *colv = nullptr;
    askit_status rc = ASKIT_OK;
#define KTRY(x) do { rc = (x); if (rc != ASKIT_OK) goto out; } while (0)
    KTRY(tmp.alloc(&items, (size_t)nsub * n_qt));
    KTRY(tmp.alloc(&boff, nsub + 1));
    KTRY(tmp.alloc(&tgt, T));
    KTRY(tmp.alloc(&d_coff, nc + 1));
    KTRY(tmp.alloc(&d_blk, blocks.size()));
    KTRY(tmp.alloc(&d_part, nsub));
    KTRY(tmp.alloc(&colv, (size_t)nsub * 64));
    {
        const int64_t ne = std::max<int64_t>(nsub * n_qt, nsub + 1);
        knn_items_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(t->sb_row0, t->sb_nr, nsub, n_qt, T, items, boff);
        iota32_kernel<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(tgt, T);
        tc16_knn_cols_kernel<<<(unsigned)nsub, 128, 0, s>>>(t->sb_row0, t->sb_nr, t->nrmc_t, eta, colv);
        if (cudaGetLastError() != cudaSuccess) { askit_set_error("shortlist set-up launch"); rc = ASKIT_ERR_CUDA; goto out; }
        if (cudaMemcpyAsync(d_coff, coff.data(), sizeof(int32_t) * (nc + 1), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(d_blk, blocks.data(), sizeof(int32_t) * blocks.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(d_part, partner.data(), sizeof(int32_t) * nsub, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            askit_set_error("shortlist schedule copy");
            rc = ASKIT_ERR_CUDA;
            goto out;
        }
        T16State *st = nullptr;
        KTRY(t16_state(t, 1, &st));
        CUtensorMap map_q, map_q8;
        KTRY(encode_2d(st->encode, &map_q, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, Yp, T, t->d_pad, t->d_pad, 1,
                       CU_TENSOR_MAP_SWIZZLE_NONE));
        KTRY(encode_2d(st->encode, &map_q8, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, Yp, T, t->d_pad, t->d_pad, 8,
                       CU_TENSOR_MAP_SWIZZLE_NONE));
        T16Args a;
        a.items = items;
        a.block_off = boff;
        a.cta_off = d_coff;
        a.cta_blocks = d_blk;
        a.tgt = tgt;
        a.d_pad = t->d_pad;
        a.cent = t->cent;
        a.colv = colv;
        a.colw = nullptr;
        a.r = 1;
        a.f16_scale = t->f16_scale;
        a.runs = 1;
        a.partner = d_part;
        a.uni_a = a.uni_c = 0.f;
        a.knn_u = U;
        a.knn_cnt = cnt;
        a.knn_cand = cand;
        a.knn_cap = cap;
        a.knn_eta = eta;
        a.knn_m2u = -2.f / (t->f16_scale * t->f16_scale);
        a.partial = nullptr;
        a.status = t->d_status;
        a.spin = SPIN_LIMIT;
        KTRY((launch16<ASKIT_PREC_FP16X3, 1, 2, 2, 2>(st, 1, map_q, map_q8, a, nc, s)));
    }
out:
#undef KTRY
    tmp.free_all();
    return rc;
}

void eval_tc16_free(askit_tree t) {
    delete (T16State *)t->tc16;
    t->tc16 = nullptr;
}
