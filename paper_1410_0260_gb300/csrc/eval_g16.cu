// Evaluate (Algorithm 4) on the tcgen05 tensor cores with FP16x3 split
// operands, d <= 64, all operands pre-split in HBM ("global centering").
//
// Every point (target or source) is centered once on the data mean xbar and
// prescaled by a power of 2 s:  x~ = (x - xbar) s, split x~ = hi + lo in FP16.
// Then, per (target i, source j),
//
//     r^2 = n_i + n_j - 2 x~_i . x~_j / s^2,    n = |x - xbar|^2 (FP32),
//     arg = -sc_j r^2 = (2 sc_j / s^2) G + (-sc_j) n_i + (-sc_j n_j),
//     partial_i += exp2(arg) w_j,
//
// with G = x~_i . x~_j on the tensor cores as three split products
// (hi*lo + lo*hi + hi*hi, FP32 accumulation, small terms first).  No target
// row is converted on the chip: a work item's 128 target rows are copied in
// the MMA's swizzled layout straight from HBM (16-byte cp.async, eight lanes
// per 128-byte row; a TMA tile::gather4 issue costs about 75 cycles per four
// rows on this part, which made the copies the bottleneck), so the kernel
// has no loader warps, only the exponentials and weight sums of the epilogue
// beside the MMAs.  The price is precision: the terms n_i, n_j and 2G are of the
// size of the data's spread R^2 around xbar and are rounded in FP32, so the
// exponent carries an error of a few 2^-24 sc R^2; the per-sub-block centered
// kernel (eval_tc16.cu) keeps these terms at the size of a node instead.  The
// tree picks this kernel only while sc_max R^2_max stays below a bound that
// keeps the FP16x3 result at FP32 grade (build_tc_operands), and falls back
// otherwise; askit_set_fp16_centering overrides the choice.  Measured: about
// 1e-5 relative L2 error of u (the per-sub-block kernel: about 1e-6), inside
// the split-product tolerance 1e-4.
//
// Work item = one source sub-block (or two sub-blocks of one node: a paired
// 256-column item) against up to 128 targets needing it (eval_lists.cu).
// One CTA per SM, 352 threads:
//   warps 0-7  two epilogue groups, each summing whole sub-blocks (alternate
//              items, or the two sub-blocks of a paired item): tcgen05.ld of
//              their 32 TMEM lanes (two buffers), ex2 on MUFU, weight sums,
//              one partial sum per (target, sub-block) entry;
//   warp 8     TMEM allocation; lane 0 loads each sub-block (TMA tiles of its
//              pre-split rows, bulk copies of its column data) and issues the
//              tcgen05.mma instructions;
//   warps 9-10 copy each item's target rows into NA stages (NA - 2 items in
//              flight) and the targets' n_i into shared memory.
// Every mbarrier wait is bounded (ASK_DEV_TIMEOUT on expiry, all roles leave,
// copies and MMAs in flight are waited for, TMEM is freed).
#include <cuda.h>
#include <cuda_fp16.h>

#include <mutex>

#include "askit_impl.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace tcx;

constexpr int G_ROWS = 128;
constexpr int G_REGION = G_ROWS * 128;   // 128 rows x 128 bytes (64 FP16), 128-byte swizzle
constexpr uint32_t G_TMEM_COLS = 512;    // four 128-column (two 256-column) FP32 accumulators

// NA: target-row stages; NB: sub-blocks per item (1, or 2 for paired items);
// NACC = 4 / NB TMEM accumulators of 128 NB columns.
template <int RC, int NA, int NB>
struct SG {
    static constexpr int NACC = 4 / NB;
    static constexpr int B_HI = 0, B_LO = NB * G_REGION;    // NB x 128 rows each, contiguous
    static constexpr int A0 = 2 * NB * G_REGION;            // stage s: hi at A0 + 2 s REGION, lo at + REGION
    static constexpr int BLK = A0 + NA * 2 * G_REGION;      // [2] per-block column-data slots
    static constexpr int BLK_COLV = 0;                      // float4 [128 NB] column data
    static constexpr int BLK_COLW = NB * 128 * 16;          // float [128 NB][RC] weights (RC > 1)
    static constexpr int COLW_BYTES = RC > 1 ? NB * 128 * RC * 4 : 0;
    static constexpr int BLKSLOT = BLK_COLW + COLW_BYTES;
    static constexpr int PT = BLK + 2 * BLKSLOT;            // float [NA][128] n_i of each stage's targets
    static constexpr int BAR = PT + NA * 128 * 4;           // 48 mbarriers
    static constexpr int MISC = BAR + 48 * 8;               // tmem address, abort flag
    static constexpr int BYTES = MISC + 16;
    static constexpr int THREADS = 352;
};

struct G16Args {
    const EvalItem *items;
    const int32_t *block_off;
    const int32_t *cta_off, *cta_blocks;
    const int32_t *tgt;       // entry -> target slot (row of the query operand)
    const uint16_t *q_hi, *q_lo; // [query rows, 64] pre-split target rows
    const float *qn;          // [query rows] n_i = |x_i - xbar|^2
    const float4 *colv;       // [n_sub, 128] column data (UNI: [n_sub, 64])
    const float *colw;        // [n_sub, 128, RC] (RC > 1)
    const int32_t *partner;   // [n_blocks] paired follower block, or -1 (NB == 2)
    int r;
    float uni_a, uni_c;       // UNI: A = 2 sc / s^2 and C = -sc
    float *partial;
    int *status;
    int spin;
};

template <int RC, int NA, int NB, int UNI>
__global__ void __launch_bounds__(352, 1)
eval_g16_kernel(const __grid_constant__ CUtensorMap map_t_hi, const __grid_constant__ CUtensorMap map_t_lo,
                const __grid_constant__ CUtensorMap map_s_hi, const __grid_constant__ CUtensorMap map_s_lo,
                const G16Args args) {
    using S = SG<RC, NA, NB>;
    constexpr int NACC = S::NACC;
    constexpr int NEPI = 256;                    // epilogue threads (two groups of 128)
    // readers of an item's n_i and drainers of its accumulator: one group
    // (alternate items) or both (paired items)
    constexpr int NITEM = NB == 2 ? 256 : 128;
    constexpr int W_MMA = 8, W_CP0 = 9;          // MMA warp, first of the two copier warps
    static_assert(NA >= 3 && NA <= 4, "the copiers keep NA - 2 items in flight");
    static_assert(!UNI || RC == 1, "the uniform-bandwidth layout serves r = 1");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(sm);
    float *ptbuf = reinterpret_cast<float *>(sm + S::PT);
    const uint32_t bar0 = sbase + S::BAR;
    auto BAR_A_FULL = [&](int s) { return bar0 + 8 * s; };            // target rows of stage s landed (64)
    auto BAR_A_EMPTY = [&](int s) { return bar0 + 8 * (4 + s); };     // MMAs reading stage s done (commit)
    auto BAR_P_FULL = [&](int s) { return bar0 + 8 * (8 + s); };      // n_i of stage s's item stored (64)
    auto BAR_P_EMPTY = [&](int s) { return bar0 + 8 * (12 + s); };    // epilogue read them (NITEM)
    const uint32_t BAR_B_FULL = bar0 + 8 * 16, BAR_B_EMPTY = bar0 + 8 * 17;
    auto BAR_BLK_FULL = [&](int s) { return bar0 + 8 * (18 + s); };   // column data of slot s landed
    auto BAR_BLK_EMPTY = [&](int s) { return bar0 + 8 * (20 + s); };  // epilogue done with slot s (NEPI)
    auto BAR_T_FULL = [&](int a) { return bar0 + 8 * (24 + a); };     // accumulator a complete (commit)
    auto BAR_T_EMPTY = [&](int a) { return bar0 + 8 * (28 + a); };    // epilogue drained accumulator a (NITEM)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + S::MISC);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + S::MISC + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < NA; ++s) {
            mbar_init(BAR_A_FULL(s), 64);
            mbar_init(BAR_A_EMPTY(s), 1);
            mbar_init(BAR_P_FULL(s), 64);
            mbar_init(BAR_P_EMPTY(s), NITEM);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(BAR_BLK_FULL(s), 1);
            mbar_init(BAR_BLK_EMPTY(s), NEPI);
        }
        mbar_init(BAR_B_FULL, 1);
        mbar_init(BAR_B_EMPTY, 1);
        for (int a = 0; a < NACC; ++a) {
            mbar_init(BAR_T_FULL(a), 1);
            mbar_init(BAR_T_EMPTY(a), NITEM);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == W_MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(G_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int c_begin = args.cta_off[blockIdx.x], c_end = args.cta_off[blockIdx.x + 1];

    if (warp < W_MMA) {
        // ----------------------------------------------------------- epilogue
        // Each group sums whole sub-blocks: with single sub-blocks (NB == 1)
        // the two groups take alternate items; with paired items (NB == 2)
        // group 0 takes the leader's 128 columns and group 1 the follower's,
        // and each writes its own entry's partial sum -- so every entry's
        // partial is formed the same way in both layouts, and the groups
        // never wait for each other.  A paired-layout item without a follower
        // is summed by group 0 alone.
        const int q = warp & 3;                    // this warp's TMEM lane quadrant
        const int row = q * 32 + lane;             // TMEM lane = target row of the item
        const int eg = warp >> 2;                  // group
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
            // this group's columns of every item of the block
            const int nrows_l = args.items[i0].nrows & 0x7fffffff;
            int c_lo = 0, c_hi = (nrows_l + 31) >> 5;
            if (NB == 2 && eg == 1) {
                c_lo = 4;
                c_hi = pb >= 0 ? 4 + ((ncols_f + 31) >> 5) : 4;
            }
            for (int it = i0; it < i1; ++it, ++li) {
                if (NB == 1 && (li & 1) != eg) continue;   // the other group's item
                const int a4 = li % NACC, sp = li % NA;
                const EvalItem item = args.items[it];
                const int e_out = (NB == 2 && eg == 1) ? (pb >= 0 ? args.items[f0 + (it - i0)].e0 : 0) : item.e0;
                if (!mbar_wait(BAR_P_FULL(sp), (li / NA) & 1, abort_flag, args.status, args.spin)) goto epi_done;
                const float pt = ptbuf[sp * 128 + row];
                mbar_arrive(BAR_P_EMPTY(sp));
                if (!mbar_wait(BAR_T_FULL(a4), (li / NACC) & 1, abort_flag, args.status, args.spin)) goto epi_done;
                tc_fence_after();
                float acc[RC];
#pragma unroll
                for (int z = 0; z < RC; ++z) acc[z] = 0.f;
                float2 acc2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};   // RC == 1
                float2 accw[RC > 1 ? RC / 2 : 1];                                    // RC > 1
#pragma unroll
                for (int z = 0; z < (RC > 1 ? RC / 2 : 1); ++z) accw[z] = make_float2(0.f, 0.f);
                if (q * 32 < item.cnt && c_lo < c_hi) {   // warp-uniform
                    const float2 pt2 = make_float2(pt, pt);
                    // arg = G A + (C n_i + B); columns past the rows carry B = -inf
                    // (UNI) or A = B = C = w = 0
                    auto cols = [&](int c, const uint32_t (&gr)[32]) {
                        if constexpr (RC == 1 && UNI) {
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
                    // 32-column chunks with two register buffers: the TMEM load
                    // of chunk c + 1 is in flight while chunk c is computed
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
                mbar_arrive(BAR_T_EMPTY(a4));
                if (row < item.cnt && c_lo < c_hi) {
                    float *p = args.partial + (int64_t)(e_out + row) * args.r;
#pragma unroll
                    for (int z = 0; z < RC; ++z)
                        if (z < args.r) p[z] = acc[z];
                }
            }
            mbar_arrive(BAR_BLK_EMPTY(bs));
        }
    epi_done:;
    } else if (warp >= W_CP0) {
        // ----------------------------------------------------- target-row copiers
        // Copier warp w takes rows 64 w .. 64 w + 63 of every item: lane l
        // holds the target slots of rows 64 w + 2 l and + 1, and each 16-byte
        // copy instruction covers four whole rows (eight lanes per 128-byte
        // row, coalesced), into the 128-byte swizzled K-major layout.  The
        // item's copies form one commit group; the stage is reported full
        // (after a proxy fence) DLAG items later, so NA - 1 items' copies are
        // in flight.  The loads an item needs -- its descriptor, its target
        // slots, their n_i -- run as a pipeline three items deep.
        constexpr int DLAG = NA - 2;
        const int cw = warp - W_CP0;
        const int u = lane >> 3, j = lane & 7;           // row within a group of four, 16-byte chunk
        const char *qhi = reinterpret_cast<const char *>(args.q_hi);
        const char *qlo = reinterpret_cast<const char *>(args.q_lo);
        // cursor over this CTA's items in order: block index, item, end of
        // the block's items (loaded once per block)
        int cc = c_begin, cit = 0, cend = 0;
        if (cc < c_end) {
            const int b = args.cta_blocks[cc];
            cit = args.block_off[b];
            cend = args.block_off[b + 1];
        }
        auto advance = [&]() {
            if (cc >= c_end) return;
            if (++cit < cend) return;
            while (++cc < c_end) {
                const int b = args.cta_blocks[cc];
                cit = args.block_off[b];
                cend = args.block_off[b + 1];
                if (cit < cend) return;
            }
        };
        struct Desc { int e0, cnt; bool ok; };
        auto load_desc = [&]() -> Desc {
            Desc dd = {0, 0, cc < c_end};
            if (dd.ok) {
                const EvalItem item = args.items[cit];
                dd.e0 = item.e0;
                dd.cnt = item.cnt;
            }
            advance();
            return dd;
        };
        // this lane's two rows; rows past cnt repeat the first target
        auto load_rows = [&](const Desc &dd, int (&r)[2]) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int rw = 64 * cw + 2 * lane + k;
                r[k] = dd.ok ? args.tgt[dd.e0 + (rw < dd.cnt ? rw : 0)] : 0;
            }
        };
        auto load_p = [&](bool ok, const int (&r)[2], float (&p)[2]) {
#pragma unroll
            for (int k = 0; k < 2; ++k) p[k] = ok ? args.qn[r[k]] : 0.f;
        };
        Desc d0 = load_desc(), d1 = load_desc(), d2 = load_desc();
        int r0[2], r1[2], r2[2];
        float p0[2], p1[2];
        load_rows(d0, r0);
        load_rows(d1, r1);
        load_p(d0.ok, r0, p0);
        int li = 0;
        for (; d0.ok && !*abort_flag; ++li) {
            const Desc d3 = load_desc();      // item li + 3
            load_rows(d2, r2);                // item li + 2
            load_p(d1.ok, r1, p1);            // item li + 1
            const int sa = li % NA;
            // n_i of this item's targets: the slot is free once the epilogue
            // of the item NA back has read it
            if (!mbar_wait(BAR_P_EMPTY(sa), ((li / NA) & 1) ^ 1, abort_flag, args.status, args.spin)) goto copy_done;
            *reinterpret_cast<float2 *>(ptbuf + sa * 128 + 64 * cw + 2 * lane) = make_float2(p0[0], p0[1]);
            mbar_arrive(BAR_P_FULL(sa));
            if (!mbar_wait(BAR_A_EMPTY(sa), ((li / NA) & 1) ^ 1, abort_flag, args.status, args.spin)) goto copy_done;
            {
                const uint32_t a_hi = sbase + S::A0 + sa * 2 * G_REGION;
#pragma unroll
                for (int g = 0; g < 16; ++g) {
                    // rows 64 cw + 4 g + u: slot held by lane 2 g + (u >> 1)
                    const int src_lane = 2 * g + (u >> 1);
                    const int s0 = __shfl_sync(0xffffffffu, r0[0], src_lane);
                    const int s1 = __shfl_sync(0xffffffffu, r0[1], src_lane);
                    const int slot = (u & 1) ? s1 : s0;
                    const int row = 64 * cw + 4 * g + u;
                    const uint32_t off = (uint32_t)(row * 128 + ((j ^ (row & 7)) << 4));
                    cp_async16(a_hi + off, qhi + (int64_t)slot * 128 + 16 * j);
                    cp_async16(a_hi + G_REGION + off, qlo + (int64_t)slot * 128 + 16 * j);
                }
                cp_async_commit();
            }
            if (li >= DLAG) {
                cp_async_wait<DLAG>();            // the copies of item li - DLAG have landed
                fence_proxy_async();
                mbar_arrive(BAR_A_FULL((li - DLAG) % NA));
            }
            d0 = d1;
            d1 = d2;
            d2 = d3;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                r0[k] = r1[k];
                r1[k] = r2[k];
                p0[k] = p1[k];
            }
        }
        // the last items' copies
        cp_async_wait<0>();
        fence_proxy_async();
        if (!*abort_flag)
            for (int k = li - DLAG > 0 ? li - DLAG : 0; k < li; ++k) mbar_arrive(BAR_A_FULL(k % NA));
    copy_done:
        // nothing may land in this CTA's shared memory after it exits
        cp_async_wait<0>();
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
            const uint32_t idesc = make_idesc(0u, G_ROWS, (ncols + 31) & ~31);
            if (!mbar_wait(BAR_B_EMPTY, (lb & 1) ^ 1, abort_flag, args.status, args.spin)) goto mma_done;
            if (!mbar_wait(BAR_BLK_EMPTY(bs), ((lb >> 1) & 1) ^ 1, abort_flag, args.status, args.spin)) goto mma_done;
            b_issued = lb + 1;
            blk_last[bs] = lb;
            mbar_expect_tx(BAR_B_FULL, (uint32_t)(2 * nsb * G_REGION));
            for (int h = 0; h < nsb; ++h) {
                tma_load_2d(sbase + S::B_HI + h * G_REGION, far ? &map_s_hi : &map_t_hi, 0, first.row0 + 128 * h,
                            BAR_B_FULL);
                tma_load_2d(sbase + S::B_LO + h * G_REGION, far ? &map_s_lo : &map_t_lo, 0, first.row0 + 128 * h,
                            BAR_B_FULL);
            }
            const uint32_t slot = sbase + S::BLK + bs * S::BLKSLOT;
            const uint32_t colw_bytes = RC > 1 ? (uint32_t)(nsb * 128 * RC * 4) : 0u;
            constexpr int CV = UNI ? 64 : 128;   // float4 of column data per sub-block
            mbar_expect_tx(BAR_BLK_FULL(bs), (uint32_t)(nsb * CV * 16) + colw_bytes);
            bulk_copy(slot + S::BLK_COLV, args.colv + (int64_t)first.cidx * CV, nsb * CV * 16, BAR_BLK_FULL(bs));
            if constexpr (RC > 1)
                bulk_copy(slot + S::BLK_COLW, args.colw + (int64_t)first.cidx * 128 * RC, colw_bytes, BAR_BLK_FULL(bs));
            for (int it = i0; it < i1; ++it, ++li) {
                const int sa = li % NA, a4 = li % NACC;
                if (!mbar_wait(BAR_A_FULL(sa), (li / NA) & 1, abort_flag, args.status, args.spin)) goto mma_done;
                if (it == i0 && !mbar_wait(BAR_B_FULL, lb & 1, abort_flag, args.status, args.spin)) goto mma_done;
                if (!mbar_wait(BAR_T_EMPTY(a4), ((li / NACC) & 1) ^ 1, abort_flag, args.status, args.spin)) goto mma_done;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(a4 * 128 * NB);
                const uint32_t a_hi = sbase + S::A0 + sa * 2 * G_REGION, a_lo = a_hi + G_REGION;
                const uint32_t b_hi = sbase + S::B_HI, b_lo = sbase + S::B_LO;
                // the tensor core rounds each accumulation step to the running sum's
                // precision: the small cross terms first, the hi*hi products last
#pragma unroll
                for (int k = 0; k < 4; ++k) {   // K = 16 per MMA: 32 bytes into the 128-byte rows
                    const uint32_t off = (uint32_t)(k * 32);
                    tc_mma<ASKIT_PREC_FP16X3>(d_tmem, sw128_desc(a_hi + off), sw128_desc(b_lo + off), idesc, k > 0);
                    tc_mma<ASKIT_PREC_FP16X3>(d_tmem, sw128_desc(a_lo + off), sw128_desc(b_hi + off), idesc, 1);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t off = (uint32_t)(k * 32);
                    tc_mma<ASKIT_PREC_FP16X3>(d_tmem, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc, 1);
                }
                tc_commit(BAR_A_EMPTY(sa));
                tc_commit(BAR_T_FULL(a4));
                if (it == i1 - 1) tc_commit(BAR_B_EMPTY);
                li_done = li;
            }
        }
    mma_done:
        // after an abort: the last sub-block's tiles and the latest column
        // data of each slot may still be landing, and MMAs may still be
        // writing TMEM -- wait for them before TMEM is freed and the CTA
        // exits (no-ops on the normal path)
        if (b_issued > 0) mbar_drain(BAR_B_FULL, (b_issued - 1) & 1);
        for (int k = 0; k < 2; ++k)
            if (blk_last[k] >= 0) mbar_drain(BAR_BLK_FULL(k), (blk_last[k] >> 1) & 1);
        if (li_done >= 0) mbar_drain(BAR_T_FULL(li_done % NACC), (li_done / NACC) & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == W_MMA) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G_TMEM_COLS) : "memory");
    }
}

// Column data of every sub-block for one Evaluate, from the global-centered
// norms: thread t of block b takes source row t of sub-block b.  General
// layout, rows (2p, 2p+1): {A_2p, A_2p+1, B_2p, B_2p+1}, {C_2p, C_2p+1, w_2p,
// w_2p+1} with A = 2 sc / s^2, B = -sc n_j, C = -sc (zeros past the rows);
// UNI (one bandwidth): {B_j, B_j+1, w_j, w_j+1} with B = -inf past the rows.
template <int RC, int UNI>
__global__ void g16_cols_kernel(const int64_t *sb_row0, const int32_t *sb_nr, int64_t n_leaf_sub, const float *sc_t,
                                const float *sc_s, const float *ng_t, const float *ng_s, const float *Wt,
                                const float *Ws, int r, float g_unscale, float4 *colv, float *colw) {
    const int64_t b = blockIdx.x;
    const int t = threadIdx.x;
    const bool far = b >= n_leaf_sub;
    const int64_t row = sb_row0[b] + t;
    const bool valid = t < sb_nr[b];
    const float sc = valid ? (far ? sc_s : sc_t)[row] : 0.f;
    const float nrm = valid ? (far ? ng_s : ng_t)[row] : 0.f;
    const float *w = (far ? Ws : Wt) + row * r;
    const int o = t & 1;
    if (UNI) {
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

// Tensor maps over the tree's pre-split operands (64 x 128 boxes, 128-byte
// swizzle): [t_hi, t_lo, s_hi, s_lo].
struct G16State {
    CUtensorMap map[4];
    bool ready = false;
    EncodeTiledFn encode = nullptr;
};

std::mutex g_g16_mu;

askit_status g16_state(askit_tree t, G16State **out) {
    std::lock_guard<std::mutex> lock(g_g16_mu);
    if (!t->g16) t->g16 = new G16State();
    G16State *st = (G16State *)t->g16;
    if (!st->encode) ASK_TRY(encode_fn(&st->encode));
    if (!st->ready) {
        const void *arr[4] = {t->Xg_hi, t->Xg_lo, t->Sg_hi, t->Sg_lo};
        for (int i = 0; i < 4; ++i)
            ASK_TRY(encode_2d(st->encode, &st->map[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, arr[i],
                              i < 2 ? t->N_pad : t->srows, TC_K, 64, G_ROWS, CU_TENSOR_MAP_SWIZZLE_128B));
        st->ready = true;
    }
    *out = st;
    return ASKIT_OK;
}

template <int RC, int NA, int NB, int UNI>
askit_status launch_g16(G16State *st, const G16Args &a, int grid, cudaStream_t s) {
    using S = SG<RC, NA, NB>;
    constexpr size_t smem = S::BYTES + 1024;
    static_assert(smem <= 232448, "shared-memory plan exceeds 227 KB");
    static const cudaError_t attr = cudaFuncSetAttribute(eval_g16_kernel<RC, NA, NB, UNI>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ASK_CUDA(attr);
    eval_g16_kernel<RC, NA, NB, UNI><<<(unsigned)grid, S::THREADS, smem, s>>>(
        st->map[0], st->map[1], st->map[2], st->map[3], a);
    ASK_LAUNCH();
    return ASKIT_OK;
}

template <int RC, int UNI>
askit_status pick_g16(askit_tree t, G16State *st, G16Args a, const WorkLists &w, int stages, bool pairs,
                      cudaStream_t s) {
    // three or four target-row stages (one or two items' copies in flight);
    // paired 256-column items up to r = 4
    if constexpr (RC <= 4) {
        if (pairs && w.sched_off[2]) {
            a.cta_off = w.sched_off[2];
            a.cta_blocks = w.sched_blocks[2];
            a.partner = w.partner;
            if (stages <= 3) return launch_g16<RC, 3, 2, UNI>(st, a, w.n_ctas, s);
            return launch_g16<RC, 4, 2, UNI>(st, a, w.n_ctas, s);
        }
    }
    if (stages <= 3) return launch_g16<RC, 3, 1, UNI>(st, a, w.n_ctas, s);
    return launch_g16<RC, 4, 1, UNI>(st, a, w.n_ctas, s);
}

template <int RC>
askit_status run_g16(askit_tree t, const WeightCtx &c, G16State *st, G16Args a, const WorkLists &w,
                     cudaStream_t s) {
    const float g_unscale = 1.f / (t->g_scale * t->g_scale);
    const bool uni = RC == 1 && t->prm.bw_mode == ASKIT_BW_CONSTANT;
    if (uni) {
        // the same rounding as the per-row values (h held in FP32)
        const double hf = (double)(float)t->prm.h;
        const float sc = (float)(t->prm.kernel_scale * 1.4426950408889634 / (hf * hf));
        a.uni_a = 2.f * g_unscale * sc;
        a.uni_c = -sc;
        g16_cols_kernel<RC, 1><<<(unsigned)t->n_sub, 128, 0, s>>>(t->sb_row0, t->sb_nr, t->n_leaf_sub, t->sc_t, t->sc_s,
                                                                  t->ng_t, t->ng_s, c.Wt, c.Ws, c.r, g_unscale, c.colv,
                                                                  c.colw);
    } else {
        g16_cols_kernel<RC, 0><<<(unsigned)t->n_sub, 128, 0, s>>>(t->sb_row0, t->sb_nr, t->n_leaf_sub, t->sc_t, t->sc_s,
                                                                  t->ng_t, t->ng_s, c.Wt, c.Ws, c.r, g_unscale, c.colv,
                                                                  c.colw);
    }
    ASK_LAUNCH();
    a.colv = c.colv;
    a.colw = c.colw;
    ASK_TRY(ktimer_mark(t, s, false));
    if constexpr (RC == 1) {
        if (uni) ASK_TRY((pick_g16<RC, 1>(t, st, a, w, t->tune_stages, t->tune_pairs, s)));
        else ASK_TRY((pick_g16<RC, 0>(t, st, a, w, t->tune_stages, t->tune_pairs, s)));
    } else {
        ASK_TRY((pick_g16<RC, 0>(t, st, a, w, t->tune_stages, t->tune_pairs, s)));
    }
    return ktimer_mark(t, s, true);
}

}  // namespace

askit_status eval_g16(askit_tree t, const WeightCtx &c, const QuerySplit &q, const WorkLists &w, float *partial,
                      cudaStream_t s) {
    if (c.r > 16) {
        askit_set_error("tensor-core evaluation covers r <= 16; use ASKIT_PREC_SIMT_FP32");
        return ASKIT_ERR_UNSUPPORTED;
    }
    if (w.n_blocks == 0) return ASKIT_OK;
    if (!t->Xg_hi || !q.hi || !q.lo || !q.n || !c.colv || (c.r > 1 && !c.colw)) {
        askit_set_error("the global-centered FP16x3 operands are missing");
        return ASKIT_ERR_INVALID_ARG;
    }
    G16State *st = nullptr;
    ASK_TRY(g16_state(t, &st));
    G16Args a;
    a.items = w.items;
    a.block_off = w.block_off;
    a.cta_off = w.cta_off;
    a.cta_blocks = w.cta_blocks;
    a.tgt = w.tgt;
    a.q_hi = q.hi;
    a.q_lo = q.lo;
    a.qn = q.n;
    a.colv = nullptr;
    a.colw = nullptr;
    a.partner = nullptr;
    a.r = c.r;
    a.uni_a = a.uni_c = 0.f;
    a.partial = partial;
    a.status = t->d_status;
    a.spin = t->spin_limit > 0 ? t->spin_limit : SPIN_LIMIT;
    if (c.r == 1) return run_g16<1>(t, c, st, a, w, s);
    if (c.r <= 4) return run_g16<4>(t, c, st, a, w, s);
    return run_g16<16>(t, c, st, a, w, s);
}

void eval_g16_free(askit_tree t) {
    delete (G16State *)t->g16;
    t->g16 = nullptr;
}

// ---------------------------------------------------------------------------
// Global-centered operands: x~ = (x - xbar) s split into FP16 hi + lo, and
// n = |x - xbar|^2, one warp per row (lanes over the TC_K columns; the sum of
// squares in FP64 over a fixed butterfly, then rounded).  Rows past `rows`
// are left as they are (zeros from the caller's memset).  A row whose scaled
// value leaves the FP16-safe range raises *overflow.
// ---------------------------------------------------------------------------
__global__ void gsplit_kernel(const float *X, int64_t ldx, int d, int64_t rows, const float *xbar, float scale,
                              uint16_t *hi, uint16_t *lo, float *n, int *overflow) {
    const int lane = threadIdx.x & 31;
    const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows) return;
    double acc = 0.0;
    bool bad = false;
#pragma unroll
    for (int h = 0; h < TC_K / 32; ++h) {
        const int k = lane + 32 * h;
        const float x = k < d ? X[row * ldx + k] - xbar[k] : 0.f;
        acc += (double)x * (double)x;
        const float v = x * scale;
        bad |= !(fabsf(v) <= 30000.f);
        const __half vh = __float2half_rn(v);
        const __half vl = __float2half_rn(v - __half2float(vh));
        hi[row * TC_K + k] = __half_as_ushort(vh);
        lo[row * TC_K + k] = __half_as_ushort(vl);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) n[row] = (float)acc;
    if (__any_sync(0xffffffffu, bad) && lane == 0 && overflow) atomicExch(overflow, 1);
}

askit_status g16_split_rows(const float *X, int64_t ldx, int d, int64_t rows, const float *xbar, float scale,
                            uint16_t *hi, uint16_t *lo, float *n, int *overflow, cudaStream_t s) {
    if (rows <= 0) return ASKIT_OK;
    gsplit_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(X, ldx, d, rows, xbar, scale, hi, lo, n, overflow);
    ASK_LAUNCH();
    return ASKIT_OK;
}

namespace {

// Column sums of the first n rows of X [*, ldx] in FP64 (thread-strided
// partial sums, then a fixed tree over the block): mean[k] = sum / n, FP32.
__global__ void col_mean_kernel(const float *X, int64_t ldx, int64_t n, float *mean) {
    __shared__ double part[256];
    const int k = blockIdx.x;
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) acc += (double)X[r * ldx + k];
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) mean[k] = (float)(part[0] / (double)n);
}

// Largest |x_k - xbar_k| over the first n rows (non-negative floats compare
// as their bit patterns).
__global__ void dev_extent_kernel(const float *X, int64_t ldx, int d, int64_t n, const float *xbar, float *ext) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float v = 0.f;
    if (e < n * d) v = fabsf(X[(e / d) * ldx + e % d] - xbar[e % d]);
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(ext), __float_as_int(v));
}

// Largest value of a non-negative array.
__global__ void max_kernel(const float *a, int64_t n, float *out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float v = e < n ? fmaxf(a[e], 0.f) : 0.f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(out), __float_as_int(v));
}

}  // namespace

// The global-centered FP16x3 operands of a narrow tree (d <= TC_K): xbar (the
// FP64 mean of the points), the prescale (a power of 2 mapping the largest
// |x_k - xbar_k| to at most 2^12, so targets up to 7 times farther out still
// fit FP16), the split rows of the tree points and of the skeleton pool, their
// n = |x - xbar|^2, and the accuracy figure rho = max_j sc_j max_i n_i: the
// exponent's FP32 rounding error is a few 2^-24 rho, so g_ok (the automatic
// choice of this kernel) holds while rho <= 512 (relative error of u about
// 1e-5 at rho = 150, within the split-product tolerance 1e-4 up to the bound).
askit_status build_g16_operands(askit_tree t, cudaStream_t s) {
    constexpr double RHO_MAX = 512.0;
    const int d = t->d;
    ASK_TRY(t->arena.alloc(&t->g_xbar, TC_K));
    ASK_CUDA(cudaMemsetAsync(t->g_xbar, 0, sizeof(float) * TC_K, s));
    col_mean_kernel<<<(unsigned)d, 256, 0, s>>>(t->Xt, t->d_pad, t->N, t->g_xbar);
    ASK_LAUNCH();
    float *red = nullptr;   // [3]: extent, max n, max sc
    ASK_CUDA(cudaMallocAsync(&red, 3 * sizeof(float), s));
    ASK_CUDA(cudaMemsetAsync(red, 0, 3 * sizeof(float), s));
    dev_extent_kernel<<<(unsigned)((t->N * d + 255) / 256), 256, 0, s>>>(t->Xt, t->d_pad, d, t->N, t->g_xbar, red);
    ASK_LAUNCH();
    float hred[3] = {0.f, 0.f, 0.f};
    ASK_CUDA(cudaMemcpyAsync(hred, red, sizeof(float), cudaMemcpyDeviceToHost, s));
    ASK_CUDA(cudaStreamSynchronize(s));
    int e = 0;
    if (hred[0] > 0.f) frexpf(4096.f / hred[0], &e);
    t->g_scale = ldexpf(1.f, e - 1);
    const size_t et = (size_t)t->N_pad * TC_K, es = (size_t)t->srows * TC_K;
    ASK_TRY(t->arena.alloc(&t->Xg_hi, et));
    ASK_TRY(t->arena.alloc(&t->Xg_lo, et));
    ASK_TRY(t->arena.alloc(&t->Sg_hi, es));
    ASK_TRY(t->arena.alloc(&t->Sg_lo, es));
    ASK_TRY(t->arena.alloc(&t->ng_t, t->N_pad));
    ASK_TRY(t->arena.alloc(&t->ng_s, t->srows));
    // every row, padding included, holds finite values: a 128-row tile read
    // past a short sub-block multiplies them by zero column data
    ASK_TRY(g16_split_rows(t->Xt, t->d_pad, d, t->N_pad, t->g_xbar, t->g_scale, t->Xg_hi, t->Xg_lo, t->ng_t, nullptr,
                           s));
    ASK_TRY(g16_split_rows(t->Xs, t->d_pad, d, t->srows, t->g_xbar, t->g_scale, t->Sg_hi, t->Sg_lo, t->ng_s, nullptr,
                           s));
    max_kernel<<<(unsigned)((t->N + 255) / 256), 256, 0, s>>>(t->ng_t, t->N, red + 1);
    max_kernel<<<(unsigned)((t->N + 255) / 256), 256, 0, s>>>(t->sc_t, t->N, red + 2);
    ASK_LAUNCH();
    ASK_CUDA(cudaMemcpyAsync(hred, red, 3 * sizeof(float), cudaMemcpyDeviceToHost, s));
    ASK_CUDA(cudaStreamSynchronize(s));
    cudaFreeAsync(red, s);
    t->g_rho = (double)hred[1] * (double)hred[2];
    t->g_ok = t->g_rho <= RHO_MAX;
    return ASKIT_OK;
}
