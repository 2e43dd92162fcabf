// Evaluate (Algorithm 4) on the tcgen05 tensor cores with FP16x3 split
// operands, d <= 64, every operand pre-split in HBM ("global centering"),
// and the whole exponent argument formed by the tensor cores.
//
// Every point is centered once on the data mean xbar.  With n = |x - xbar|^2
// and sc_j = c log2(e) / h_j^2 (the source's bandwidth),
//
//     arg_ij = -sc_j |x_i - y_j|^2
//            = 2 sc_j (x_i - xbar).(y_j - xbar) - sc_j n_i - sc_j n_j,
//     partial_i += exp2(arg_ij) w_j.
//
// The MMA accumulator receives arg_ij itself:
//   - the main K = 64 block: targets a_i = (x_i - xbar) sigma, sources
//     b_j = (y_j - xbar) 2 sc_j / sigma, each split into FP16 hi + lo and
//     multiplied as hi*lo + lo*hi + hi*hi (FP32 accumulation, small terms
//     first); sigma is a power of 2 near sqrt(2 sc_max), so both sides have
//     similar magnitudes well inside the FP16 range;
//   - one extra K = 16 block holding the norm terms already split:
//     targets [h(n_i tau), h(n_i tau), l(n_i tau), kappa, kappa, 0 ...],
//     sources [h(m_j), l(m_j), h(m_j), h(v_j), l(v_j), 0 ...] with
//     m_j = -sc_j / tau, v_j = -sc_j n_j / kappa (tau, kappa powers of 2
//     balancing the factors), whose product is -sc_j (n_i + n_j) to the
//     split's precision.
// So the epilogue is an ex2 on MUFU and, for r <= 4, r weight FMAs per pair.
// For r > 4 the weight sums run on the tensor cores as well: the epilogue
// writes k 2^14, split into FP16 hi + lo, back over the argument's TMEM
// columns, and a second MMA with A read from TMEM multiplies it with the
// sub-block's weights, split the same way after scaling every vector by a
// power of 2 (k hi against [w' hi | w' lo] and k lo against w' hi, FP32
// accumulation), into a 32-column accumulator whose halves the epilogue adds:
// one ex2 and a few conversions per pair instead of r FMAs and r/4
// shared-memory loads of the weights.  An argument accumulator is free again
// once its item's weight MMAs have read it, so the tensor cores never wait
// for the epilogue's write-out.  The price
// is precision: the terms 2 sc (x - xbar).(y - xbar) and sc n are of the size
// of sc R^2 (R = the data's spread around xbar) and are rounded in FP32, so
// the exponent carries an error of a few 2^-24 sc R^2; the per-sub-block
// centered kernel (eval_tc16.cu) keeps these terms at the size of a node.
// The tree takes this kernel only while rho = sc_max R^2_max <= 512
// (build_g16_operands), and askit_set_fp16_centering overrides the choice.
// Measured: relative L2 error of u about 1e-5 (the per-sub-block kernel
// about 1e-6), within the split-product tolerance 1e-4.
//
// No target row is converted on the chip: each work item's 128 target rows
// are copied in the MMA's layouts straight from HBM (16-byte cp.async, eight
// lanes per 128-byte row; a TMA tile::gather4 costs about 75 cycles of issue
// per four rows on this part, which made the copies the bottleneck).
//
// Work item = one source sub-block (or two sub-blocks of one node: a paired
// 256-column item) against up to 128 targets needing it (eval_lists.cu).
// One CTA per SM, 384 threads:
//   warps 0-7  two epilogue groups, each summing whole sub-blocks (alternate
//              items, or the two sub-blocks of a paired item): tcgen05.ld of
//              their 32 TMEM lanes (two buffers), ex2 on MUFU, weight sums
//              (r > 4: the split exponentials stored back to TMEM, then the
//              weight MMA's sums loaded), one partial sum per (target,
//              sub-block) entry;
//   warp 8     TMEM allocation; lane 0 loads each sub-block (TMA tiles of its
//              split rows, bulk copies of its norm block and weights) and
//              issues the argument MMAs (r <= 4: of the even items; r > 4: of
//              every item);
//   warps 9-10 copy each item's target rows into NA stages (NA - 2 items'
//              copies in flight);
//   warp 11    lane 0 issues the odd items' argument MMAs (r <= 4), or every
//              item's weight MMAs once the epilogue has stored its
//              exponentials (r > 4): a tcgen05.mma costs its issuing thread
//              about a hundred cycles.
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
constexpr int GX_REGION = G_ROWS * 32;   // 128 rows x 32 bytes (16 FP16): the norm block
constexpr int GX_K = 16;                 // columns of the norm block
constexpr uint32_t G_TMEM_COLS = 512;    // 4 x 128 (2 x 256) columns; r > 4: 3 x 128 + 4 x 32

// Shared-memory descriptor of a K-major operand without swizzle: 8-row x
// 16-byte core matrices stored contiguously, the next core matrix along K
// 128 bytes on (leading-byte offset), along M/N 256 bytes on (stride-byte
// offset); version bit 46, layout type 0 (no swizzle).
__device__ __forceinline__ uint64_t ns_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
           ((uint64_t)1 << 46);
}
// Byte offset of row r, 16-byte chunk c of a norm block in that layout.
__host__ __device__ __forceinline__ uint32_t nx_off(int r, int c) {
    return (uint32_t)((r >> 3) * 256 + c * 128 + (r & 7) * 16);
}

// Weights of a sub-block for the weight MMA (r > 4): W' = w 2^-e_z split into
// FP16 hi and lo, each [16 vectors x 128 source rows] K-major without swizzle
// (core matrices of 8 vectors x 8 rows; the next along the rows 128 bytes on,
// the next 8 vectors 2048 bytes on), then 16 FP32 factors 2^(e_z - G_KSHIFT).
constexpr int GW_SPLIT = 4096;                  // bytes of one split
constexpr int GW_BYTES = 2 * GW_SPLIT + 64;     // hi, lo, factors
constexpr int G_KSHIFT = 14;                    // exponentials enter the MMA as k 2^14
constexpr int GW_NDW = 4;                       // weight-sum accumulators (32 columns each)
__host__ __device__ __forceinline__ uint32_t gw_off(int z, int row) {
    return (uint32_t)((z >> 3) * 2048 + (row >> 3) * 128 + (z & 7) * 16 + (row & 7) * 2);
}
__device__ __forceinline__ uint64_t gw_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(2048 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// NA: target-row stages; NB: sub-blocks per item (1, or 2 for paired items).
// r <= 4 (WMMA false): NACC = 4 / NB TMEM accumulators of 128 NB columns and
// the weight sums on the FP32 pipe.  r > 4 (WMMA, NB = 1): three 128-column
// accumulators for the exponent's argument (later overwritten by the split
// exponentials, the A operand of the weight MMA) and GW_NDW 32-column
// accumulators of the weight sums from column 384 (columns 0-15: k hi w' hi +
// k lo w' hi, 16-31: k hi w' lo).
template <int RC, int NA, int NB>
struct SG {
    static constexpr bool WMMA = RC > 4;
    static_assert(!WMMA || NB == 1, "weight MMAs take single sub-blocks");
    static constexpr int NACC = WMMA ? 3 : 4 / NB;
    static constexpr int B_HI = 0, B_LO = NB * G_REGION;    // NB x 128 rows each, contiguous
    static constexpr int B_X = 2 * NB * G_REGION;           // NB x 128 rows of the norm block
    static constexpr int A0 = B_X + NB * GX_REGION;         // stage s at A0 + s ASTAGE: hi, lo, norm block
    static constexpr int ASTAGE = 2 * G_REGION + GX_REGION;
    static constexpr int BLK = A0 + NA * ASTAGE;            // [2] per-block weight slots
    static constexpr int BLKSLOT = WMMA ? GW_BYTES : NB * 128 * RC * 4;   // float [128 NB][RC], or split weights
    static constexpr int BAR = BLK + 2 * BLKSLOT;           // 40 mbarriers
    static constexpr int MISC = BAR + 40 * 8;               // tmem address, abort flag
    static constexpr int BYTES = MISC + 16;
    static constexpr int THREADS = 384;    // warp 11: the second MMA issuer (r <= 4) or the weight MMAs' (r > 4)
    static_assert(A0 % 1024 == 0 && ASTAGE % 1024 == 0, "swizzled stages need 1024-byte alignment");
};

struct G16Args {
    const EvalItem *items;
    const int32_t *block_off;
    const int32_t *cta_off, *cta_blocks;
    const int32_t *tgt;            // entry -> target slot (row of the query operand)
    const uint16_t *q_hi, *q_lo;   // [query rows, 64] split target rows
    const uint16_t *q_x;           // [query rows, 16] target norm blocks
    const uint16_t *bx;            // [n_sub, 128 x 16] source norm blocks (core-matrix layout)
    const float *colw;             // [n_sub, 128, RC] weights (zeros past the rows)
    const int32_t *partner;        // [n_blocks] paired follower block, or -1 (NB == 2)
    int r;
    float *partial;
    int *status;
    int spin;
};

template <int RC, int NA, int NB>
__global__ void __launch_bounds__(SG<RC, NA, NB>::THREADS, 1)
eval_g16_kernel(const __grid_constant__ CUtensorMap map_t_hi, const __grid_constant__ CUtensorMap map_t_lo,
                const __grid_constant__ CUtensorMap map_s_hi, const __grid_constant__ CUtensorMap map_s_lo,
                const G16Args args) {
    using S = SG<RC, NA, NB>;
    constexpr int NACC = S::NACC;
    constexpr int NEPI = 256;                    // epilogue threads (two groups of 128)
    // drainers of an item's accumulator: one group (alternate items) or both
    // (paired items)
    constexpr int NITEM = NB == 2 ? 256 : 128;
    constexpr int W_MMA = 8, W_CP0 = 9;          // MMA warp, first of the two copier warps
    constexpr int W_WI = 11;                     // r <= 4: odd items' argument MMAs; r > 4: the weight MMAs
    // r <= 4: two threads issue the argument MMAs, alternate items (a
    // tcgen05.mma costs its issuing thread about a hundred cycles, close to
    // what a 128-row, 256-column, K = 16 MMA takes on the tensor core)
    constexpr bool SPLIT = !S::WMMA;
    static_assert(NA >= 3 && NA <= 4, "the copiers keep NA - 2 items in flight");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(sm);
    const uint32_t bar0 = sbase + S::BAR;
    auto BAR_A_FULL = [&](int s) { return bar0 + 8 * s; };            // target rows of stage s landed (64)
    auto BAR_A_EMPTY = [&](int s) { return bar0 + 8 * (4 + s); };     // MMAs reading stage s done (commit)
    const uint32_t BAR_B_FULL = bar0 + 8 * 8, BAR_B_EMPTY = bar0 + 8 * 9;
    auto BAR_BLK_FULL = [&](int s) { return bar0 + 8 * (10 + s); };   // weights of slot s landed
    auto BAR_BLK_EMPTY = [&](int s) { return bar0 + 8 * (12 + s); };  // epilogue done with slot s (NEPI)
    auto BAR_T_FULL = [&](int a) { return bar0 + 8 * (16 + a); };     // accumulator a complete (commit)
    // accumulator a free: drained by the epilogue (NITEM), or, r > 4, read by
    // the item's weight MMAs (commit)
    auto BAR_T_EMPTY = [&](int a) { return bar0 + 8 * (20 + a); };
    auto BAR_K_READY = [&](int a) { return bar0 + 8 * (24 + a); };    // split exponentials of a in TMEM (128)
    auto BAR_DW_FULL = [&](int k) { return bar0 + 8 * (28 + k); };    // weight sums k complete (commit)
    auto BAR_DW_EMPTY = [&](int k) { return bar0 + 8 * (32 + k); };   // weight sums k read (128)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + S::MISC);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + S::MISC + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < NA; ++s) {
            mbar_init(BAR_A_FULL(s), 64);
            mbar_init(BAR_A_EMPTY(s), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(BAR_BLK_FULL(s), 1);
            mbar_init(BAR_BLK_EMPTY(s), NEPI);
        }
        mbar_init(BAR_B_FULL, 1);
        mbar_init(BAR_B_EMPTY, SPLIT ? 2 : 1);      // one commit per issuer and block
        for (int a = 0; a < NACC; ++a) {
            mbar_init(BAR_T_FULL(a), 1);
            mbar_init(BAR_T_EMPTY(a), S::WMMA ? 1 : NITEM);
            if constexpr (S::WMMA) mbar_init(BAR_K_READY(a), 128);
        }
        if constexpr (S::WMMA)
            for (int k = 0; k < GW_NDW; ++k) {
                mbar_init(BAR_DW_FULL(k), 1);
                mbar_init(BAR_DW_EMPTY(k), 128);
            }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the copiers write only the first 16-byte chunk of each target row's
    // norm block: the second (columns 8-15) stays zero
    for (int e = tid; e < NA * G_ROWS; e += S::THREADS) {
        const int s = e / G_ROWS, rr = e % G_ROWS;
        *reinterpret_cast<uint4 *>(sm + S::A0 + s * S::ASTAGE + 2 * G_REGION + nx_off(rr, 1)) = make_uint4(0, 0, 0, 0);
    }
    fence_proxy_async();
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

    // The argument MMAs of item li (stage li % NA, accumulator li % NACC)
    // against the block's sub-block tiles; false when a wait gave up.
    auto issue_arg = [&](int li, uint32_t idesc) -> bool {
        const int sa = li % NA, a4 = li % NACC;
        if (!mbar_wait(BAR_A_FULL(sa), (li / NA) & 1, abort_flag, args.status, args.spin)) return false;
        if (!mbar_wait(BAR_T_EMPTY(a4), ((li / NACC) & 1) ^ 1, abort_flag, args.status, args.spin)) return false;
        tc_fence_after();
        const uint32_t d_tmem = tmem + (uint32_t)(a4 * 128 * NB);
        const uint32_t a_hi = sbase + S::A0 + sa * S::ASTAGE, a_lo = a_hi + G_REGION;
        const uint32_t a_x = a_hi + 2 * G_REGION;
        const uint32_t b_hi = sbase + S::B_HI, b_lo = sbase + S::B_LO, b_x = sbase + S::B_X;
        // the tensor core rounds each accumulation step to the running sum's
        // precision: the small cross terms first, then the hi*hi products,
        // then the norm block, which brings the sum down to the exponent's
        // argument
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
        tc_mma<ASKIT_PREC_FP16X3>(d_tmem, ns_desc(a_x), ns_desc(b_x), idesc, 1);
        tc_commit(BAR_A_EMPTY(sa));
        tc_commit(BAR_T_FULL(a4));
        return true;
    };
    // N of a block's argument MMAs: every 32-column chunk the epilogue reads
    // (a paired follower's columns follow the leader's), so no column it
    // reads holds a stale accumulator
    auto block_idesc = [&](int b, int i0) -> uint32_t {
        const int pb = NB == 2 ? args.partner[b] : -1;
        const int ncols = (args.items[i0].nrows & 0x7fffffff) +
                          (pb >= 0 ? (args.items[args.block_off[pb]].nrows & 0x7fffffff) : 0);
        return make_idesc(0u, G_ROWS, (ncols + 31) & ~31);
    };

    if (warp < W_MMA) {
        // ----------------------------------------------------------- epilogue
        // Each group sums whole sub-blocks: with single sub-blocks (NB == 1)
        // the two groups take alternate items; with paired items (NB == 2)
        // group 0 takes the leader's 128 columns and group 1 the follower's,
        // and each writes its own entry's partial sum -- so every entry's
        // partial is formed the same way in both layouts.  A paired-layout
        // item without a follower is summed by group 0 alone.
        const int q = warp & 3;                    // this warp's TMEM lane quadrant
        const int row = q * 32 + lane;             // TMEM lane = target row of the item
        const int eg = warp >> 2;                  // group
        // r > 4: an item's weight sums are written out after the group has
        // split its next item of the same block (their MMAs are issued after
        // that item's argument MMAs), or at the end of the block
        int pend_li = -1, pend_e0 = 0, pend_cnt = 0;
        auto wout = [&](int pl, int e0, int cnt, const float *cw) -> bool {
            const int k = pl % GW_NDW;
            if (!mbar_wait(BAR_DW_FULL(k), (pl / GW_NDW) & 1, abort_flag, args.status, args.spin)) return false;
            tc_fence_after();
            uint32_t g[32];
            if (q * 32 < cnt) {   // warp-uniform
                tmem_ld32_async(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(3 * 128 + k * 32), g);
                tmem_wait_pin(g);
            }
            tc_fence_before();
            mbar_arrive(BAR_DW_EMPTY(k));
            if (row < cnt) {
                // the sums of w' k 2^14 back to w k: the sub-block's factors
                const float4 *fac = reinterpret_cast<const float4 *>(cw + 2 * GW_SPLIT / 4);
                float *p = args.partial + (int64_t)(e0 + row) * args.r;
                auto u = [&](int z, float f) { return (__uint_as_float(g[z]) + __uint_as_float(g[16 + z])) * f; };
#pragma unroll
                for (int z = 0; z < 16; z += 4) {
                    const float4 f = fac[z / 4];
                    const float4 v = make_float4(u(z, f.x), u(z + 1, f.y), u(z + 2, f.z), u(z + 3, f.w));
                    if (args.r == 16) {
                        *reinterpret_cast<float4 *>(p + z) = v;
                    } else {
                        if (z < args.r) p[z] = v.x;
                        if (z + 1 < args.r) p[z + 1] = v.y;
                        if (z + 2 < args.r) p[z + 2] = v.z;
                        if (z + 3 < args.r) p[z + 3] = v.w;
                    }
                }
            }
            return true;
        };
        int li = 0, lb = 0;
        for (int ci = c_begin; ci < c_end && !*abort_flag; ++ci, ++lb) {
            const int b = args.cta_blocks[ci];
            const int bs = lb & 1;
            if (!mbar_wait(BAR_BLK_FULL(bs), (lb >> 1) & 1, abort_flag, args.status, args.spin)) goto epi_done;
            const float *cwp = reinterpret_cast<const float *>(sm + S::BLK + bs * S::BLKSLOT);
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
                const int a4 = li % NACC;
                const EvalItem item = args.items[it];
                const int e_out = (NB == 2 && eg == 1) ? (pb >= 0 ? args.items[f0 + (it - i0)].e0 : 0) : item.e0;
                if (!mbar_wait(BAR_T_FULL(a4), (li / NACC) & 1, abort_flag, args.status, args.spin)) goto epi_done;
                tc_fence_after();
                if constexpr (S::WMMA) {
                    // k 2^14 split into FP16 hi + lo, stored over the argument
                    // columns it came from: chunk c's 32 columns take its 32 hi
                    // values (two per column), then its 32 lo values; the MMA
                    // warp multiplies them with the sub-block's split weights
                    const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a4 * 128);
                    if (q * 32 < item.cnt) {   // warp-uniform
                        auto split_store = [&](int c, const uint32_t (&gr)[32]) {
                            uint32_t hw[16], lw[16];
#pragma unroll
                            for (int m = 0; m < 16; ++m) {
                                const float k0 = ex2_approx(__uint_as_float(gr[2 * m])) * (float)(1 << G_KSHIFT);
                                const float k1 = ex2_approx(__uint_as_float(gr[2 * m + 1])) * (float)(1 << G_KSHIFT);
                                const __half2 h = __floats2half2_rn(k0, k1);
                                const float2 hf = __half22float2(h);
                                const __half2 l = __floats2half2_rn(k0 - hf.x, k1 - hf.y);
                                hw[m] = *reinterpret_cast<const uint32_t *>(&h);
                                lw[m] = *reinterpret_cast<const uint32_t *>(&l);
                            }
                            tmem_st16(tbase + (uint32_t)(c * 32), hw);
                            tmem_st16(tbase + (uint32_t)(c * 32 + 16), lw);
                        };
                        // one chunk at a time (the other group's warp on the same
                        // sub-partition covers the load's latency); a chunk's
                        // stores go to its own, already loaded, columns
#pragma unroll 1
                        for (int c = 0; c < c_hi; ++c) {
                            uint32_t ga[32];
                            tmem_ld32_async(tbase + (uint32_t)(c * 32), ga);
                            tmem_wait_pin(ga);
                            split_store(c, ga);
                        }
                        tmem_st_wait();
                    }
                    tc_fence_before();
                    mbar_arrive(BAR_K_READY(a4));
                    if (pend_li >= 0 && !wout(pend_li, pend_e0, pend_cnt, cwp)) goto epi_done;
                    pend_li = li;
                    pend_e0 = item.e0;
                    pend_cnt = item.cnt;
                } else {
                float acc[RC];
#pragma unroll
                for (int z = 0; z < RC; ++z) acc[z] = 0.f;
                float2 acc2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};   // RC == 1
                float2 accw[RC > 1 ? RC / 2 : 1];                                    // RC > 1
#pragma unroll
                for (int z = 0; z < (RC > 1 ? RC / 2 : 1); ++z) accw[z] = make_float2(0.f, 0.f);
                if (q * 32 < item.cnt && c_lo < c_hi) {   // warp-uniform
                    // the accumulator holds the exponent's argument; columns
                    // past the rows carry w = 0
                    auto cols = [&](int c, const uint32_t (&gr)[32]) {
                        if constexpr (RC == 1) {
#pragma unroll
                            for (int jj = 0; jj < 32; jj += 4) {
                                const float4 w4 = *reinterpret_cast<const float4 *>(cwp + c * 32 + jj);
                                const float2 k0 = make_float2(ex2_approx(__uint_as_float(gr[jj])),
                                                              ex2_approx(__uint_as_float(gr[jj + 1])));
                                const float2 k1 = make_float2(ex2_approx(__uint_as_float(gr[jj + 2])),
                                                              ex2_approx(__uint_as_float(gr[jj + 3])));
                                acc2[0] = __ffma2_rn(k0, make_float2(w4.x, w4.y), acc2[0]);
                                acc2[1] = __ffma2_rn(k1, make_float2(w4.z, w4.w), acc2[1]);
                            }
                        } else {
#pragma unroll
                            for (int jj = 0; jj < 32; ++jj) {
                                const int j = c * 32 + jj;
                                const float k = ex2_approx(__uint_as_float(gr[jj]));
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
            }
            if constexpr (S::WMMA) {
                if (pend_li >= 0 && !wout(pend_li, pend_e0, pend_cnt, cwp)) goto epi_done;
                pend_li = -1;
            }
            mbar_arrive(BAR_BLK_EMPTY(bs));
        }
    epi_done:;
    } else if (warp >= W_CP0 && warp < W_CP0 + 2) {
        // ----------------------------------------------------- target-row copiers
        // Copier warp w takes rows 64 w .. 64 w + 63 of every item: lane l
        // holds the target slots of rows 64 w + 2 l and + 1.  Each 16-byte copy
        // instruction of the split rows covers four whole rows (eight lanes per
        // 128-byte row, coalesced) into the 128-byte swizzled K-major layout;
        // the norm blocks' first chunks follow, one row per lane.  An item's
        // copies form one commit group; the stage is reported full (after a
        // proxy fence) NA - 2 items later.  The loads an item needs -- its
        // descriptor, then its target slots -- run as a pipeline two items
        // ahead.
        constexpr int DLAG = NA - 2;
        const int cw = warp - W_CP0;
        const int u = lane >> 3, j = lane & 7;           // row within a group of four, 16-byte chunk
        const char *qhi = reinterpret_cast<const char *>(args.q_hi);
        const char *qlo = reinterpret_cast<const char *>(args.q_lo);
        const char *qx = reinterpret_cast<const char *>(args.q_x);
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
        Desc d0 = load_desc(), d1 = load_desc();
        int r0[2], r1[2];
        load_rows(d0, r0);
        int li = 0;
        for (; d0.ok && !*abort_flag; ++li) {
            const Desc d2 = load_desc();      // item li + 2
            load_rows(d1, r1);                // item li + 1
            const int sa = li % NA;
            if (!mbar_wait(BAR_A_EMPTY(sa), ((li / NA) & 1) ^ 1, abort_flag, args.status, args.spin)) goto copy_done;
            {
                const uint32_t a_hi = sbase + S::A0 + sa * S::ASTAGE;
#pragma unroll
                for (int g = 0; g < 16; ++g) {
                    // rows 64 cw + 4 g + u: slot held by lane 2 g + (u >> 1)
                    const int src_lane = 2 * g + (u >> 1);
                    const int s0 = __shfl_sync(0xffffffffu, r0[0], src_lane);
                    const int s1 = __shfl_sync(0xffffffffu, r0[1], src_lane);
                    const int slot = (u & 1) ? s1 : s0;
                    const int rr = 64 * cw + 4 * g + u;
                    const uint32_t off = (uint32_t)(rr * 128 + ((j ^ (rr & 7)) << 4));
                    cp_async16(a_hi + off, qhi + (int64_t)slot * 128 + 16 * j);
                    cp_async16(a_hi + G_REGION + off, qlo + (int64_t)slot * 128 + 16 * j);
                }
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int rr = 64 * cw + 2 * lane + k;
                    cp_async16(a_hi + 2 * G_REGION + nx_off(rr, 0), qx + (int64_t)r0[k] * (2 * GX_K));
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
#pragma unroll
            for (int k = 0; k < 2; ++k) r0[k] = r1[k];
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
        int blk_last[2] = {-1, -1};   // last block whose weights went to slot 0 / 1
        int li_done = -1;             // last item whose MMAs were committed
        for (int ci = c_begin; ci < c_end && !*abort_flag; ++ci, ++lb) {
            const int b = args.cta_blocks[ci];
            const int i0 = args.block_off[b], i1 = args.block_off[b + 1];
            const EvalItem first = args.items[i0];
            const bool far = first.nrows < 0;
            const int bs = lb & 1;
            // a paired follower (NB == 2) is the next sub-block of the same
            // node: its rows, norm block and weights follow the leader's
            const int pb = NB == 2 ? args.partner[b] : -1;
            const int nsb = pb >= 0 ? 2 : 1;
            const uint32_t idesc = block_idesc(b, i0);
            if (!mbar_wait(BAR_B_EMPTY, (lb & 1) ^ 1, abort_flag, args.status, args.spin)) goto mma_done;
            if (!mbar_wait(BAR_BLK_EMPTY(bs), ((lb >> 1) & 1) ^ 1, abort_flag, args.status, args.spin)) goto mma_done;
            b_issued = lb + 1;
            blk_last[bs] = lb;
            mbar_expect_tx(BAR_B_FULL, (uint32_t)(nsb * (2 * G_REGION + GX_REGION)));
            for (int h = 0; h < nsb; ++h) {
                tma_load_2d(sbase + S::B_HI + h * G_REGION, far ? &map_s_hi : &map_t_hi, 0, first.row0 + 128 * h,
                            BAR_B_FULL);
                tma_load_2d(sbase + S::B_LO + h * G_REGION, far ? &map_s_lo : &map_t_lo, 0, first.row0 + 128 * h,
                            BAR_B_FULL);
            }
            bulk_copy(sbase + S::B_X, args.bx + (int64_t)first.cidx * G_ROWS * GX_K, (uint32_t)(nsb * GX_REGION),
                      BAR_B_FULL);
            const uint32_t wbytes = S::WMMA ? (uint32_t)GW_BYTES : (uint32_t)(nsb * 128 * RC * 4);
            mbar_expect_tx(BAR_BLK_FULL(bs), wbytes);
            bulk_copy(sbase + S::BLK + bs * S::BLKSLOT,
                      reinterpret_cast<const uint8_t *>(args.colw) + (int64_t)first.cidx * S::BLKSLOT / NB, wbytes,
                      BAR_BLK_FULL(bs));
            // every block's tiles are waited for, items of this thread or not:
            // a parity wait may fall at most one phase behind the loads
            if (!mbar_wait(BAR_B_FULL, lb & 1, abort_flag, args.status, args.spin)) goto mma_done;
            for (int it = i0; it < i1; ++it, ++li) {
                if (SPLIT && (li & 1)) continue;            // the second issuer's item
                if (!issue_arg(li, idesc)) goto mma_done;
                li_done = li;
            }
            tc_commit(BAR_B_EMPTY);     // this thread's MMAs of the block have read the tiles
        }
    mma_done:
        // after an abort: the last sub-block's tiles and the latest weights of
        // each slot may still be landing, and MMAs may still be writing TMEM
        // -- wait for them before TMEM is freed and the CTA exits (no-ops on
        // the normal path)
        if (b_issued > 0) mbar_drain(BAR_B_FULL, (b_issued - 1) & 1);
        for (int k = 0; k < 2; ++k)
            if (blk_last[k] >= 0) mbar_drain(BAR_BLK_FULL(k), (blk_last[k] >> 1) & 1);
        if (li_done >= 0) mbar_drain(BAR_T_FULL(li_done % NACC), (li_done / NACC) & 1);
    } else if (SPLIT && warp == W_WI && lane == 0) {
        // ---------------------------------------- second argument-MMA issuer
        int li = 0, lb = 0, li_done = -1;
        for (int ci = c_begin; ci < c_end && !*abort_flag; ++ci, ++lb) {
            const int b = args.cta_blocks[ci];
            const int i0 = args.block_off[b], i1 = args.block_off[b + 1];
            const uint32_t idesc = block_idesc(b, i0);
            // this block's tiles have landed (waited for even without items
            // here, so that no later parity wait can pass on an old phase)
            if (!mbar_wait(BAR_B_FULL, lb & 1, abort_flag, args.status, args.spin)) goto mma2_done;
            for (int it = i0; it < i1; ++it, ++li) {
                if (!(li & 1)) continue;                   // the first issuer's item
                if (!issue_arg(li, idesc)) goto mma2_done;
                li_done = li;
            }
            tc_commit(BAR_B_EMPTY);
        }
    mma2_done:
        if (li_done >= 0) mbar_drain(BAR_T_FULL(li_done % NACC), (li_done / NACC) & 1);
    } else if (S::WMMA && warp == W_WI && lane == 0) {
        // ------------------------------------------ weight-MMA issuer (r > 4)
        // A thread of its own: each tcgen05.mma costs its issuing thread about
        // a hundred cycles, and an item's 16 small weight MMAs would otherwise
        // delay the next item's argument MMAs.  Item by item: once the
        // epilogue has stored the split exponentials (K_READY) and the item's
        // weight-sum accumulator is free, 16 source rows per step: k hi
        // against [w' hi | w' lo] (N = 32: the lo split's rows follow the hi
        // split's), then k lo against w' hi into the first 16 columns.
        constexpr uint32_t idesc32 = make_idesc(0u, G_ROWS, 32), idesc16 = make_idesc(0u, G_ROWS, 16);
        int li = 0, lb = 0, w_done = -1;
        for (int ci = c_begin; ci < c_end && !*abort_flag; ++ci, ++lb) {
            const int b = args.cta_blocks[ci];
            const int i0 = args.block_off[b], i1 = args.block_off[b + 1];
            const int bs = lb & 1;
            const int nk = 2 * (((args.items[i0].nrows & 0x7fffffff) + 31) >> 5);   // the chunks the epilogue split
            if (!mbar_wait(BAR_BLK_FULL(bs), (lb >> 1) & 1, abort_flag, args.status, args.spin)) goto wi_done;
            const uint32_t wh = sbase + S::BLK + bs * S::BLKSLOT;
            for (int it = i0; it < i1; ++it, ++li) {
                const int a = li % NACC, k = li % GW_NDW;
                if (!mbar_wait(BAR_K_READY(a), (li / NACC) & 1, abort_flag, args.status, args.spin)) goto wi_done;
                if (!mbar_wait(BAR_DW_EMPTY(k), ((li / GW_NDW) & 1) ^ 1, abort_flag, args.status, args.spin))
                    goto wi_done;
                tc_fence_after();
                const uint32_t dw = tmem + (uint32_t)(3 * 128 + k * 32), ak = tmem + (uint32_t)(a * 128);
                for (int ks = 0; ks < nk; ++ks) {
                    const uint32_t ch = (uint32_t)(32 * (ks >> 1) + 8 * (ks & 1));
                    tc_mma_ts(dw, ak + ch, gw_desc(wh + 256 * ks), idesc32, ks > 0);
                    tc_mma_ts(dw, ak + ch + 16, gw_desc(wh + 256 * ks), idesc16, 1);
                }
                tc_commit(BAR_DW_FULL(k));
                tc_commit(BAR_T_EMPTY(a));     // the argument's columns are free again
                w_done = li;
            }
        }
    wi_done:
        // weight MMAs in flight after an abort finish before TMEM is freed
        if (w_done >= 0) mbar_drain(BAR_DW_FULL(w_done % GW_NDW), (w_done / GW_NDW) & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == W_MMA) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G_TMEM_COLS) : "memory");
    }
}

// Weights of every sub-block for one Evaluate: thread t of block b takes
// source row t of sub-block b: colw [b, t, z] = w_z (zeros past the rows and
// past r).
template <int RC>
__global__ void g16_cols_kernel(const int64_t *sb_row0, const int32_t *sb_nr, int64_t n_leaf_sub, const float *Wt,
                                const float *Ws, int r, float *colw) {
    const int64_t b = blockIdx.x;
    const int t = threadIdx.x;
    const bool far = b >= n_leaf_sub;
    const int64_t row = sb_row0[b] + t;
    const bool valid = t < sb_nr[b];
    const float *w = (far ? Ws : Wt) + row * r;
#pragma unroll
    for (int z = 0; z < RC; ++z) colw[(b * 128 + t) * RC + z] = (valid && z < r) ? w[z] : 0.f;
}

// Split weights of every sub-block for the weight MMA (r > 4): thread t of
// block b takes source row t.  Per vector z the sub-block's largest |w| sets
// e_z with max |w| 2^-e_z in [2^13, 2^14); w' = w 2^-e_z (exact) is split into
// FP16 hi = rn(w') and lo = rn(w' - hi), and the factor 2^(e_z - 14) turns the
// MMA's sums of (k 2^14) w' back into sums of k w.  Rows past the sub-block
// and vectors past r are zero.
__global__ void g16_wcols_kernel(const int64_t *sb_row0, const int32_t *sb_nr, int64_t n_leaf_sub, const float *Wt,
                                 const float *Ws, int r, uint8_t *colw) {
    __shared__ float wmax[4][16];
    const int64_t b = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const bool valid = t < sb_nr[b];
    const float *w = (b >= n_leaf_sub ? Ws : Wt) + (sb_row0[b] + t) * r;
    float v[16];
#pragma unroll
    for (int z = 0; z < 16; ++z) {
        v[z] = (valid && z < r) ? w[z] : 0.f;
        float m = fabsf(v[z]);
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) wmax[warp][z] = m;
    }
    __syncthreads();
    uint8_t *out = colw + b * GW_BYTES;
#pragma unroll
    for (int z = 0; z < 16; ++z) {
        const float m = fmaxf(fmaxf(wmax[0][z], wmax[1][z]), fmaxf(wmax[2][z], wmax[3][z]));
        int e = 0;
        if (m > 0.f) {
            int ex;
            frexpf(m, &ex);              // m = f 2^ex, f in [1/2, 1)
            e = ex - G_KSHIFT;
        }
        const float wp = ldexpf(v[z], -e);
        const __half hi = __float2half_rn(wp);
        const __half lo = __float2half_rn(wp - __half2float(hi));
        *reinterpret_cast<__half *>(out + gw_off(z, t)) = hi;
        *reinterpret_cast<__half *>(out + GW_SPLIT + gw_off(z, t)) = lo;
        if (t == 0) reinterpret_cast<float *>(out + 2 * GW_SPLIT)[z] = ldexpf(1.f, e - G_KSHIFT);
    }
}

// Tensor maps over the tree's split source rows (64 x 128 boxes, 128-byte
// swizzle): [leaf rows hi, lo, skeleton rows hi, lo].
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
        const void *arr[4] = {t->Xb_hi, t->Xb_lo, t->Sb_hi, t->Sb_lo};
        for (int i = 0; i < 4; ++i)
            ASK_TRY(encode_2d(st->encode, &st->map[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, arr[i],
                              i < 2 ? t->N_pad : t->srows, TC_K, 64, G_ROWS, CU_TENSOR_MAP_SWIZZLE_128B));
        st->ready = true;
    }
    *out = st;
    return ASKIT_OK;
}

template <int RC, int NA, int NB>
askit_status launch_g16(G16State *st, const G16Args &a, int grid, cudaStream_t s) {
    using S = SG<RC, NA, NB>;
    constexpr size_t smem = S::BYTES + 1024;
    static_assert(smem <= 232448, "shared-memory plan exceeds 227 KB");
    static const cudaError_t attr = cudaFuncSetAttribute(eval_g16_kernel<RC, NA, NB>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ASK_CUDA(attr);
    eval_g16_kernel<RC, NA, NB><<<(unsigned)grid, S::THREADS, smem, s>>>(st->map[0], st->map[1], st->map[2],
                                                                         st->map[3], a);
    ASK_LAUNCH();
    return ASKIT_OK;
}

template <int RC>
askit_status run_g16(askit_tree t, const WeightCtx &c, G16State *st, G16Args a, const WorkLists &w,
                     cudaStream_t s) {
    // weights in the sub-blocks' row order: r = 1 in the first 128 floats of
    // each sub-block's column-data slot, 1 < r <= 4 in the per-sub-block
    // weights, r > 4 split for the weight MMA
    float *colw = RC == 1 ? reinterpret_cast<float *>(c.colv) : c.colw;
    if constexpr (SG<RC, 3, 1>::WMMA)
        g16_wcols_kernel<<<(unsigned)t->n_sub, 128, 0, s>>>(t->sb_row0, t->sb_nr, t->n_leaf_sub, c.Wt, c.Ws, c.r,
                                                            reinterpret_cast<uint8_t *>(colw));
    else
        g16_cols_kernel<RC><<<(unsigned)t->n_sub, 128, 0, s>>>(t->sb_row0, t->sb_nr, t->n_leaf_sub, c.Wt, c.Ws, c.r,
                                                               colw);
    ASK_LAUNCH();
    a.colw = colw;
    ASK_TRY(ktimer_mark(t, s, false));
    // three or four target-row stages (one or two items' copies in flight);
    // paired 256-column items up to r = 4
    bool done = false;
    if constexpr (RC <= 4) {
        if (t->tune_pairs && w.sched_off[2]) {
            a.cta_off = w.sched_off[2];
            a.cta_blocks = w.sched_blocks[2];
            a.partner = w.partner;
            if (t->tune_stages <= 3) ASK_TRY((launch_g16<RC, 3, 2>(st, a, w.n_ctas, s)));
            else ASK_TRY((launch_g16<RC, 4, 2>(st, a, w.n_ctas, s)));
            done = true;
        }
    }
    if (!done) {
        if (t->tune_stages <= 3) ASK_TRY((launch_g16<RC, 3, 1>(st, a, w.n_ctas, s)));
        else ASK_TRY((launch_g16<RC, 4, 1>(st, a, w.n_ctas, s)));
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
    if (!t->Xb_hi || !t->g_bx || !q.hi || !q.lo || !q.x || !c.colv || (c.r > 1 && !c.colw)) {
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
    a.q_x = q.x;
    a.bx = t->g_bx;
    a.colw = nullptr;
    a.partner = nullptr;
    a.r = c.r;
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
// Operands.  FP16 split of v: hi = fp16(v), lo = fp16(v - hi).
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ void split16(float v, uint16_t &h, uint16_t &l) {
    const __half vh = __float2half_rn(v);
    const __half vl = __float2half_rn(v - __half2float(vh));
    h = __half_as_ushort(vh);
    l = __half_as_ushort(vl);
}

// Target rows: a = (x - xbar) sigma split, and the norm block [h(n tau),
// h(n tau), l(n tau), kappa, kappa, 0 ...] with n = |x - xbar|^2 (FP64 sum
// over a fixed butterfly, rounded).  One warp per row.  A value outside the
// FP16-safe range raises *overflow.
__global__ void gsplit_targets_kernel(const float *X, int64_t ldx, int d, int64_t rows, const float *xbar, float sigma,
                                      float tau, float kappa, uint16_t *hi, uint16_t *lo, uint16_t *nx,
                                      int *overflow) {
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
        const float v = x * sigma;
        bad |= !(fabsf(v) <= 30000.f);
        split16(v, hi[row * TC_K + k], lo[row * TC_K + k]);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const float nt = (float)acc * tau;
    bad |= !(nt <= 30000.f);
    if (lane < GX_K) {
        uint16_t h = 0, l = 0;
        split16(nt, h, l);
        const uint16_t kk = __half_as_ushort(__float2half_rn(kappa));
        const uint16_t v = lane <= 1 ? h : lane == 2 ? l : lane <= 4 ? kk : (uint16_t)0;
        nx[row * GX_K + lane] = v;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0 && overflow) atomicExch(overflow, 1);
}

// Source rows: b = (y - xbar) 2 sc_j / sigma split (sc_j the row's exponent
// scale; padding rows carry sc = 0) and n_j.  One warp per row.
__global__ void gsplit_sources_kernel(const float *X, int64_t ldx, int d, int64_t rows, const float *xbar,
                                      const float *sc, float inv_sigma, uint16_t *hi, uint16_t *lo, float *nrm) {
    const int lane = threadIdx.x & 31;
    const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows) return;
    const float f = 2.f * sc[row] * inv_sigma;
    double acc = 0.0;
#pragma unroll
    for (int h = 0; h < TC_K / 32; ++h) {
        const int k = lane + 32 * h;
        const float x = k < d ? X[row * ldx + k] - xbar[k] : 0.f;
        acc += (double)x * (double)x;
        split16(x * f, hi[row * TC_K + k], lo[row * TC_K + k]);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) nrm[row] = (float)acc;
}

// Source norm blocks, one 128-row block per sub-block in the core-matrix
// layout: row t = [h(m), l(m), h(m), h(v), l(v), 0 ...], m = -sc / tau,
// v = -sc n / kappa.
__global__ void gsplit_bx_kernel(const int64_t *sb_row0, const int32_t *sb_nr, int64_t n_leaf_sub, const float *sc_t,
                                 const float *sc_s, const float *n_t, const float *n_s, float inv_tau, float inv_kappa,
                                 uint16_t *bx) {
    const int64_t b = blockIdx.x;
    const int t = threadIdx.x;
    const bool far = b >= n_leaf_sub;
    const int64_t row = sb_row0[b] + t;
    const bool valid = t < sb_nr[b];
    uint16_t e[GX_K];
#pragma unroll
    for (int k = 0; k < GX_K; ++k) e[k] = 0;
    // a row past the sub-block (the tile's next rows hold other points, whose
    // main products may be large and positive) gets kappa v = -60000 kappa:
    // its argument stays far below zero, so ex2 is finite (0) and the zero
    // weight leaves no trace
    e[3] = __half_as_ushort(__float2half_rn(-60000.f));
    if (valid) {
        const float sc = (far ? sc_s : sc_t)[row], n = (far ? n_s : n_t)[row];
        uint16_t mh, ml, vh, vl;
        split16(-sc * inv_tau, mh, ml);
        split16(-sc * n * inv_kappa, vh, vl);
        e[0] = mh;
        e[1] = ml;
        e[2] = mh;
        e[3] = vh;
        e[4] = vl;
    }
    uint8_t *blk = reinterpret_cast<uint8_t *>(bx + b * G_ROWS * GX_K);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        uint4 v;
        v.x = (uint32_t)e[8 * c] | ((uint32_t)e[8 * c + 1] << 16);
        v.y = (uint32_t)e[8 * c + 2] | ((uint32_t)e[8 * c + 3] << 16);
        v.z = (uint32_t)e[8 * c + 4] | ((uint32_t)e[8 * c + 5] << 16);
        v.w = (uint32_t)e[8 * c + 6] | ((uint32_t)e[8 * c + 7] << 16);
        *reinterpret_cast<uint4 *>(blk + nx_off(t, c)) = v;
    }
}

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

// The power of 2 nearest to v (in the exponent).
float pow2_near(double v) {
    if (!(v > 0.0)) return 1.f;
    return ldexpf(1.f, (int)lround(log2(v)));
}

}  // namespace

askit_status g16_split_rows(const float *X, int64_t ldx, int d, int64_t rows, const askit_tree_s *t, uint16_t *hi,
                            uint16_t *lo, uint16_t *nx, int *overflow, cudaStream_t s) {
    if (rows <= 0) return ASKIT_OK;
    gsplit_targets_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(X, ldx, d, rows, t->g_xbar, t->g_sigma, t->g_tau,
                                                                    t->g_kappa, hi, lo, nx, overflow);
    ASK_LAUNCH();
    return ASKIT_OK;
}

// The global-centered FP16x3 operands of a narrow tree (d <= TC_K): xbar (the
// FP64 mean of the points), the scales sigma (a power of 2 near sqrt(2 sc_max),
// kept so that every |x_k - xbar_k| sigma <= 2^12: targets up to about 7 times
// farther out still fit FP16), tau near sqrt(sc_max / R^2_max) and kappa near
// sqrt(sc_max R^2_max), the split target rows of the tree points, the split
// source rows of the points and of the skeleton pool, the source norm blocks
// of every sub-block, and the accuracy figure rho = sc_max R^2_max: the
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
    max_kernel<<<(unsigned)((t->N + 255) / 256), 256, 0, s>>>(t->sc_t, t->N, red + 2);
    ASK_LAUNCH();
    float hred[3] = {0.f, 0.f, 0.f};
    ASK_CUDA(cudaMemcpyAsync(hred, red, 3 * sizeof(float), cudaMemcpyDeviceToHost, s));
    ASK_CUDA(cudaStreamSynchronize(s));
    const double ext = hred[0], sc_max = hred[2];
    float sigma = pow2_near(sqrt(2.0 * sc_max));
    while (ext * sigma > 4096.0) sigma *= 0.5f;
    t->g_sigma = sigma;
    // the sources' split rows and every row's n; every row, padding
    // included, holds finite values (a 128-row tile read past a short
    // sub-block multiplies them by zero weights)
    const size_t et = (size_t)t->N_pad * TC_K, es = (size_t)t->srows * TC_K;
    ASK_TRY(t->arena.alloc(&t->ng_t, t->N_pad));
    ASK_TRY(t->arena.alloc(&t->ng_s, t->srows));
    ASK_TRY(t->arena.alloc(&t->Xb_hi, et));
    ASK_TRY(t->arena.alloc(&t->Xb_lo, et));
    ASK_TRY(t->arena.alloc(&t->Sb_hi, es));
    ASK_TRY(t->arena.alloc(&t->Sb_lo, es));
    gsplit_sources_kernel<<<(unsigned)((t->N_pad + 7) / 8), 256, 0, s>>>(t->Xt, t->d_pad, d, t->N_pad, t->g_xbar,
                                                                        t->sc_t, 1.f / sigma, t->Xb_hi, t->Xb_lo,
                                                                        t->ng_t);
    gsplit_sources_kernel<<<(unsigned)((t->srows + 7) / 8), 256, 0, s>>>(t->Xs, t->d_pad, d, t->srows, t->g_xbar,
                                                                        t->sc_s, 1.f / sigma, t->Sb_hi, t->Sb_lo,
                                                                        t->ng_s);
    max_kernel<<<(unsigned)((t->N + 255) / 256), 256, 0, s>>>(t->ng_t, t->N, red + 1);
    ASK_LAUNCH();
    ASK_CUDA(cudaMemcpyAsync(hred, red, 3 * sizeof(float), cudaMemcpyDeviceToHost, s));
    ASK_CUDA(cudaStreamSynchronize(s));
    cudaFreeAsync(red, s);
    const double r2max = hred[1];
    t->g_tau = pow2_near(r2max > 0.0 ? sqrt(sc_max / r2max) : 1.0);
    t->g_kappa = pow2_near(sqrt(sc_max * r2max));
    t->g_rho = sc_max * r2max;
    t->g_ok = t->g_rho <= RHO_MAX;
    // the tree points as targets, and the sources' norm blocks
    ASK_TRY(t->arena.alloc(&t->Xg_hi, et));
    ASK_TRY(t->arena.alloc(&t->Xg_lo, et));
    ASK_TRY(t->arena.alloc(&t->Xg_x, (size_t)t->N_pad * GX_K));
    ASK_TRY(t->arena.alloc(&t->g_bx, (size_t)std::max<int64_t>(1, t->n_sub) * G_ROWS * GX_K));
    ASK_TRY(g16_split_rows(t->Xt, t->d_pad, d, t->N_pad, t, t->Xg_hi, t->Xg_lo, t->Xg_x, nullptr, s));
    if (t->n_sub > 0)
        gsplit_bx_kernel<<<(unsigned)t->n_sub, 128, 0, s>>>(t->sb_row0, t->sb_nr, t->n_leaf_sub, t->sc_t, t->sc_s,
                                                            t->ng_t, t->ng_s, 1.f / t->g_tau, 1.f / t->g_kappa,
                                                            t->g_bx);
    ASK_LAUNCH();
    ASK_CUDA(cudaStreamSynchronize(s));
    return ASKIT_OK;
}
