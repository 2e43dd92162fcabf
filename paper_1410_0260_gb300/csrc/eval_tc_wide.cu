// Evaluate (Algorithm 4) on the tcgen05 tensor cores for wide points
// (64 < d): the distance contraction runs over K = d in chunks of 32.
//
// Work items are the same as for the narrow kernels (one source sub-block of
// <= 128 rows against <= 128 targets that need it), optionally paired: the
// two sub-blocks of one node need the same targets and share the node's
// center c_B, so one 256-column item serves both with a single copy and split
// of its target rows.  Both sides are centered on c_B:
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
// Operands in shared memory use the tensor core's layout without swizzle:
// 8-row x 16-byte core matrices, a chunk's four K groups of 8 elements one
// after another ([K group][rows][16 B]).  The pre-split sub-block rows are
// stored in HBM as planes of K groups, so each split's chunk arrives in that
// layout from one 3-D TMA box ({8 rows x 8 elements, rows / 8, 4 K
// groups}); the
// loaders write the split target rows the same way (16 bytes a row, no bank
// conflicts).
//
// One CTA per SM, 448 threads:
//   warps 0-7  loaders.  Copy: warp w brings half w >> 2 of rows
//              32 (w & 3) .. + 31 of a chunk's FP32 target rows into a raw
//              buffer (4 lanes along a half row, 8 rows an instruction), three
//              (r > 4: one) chunks ahead of the split;
//              split: thread t takes half (t >> 7) of row t & 127 of the
//              chunk, subtracts c_B (from the warp's copy of its half of c_B
//              in shared memory; from global memory past kw = 1024 or r = 4),
//              accumulates |a|^2, splits into FP16/BF16 hi + lo; they also
//              write the item's column data (c log2(e) / h^2, |b|^2, w) for
//              the epilogue, double-buffered so that they run on into the
//              next item while the epilogue drains the last;
//   warps 8-11 epilogue (TMEM lane quadrant = warp & 3);
//   warp 12    TMEM allocation; lane 0 issues the tcgen05.mma instructions;
//   warp 13    producer: TMA of the sub-block's hi and lo chunk.
// Chunk stages in two rings, released separately by the MMAs' commits: three
// of the split targets and three of the sub-block's chunk, requested two
// chunks' MMAs before it is needed.  Single sub-blocks: two items' accumulators (main +
// cross) fill TMEM's 512 columns, so the MMAs of item i+1 overlap the
// epilogue of item i; paired items: one item's 256-column accumulators fill
// it.  Every mbarrier wait is bounded: on timeout the kernel records
// ASK_DEV_TIMEOUT, every role leaves its loop, copies in flight are waited
// for, and TMEM is freed.
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
constexpr int W_KC = 32;                        // K elements per chunk
constexpr int W_KG = 4;                         // K groups of 8 elements per chunk
constexpr int W_REGION = W_ROWS * W_KC * 2;     // one 16-bit split of 128 rows (8 KB)
constexpr uint32_t W_TMEM_COLS = 512;           // main accumulators, then cross accumulators

// Shared-memory descriptor of a K-major operand without swizzle: the next
// core matrix along K `lbo` bytes on, along M/N 128 bytes on (8 rows of 16
// bytes); version bit 46, layout type 0.
__device__ __forceinline__ uint64_t nsw_desc(uint32_t saddr, uint32_t lbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(128 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

template <int RC, int NB>
struct WSmem {
    static constexpr int NSLOT = NB == 1 ? 2 : 1;   // items in flight in TMEM
    static constexpr int NCOL = NB * W_ROWS;        // columns of an item
    // Two rings of chunk stages, released separately by the MMAs' commits:
    // NSA stages of the split targets (A hi, A lo: [4][128][16 B] each),
    // NSB of the sub-block's (B hi, B lo: [4][NCOL][16 B] each).
    static constexpr int NSA = 3;
    static constexpr int NSB = 3;
    static constexpr int NRAW = RC <= 4 ? 3 : 2;    // raw target-row buffers: NRAW - 1 chunks read ahead
    // each loader warp's copy of its half of c_B (kw / 2 floats) while kw <=
    // CEN_KW; else c_B is read from global memory
    static constexpr int CEN_KW = RC <= 4 ? 1024 : 0;
    static constexpr int A_STAGE = 2 * W_REGION, B_STAGE = 2 * NB * W_REGION;
    static constexpr int A_LO = W_REGION, B_LO = NB * W_REGION;   // within a stage
    static constexpr int B0 = NSA * A_STAGE;
    // NRAW buffers of a chunk's raw FP32 target rows [128 rows][32], a
    // row's 16-byte pieces XOR-permuted by (row & 7) for conflict-free reads
    static constexpr int RAW0 = B0 + NSB * B_STAGE;
    static constexpr int RAW_BYTES = W_ROWS * W_KC * 4;
    // the column data and |a|^2 of two items (item li in buffer li & 1), so
    // that the loaders move on to the next item while the epilogue runs
    static constexpr int CENW = RAW0 + NRAW * RAW_BYTES;       // float [8 warps][CEN_KW / 2]
    static constexpr int ANORM = CENW + 8 * CEN_KW * 2;        // float [2][2 halves][128]
    static constexpr int COLV = ANORM + 2 * 2 * 128 * 4;       // float4 [2][NCOL]
    static constexpr int COLW = COLV + 2 * NCOL * 16;          // float [2][NCOL][RC]
    static constexpr int BAR = COLW + 2 * NCOL * RC * 4;       // 32 mbarriers
    static constexpr int MISC = BAR + 32 * 8;                  // tmem address, abort flag
    static constexpr int BYTES = MISC + 16;
    static constexpr uint32_t TX = 2 * NB * W_REGION;   // bytes landing per chunk
};

struct TcwArgs {
    const EvalItem *items;
    const int32_t *block_off;
    const int32_t *cta_off, *cta_blocks;
    const int32_t *partner;   // [n_blocks] paired follower block, or -1 (NB == 2)
    const int32_t *tgt;       // entry -> target slot
    int nkc;                  // K chunks (kw / 32)
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

template <int P, int RC, int NB>
__global__ void __launch_bounds__(W_THREADS, 1)
eval_tcw_kernel(const __grid_constant__ CUtensorMap map_t_hi, const __grid_constant__ CUtensorMap map_t_lo,
                const __grid_constant__ CUtensorMap map_s_hi, const __grid_constant__ CUtensorMap map_s_lo,
                const __grid_constant__ CUtensorMap map_t_hi1, const __grid_constant__ CUtensorMap map_t_lo1,
                const TcwArgs args) {
    using S = WSmem<RC, NB>;
    constexpr int NSLOT = S::NSLOT, NCOL = S::NCOL, NSA = S::NSA, NSB = S::NSB, NRAW = S::NRAW;
    constexpr uint32_t FMT = P == ASKIT_PREC_BF16X3 ? 1u : 0u;
    constexpr uint32_t IDESC = make_idesc(FMT, W_ROWS, NCOL);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    const uint32_t sbase = smem_u32(sm);
    float *a_norm = reinterpret_cast<float *>(sm + S::ANORM);
    float4 *colv = reinterpret_cast<float4 *>(sm + S::COLV);
    float *colw = reinterpret_cast<float *>(sm + S::COLW);
    const uint32_t bar0 = sbase + S::BAR;
    auto BAR_A_FULL = [&](int s) { return bar0 + 8 * s; };          // loaders stored A stage s (256)
    auto BAR_A_FREE = [&](int s) { return bar0 + 8 * (4 + s); };    // MMAs reading A stage s finished (commit)
    auto BAR_L_FULL = [&](int s) { return bar0 + 8 * (8 + s); };    // B stage s landed
    auto BAR_B_FREE = [&](int s) { return bar0 + 8 * (12 + s); };   // MMAs reading B stage s finished (commit)
    auto BAR_COL_EMPTY = [&](int c) { return bar0 + 8 * (16 + c); };// epilogue done with column buffer c (128)
    auto BAR_T_FULL = [&](int a) { return bar0 + 8 * (18 + a); };   // accumulators of item slot a complete
    auto BAR_T_EMPTY = [&](int a) { return bar0 + 8 * (20 + a); };  // epilogue drained slot a (128)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + S::MISC);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + S::MISC + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < NSA; ++s) {
            mbar_init(BAR_A_FULL(s), 256);
            mbar_init(BAR_A_FREE(s), 1);
        }
        for (int s = 0; s < NSB; ++s) {
            mbar_init(BAR_L_FULL(s), 1);
            mbar_init(BAR_B_FREE(s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(BAR_T_FULL(a), 1);
            mbar_init(BAR_T_EMPTY(a), 128);
            mbar_init(BAR_COL_EMPTY(a), 128);
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
    // rows of the follower of block b's pair (0: none)
    auto follower_rows = [&](int b, int &f0) -> int {
        const int pb = NB == 2 ? args.partner[b] : -1;
        f0 = pb >= 0 ? args.block_off[pb] : 0;
        return pb >= 0 ? (args.items[f0].nrows & 0x7fffffff) : 0;
    };

    if (warp < 8) {
        // ------------------------------------------------------------ loaders
        // Thread t splits half h = t >> 7 of row t & 127 of every chunk, so
        // warp w splits half w >> 2 of rows 32 (w & 3) .. + 31; it also copies
        // exactly those bytes (lanes: 4 pieces of 16 B along a half row x 8
        // rows an instruction), so a raw buffer is private to the warp and
        // its copies need no block-wide barrier: cp.async groups and
        // __syncwarp.  Copies run NRAW - 1 chunks ahead of the split on a fill
        // cursor of their own (item and chunk in this CTA's order); the copy
        // slots of the item after the fill cursor's are read one item ahead,
        // and the header of the item after that one item before them.
        const int row = tid & 127, h = tid >> 7;
        const int cpiece = 4 * h + (lane & 3);            // 16-byte piece of a row's 128-byte chunk
        const int crow0 = 32 * (warp & 3) + (lane >> 2);  // copy rows crow0 + 8 i
        struct Cur { int ci, it, i1; };    // cta_blocks index, item, end of its block
        auto advance = [&](Cur &c) {
            if (++c.it < c.i1) return;
            while (++c.ci < c_end) {
                const int b = args.cta_blocks[c.ci];
                c.it = args.block_off[b];
                c.i1 = args.block_off[b + 1];
                if (c.it < c.i1) return;
            }
        };
        auto copy_slots = [&](const Cur &c, int (&sl)[4], uint32_t &mask) {
            mask = 0;
            if (c.ci >= c_end) return;
            const EvalItem nx = args.items[c.it];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = crow0 + 8 * i;
                sl[i] = r < nx.cnt ? args.tgt[nx.e0 + r] : 0;
                if (r < nx.cnt) mask |= 1u << i;
            }
        };
        Cur fc{c_begin - 1, 0, 0};
        advance(fc);               // the CTA's first item
        Cur nc = fc;
        advance(nc);
        int fs[4], ns[4];
        uint32_t fmask = 0, nmask = 0;
        copy_slots(fc, fs, fmask);
        copy_slots(nc, ns, nmask);
        // the header (first entry, count) of the item after nc, read one item
        // before its slots, so that no slot load waits on it
        Cur hc = nc;
        advance(hc);
        int2 nh = make_int2(0, 0);
        if (hc.ci < c_end) nh = make_int2(args.items[hc.it].e0, args.items[hc.it].cnt);
        int fkc = 0, gf = 0;       // fill cursor's chunk; chunks filled so far
        // the fill cursor's chunk into raw buffer gf % NRAW (its last chunk,
        // gf - NRAW, split by this warp); one cp.async group per call, empty
        // past the CTA's last item
        auto fill_one = [&]() {
            if (fc.ci < c_end) {
                const uint32_t dst0 = sbase + S::RAW0 + (gf % NRAW) * S::RAW_BYTES;
                const int64_t col = (int64_t)fkc * W_KC + 4 * cpiece;
                const bool in_row = col < args.ldq;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = crow0 + 8 * i;
                    const bool ok = in_row && ((fmask >> i) & 1u);
                    const float *src = ok ? args.q + (int64_t)fs[i] * args.ldq + col : args.q;
                    cp_async16_zfill(dst0 + (uint32_t)(r * W_KC * 4 + ((cpiece ^ (r & 7)) << 4)), src, ok ? 16u : 0u);
                }
                ++gf;
                if (++fkc == nkc) {
                    fkc = 0;
                    fc = nc;
#pragma unroll
                    for (int i = 0; i < 4; ++i) fs[i] = ns[i];
                    fmask = nmask;
                    nc = hc;
                    nmask = 0;
                    if (nc.ci < c_end) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int r = crow0 + 8 * i;
                            ns[i] = r < nh.y ? args.tgt[nh.x + r] : 0;
                            if (r < nh.y) nmask |= 1u << i;
                        }
                    }
                    advance(hc);
                    if (hc.ci < c_end) nh = make_int2(args.items[hc.it].e0, args.items[hc.it].cnt);
                }
            }
            cp_async_commit();
        };
        int g = 0, li = 0;
        for (int k = 0; k < NRAW - 1; ++k) fill_one();
        const float2 neg1 = make_float2(-1.f, -1.f);
        const float2 sc2 = make_float2(args.f16_scale, args.f16_scale);
        // every exit below is taken by the whole warp (warp-wide votes), so
        // that no __syncwarp waits for a lane that has left
        for (int ci = c_begin; ci < c_end && !__shfl_sync(0xffffffffu, *abort_flag, 0); ++ci) {
            const int b = args.cta_blocks[ci];
            const int i0 = args.block_off[b], i1 = args.block_off[b + 1];
            const EvalItem first = args.items[i0];
            const bool far = first.nrows < 0;
            int f0 = 0;
            const int nrows_f = follower_rows(b, f0);
            // the source column this thread describes: single sub-blocks,
            // column `row` (half 0 only); pairs, column 128 h + row
            const int col = NB == 2 ? 128 * h + row : row;
            const bool writes_col = NB == 2 || h == 0;
            const int nrows_c = (NB == 2 && h == 1) ? nrows_f : (first.nrows & 0x7fffffff);
            const bool has_src = row < nrows_c;
            const int64_t srow = (int64_t)first.row0 + (NB == 2 ? 128 * h : 0) + row;
            const float sc = has_src ? __ldg((far ? args.sc_s : args.sc_t) + srow) : 0.f;
            const float qn = has_src ? __ldg((far ? args.nrm_s : args.nrm_t) + srow) : 0.f;
            const float *wrow = (far ? args.Ws : args.Wt) + srow * args.r;
            // c_B: this thread's 16 elements of chunk kc at cen[8 kc .. 8 kc + 3]
            // (global memory; the same 64 bytes for a warp), or at
            // cenw[4 kc .. 4 kc + 3] in the warp's copy
            const float4 *cen = reinterpret_cast<const float4 *>(args.cent + (int64_t)first.cidx * args.kw) + 4 * h;
            float4 *cenw = reinterpret_cast<float4 *>(sm + S::CENW) + warp * (S::CEN_KW / 8);
            const bool cen_sm = args.kw <= S::CEN_KW;
            if (cen_sm) {
                __syncwarp();                   // no lane still reads the last segment's copy
                for (int q = lane; q < 4 * nkc; q += 32) cenw[q] = __ldg(cen + 8 * (q >> 2) + (q & 3));
                __syncwarp();
            }
            for (int it = i0; it < i1; ++it, ++li) {
                const int cbuf = li & 1;
                const int cnt = args.items[it].cnt;
                const bool has_tgt = row < cnt;
                if (!__all_sync(0xffffffffu, mbar_wait(BAR_COL_EMPTY(cbuf), ((li >> 1) & 1) ^ 1, abort_flag, args.status)))
                    goto loader_done;
                // column data of source column `col` for this item's buffer:
                // arg = g A + (C p + B) = -sc (p + q - 2 g / scale^2)
                if (writes_col) {
                    float *cp = reinterpret_cast<float *>(colv + cbuf * NCOL + 2 * (col >> 1));
                    const int o = col & 1;
                    cp[0 + o] = 2.f * args.g_unscale * sc;
                    cp[2 + o] = -sc * qn;
                    cp[4 + o] = -sc;
                    cp[6 + o] = has_src ? __ldg(wrow) : 0.f;
                    if (RC > 1) {
#pragma unroll
                        for (int z = 0; z < RC; ++z)
                            colw[(cbuf * NCOL + col) * RC + z] = (has_src && z < args.r) ? __ldg(wrow + z) : 0.f;
                    }
                }
                float2 nn2 = make_float2(0.f, 0.f);
                for (int kc = 0; kc < nkc; ++kc, ++g) {
                    const int s = g % NSA;
                    const uint32_t par = (g / NSA) & 1;
                    __syncwarp();                       // every lane done with chunk g - 1's buffer
                    fill_one();                         // chunk g + NRAW - 1
                    cp_async_wait<NRAW - 1>();          // this thread's copies of chunk g landed
                    if (!__all_sync(0xffffffffu, mbar_wait(BAR_A_FREE(s), par ^ 1, abort_flag, args.status)))
                        goto loader_done;
                    __syncwarp();                       // ... and every lane's
                    uint8_t *st = sm + s * S::A_STAGE;
                    const uint8_t *raw = sm + S::RAW0 + (g % NRAW) * S::RAW_BYTES + row * W_KC * 4;
#pragma unroll
                    for (int kg2 = 0; kg2 < 2; ++kg2) {
                        // K group kg = 2 h + kg2: elements 8 kg .. 8 kg + 7 of the chunk,
                        // raw pieces 2 kg and 2 kg + 1 (stored at piece ^ (row & 7))
                        const int kg = 2 * h + kg2;
                        const float4 xl = *reinterpret_cast<const float4 *>(raw + (((2 * kg) ^ (row & 7)) << 4));
                        const float4 xh = *reinterpret_cast<const float4 *>(raw + (((2 * kg + 1) ^ (row & 7)) << 4));
                        float4 ml, mh;
                        if (cen_sm) {
                            ml = cenw[4 * kc + 2 * kg2];
                            mh = cenw[4 * kc + 2 * kg2 + 1];
                        } else {
                            ml = __ldg(cen + 8 * kc + 2 * kg2);
                            mh = __ldg(cen + 8 * kc + 2 * kg2 + 1);
                        }
                        // a = x - c_B, two elements an instruction
                        float2 v[4] = {__ffma2_rn(make_float2(ml.x, ml.y), neg1, make_float2(xl.x, xl.y)),
                                       __ffma2_rn(make_float2(ml.z, ml.w), neg1, make_float2(xl.z, xl.w)),
                                       __ffma2_rn(make_float2(mh.x, mh.y), neg1, make_float2(xh.x, xh.y)),
                                       __ffma2_rn(make_float2(mh.z, mh.w), neg1, make_float2(xh.z, xh.w))};
                        if (!has_tgt) {
#pragma unroll
                            for (int e = 0; e < 4; ++e) v[e] = make_float2(0.f, 0.f);
                        }
                        uint32_t hv[4], lv[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            nn2 = __ffma2_rn(v[e], v[e], nn2);
                            if constexpr (P == ASKIT_PREC_FP16X3) {
                                const float2 vs = __fmul2_rn(v[e], sc2);
                                const __half2 hh = __floats2half2_rn(vs.x, vs.y);
                                const float2 r2 = __ffma2_rn(__half22float2(hh), neg1, vs);
                                const __half2 ll = __floats2half2_rn(r2.x, r2.y);
                                hv[e] = *reinterpret_cast<const uint32_t *>(&hh);
                                lv[e] = *reinterpret_cast<const uint32_t *>(&ll);
                            } else {
                                const __nv_bfloat162 hh = __floats2bfloat162_rn(v[e].x, v[e].y);
                                const float2 r2 = __ffma2_rn(__bfloat1622float2(hh), neg1, v[e]);
                                const __nv_bfloat162 ll = __floats2bfloat162_rn(r2.x, r2.y);
                                hv[e] = *reinterpret_cast<const uint32_t *>(&hh);
                                lv[e] = *reinterpret_cast<const uint32_t *>(&ll);
                            }
                        }
                        // core-matrix layout: K group kg, row `row`, 16 bytes
                        const int off = kg * (W_ROWS * 16) + row * 16;
                        *reinterpret_cast<uint4 *>(st + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                        *reinterpret_cast<uint4 *>(st + S::A_LO + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
                    }
                    if (kc == nkc - 1) a_norm[(cbuf * 2 + h) * 128 + row] = nn2.x + nn2.y;
                    // generic-proxy stores -> visible to the tensor core's async proxy
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_arrive(BAR_A_FULL(s));
                }
            }
        }
    loader_done:
        // no copy may land in shared memory after the CTA exits (also after
        // an abort)
        cp_async_wait<0>();
    } else if (warp < 12) {
        // ----------------------------------------------------------- epilogue
        // Row `row` of every item; columns 0-127 belong to the item's
        // sub-block (the leader of a pair), 128-255 to the pair's follower,
        // each summed into its own entry's partial.
        const int row = tid - 256;
        const int q = warp & 3;
        int li = 0;
        for (int ci = c_begin; ci < c_end && !*abort_flag; ++ci) {
            const int b = args.cta_blocks[ci];
            const int i0 = args.block_off[b], i1 = args.block_off[b + 1];
            int f0 = 0;
            const int nrows_f = follower_rows(b, f0);
            for (int it = i0; it < i1; ++it, ++li) {
                const int a = li % NSLOT, cbuf = li & 1;
                const EvalItem item = args.items[it];
                const int nrows = item.nrows & 0x7fffffff;
                if (!mbar_wait(BAR_T_FULL(a), (li / NSLOT) & 1, abort_flag, args.status)) goto epi_done;
                tc_fence_after();
                float acc[NB][RC];
#pragma unroll
                for (int hb = 0; hb < NB; ++hb)
#pragma unroll
                    for (int z = 0; z < RC; ++z) acc[hb][z] = 0.f;
                if (q * 32 < item.cnt) {
                    const float pt = a_norm[(cbuf * 2) * 128 + row] + a_norm[(cbuf * 2 + 1) * 128 + row];
                    const float2 pt2 = make_float2(pt, pt);
                    const float4 *cv4 = colv + cbuf * NCOL;
                    const float *cwp = colw + cbuf * NCOL * RC;
                    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
                    if constexpr (RC == 1) {
                        // 16-column steps; the next step's TMEM loads (main in
                        // r[0..15], cross in r[16..31]) are in flight while this
                        // step's columns are summed
#pragma unroll
                        for (int hb = 0; hb < NB; ++hb) {
                            const int nst = ((hb == 0 ? nrows : nrows_f) + 15) >> 4;
                            float2 acc2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                            uint32_t ra[32], rb[32];
                            auto issue = [&](int c, uint32_t (&r)[32]) {
                                const uint32_t col = (uint32_t)(a * NCOL + hb * 128 + 16 * c);
                                tmem_ld16_async_at<0>(lane_base + col, r);
                                tmem_ld16_async_at<16>(lane_base + 256 + col, r);
                            };
                            auto sum = [&](int c, const uint32_t (&r)[32]) {
                                const int cb = hb * 128 + 16 * c;
#pragma unroll
                                for (int jj = 0; jj < 16; jj += 2) {
                                    const float4 ab = cv4[cb + jj];
                                    const float4 cw = cv4[cb + jj + 1];
                                    const float2 gg = make_float2(__uint_as_float(r[jj]) + __uint_as_float(r[16 + jj]),
                                                                  __uint_as_float(r[jj + 1]) + __uint_as_float(r[17 + jj]));
                                    const float2 inner = __ffma2_rn(make_float2(cw.x, cw.y), pt2, make_float2(ab.z, ab.w));
                                    const float2 arg = __ffma2_rn(gg, make_float2(ab.x, ab.y), inner);
                                    const float2 k = make_float2(ex2_approx(arg.x), ex2_approx(arg.y));
                                    acc2[(jj >> 1) & 1] = __ffma2_rn(k, make_float2(cw.z, cw.w), acc2[(jj >> 1) & 1]);
                                }
                            };
                            if (nst > 0) {
                                issue(0, ra);
                                tmem_wait_pin(ra);
                            }
#pragma unroll 1
                            for (int c = 0; c < nst; c += 2) {
                                if (c + 1 < nst) issue(c + 1, rb);
                                sum(c, ra);
                                if (c + 1 < nst) {
                                    tmem_wait_pin(rb);
                                    if (c + 2 < nst) issue(c + 2, ra);
                                    sum(c + 1, rb);
                                    if (c + 2 < nst) tmem_wait_pin(ra);
                                }
                            }
                            acc[hb][0] = (acc2[0].x + acc2[0].y) + (acc2[1].x + acc2[1].y);
                        }
                    } else {
#pragma unroll
                        for (int hb = 0; hb < NB; ++hb) {
                            const int ncols = hb == 0 ? nrows : nrows_f;
#pragma unroll 1
                            for (int c = 0; c < 4 && c * 32 < ncols; ++c) {
                                const int cb = hb * 128 + c * 32;   // first column of the chunk
                                float g[32], gx[32];
                                tmem_ld32(lane_base + (uint32_t)(a * NCOL + cb), g);
                                tmem_ld32(lane_base + (uint32_t)(256 + a * NCOL + cb), gx);
#pragma unroll
                                for (int jj = 0; jj < 32; ++jj) g[jj] += gx[jj];
#pragma unroll
                                for (int jj = 0; jj < 32; ++jj) {
                                    const int j = cb + jj;
                                    const float4 ab = cv4[j & ~1];
                                    const float4 cw = cv4[(j & ~1) + 1];
                                    const bool o = j & 1;
                                    const float A = o ? ab.y : ab.x, B = o ? ab.w : ab.z, Cc = o ? cw.y : cw.x;
                                    const float k = ex2_approx(fmaf(g[jj], A, fmaf(Cc, pt, B)));
#pragma unroll
                                    for (int z = 0; z < RC; ++z) acc[hb][z] = fmaf(k, cwp[j * RC + z], acc[hb][z]);
                                }
                            }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(BAR_T_EMPTY(a));
                mbar_arrive(BAR_COL_EMPTY(cbuf));
                if (row < item.cnt) {
#pragma unroll
                    for (int hb = 0; hb < NB; ++hb) {
                        if (hb == 1 && nrows_f == 0) break;
                        const int e0 = hb == 0 ? item.e0 : args.items[f0 + (it - i0)].e0;
                        float *p = args.partial + (int64_t)(e0 + row) * args.r;
#pragma unroll
                        for (int z = 0; z < RC; ++z)
                            if (z < args.r) p[z] = acc[hb][z];
                    }
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
            // 8-row groups where the sub-block starts on one (every skeleton),
            // else single rows (a leaf anywhere in tree order)
            const bool rg = (first.row0 & 7) == 0;
            const CUtensorMap *mh = far ? &map_s_hi : (rg ? &map_t_hi : &map_t_hi1);
            const CUtensorMap *ml = far ? &map_s_lo : (rg ? &map_t_lo : &map_t_lo1);
            const int y = rg ? first.row0 >> 3 : first.row0;
            for (int it = i0; it < i1; ++it) {
                for (int kc = 0; kc < nkc; ++kc, ++g) {
                    const int s = g % NSB;
                    const uint32_t par = ((g / NSB) & 1) ^ 1;
                    if (!mbar_wait(BAR_B_FREE(s), par, abort_flag, args.status)) goto prod_done;
                    const uint32_t st = sbase + S::B0 + s * S::B_STAGE;
                    ++issued;
                    mbar_expect_tx(BAR_L_FULL(s), S::TX);
                    // [4 K groups][NCOL rows][16 B]: the core-matrix layout (a
                    // pair's follower rows follow the leader's)
                    tma_load_3d(st, mh, 0, y, kc * W_KG, BAR_L_FULL(s));
                    tma_load_3d(st + S::B_LO, ml, 0, y, kc * W_KG, BAR_L_FULL(s));
                }
            }
        }
    prod_done:
        // copies of the last NSB chunks may still be landing after an abort
        for (int gg = issued > NSB ? issued - NSB : 0; gg < issued; ++gg)
            mbar_drain(BAR_L_FULL(gg % NSB), (gg / NSB) & 1);
    } else if (warp == 12 && lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        int g = 0, li = 0;
        for (int ci = c_begin; ci < c_end && !*abort_flag; ++ci) {
            const int b = args.cta_blocks[ci];
            for (int it = args.block_off[b]; it < args.block_off[b + 1]; ++it, ++li) {
                const int a = li % NSLOT;
                const uint32_t d_main = tmem + (uint32_t)(a * NCOL), d_cross = tmem + (uint32_t)(256 + a * NCOL);
                for (int kc = 0; kc < nkc; ++kc, ++g) {
                    const int sa = g % NSA, sb = g % NSB;
                    if (!mbar_wait(BAR_A_FULL(sa), (g / NSA) & 1, abort_flag, args.status)) goto mma_done;
                    if (!mbar_wait(BAR_L_FULL(sb), (g / NSB) & 1, abort_flag, args.status)) goto mma_done;
                    if (kc == 0 && !mbar_wait(BAR_T_EMPTY(a), ((li / NSLOT) & 1) ^ 1, abort_flag, args.status))
                        goto mma_done;
                    tc_fence_after();
                    const uint32_t a_hi = sbase + sa * S::A_STAGE, a_lo = a_hi + S::A_LO;
                    const uint32_t b_hi = sbase + S::B0 + sb * S::B_STAGE, b_lo = b_hi + S::B_LO;
                    constexpr uint32_t LA = W_ROWS * 16, LB = NCOL * 16;   // bytes between K groups
#pragma unroll
                    for (int k = 0; k < 2; ++k) {   // K = 16 per MMA: two K groups
                        const uint32_t oa = (uint32_t)(2 * k) * LA, ob = (uint32_t)(2 * k) * LB;
                        tc_mma<P>(d_cross, nsw_desc(a_hi + oa, LA), nsw_desc(b_lo + ob, LB), IDESC, (kc | k) != 0);
                        tc_mma<P>(d_cross, nsw_desc(a_lo + oa, LA), nsw_desc(b_hi + ob, LB), IDESC, 1);
                        tc_mma<P>(d_main, nsw_desc(a_hi + oa, LA), nsw_desc(b_hi + ob, LB), IDESC, (kc | k) != 0);
                    }
                    tc_commit(BAR_A_FREE(sa));
                    tc_commit(BAR_B_FREE(sb));
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

// 3-D tensor maps of the pre-split source arrays (16-bit planes of K groups,
// [kw / 8][rows][8]), each box four contiguous runs of 2 or 4 KB landing in
// the core-matrix layout:
//   row groups: {64 elements = 8 rows of a K group, rows / 8, kw / 8 K
//     groups}, boxes {64, 16 NB, 4} (128-byte requests), for sub-blocks that
//     start on a multiple of 8 rows (skeletons start on multiples of 32);
//   rows: {8, rows, kw / 8}, boxes {8, 128 NB, 4} (16-byte requests), for
//     leaf sub-blocks that do not.
// [precision (BF16, FP16)][NB - 1][t_hi, t_lo, s_hi, s_lo (row groups), t_hi, t_lo (rows)].
struct TcwState {
    CUtensorMap map[2][2][6];
    bool ready[2] = {false, false};
    EncodeTiledFn encode = nullptr;
};

std::mutex g_tcw_mu;

askit_status encode_kgroups(EncodeTiledFn fn, CUtensorMap *m, CUtensorMapDataType ty, const void *base, int64_t rows,
                            int64_t kw, int box_rows, bool row_groups) {
    const int rg = row_groups ? 8 : 1;
    cuuint64_t dims[3] = {(cuuint64_t)(8 * rg), (cuuint64_t)(rows / rg), (cuuint64_t)(kw / 8)};
    cuuint64_t strides[2] = {(cuuint64_t)(16 * rg), (cuuint64_t)rows * 16};  // bytes: next row (group), next K group
    cuuint32_t box[3] = {(cuuint32_t)(8 * rg), (cuuint32_t)(box_rows / rg), (cuuint32_t)W_KG};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, ty, 3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        askit_set_error("cuTensorMapEncodeTiled (K groups) failed (%d)", (int)r);
        return ASKIT_ERR_CUDA;
    }
    return ASKIT_OK;
}

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
        for (int nb = 0; nb < 2; ++nb)
            for (int i = 0; i < 6; ++i)
                ASK_TRY(encode_kgroups(st->encode, &st->map[pi][nb][i], ty, arr[i & 3],
                                       (i & 3) < 2 ? t->N_pad : t->srows, t->kw, W_ROWS * (nb + 1), i < 4));
        st->ready[pi] = true;
    }
    *out = st;
    return ASKIT_OK;
}

template <int P, int RC, int NB>
askit_status launch_w(askit_tree t, TcwState *st, int pi, const TcwArgs &a, int grid, cudaStream_t s) {
    using S = WSmem<RC, NB>;
    constexpr size_t smem = S::BYTES + 128;
    static_assert(smem <= 232448, "shared-memory plan exceeds 227 KB");
    static const cudaError_t attr =
        cudaFuncSetAttribute(eval_tcw_kernel<P, RC, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ASK_CUDA(attr);
    ASK_TRY(ktimer_mark(t, s, false));
    const CUtensorMap *m = st->map[pi][NB - 1];
    eval_tcw_kernel<P, RC, NB><<<(unsigned)grid, W_THREADS, smem, s>>>(m[0], m[1], m[2], m[3], m[4], m[5], a);
    ASK_LAUNCH();
    return ktimer_mark(t, s, true);
}

template <int P, int RC>
askit_status run_w(askit_tree t, TcwState *st, int pi, TcwArgs a, const WorkLists &w, cudaStream_t s) {
    // paired items: the two sub-blocks of a node (same targets, same center)
    // in one 256-column item, on the segments' schedule (several CTAs on one
    // block at a time, so that its source rows stay in L2 across its items)
    if (t->tune_pairs && w.seg_sched_off) {
        a.block_off = w.seg_off;
        a.partner = w.seg_partner;
        a.cta_off = w.seg_sched_off;
        a.cta_blocks = w.seg_sched;
        return launch_w<P, RC, 2>(t, st, pi, a, w.n_ctas, s);
    }
    return launch_w<P, RC, 1>(t, st, pi, a, w.n_ctas, s);
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
    if ((reinterpret_cast<uintptr_t>(Xq) & 15) != 0 || t->kw % W_KC != 0) {
        askit_set_error("target rows must be 16-byte aligned and the row width a multiple of %d", W_KC);
        return ASKIT_ERR_INVALID_ARG;
    }
    (void)q_rows;
    const int pi = precision == ASKIT_PREC_BF16X3 ? 0 : 1;
    TcwState *st = nullptr;
    ASK_TRY(tcw_state(t, pi, &st));
    TcwArgs a;
    a.q = Xq;
    a.ldq = ldq;
    a.items = w.items;
    a.block_off = w.block_off;
    a.cta_off = w.cta_off;
    a.cta_blocks = w.cta_blocks;
    a.partner = nullptr;
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
        if (c.r == 1) return run_w<ASKIT_PREC_BF16X3, 1>(t, st, pi, a, w, s);
        if (c.r <= 4) return run_w<ASKIT_PREC_BF16X3, 4>(t, st, pi, a, w, s);
        return run_w<ASKIT_PREC_BF16X3, 16>(t, st, pi, a, w, s);
    }
    if (c.r == 1) return run_w<ASKIT_PREC_FP16X3, 1>(t, st, pi, a, w, s);
    if (c.r <= 4) return run_w<ASKIT_PREC_FP16X3, 4>(t, st, pi, a, w, s);
    return run_w<ASKIT_PREC_FP16X3, 16>(t, st, pi, a, w, s);
}

void eval_tc_wide_free(askit_tree t) {
    delete (TcwState *)t->tcw;
    t->tcw = nullptr;
}
