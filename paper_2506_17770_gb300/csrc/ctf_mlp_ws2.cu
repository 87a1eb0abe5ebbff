// ctf_mlp_ws2.cu -- learned-decode filter for STF, Box and Mask Sampling on
// single views: warps specialised by role, with the texel features computed
// by the warps that select the texels.
//
// A CTA of 256 threads (four per SM) takes the groups of 8 pixel tiles g0,
// g0 + G, ... (G = gridDim.x) in turn:
//   - warpgroup 1 (warps 4-7, the producers, two tiles of the group each)
//     runs step 1 of the collaborative flow (Sec. 3) on its tiles, packs the
//     texel lists of the group into consecutive rows (tile order, list order
//     within a tile), and writes the features of its own rows straight into
//     the group's layer-1 operand buffer in the tensor cores' layout;
//   - warpgroup 0 (warps 0-3, the consumer) owns the 128 TMEM lanes and runs
//     the tcgen05 MLP chain(s) over the group's rows: three MMA layers, the
//     two hidden epilogues (bias, ReLU, conversion to the next operand) and
//     the output epilogue into the row values; then it gathers, filters and
//     stores the group's pixels from the row values (warp w the tiles w and
//     4 + w).
// One consumer thread issues the MMAs and polls their barrier; the other
// consumer threads wait at a named barrier (no polling).  Warps whose 32
// rows all lie past the group's last row skip their epilogues.  The hidden
// activations stay in tensor memory: each epilogue writes them next to the
// accumulator, and the next layer's MMAs read their A operand from there.
// Three stages of group buffers (operand rows, whose first 4 KB the row
// values overwrite once the rows have been consumed, per-pixel words, counts
// and first rows) rotate over consecutive groups, so the producers may run
// two groups ahead of the consumer.  The producers hand a stage over with a
// full barrier (four arrivals) and get it back with a done barrier (one
// arrival, after the gather); a named barrier among the producers at the
// start of each group orders their reuse of the texel lists.  Every wait is
// bounded; a wait that gives up records CTF_ERR_TIMEOUT and both roles
// leave.  The CTA starts with 64 registers per thread; setmaxnreg gives the
// producers 72 and the consumer 56 (128 x 72 + 128 x 56 = 256 x 64).
// Each pixel gets the same texels, texel values, image and counts as the
// other learned kernels: the rows of an MMA are independent, so where a
// texel's row sits does not change its value, and an MMA's result does not
// depend on whether its A operand comes from shared or tensor memory.
#include <cstdint>
#include <mutex>
#include <set>
#include <utility>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "ctf_device.cuh"
#include "ctf_internal.h"
#include "ctf_mlp.cuh"
#include "ctf_select.cuh"
#include "tc_ops.cuh"
#include "ctf_mlp_chain.cuh"
#include "ctf_exact_tile.cuh"

namespace ctf {
namespace {

constexpr int kPProducerWarps = 4;
constexpr int kPProducerThreads = 32 * kPProducerWarps;
constexpr int kPThreads = kRows + kPProducerThreads;
constexpr int kPSlots = kGroupTiles / kPProducerWarps;  // pixel tiles of the group per producer warp
constexpr int kPCtasPerSm = kPProducerWarps == 4 ? 4 : 3;
constexpr int kPLaunchRegs = (65536 / (kPThreads * kPCtasPerSm)) & ~7;
// with four producer warps setmaxnreg moves registers from the consumer to them
constexpr bool kPSplitRegs = kPProducerWarps == 4;
constexpr int kPConsumerRegs = 56, kPProducerRegs = 72;
static_assert(!kPSplitRegs || kRows * kPConsumerRegs + kPProducerThreads * kPProducerRegs == kPThreads * kPLaunchRegs,
              "the register split adds up to the launch's registers");
static_assert(kGroupTiles % kPProducerWarps == 0 && 2 * kRows % kPProducerThreads == 0, "role shapes");
constexpr int kPFeatRounds = 2 * kRows / kPProducerThreads;  // rows per producer thread, at most

// Shared memory (bytes).  The operand image sits at 0 with the offsets of
// ctf_mlp.cuh; then the MMA barrier and TMEM slot, the stage hand-over
// barriers, the producers' Mask rank slots and texel lists, in the variant
// with fallbacks C / C+ one texel table per warp, and the stages.
// Tensor memory (128 columns): every layer's accumulator D at columns
// [0, 64), the hidden activations at [64, 96).
constexpr int kPMaxStages = 3;
constexpr int kPBar = kImgBytes;                 // MMA barrier (8 B), TMEM base (4 B)
constexpr int kPTmem = kPBar + 8;
constexpr int kPHand = kPBar + 16;               // full[kPMaxStages], done[kPMaxStages]
// producer warps x 64 rank slots (two texels per lane may rank 64 texels a tile)
constexpr int kPRanks = kPHand + 16 * kPMaxStages;
constexpr int kPList = kPRanks + kPProducerWarps * 64 * 4;  // 8 slots x 32 (or 4 x 64) int2 texel lists
constexpr int kPFbTab = kPList + kGroupTiles * 32 * 8;      // fallback variant: 8 warps' texel tables
// one stage
constexpr int kPX = 0;                           // 256 rows x 32 B layer-1 operand; row values overlay 0..4095
constexpr int kPST = kPX + 8192;                 // 256 x float2 (s, t)
constexpr int kPInfo = kPST + 2048;              // 256 x uint32 per-pixel words
constexpr int kPCount = kPInfo + 1024;           // 8 x int texels per tile
constexpr int kPBase = kPCount + 32;             // 8 x int first row per tile
constexpr int kPRows = kPBase + 32;              // int: rows of the group
constexpr int kPQ = kPRows + 16;                 // fallback variant: 256 x int2 texel a pixel's lane produces
constexpr int kPUL = kPQ + 2048;                 // fallback variant: 256 x int2 upper-left texel of the footprint

// kFb: the variant with fallbacks C / C+ (two stages, to make room for the
// texel tables and the per-pixel texels the blend of eq. 1 needs); kList:
// List Merge (two stages and a List Merge table per producer warp, at the
// place of the fallback tables).
// kBatch: the persistent batch kernel, whose stages also carry the group's
// view (at kPBat: its slot, the group's first tile, copies of its
// parameters and network).
constexpr int kPBat = kPRows + 16;
constexpr int kPBatBytes = 16 + (int)sizeof(ExactParams) + (((int)sizeof(MlpDevice) + 15) & ~15);
template <bool kFb, bool kList = false, bool kBatch = false>
struct PLayout {
    static_assert(!(kFb && kList), "List Merge with fallbacks runs on the extension kernel");
    static_assert(!(kFb && kBatch), "batches take no fallbacks on learned views");
    static constexpr int kStages = (kFb || kList) ? 2 : 3;
    static constexpr int kStage0 = kFb ? kPFbTab + 8 * (int)sizeof(FbTable)
                                       : (kList ? kPFbTab + kPProducerWarps * (int)sizeof(ListTable) : kPFbTab);
    static constexpr int kStageBytes = kFb ? kPUL + 2048 : kPRows + 16 + (kBatch ? kPBatBytes : 0);
    static constexpr int kBytes = kStage0 + kStages * kStageBytes;
    static_assert(kStage0 % 16 == 0 && kStageBytes % 16 == 0 && kPFbTab % 16 == 0, "16-byte operand buffers");
    // kPCtasPerSm CTAs per SM fit, and no more than four (4 x 128 TMEM columns)
    static_assert(kPCtasPerSm * (kBytes + 1024 + 128) <= 228 * 1024, "the CTAs of an SM fit in shared memory");
};
static_assert(65536 / (kPThreads * kPLaunchRegs) <= 4, "at most four CTAs share an SM's TMEM");

template <bool kFb, bool kList, bool kBatch = false>
__device__ __forceinline__ unsigned char *p_stage(unsigned char *sm, int s) {
    return sm + PLayout<kFb, kList, kBatch>::kStage0 + s * PLayout<kFb, kList, kBatch>::kStageBytes;
}
__device__ __forceinline__ uint64_t *p_full(unsigned char *sm, int s) {
    return reinterpret_cast<uint64_t *>(sm + kPHand) + s;
}
__device__ __forceinline__ uint64_t *p_done(unsigned char *sm, int s) {
    return reinterpret_cast<uint64_t *>(sm + kPHand) + kPMaxStages + s;
}

__device__ __forceinline__ void p_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(bar)) : "memory");
}

// Named barriers: 1 among the 128 consumer threads, 2 among the producer
// threads (0 stays __syncthreads).
__device__ __forceinline__ void cons_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__device__ __forceinline__ void prod_bar() { asm volatile("bar.sync 2, %0;" ::"n"(kPProducerThreads) : "memory"); }

// Barrier `id` among n threads, returning whether any of them passed true.
template <int id, int n>
__device__ __forceinline__ bool bar_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(id), "n"(n)
        : "memory");
    return r != 0;
}

// Hidden epilogue of a warp's 32 rows: TMEM columns [taddr, taddr + 64) of
// this thread's row -> bias, ReLU -> the next layer's A operand, written to
// TMEM columns from hcol on (FP16 pairs, or E4M3 quadruples, per 32-bit
// column in K order).
__device__ __forceinline__ void p_hidden_epilogue(uint32_t hcol, uint32_t taddr, const float *bias,
                                                  const float *oscale, bool fp8) {
    const float4 *b4 = reinterpret_cast<const float4 *>(bias);
    const float4 *o4 = reinterpret_cast<const float4 *>(oscale);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float d[16];
        tc::tmem_ld16(taddr + 16 * q, d);
        tc::tmem_wait_ld();
        tc::regs_after_wait<16>(d);
        if (!fp8) {
            uint32_t w[8];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 4 * i;
                const float4 b = b4[(16 * q + k) / 4];
                const float2 t0 = __fadd2_rn(make_float2(d[k], d[k + 1]), make_float2(b.x, b.y));
                const float2 t1 = __fadd2_rn(make_float2(d[k + 2], d[k + 3]), make_float2(b.z, b.w));
                w[2 * i] = relu_half2(t0.x, t0.y);
                w[2 * i + 1] = relu_half2(t1.x, t1.y);
            }
            tc::tmem_st8(hcol + 8 * q, w);
        } else {
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 4 * i;
                const float4 b = b4[(16 * q + k) / 4], o = o4[(16 * q + k) / 4];
                const float2 t0 = __ffma2_rn(make_float2(d[k], d[k + 1]), make_float2(o.x, o.y), make_float2(b.x, b.y));
                const float2 t1 =
                    __ffma2_rn(make_float2(d[k + 2], d[k + 3]), make_float2(o.z, o.w), make_float2(b.z, b.w));
                w[i] = (uint32_t)relu_e4m3x2(t0.x, t0.y) | ((uint32_t)relu_e4m3x2(t1.x, t1.y) << 16);
            }
            tc::tmem_st4(hcol + 4 * q, w);
        }
    }
    tc::tmem_wait_st();
}

// One MMA layer's completion: thread 0 polls the barrier, the other
// consumer threads wait at the consumer barrier, which also carries the
// outcome to all of them.  Returns false (for every consumer thread alike)
// if the MMAs did not complete within the bound.
__device__ __forceinline__ bool p_layer_done(uint64_t *bar, uint32_t &phase, int *err) {
    bool ok = true;
    if (threadIdx.x == 0) ok = tc::mbar_wait(bar, phase, kMaxTries);
    phase ^= 1u;
    __syncwarp();  // the barrier below is .aligned: warp 0 reconverges first
    if (bar_or<1, kRows>(!ok)) {
        if (threadIdx.x == 0) atomicExch(err, CTF_ERR_TIMEOUT);
        return false;
    }
    tc::fence_after_sync();
    return true;
}

// The three layers for the 128 rows of chain c of a stage (layer-1 operand
// at sX).  TMEM columns: D (every layer's accumulator) at [0, 64), the
// hidden activations H at [64, 96).  `live`: this warp has rows below the
// group's row count (else it skips its epilogues).  Consumer threads only.
__device__ __forceinline__ bool p_chain(unsigned char *sm, uint32_t tmem, uint64_t *bar, uint32_t &phase,
                                        uint32_t sX, bool fp8, bool live, float4 &out, int *err) {
    const int tid = threadIdx.x, warp = tid >> 5;
    const float *b1 = reinterpret_cast<const float *>(sm + kImgB1);
    const float *b2 = reinterpret_cast<const float *>(sm + kImgB2);
    const float *b3 = reinterpret_cast<const float *>(sm + kImgB3);
    const float *s1 = reinterpret_cast<const float *>(sm + kImgS1);
    const float *s2 = reinterpret_cast<const float *>(sm + kImgS2);
    const float *s3 = reinterpret_cast<const float *>(sm + kImgS3);
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    const uint32_t sW1 = tc::smem_addr(sm + kImgW1), sW2 = tc::smem_addr(sm + kImgW2),
                   sW3 = tc::smem_addr(sm + kImgW3);
    const uint32_t kstep = 256;              // 32 bytes of K per 8-row group
    const uint32_t sboX = 256u;              // K = 32 bytes per row, FP16 and E4M3 alike
    const uint32_t sboH = fp8 ? 512u : 1024u;  // 64 elements per row
    const int nk = fp8 ? 2 : 4;              // MMAs over K = 64
    const uint32_t id64 = fp8 ? tc::idesc_e4m3(128, 64) : tc::idesc_f16(128, 64);
    const uint32_t id16 = fp8 ? tc::idesc_e4m3(128, 16) : tc::idesc_f16(128, 16);
    const uint32_t tH = tmem + 64;

    // ---- layer 1: D = X W1^T
    if (tid == 0) {
        tc::fence_after_sync();
        const uint64_t a = tc::smem_desc(sX, 128, sboX), b = tc::smem_desc(sW1, 128, sboX);
        if (fp8) tc::mma_e4m3(tmem, a, b, id64, false);
        else tc::mma_f16(tmem, a, b, id64, false);
        tc::commit(bar);
    }
    if (!p_layer_done(bar, phase, err)) return false;
    if (live) p_hidden_epilogue(lane_base + 64, lane_base + 0, b1, s1, fp8);
    tc::fence_before_sync();
    cons_bar();
    // ---- layer 2: D = H1 W2^T (D1 has been read)
    if (tid == 0) {
        tc::fence_after_sync();
        for (int j = 0; j < nk; ++j) {
            const uint64_t b = tc::smem_desc(sW2 + j * kstep, 128, sboH);
            if (fp8) tc::mma_e4m3_ts(tmem, tH + 8 * j, b, id64, j > 0);
            else tc::mma_f16_ts(tmem, tH + 8 * j, b, id64, j > 0);
        }
        tc::commit(bar);
    }
    if (!p_layer_done(bar, phase, err)) return false;
    // the layer-2 MMAs have read H1, so H2 may overwrite it
    if (live) p_hidden_epilogue(lane_base + 64, lane_base + 0, b2, s2, fp8);
    tc::fence_before_sync();
    cons_bar();
    // ---- layer 3: D[0..16) = H2 W3^T
    if (tid == 0) {
        tc::fence_after_sync();
        for (int j = 0; j < nk; ++j) {
            const uint64_t b = tc::smem_desc(sW3 + j * kstep, 128, sboH);
            if (fp8) tc::mma_e4m3_ts(tmem, tH + 8 * j, b, id16, j > 0);
            else tc::mma_f16_ts(tmem, tH + 8 * j, b, id16, j > 0);
        }
        tc::commit(bar);
    }
    if (!p_layer_done(bar, phase, err)) return false;
    if (live) {
        uint32_t r[4];
        tc::tmem_ld4(lane_base + 0, r);
        tc::tmem_wait_ld();
        tc::regs_after_wait<4>(r);
        float o[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float d = __uint_as_float(r[c]);
            const float v = fp8 ? __fmaf_rn(d, s3[c], b3[c]) : __fadd_rn(d, b3[c]);
            o[c] = fminf(fmaxf(v, 0.f), 1.f);
        }
        out = make_float4(o[0], o[1], o[2], o[3]);
    }
    tc::fence_before_sync();
    return true;
}

// Producer: step 1 on tile slot g of the group at `first` into stage st:
// per pixel (s, t) and the packed word of the other learned kernels (bits
// 0-19 the list indices of its 4 taps on success, else of its own texel;
// 20-22 its count; 23 active; 24 inside; 25 success), the slot's texel count,
// and the slot's texel list (clamped) at list[32 g + rank].
// kStats: the variant that keeps the outcome counters (p.stats set).
// kFb: the variant with fallbacks C / C+: an over-budget magnified tile
// takes its texels from fb_choose (the exact path's choice, with the warp's
// table fbt); each lane's produced texel gets the rank of the lane among
// the producing lanes, and the pixel's word carries bit 26 (fallback tile)
// and bit 27 (this lane produces); the produced texel and the footprint's
// upper-left texel go to the stage for the blend of eq. 1.
// kTwo: the variant with two texels per lane (groups of 4 tiles of up to 64
// texels): the tile's list at list[64 g + rank]; the pixel's word holds the
// 6-bit list indices of its taps (bits 0-23, or of its own texel), its count
// (24-25), active (26), inside (27) and success (28).
template <int ALG, int TW, int MD, bool kStats, bool kFb, bool kTwo = false>
__device__ __forceinline__ void p_step1(const ExactParams &p, const TilePos &tp, long long first, int g,
                                        unsigned char *st, int2 *list, int lane, uint32_t lt, int *ranks,
                                        Counters &cnt, FbTable *fbt, ListTable *T) {
    constexpr int TH = 32 / TW;
    const int tx = lane % TW, ty = lane / TW;
    float2 *pix_st = reinterpret_cast<float2 *>(st + kPST);
    uint32_t *pix_info = reinterpret_cast<uint32_t *>(st + kPInfo);
    const long long tile = first + g;
    const bool valid = tile < p.n_tiles;
    int bx = 0, by = 0;
    if (valid) tile_pos(tp, g, bx, by);
    const int px = bx * TW + tx, py = by * TH + ty;
    const bool inside = valid && px < p.W && py < p.H;
    const uint32_t idx = ck(inside ? (uint32_t)py * (uint32_t)p.W + (uint32_t)px : 0u, view_pixels(p), p.err,
                            kBndPixel);
    float2 uv = make_float2(0.f, 0.f);
    float4 jac = make_float4(0.f, 0.f, 0.f, 0.f);
    bool covered = inside;
    if (inside) {
        uv = __ldcs(p.uv + idx);
        if (ALG >= ALG_LIST) jac = __ldcs(p.jac + idx);
        if (p.cov) covered = __ldcs(p.cov + idx) != 0;
    }
    PixelSetup ps;
    ps.active = covered;
    setup_coords(uv, (float)p.Wt, (float)p.Ht, ps);
    Selection sel;
    if (valid) {
        sel = select_tile<ALG, MD, kStats, false, kTwo>(p, ps, jac, px, py, lane, lt, T, ranks, cnt);
    } else {
        sel.path = PATH_EMPTY;
        sel.A = 0;
        sel.produce = sel.produce2 = false;
        sel.count = 0;
        sel.my_rank = sel.my_rank2 = 0;
    }
    if (kTwo) {
        auto clamp_xy = [&](int x, int y) { return make_int2(min(max(x, 0), p.Wt - 1), min(max(y, 0), p.Ht - 1)); };
        if (sel.produce) list[64 * g + ck(sel.my_rank, 64, p.err, kBndTexList)] = clamp_xy(sel.tx, sel.ty);
        if (sel.produce2) list[64 * g + ck(sel.my_rank2, 64, p.err, kBndTexList)] = clamp_xy(sel.tx2, sel.ty2);
        const bool succ = sel.path == PATH_SUCCESS;
        if (lane == 0) reinterpret_cast<int *>(st + kPCount)[g] = succ ? sel.n : __popc(sel.A);
        uint32_t info = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) info |= ((uint32_t)sel.rk[k] & 63u) << (6 * k);
        info = succ ? info : ((uint32_t)sel.my_rank & 63u);
        info |= ((uint32_t)sel.count << 24) | (ps.active ? 1u << 26 : 0u) | (inside ? 1u << 27 : 0u) |
                (succ ? 1u << 28 : 0u);
        reinterpret_cast<float2 *>(st + kPST)[32 * g + lane] = make_float2(ps.s, ps.t);
        reinterpret_cast<uint32_t *>(st + kPInfo)[32 * g + lane] = info;
        return;
    }
    if (kFb && p.fallback != 0 && sel.path == PATH_FALLBACK_BUDGET) {  // warp-uniform
        const FbChoice c = fb_choose(p.fallback, p.view, p.y0, p.k0, p.k1, ps.ulx, ps.uly, ps.s, ps.t, ps.active, px,
                                     py, sel.A, lane, lt, fbt);
        const uint32_t pm = __ballot_sync(FULL, c.produce);
        const int rank = __popc(pm & lt), n = __popc(pm);
        if (c.produce)
            list[32 * g + ck(rank, 32, p.err, kBndTexList)] =
                make_int2(min(max(c.qx, 0), p.Wt - 1), min(max(c.qy, 0), p.Ht - 1));
        if (lane == 0) reinterpret_cast<int *>(st + kPCount)[g] = n;
        // select_tile counted one evaluation per active lane
        if (kStats) cnt.v[kStatTexelEvals] += n - __popc(sel.A);
        const uint32_t info = (uint32_t)rank | ((c.produce ? 1u : 0u) << 20) | (ps.active ? 1u << 23 : 0u) |
                              (inside ? 1u << 24 : 0u) | (1u << 26) | (c.produce ? 1u << 27 : 0u);
        pix_st[32 * g + lane] = make_float2(ps.s, ps.t);
        pix_info[32 * g + lane] = info;
        reinterpret_cast<int2 *>(st + kPQ)[32 * g + lane] = make_int2(c.qx, c.qy);
        reinterpret_cast<int2 *>(st + kPUL)[32 * g + lane] = make_int2(ps.ulx, ps.uly);
        return;
    }
    if (sel.produce)
        list[32 * g + ck(sel.my_rank, 32, p.err, kBndTexList)] =
            make_int2(min(max(sel.tx, 0), p.Wt - 1), min(max(sel.ty, 0), p.Ht - 1));
    const bool succ = sel.path == PATH_SUCCESS;
    const int n = succ ? sel.n : __popc(sel.A);
    if (lane == 0) reinterpret_cast<int *>(st + kPCount)[g] = n;
    uint32_t info = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) info |= ((uint32_t)sel.rk[k] & 31u) << (5 * k);
    info = succ ? info : ((uint32_t)sel.my_rank & 31u);
    info |= ((uint32_t)sel.count << 20) | (ps.active ? 1u << 23 : 0u) | (inside ? 1u << 24 : 0u) |
            (succ ? 1u << 25 : 0u);
    pix_st[32 * g + lane] = make_float2(ps.s, ps.t);
    pix_info[32 * g + lane] = info;
}

// Consumer: step 3 for tile slot g of the group at `first` from stage st
// (its row values in place): gather, filter, store; `lane` is the pixel.
template <int TW, bool kFb, bool kTwo = false>
__device__ __forceinline__ void p_gather(const ExactParams &p, const TilePos &tp, int g, const unsigned char *st,
                                         int lane, FbTable *fbt) {
    constexpr int TH = 32 / TW;
    const int tx = lane % TW, ty = lane / TW;
    const uint32_t info = reinterpret_cast<const uint32_t *>(st + kPInfo)[32 * g + lane];
    const float4 *outrow = reinterpret_cast<const float4 *>(st + kPX);
    const int base = reinterpret_cast<const int *>(st + kPBase)[g];
    // row of list entry i of this tile (the row values fill the stage's first 4 KB: 256 rows)
    auto row_of = [&](uint32_t i) { return ck(base + (int)i, 2 * kRows, p.err, kBndRow); };
    int bx, by;
    tile_pos(tp, g, bx, by);
    // the word's fields (kTwo: 6-bit list indices)
    constexpr int kIdxBits = kTwo ? 6 : 5, kCnt = kTwo ? 24 : 20, kAct = kTwo ? 26 : 23, kIns = kTwo ? 27 : 24,
                  kSucc = kTwo ? 28 : 25;
    constexpr uint32_t kIdxMask = (1u << kIdxBits) - 1u, kCntMask = kTwo ? 3u : 7u;
    const bool inside = ((info >> kIns) & 1u) != 0;  // (pixels outside the frame take part in the blend only)
    const uint32_t idx = ck(inside ? (uint32_t)(by * TH + ty) * (uint32_t)p.W + (uint32_t)(bx * TW + tx) : 0u,
                            view_pixels(p), p.err, kBndPixel);
    if (kFb && ((info >> 26) & 1u)) {
        // fallback C / C+ (the whole warp: the blend is warp-collective):
        // eq. 1 over the produced texels of the footprint, their values the
        // rows of the tile's list
        FbChoice c;
        c.produce = ((info >> 27) & 1u) != 0;
        const int2 q = reinterpret_cast<const int2 *>(st + kPQ)[32 * g + lane];
        const int2 ul = reinterpret_cast<const int2 *>(st + kPUL)[32 * g + lane];
        const float2 s = reinterpret_cast<const float2 *>(st + kPST)[32 * g + lane];
        c.qx = q.x;
        c.qy = q.y;
        const float4 val = c.produce ? outrow[row_of(info & 31u)] : make_float4(0.f, 0.f, 0.f, 0.f);
        const FallbackOut fo = fb_blend<false>(val, c, ul.x, ul.y, s.x, s.y, ((info >> 23) & 1u) != 0, lane, fbt);
        if (inside) {
            __stcs(p.out + idx, fo.res);
            if (p.evals) p.evals[idx] = (uint8_t)fo.count;
        }
        return;
    }
    if (!inside) return;  // outside the frame (or no tile)
    float4 result = make_float4(0.f, 0.f, 0.f, 0.f);
    uint8_t cv = 0;
    if ((info >> kAct) & 1u) {
        if ((info >> kSucc) & 1u) {
            const float2 s = reinterpret_cast<const float2 *>(st + kPST)[32 * g + lane];
            float w[4];
            bilinear_weights(s.x, s.y, w);
            float2 rg = make_float2(0.f, 0.f), ba = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 t = outrow[row_of((info >> (kIdxBits * k)) & kIdxMask)];
                const float2 wk = make_float2(w[k], w[k]);
                rg = __ffma2_rn(wk, make_float2(t.x, t.y), rg);
                ba = __ffma2_rn(wk, make_float2(t.z, t.w), ba);
            }
            result = make_float4(rg.x, rg.y, ba.x, ba.y);
            cv = (uint8_t)((info >> kCnt) & kCntMask);
        } else {
            result = outrow[row_of(info & kIdxMask)];
            cv = 1;
        }
    }
    __stcs(p.out + idx, result);
    if (p.evals) p.evals[idx] = cv;
}

template <int ALG, int TW, int MD, bool kStats, bool kFb, bool kTwo>
__global__ void __launch_bounds__(kPThreads, kPCtasPerSm) mlp_filter_pf_kernel(const ExactParams p, const MlpDevice m, int *err) {
    static_assert(!(kFb && kTwo), "fallbacks with two texels per lane run on the extension kernel");
    constexpr bool kList = ALG == ALG_LIST;
    constexpr int kPStages = PLayout<kFb, kList>::kStages;
    // tiles per group: two texels per lane may need 64 rows a tile
    constexpr int kGT = kTwo ? kGroupTiles / 2 : kGroupTiles;
    constexpr int kSlots = kGT / kPProducerWarps;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ unsigned long long block_stats[kNumStats];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // fallback variant: warp w's texel table (empty between tiles)
    FbTable *fbt = kFb ? reinterpret_cast<FbTable *>(sm + kPFbTab) + warp : nullptr;
    if (kFb) fb_clear(fbt, lane);
    // List Merge: producer warp w - 4's table (empty between tiles)
    ListTable *T = kList && warp >= 4 ? reinterpret_cast<ListTable *>(sm + kPFbTab) + (warp - 4) : nullptr;
    if (kList && warp >= 4) {
#pragma unroll
        for (int q = 0; q < 8; ++q) T->keys[lane * 8 + q] = kEmpty;
    }
    uint64_t *mma_bar = reinterpret_cast<uint64_t *>(sm + kPBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + kPTmem);
    if (threadIdx.x < kNumStats) block_stats[threadIdx.x] = 0;
    {
        const uint4 *src = m.img;
        uint4 *dst = reinterpret_cast<uint4 *>(sm + kImgW1);
        for (int i = threadIdx.x; i < kImgBytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
        // every thread's part of the image, written through the generic
        // proxy, ordered before the MMAs that read it through the async proxy
        tc::fence_proxy_async();
    }
    if (threadIdx.x == 0) {
        tc::mbar_init(mma_bar, 1);
        for (int s = 0; s < kPStages; ++s) {
            tc::mbar_init(p_full(sm, s), kPProducerWarps);
            tc::mbar_init(p_done(sm, s), 1);
        }
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const float *inv_a1 = reinterpret_cast<const float *>(sm + kImgA1);
    Counters cnt;
#pragma unroll
    for (int i = 0; i < kNumStats; ++i) cnt.v[i] = 0;
    const long long n_groups = (p.n_tiles + kGT - 1) / kGT;
    const long long G = gridDim.x;
    const bool fp8 = m.fp8 != 0;

    if (warp < 4) {
        // ---------------- consumer ----------------
        if (kPSplitRegs) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kPConsumerRegs));
        const int tid = threadIdx.x;
        uint32_t phase = 0;
        for (long long j = 0;; ++j) {
            const long long grp = blockIdx.x + j * G;
            if (grp >= n_groups) break;
            const int s = (int)(j % kPStages);
            const uint32_t par = (uint32_t)((j / kPStages) & 1);
            unsigned char *st = p_stage<kFb, kList>(sm, s);
            bool ok = true;
            if (tid == 0) ok = tc::mbar_wait(p_full(sm, s), par, kMaxTries);
            __syncwarp();
            if (bar_or<1, kRows>(!ok)) {
                if (tid == 0) atomicExch(err, CTF_ERR_TIMEOUT);
                break;
            }
            const int R = *reinterpret_cast<const int *>(st + kPRows);
            const int passes = (R + kRows - 1) / kRows;
            float4 *outrow = reinterpret_cast<float4 *>(st + kPX);
            const uint32_t sX = tc::smem_addr(st + kPX);
            for (int c = 0; c < passes && ok; ++c) {
                const bool live = kRows * c + 32 * warp < R;
                float4 v;
                ok = p_chain(sm, tmem, mma_bar, phase, sX + 4096u * (uint32_t)c, fp8, live, v, err);
                // chain c's outputs overwrite operand rows of chain 0, which its
                // layer-1 MMA has read; chain 1's operand rows (bytes 4096 on)
                // are untouched
                if (ok && live) outrow[ck(kRows * c + tid, 2 * kRows, p.err, kBndRow)] = v;
                cons_bar();
            }
            if (!ok) break;
            {
                // step 3 for the group: warp w the tiles w and 4 + w
                const TilePos tpc = tile_pos0(p, grp * kGT);
#pragma unroll 1
                for (int k = 0; k < kSlots; ++k) p_gather<TW, kFb, kTwo>(p, tpc, 4 * k + warp, st, tid & 31, fbt);
            }
            __syncwarp();
            cons_bar();  // every consumer warp has read the stage
            if (tid == 0) p_arrive(p_done(sm, s));
        }
    } else {
        // ---------------- producers: kPSlots tile slots per warp ----------------
        if (kPSplitRegs) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kPProducerRegs));
        const int pw = warp - 4;
        const uint32_t lt = lanemask_lt();
        int *ranks = reinterpret_cast<int *>(sm + kPRanks) + 64 * pw;
        int2 *list = reinterpret_cast<int2 *>(sm + kPList);
        const int pt = threadIdx.x - kRows;  // producer thread
        for (long long j = 0;; ++j) {
            const long long grp = blockIdx.x + j * G;
            const bool have = grp < n_groups;  // uniform over the CTA
            if (!have) break;
            {
                const int s = (int)(j % kPStages);
                unsigned char *st = p_stage<kFb, kList>(sm, s);
                if (j >= kPStages) {
                    // the consumer has gathered group j - kPStages from this stage
                    bool okd = true;
                    if (lane == 0) okd = tc::mbar_wait(p_done(sm, s), (uint32_t)(((j - kPStages) / kPStages) & 1), kMaxTries);
                    __syncwarp();
                    if (bar_or<2, kPProducerThreads>(!okd)) {
                        if (threadIdx.x == 128) atomicExch(err, CTF_ERR_TIMEOUT);
                        break;
                    }
                }
                // every producer warp has read the texel lists of group j - 1
                __syncwarp();
                prod_bar();
                const long long first = grp * kGT;
                const TilePos tp = tile_pos0(p, first);
#pragma unroll 1
                for (int k = 0; k < kSlots; ++k)
                    p_step1<ALG, TW, MD, kStats, kFb, kTwo>(p, tp, first, kSlots * pw + k, st, list, lane, lt, ranks,
                                                            cnt, fbt, T);
                __syncwarp();
                prod_bar();  // every slot's list and count is in place
                // rows: slot g owns [start_g, start_g + count_g) in slot order;
                // this thread's rows pt and pt + kPProducerThreads fall in slots
                // g0 and g1
                const int *count = reinterpret_cast<const int *>(st + kPCount);
                int R = 0, g0 = 0, b0 = 0, g1 = 0, b1 = 0, mybase = 0;
#pragma unroll
                for (int g = 0; g < kGT; ++g) {
                    if (pt >= R) {
                        g0 = g;
                        b0 = R;
                    }
                    if (pt + kPProducerThreads >= R) {
                        g1 = g;
                        b1 = R;
                    }
                    if (pt == g) mybase = R;
                    R += count[g];
                }
                if (pt < kGT) reinterpret_cast<int *>(st + kPBase)[pt] = mybase;
                if (pt == 0) {
                    *reinterpret_cast<int *>(st + kPRows) = R;
                    if (kStats) cnt.v[kStatTexelEvalsUnique] += R;
                }
                // features of rows pt and pt + kPProducerThreads, in the tensor
                // cores' operand layout
#pragma unroll 1
                for (int c = 0; c < kPFeatRounds; ++c) {
                    const int row = pt + kPProducerThreads * c;
                    if (row >= R) break;
                    constexpr int kLs = kTwo ? 64 : 32;  // list entries a tile
                    const int2 t = c == 0 ? list[kLs * g0 + ck(row - b0, kLs, p.err, kBndTexList)]
                                          : list[kLs * g1 + ck(row - b1, kLs, p.err, kBndTexList)];
                    float f[kMlpIn];
                    texel_features(m, t.x, t.y, f);
                    store_x_row_at(st + kPX, ck(row, 2 * kRows, p.err, kBndRow), f, fp8, inv_a1);
                }
                tc::fence_proxy_async();  // generic-proxy writes -> the MMAs' async proxy
                __syncwarp();
                if (lane == 0) p_arrive(p_full(sm, s));
            }
        }
    }

    if (kStats && p.stats && lane == 0) {
#pragma unroll
        for (int i = 0; i < kNumStats; ++i)
            if (cnt.v[i]) atomicAdd(&block_stats[i], (unsigned long long)cnt.v[i]);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();  // tcgen05.dealloc needs the whole warp
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
    if (p.stats && threadIdx.x < kNumStats && block_stats[threadIdx.x])
        atomicAdd(p.stats + threadIdx.x, block_stats[threadIdx.x]);
}

// Last view whose first item is <= item (views without items share the
// next view's first item, so they are skipped).
__device__ __forceinline__ int find_batch_view(const long long *begin, int nviews, long long item) {
    int lo = 0, hi = nviews - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(begin + mid) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The learned views of a batch: the packed-group kernel made persistent.
// The producers take groups (items of 8 tiles) from a global counter, find
// the group's view, copy its parameters and network into the stage and run
// step 1 and the features as for one view; the consumer runs the chains and
// the gather with the stage's copies, and reloads the operand image when a
// group's network is not the one in shared memory (between chains, when no
// MMA is in flight).  A stage whose view slot is -1 ends the CTA's work.
struct PfBatch {
    const BatchViewDev *views;
    const int *index;
    const long long *item_begin;
    int nkind, nviews;
    long long total_items;
    unsigned long long *counter;
    unsigned long long *stats;
    int *err;
};

template <int ALG, int TW, int MD, bool kStats>
__global__ void __launch_bounds__(kPThreads, kPCtasPerSm) mlp_batch_pf_kernel(const PfBatch b, const MlpDevice m0) {
    constexpr bool kList = ALG == ALG_LIST;
    constexpr int kPStages = PLayout<false, kList, true>::kStages;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ unsigned long long block_stats[kNumStats];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ListTable *T = kList && warp >= 4 ? reinterpret_cast<ListTable *>(sm + kPFbTab) + (warp - 4) : nullptr;
    if (kList && warp >= 4) {
#pragma unroll
        for (int q = 0; q < 8; ++q) T->keys[lane * 8 + q] = kEmpty;
    }
    uint64_t *mma_bar = reinterpret_cast<uint64_t *>(sm + kPBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + kPTmem);
    if (threadIdx.x < kNumStats) block_stats[threadIdx.x] = 0;
    {
        const uint4 *src = m0.img;
        uint4 *dst = reinterpret_cast<uint4 *>(sm + kImgW1);
        for (int i = threadIdx.x; i < kImgBytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
        // every thread's part of the image, written through the generic
        // proxy, ordered before the MMAs that read it through the async proxy
        tc::fence_proxy_async();
    }
    if (threadIdx.x == 0) {
        tc::mbar_init(mma_bar, 1);
        for (int s = 0; s < kPStages; ++s) {
            tc::mbar_init(p_full(sm, s), kPProducerWarps);
            tc::mbar_init(p_done(sm, s), 1);
        }
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    Counters cnt;
#pragma unroll
    for (int i = 0; i < kNumStats; ++i) cnt.v[i] = 0;
    int *err = b.err;

    if (warp < 4) {
        // ---------------- consumer ----------------
        if (kPSplitRegs) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kPConsumerRegs));
        const int tid = threadIdx.x;
        uint32_t phase = 0;
        const uint4 *loaded = m0.img;
        for (long long j = 0;; ++j) {
            const int s = (int)(j % kPStages);
            const uint32_t par = (uint32_t)((j / kPStages) & 1);
            unsigned char *st = p_stage<false, kList, true>(sm, s);
            bool ok = true;
            if (tid == 0) ok = tc::mbar_wait(p_full(sm, s), par, kMaxTries);
            __syncwarp();
            if (bar_or<1, kRows>(!ok)) {
                if (tid == 0) atomicExch(err, CTF_ERR_TIMEOUT);
                break;
            }
            const int *bm = reinterpret_cast<const int *>(st + kPBat);
            if (bm[0] < 0) break;  // no more groups
            const long long first = *reinterpret_cast<const long long *>(st + kPBat + 8);
            const ExactParams &p = *reinterpret_cast<const ExactParams *>(st + kPBat + 16);
            const MlpDevice &m = *reinterpret_cast<const MlpDevice *>(st + kPBat + 16 + sizeof(ExactParams));
            if (m.img != loaded) {
                // another network: its operand image (every MMA of the last chain is done)
                const uint4 *src = m.img;
                uint4 *dst = reinterpret_cast<uint4 *>(sm + kImgW1);
                for (int i = tid; i < kImgBytes / 16; i += kRows) dst[i] = __ldg(src + i);
                tc::fence_proxy_async();  // generic-proxy writes -> the MMAs' async proxy
                cons_bar();
                loaded = m.img;
            }
            const bool fp8 = m.fp8 != 0;
            const int R = *reinterpret_cast<const int *>(st + kPRows);
            const int passes = (R + kRows - 1) / kRows;
            float4 *outrow = reinterpret_cast<float4 *>(st + kPX);
            const uint32_t sX = tc::smem_addr(st + kPX);
            for (int c = 0; c < passes && ok; ++c) {
                const bool live = kRows * c + 32 * warp < R;
                float4 v;
                ok = p_chain(sm, tmem, mma_bar, phase, sX + 4096u * (uint32_t)c, fp8, live, v, err);
                if (ok && live) outrow[ck(kRows * c + tid, 2 * kRows, err, kBndRow)] = v;
                cons_bar();
            }
            if (!ok) break;
            {
                const TilePos tpc = tile_pos0(p, first);
#pragma unroll 1
                for (int k = 0; k < 2; ++k) p_gather<TW, false>(p, tpc, 4 * k + warp, st, tid & 31, nullptr);
            }
            __syncwarp();
            cons_bar();  // every consumer warp has read the stage
            if (tid == 0) p_arrive(p_done(sm, s));
        }
    } else {
        // ---------------- producers ----------------
        if (kPSplitRegs) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kPProducerRegs));
        const int pw = warp - 4;
        const uint32_t lt = lanemask_lt();
        int *ranks = reinterpret_cast<int *>(sm + kPRanks) + 64 * pw;
        int2 *list = reinterpret_cast<int2 *>(sm + kPList);
        const int pt = threadIdx.x - kRows;  // producer thread
        for (long long j = 0;; ++j) {
            const int s = (int)(j % kPStages);
            unsigned char *st = p_stage<false, kList, true>(sm, s);
            if (j >= kPStages) {
                // the consumer has gathered group j - kPStages from this stage
                bool okd = true;
                if (lane == 0) okd = tc::mbar_wait(p_done(sm, s), (uint32_t)(((j - kPStages) / kPStages) & 1), kMaxTries);
                __syncwarp();
                if (bar_or<2, kPProducerThreads>(!okd)) {
                    if (threadIdx.x == 128) atomicExch(err, CTF_ERR_TIMEOUT);
                    break;
                }
            }
            // every producer warp has read the texel lists of the last group
            __syncwarp();
            prod_bar();
            int *bm = reinterpret_cast<int *>(st + kPBat);
            if (pt == 0) *reinterpret_cast<long long *>(st + kPBat + 8) = (long long)atomicAdd(b.counter, 1ull);
            prod_bar();
            const long long item = *reinterpret_cast<volatile long long *>(st + kPBat + 8);
            if (item >= b.total_items) {
                if (pt == 0) bm[0] = -1;
                __syncwarp();
                if (lane == 0) p_arrive(p_full(sm, s));
                break;
            }
            const int vk = ck(find_batch_view(b.item_begin, b.nkind, item), b.nkind, err, kBndBatch);
            const BatchViewDev *V = b.views + ck(__ldg(b.index + vk), b.nviews, err, kBndBatch);
            {
                // the view's parameters and network into the stage
                const uint4 *src = reinterpret_cast<const uint4 *>(&V->p);
                uint4 *dst = reinterpret_cast<uint4 *>(st + kPBat + 16);
                if (pt < (int)(sizeof(ExactParams) / 16)) dst[pt] = __ldg(src + pt);
                const uint2 *msrc = reinterpret_cast<const uint2 *>(&V->m);
                uint2 *mdst = reinterpret_cast<uint2 *>(st + kPBat + 16 + sizeof(ExactParams));
                if (pt < (int)(sizeof(MlpDevice) / 8)) mdst[pt] = __ldg(msrc + pt);
            }
            const long long first = (item - __ldg(b.item_begin + vk)) * kGroupTiles;
            prod_bar();  // the copies are in place
            if (pt == 0) {
                bm[0] = vk;
                *reinterpret_cast<long long *>(st + kPBat + 8) = first;
            }
            const ExactParams &p = *reinterpret_cast<const ExactParams *>(st + kPBat + 16);
            const MlpDevice &m = *reinterpret_cast<const MlpDevice *>(st + kPBat + 16 + sizeof(ExactParams));
            const bool fp8 = m.fp8 != 0;
            const float *inv_a1 = reinterpret_cast<const float *>(reinterpret_cast<const unsigned char *>(m.img) + kImgA1);
            const TilePos tp = tile_pos0(p, first);
#pragma unroll 1
            for (int k = 0; k < kPSlots; ++k)
                p_step1<ALG, TW, MD, kStats, false>(p, tp, first, kPSlots * pw + k, st, list, lane, lt, ranks, cnt,
                                                    nullptr, T);
            __syncwarp();
            prod_bar();  // every slot's list and count is in place
            const int *count = reinterpret_cast<const int *>(st + kPCount);
            int R = 0, g0 = 0, b0 = 0, g1 = 0, b1 = 0, mybase = 0;
#pragma unroll
            for (int g = 0; g < kGroupTiles; ++g) {
                if (pt >= R) {
                    g0 = g;
                    b0 = R;
                }
                if (pt + kPProducerThreads >= R) {
                    g1 = g;
                    b1 = R;
                }
                if (pt == g) mybase = R;
                R += count[g];
            }
            if (pt < kGroupTiles) reinterpret_cast<int *>(st + kPBase)[pt] = mybase;
            if (pt == 0) {
                *reinterpret_cast<int *>(st + kPRows) = R;
                if (kStats) cnt.v[kStatTexelEvalsUnique] += R;
            }
#pragma unroll 1
            for (int c = 0; c < kPFeatRounds; ++c) {
                const int row = pt + kPProducerThreads * c;
                if (row >= R) break;
                const int2 t = c == 0 ? list[32 * g0 + ck(row - b0, 32, err, kBndTexList)]
                                      : list[32 * g1 + ck(row - b1, 32, err, kBndTexList)];
                float f[kMlpIn];
                texel_features(m, t.x, t.y, f);
                store_x_row_at(st + kPX, ck(row, 2 * kRows, err, kBndRow), f, fp8, inv_a1);
            }
            tc::fence_proxy_async();  // generic-proxy writes -> the MMAs' async proxy
            __syncwarp();
            if (lane == 0) p_arrive(p_full(sm, s));
        }
    }

    if (kStats && b.stats && lane == 0) {
#pragma unroll
        for (int i = 0; i < kNumStats; ++i)
            if (cnt.v[i]) atomicAdd(&block_stats[i], (unsigned long long)cnt.v[i]);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();  // tcgen05.dealloc needs the whole warp
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
    if (kStats && b.stats && threadIdx.x < kNumStats && block_stats[threadIdx.x])
        atomicAdd(b.stats + threadIdx.x, block_stats[threadIdx.x]);
}

using PfFn = void (*)(const ExactParams, const MlpDevice, int *);

// Variants: kPlain, kFallback (C / C+ on Box and Mask), kTwoTexels (two
// texels per lane on List Merge, Box and Mask).
enum { kPlain = 0, kFallback = 1, kTwoTexels = 2 };

template <int TW, bool kStats, int kVar>
PfFn pf_pick(int alg, int md) {
    constexpr bool kFb = kVar == kFallback, kTwo = kVar == kTwoTexels;
    switch (alg) {
    case ALG_STF: return kVar == kPlain ? mlp_filter_pf_kernel<ALG_STF, TW, 16, kStats, false, false> : nullptr;
    case ALG_LIST: return kFb ? nullptr : mlp_filter_pf_kernel<ALG_LIST, TW, 16, kStats, false, kTwo>;
    case ALG_BOX: return mlp_filter_pf_kernel<ALG_BOX, TW, 16, kStats, kFb, kTwo>;
    case ALG_MASK:
        return md == 11 ? mlp_filter_pf_kernel<ALG_MASK, TW, 11, kStats, kFb, kTwo>
                        : mlp_filter_pf_kernel<ALG_MASK, TW, 16, kStats, kFb, kTwo>;
    default: return nullptr;
    }
}

template <int TW, bool kStats>
PfFn pf_pick_var(int alg, int md, int var) {
    switch (var) {
    case kPlain: return pf_pick<TW, kStats, kPlain>(alg, md);
    case kFallback: return pf_pick<TW, kStats, kFallback>(alg, md);
    case kTwoTexels: return pf_pick<TW, kStats, kTwoTexels>(alg, md);
    default: return nullptr;
    }
}

PfFn pf_kernel(int alg, int tile_w, int mask_dim, bool st, int var) {
    switch (tile_w) {
    case 8: return st ? pf_pick_var<8, true>(alg, mask_dim, var) : pf_pick_var<8, false>(alg, mask_dim, var);
    case 4: return st ? pf_pick_var<4, true>(alg, mask_dim, var) : pf_pick_var<4, false>(alg, mask_dim, var);
    case 16: return st ? pf_pick_var<16, true>(alg, mask_dim, var) : pf_pick_var<16, false>(alg, mask_dim, var);
    default: return nullptr;
    }
}

cudaError_t pf_prepare(PfFn fn, int smem_bytes) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(dev, reinterpret_cast<const void *>(fn));
    if (done.count(key)) return cudaSuccess;
    // setmaxnreg.inc waits until the consumer has released what it asks for:
    // the split only adds up if the kernel starts with kPLaunchRegs registers
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if (kPSplitRegs ? fa.numRegs != kPLaunchRegs : fa.numRegs > kPLaunchRegs) return cudaErrorInvalidDeviceFunction;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e == cudaSuccess) done.insert(key);
    return e;
}

int pf_smem(int var, int alg) {
    return var == kFallback ? PLayout<true>::kBytes
                            : (alg == ALG_LIST ? PLayout<false, true>::kBytes : PLayout<false>::kBytes);
}

}  // namespace

bool mlp_filter_pf_fallback_applies(const ExactParams &p, int alg) {
    return (alg == ALG_BOX || alg == ALG_MASK) && p.fallback != 0 && p.tpl == 1 && !p.group_dedup;
}

bool mlp_filter_pf_two_applies(const ExactParams &p, int alg) {
    return (alg == ALG_LIST || alg == ALG_BOX || alg == ALG_MASK) && p.fallback == 0 && p.tpl == 2 && !p.group_dedup;
}

cudaError_t prepare_mlp_filter_pf(int alg, int tile_w, int mask_dim) {
    for (int var = kPlain; var <= kTwoTexels; ++var) {
        for (int st = 0; st < 2; ++st) {
            PfFn fn = pf_kernel(alg, tile_w, mask_dim, st != 0, var);
            if (!fn) continue;  // no such variant for this algorithm
            const cudaError_t e = pf_prepare(fn, pf_smem(var, alg));
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_mlp_filter_pf(const ExactParams &p, const MlpDevice &m, int alg, int tile_w, int mask_dim, int *err,
                                 cudaStream_t stream) {
    const int var = p.fallback != 0 ? kFallback : (p.tpl == 2 ? kTwoTexels : kPlain);
    if (var == kFallback && !mlp_filter_pf_fallback_applies(p, alg)) return cudaErrorInvalidValue;
    if (var == kTwoTexels && !mlp_filter_pf_two_applies(p, alg)) return cudaErrorInvalidValue;
    PfFn fn = pf_kernel(alg, tile_w, mask_dim, p.stats != nullptr, var);
    if (!fn) return cudaErrorInvalidValue;
    if (p.n_tiles == 0) return cudaSuccess;
    if (p.n_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;  // tile positions use 32-bit arithmetic
    cudaError_t e = pf_prepare(fn, pf_smem(var, alg));
    if (e != cudaSuccess) return e;
    const int gt = var == kTwoTexels ? kGroupTiles / 2 : kGroupTiles;
    const long long groups = (p.n_tiles + gt - 1) / gt;
    const long long cap = (long long)device_sm_count() * kPCtasPerSm;
    const int grid = (int)(groups < cap ? groups : cap);
    fn<<<grid, kPThreads, pf_smem(var, alg), stream>>>(p, m, err);
    return cudaGetLastError();
}

namespace {
using BatchPfFn = void (*)(const PfBatch, const MlpDevice);

template <int TW, bool kStats>
BatchPfFn batch_pf_pick(int alg, int md) {
    switch (alg) {
    case ALG_STF: return mlp_batch_pf_kernel<ALG_STF, TW, 16, kStats>;
    case ALG_LIST: return mlp_batch_pf_kernel<ALG_LIST, TW, 16, kStats>;
    case ALG_BOX: return mlp_batch_pf_kernel<ALG_BOX, TW, 16, kStats>;
    case ALG_MASK: return md == 11 ? mlp_batch_pf_kernel<ALG_MASK, TW, 11, kStats> : mlp_batch_pf_kernel<ALG_MASK, TW, 16, kStats>;
    default: return nullptr;
    }
}

BatchPfFn batch_pf_kernel(int alg, int tile_w, int md, bool st) {
    switch (tile_w) {
    case 8: return st ? batch_pf_pick<8, true>(alg, md) : batch_pf_pick<8, false>(alg, md);
    case 4: return st ? batch_pf_pick<4, true>(alg, md) : batch_pf_pick<4, false>(alg, md);
    case 16: return st ? batch_pf_pick<16, true>(alg, md) : batch_pf_pick<16, false>(alg, md);
    default: return nullptr;
    }
}

int batch_pf_smem(int alg) {
    return alg == ALG_LIST ? PLayout<false, true, true>::kBytes : PLayout<false, false, true>::kBytes;
}
}  // namespace

bool mlp_batch_pf_applies(int alg, int group_dedup) {
    return (alg == ALG_STF || alg == ALG_LIST || alg == ALG_BOX || alg == ALG_MASK) && !group_dedup;
}

cudaError_t prepare_mlp_batch_pf(int alg, int tile_w, int mask_dim) {
    for (int st = 0; st < 2; ++st) {
        BatchPfFn fn = batch_pf_kernel(alg, tile_w, mask_dim, st != 0);
        if (!fn) return cudaErrorInvalidValue;
        const cudaError_t e = pf_prepare(reinterpret_cast<PfFn>(fn), batch_pf_smem(alg));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_mlp_batch_pf(const BatchViewDev *views, int nviews, const int *index, const long long *item_begin,
                                int nkind, long long total_items, unsigned long long *counter, unsigned long long *stats,
                                int *err, const MlpDevice &m0, int alg, int tile_w, int mask_dim, cudaStream_t s) {
    BatchPfFn fn = batch_pf_kernel(alg, tile_w, mask_dim, stats != nullptr);
    if (!fn) return cudaErrorInvalidValue;
    if (total_items <= 0) return cudaSuccess;
    cudaError_t e = pf_prepare(reinterpret_cast<PfFn>(fn), batch_pf_smem(alg));
    if (e != cudaSuccess) return e;
    PfBatch b;
    b.views = views;
    b.index = index;
    b.item_begin = item_begin;
    b.nkind = nkind;
    b.nviews = nviews;
    b.total_items = total_items;
    b.counter = counter;
    b.stats = stats;
    b.err = err;
    const long long cap = (long long)device_sm_count() * kPCtasPerSm;
    const int grid = (int)(total_items < cap ? total_items : cap);
    fn<<<grid, kPThreads, batch_pf_smem(alg), s>>>(b, m0);
    return cudaGetLastError();
}

}  // namespace ctf
