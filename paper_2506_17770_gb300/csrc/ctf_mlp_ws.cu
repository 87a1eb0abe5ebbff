// ctf_mlp_ws.cu -- learned-decode filter with warps specialised by role, for
// STF, Box and Mask Sampling on single views (with or without group_dedup).
//
// A CTA of 256 threads (four per SM) takes the groups of 8 pixel tiles g0,
// g0 + G, ... (G = gridDim.x) in turn:
//   - warpgroup 0 (warps 0-3, the consumer, 80 registers) owns the 128 TMEM
//     lanes: for each group it packs the texel lists of the 8 tiles into
//     rows, computes their features and runs the tcgen05 MLP chain(s) into a
//     row-value buffer;
//   - warpgroup 1 (warps 4-7, the producers, 48 registers, two tiles of the
//     group each) runs step 1 of the collaborative flow for the next group
//     while the consumer's MMAs execute, and gathers, filters and stores the
//     pixels of the previous group from its row values.
// The CTA is launched with 64 registers per thread; the warpgroups then move
// registers from the producers to the consumer with setmaxnreg (128 x 80 +
// 128 x 48 = 256 x 64, so the increase is always granted).
// Two stages of group buffers (texel lists, per-pixel words, tile counts,
// row values, row map) alternate between consecutive groups.  Four pairs of mbarriers
// hand them over: full (step 1 done), empty (lists read), done (row values
// written), gathered (row values read).  Every wait is bounded; a wait that
// gives up records CTF_ERR_TIMEOUT and the waiting role stops, so the kernel
// always ends.  Each group gets the same rows, texel values, image and counts
// as mlp_group in ctf_mlp_chain.cuh; with group_dedup the consumer merges
// the group's lists in a hash table first, so that each distinct texel takes
// one row, and a per-stage row map sends every list entry to its row.
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

namespace ctf {
namespace {

constexpr int kWsThreads = 256;
constexpr int kWsProducerWarps = 4;
constexpr int kWsLaunchRegs = 64, kWsConsumerRegs = 80, kWsProducerRegs = 48;
static_assert(128 * kWsConsumerRegs + 32 * kWsProducerWarps * kWsProducerRegs == kWsThreads * kWsLaunchRegs,
              "the register split adds up to the launch's registers");
constexpr int kWsSlotsPerProducer = kGroupTiles / kWsProducerWarps;  // pixel tiles of the group per producer warp

// Shared memory: the chain's operand image, X, H, MMA barrier and TMEM slot
// (ctf_mlp_chain.cuh offsets below kSmList), then the producers' Mask rank
// slots, two stages of group buffers and the hand-over barriers.
constexpr int kWsRanks = kSmList;                            // producer warps x 32 ints
constexpr int kWsStage0 = kWsRanks + kWsProducerWarps * 32 * 4;
constexpr int kWsTex = 0;                                    // 256 x int2 texel lists (slot g at 32 g)
constexpr int kWsST = kWsTex + 256 * 8;                      // 256 x float2 (s, t)
constexpr int kWsInfo = kWsST + 256 * 8;                     // 256 x uint32 per-pixel words
constexpr int kWsCount = kWsInfo + 256 * 4;                  // 8 x int texels per tile (producers)
constexpr int kWsBase = kWsCount + 32;                       // 8 x int first row per tile (consumer)
constexpr int kWsOut = kWsBase + 32;                         // 256 x float4 row values
constexpr int kWsRowMap = kWsOut + 256 * 16;                 // 256 x u8 list entry -> row (group_dedup)
constexpr int kWsStageBytes = kWsRowMap + 256;
constexpr int kWsBars = kWsStage0 + 2 * kWsStageBytes;       // full[2], empty[2], done[2], gathered[2]
constexpr int kWsBytes = kWsBars + 8 * 8;
static_assert(kWsStage0 % 16 == 0 && kWsStageBytes % 16 == 0 && kWsOut % 16 == 0, "16-byte buffers");
// four CTAs per SM: 4 x 128 TMEM columns, shared memory and 256 x 64 registers each
static_assert(4 * (kWsBytes + 1024 + 128) <= 228 * 1024, "four CTAs per SM fit");
static_assert(5 * kWsThreads * kWsLaunchRegs > 65536, "a fifth CTA, which would find no free TMEM, never fits");

__device__ __forceinline__ unsigned char *ws_stage(unsigned char *sm, int s) {
    return sm + kWsStage0 + s * kWsStageBytes;
}

__device__ __forceinline__ uint64_t *ws_bar(unsigned char *sm, int kind, int s) {
    return reinterpret_cast<uint64_t *>(sm + kWsBars) + 2 * kind + s;
}
enum { kBarFull = 0, kBarEmpty = 1, kBarDone = 2, kBarGathered = 3 };

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(bar)) : "memory");
}

// Barrier 1 among the 128 consumer threads (barrier 0 stays __syncthreads).
__device__ __forceinline__ void cons_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// The same barrier, returning whether any consumer thread passed true.
__device__ __forceinline__ bool cons_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, 1, 128, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

// Hidden epilogue in two halves of 32 columns (fewer live registers than the
// one-pass form): TMEM columns [col, col + 64) of this thread's row -> bias,
// ReLU -> the next layer's A operand, as in hidden_epilogue.
__device__ __forceinline__ void ws_hidden_epilogue(unsigned char *sm, uint32_t taddr, const float *bias,
                                                   const float *oscale, bool fp8, int row) {
    unsigned char *H = sm + kSmH;
    const float2 *b2 = reinterpret_cast<const float2 *>(bias);
    const float2 *o2 = reinterpret_cast<const float2 *>(oscale);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float d[32];
        tc::tmem_ld16(taddr + 32 * half, d);
        tc::tmem_ld16(taddr + 32 * half + 16, d + 16);
        tc::tmem_wait_ld();
        tc::regs_after_wait<32>(d);
        if (!fp8) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                uint32_t w[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int k = 8 * c + 2 * i, kk = 32 * half + k;
                    const float2 t = __fadd2_rn(make_float2(d[k], d[k + 1]), b2[kk / 2]);
                    w[i] = relu_half2(t.x, t.y);
                }
                *reinterpret_cast<uint4 *>(H + core_offset(row, 32 * half + 8 * c, 64, 2)) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                uint32_t w[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int k = 16 * c + 4 * i, kk = 32 * half + k;
                    const float2 t0 = __ffma2_rn(make_float2(d[k], d[k + 1]), o2[kk / 2], b2[kk / 2]);
                    const float2 t1 = __ffma2_rn(make_float2(d[k + 2], d[k + 3]), o2[kk / 2 + 1], b2[kk / 2 + 1]);
                    w[i] = (uint32_t)relu_e4m3x2(t0.x, t0.y) | ((uint32_t)relu_e4m3x2(t1.x, t1.y) << 16);
                }
                *reinterpret_cast<uint4 *>(H + core_offset(row, 32 * half + 16 * c, 64, 1)) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    }
}

// The three layers for the 128 rows whose layer-1 operand the consumer
// threads have written; mlp_chain with the consumer barrier in place of the
// CTA barrier.  Returns false (for every consumer thread alike) if an MMA
// did not complete within the wait bound.
__device__ __forceinline__ bool ws_chain(Chain &ch, bool fp8, float4 &out, int *err) {
    const int tid = threadIdx.x, warp = tid >> 5;
    unsigned char *sm = ch.sm;
    const float *b1 = reinterpret_cast<const float *>(sm + kImgB1);
    const float *b2 = reinterpret_cast<const float *>(sm + kImgB2);
    const float *b3 = reinterpret_cast<const float *>(sm + kImgB3);
    const float *s1 = reinterpret_cast<const float *>(sm + kImgS1);
    const float *s2 = reinterpret_cast<const float *>(sm + kImgS2);
    const float *s3 = reinterpret_cast<const float *>(sm + kImgS3);
    const uint32_t lane_base = ch.tmem + ((uint32_t)(32 * warp) << 16);
    const uint32_t sX = tc::smem_addr(sm + kSmX), sH = tc::smem_addr(sm + kSmH);
    const uint32_t sW1 = tc::smem_addr(sm + kImgW1), sW2 = tc::smem_addr(sm + kImgW2),
                   sW3 = tc::smem_addr(sm + kImgW3);
    const uint32_t kstep_bytes = 256;
    const uint32_t sboX = 256u;
    const uint32_t sboH = fp8 ? 512u : 1024u;
    const int nk_h = fp8 ? 2 : 4;
    const uint32_t id64 = fp8 ? tc::idesc_e4m3(128, 64) : tc::idesc_f16(128, 64);
    const uint32_t id16 = fp8 ? tc::idesc_e4m3(128, 16) : tc::idesc_f16(128, 16);

    bool timed_out = false;
    // ---- layer 1: D[0..64) = X * W1^T
    tc::fence_proxy_async();
    tc::fence_before_sync();
    cons_sync();
    if (tid == 0) {
        tc::fence_after_sync();
        const uint64_t a = tc::smem_desc(sX, 128, sboX), b = tc::smem_desc(sW1, 128, sboX);
        if (fp8) tc::mma_e4m3(ch.tmem, a, b, id64, false);
        else tc::mma_f16(ch.tmem, a, b, id64, false);
        tc::commit(ch.bar);
    }
    timed_out |= !tc::mbar_wait(ch.bar, ch.phase, kMaxTries);
    __syncwarp();
    ch.phase ^= 1u;
    tc::fence_after_sync();
    ws_hidden_epilogue(sm, lane_base + 0, b1, s1, fp8, tid);
    // ---- layer 2: D[64..128) = H1 * W2^T
    tc::fence_proxy_async();
    tc::fence_before_sync();
    if (cons_or(timed_out)) {
        if (tid == 0) atomicExch(err, CTF_ERR_TIMEOUT);
        return false;
    }
    if (tid == 0) {
        tc::fence_after_sync();
        for (int j = 0; j < nk_h; ++j) {
            const uint64_t a = tc::smem_desc(sH + j * kstep_bytes, 128, sboH);
            const uint64_t b = tc::smem_desc(sW2 + j * kstep_bytes, 128, sboH);
            if (fp8) tc::mma_e4m3(ch.tmem + 64, a, b, id64, j > 0);
            else tc::mma_f16(ch.tmem + 64, a, b, id64, j > 0);
        }
        tc::commit(ch.bar);
    }
    timed_out |= !tc::mbar_wait(ch.bar, ch.phase, kMaxTries);
    __syncwarp();
    ch.phase ^= 1u;
    tc::fence_after_sync();
    // the layer-2 MMAs have read H1, so H2 may overwrite it
    ws_hidden_epilogue(sm, lane_base + 64, b2, s2, fp8, tid);
    // ---- layer 3: D[0..16) = H2 * W3^T
    tc::fence_proxy_async();
    tc::fence_before_sync();
    if (cons_or(timed_out)) {
        if (tid == 0) atomicExch(err, CTF_ERR_TIMEOUT);
        return false;
    }
    if (tid == 0) {
        tc::fence_after_sync();
        for (int j = 0; j < nk_h; ++j) {
            const uint64_t a = tc::smem_desc(sH + j * kstep_bytes, 128, sboH);
            const uint64_t b = tc::smem_desc(sW3 + j * kstep_bytes, 128, sboH);
            if (fp8) tc::mma_e4m3(ch.tmem, a, b, id16, j > 0);
            else tc::mma_f16(ch.tmem, a, b, id16, j > 0);
        }
        tc::commit(ch.bar);
    }
    timed_out |= !tc::mbar_wait(ch.bar, ch.phase, kMaxTries);
    __syncwarp();
    ch.phase ^= 1u;
    tc::fence_after_sync();
    float d[16];
    tc::tmem_ld16(lane_base + 0, d);
    tc::tmem_wait_ld();
    tc::regs_after_wait<16>(d);
    float o[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float v = fp8 ? __fmaf_rn(d[c], s3[c], b3[c]) : __fadd_rn(d[c], b3[c]);
        o[c] = fminf(fmaxf(v, 0.f), 1.f);
    }
    out = make_float4(o[0], o[1], o[2], o[3]);
    tc::fence_before_sync();
    if (cons_or(timed_out)) {
        if (tid == 0) atomicExch(err, CTF_ERR_TIMEOUT);
        return false;
    }
    return true;
}

// Producer: step 1 on tile slot g (this warp's) of the group whose first tile
// is `first`, into stage buffer st: the slot's texel list at texlist[32 g +
// rank], per pixel (s, t) and the packed word of mlp_group (bits 0-19 the
// list indices of its 4 taps on success, else of its own texel; 20-22 its
// count; 23 active; 24 inside; 25 success), and the slot's texel count.
template <int ALG, int TW, int MD>
__device__ __forceinline__ void ws_step1(const ExactParams &p, long long first, int g, unsigned char *st, int lane,
                                         uint32_t lt, int *ranks, Counters &cnt) {
    constexpr int TH = 32 / TW;
    const int tx = lane % TW, ty = lane / TW;
    int2 *texlist = reinterpret_cast<int2 *>(st + kWsTex);
    float2 *pix_st = reinterpret_cast<float2 *>(st + kWsST);
    uint32_t *pix_info = reinterpret_cast<uint32_t *>(st + kWsInfo);
    int *count = reinterpret_cast<int *>(st + kWsCount);
    const long long tile = first + g;
    const bool valid = tile < p.n_tiles;
    int bx = 0, by = 0;
    if (valid) tile_pos(tile_pos0(p, first), g, bx, by);
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
        sel = select_tile<ALG, MD, true, false>(p, ps, jac, px, py, lane, lt, nullptr, ranks, cnt);
    } else {
        sel.path = PATH_EMPTY;
        sel.A = 0;
        sel.produce = false;
        sel.count = 0;
        sel.my_rank = 0;
    }
    if (sel.produce)
        texlist[32 * g + ck(sel.my_rank, 32, p.err, kBndTexList)] =
            make_int2(min(max(sel.tx, 0), p.Wt - 1), min(max(sel.ty, 0), p.Ht - 1));
    const bool succ = sel.path == PATH_SUCCESS;
    if (lane == 0) count[g] = succ ? sel.n : __popc(sel.A);
    uint32_t info = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) info |= ((uint32_t)sel.rk[k] & 31u) << (5 * k);
    info = succ ? info : ((uint32_t)sel.my_rank & 31u);
    info |= ((uint32_t)sel.count << 20) | (ps.active ? 1u << 23 : 0u) | (inside ? 1u << 24 : 0u) |
            (succ ? 1u << 25 : 0u);
    pix_st[32 * g + lane] = make_float2(ps.s, ps.t);
    pix_info[32 * g + lane] = info;
}

// Producer: step 3 for tile slot g of the group at `first` from stage st
// (its row values written by the consumer): gather, filter, store.
template <int TW>
__device__ __forceinline__ void ws_gather(const ExactParams &p, long long first, int g, const unsigned char *st,
                                          int lane, bool dedup) {
    constexpr int TH = 32 / TW;
    const int tx = lane % TW, ty = lane / TW;
    const float2 *pix_st = reinterpret_cast<const float2 *>(st + kWsST);
    const uint32_t *pix_info = reinterpret_cast<const uint32_t *>(st + kWsInfo);
    const float4 *outrow = reinterpret_cast<const float4 *>(st + kWsOut);
    const uint32_t info = pix_info[32 * g + lane];
    if (!((info >> 24) & 1u)) return;  // outside the frame (or no tile)
    // the slot's first row, from the consumer (the other slots' counts may
    // already belong to a later group)
    const int base = reinterpret_cast<const int *>(st + kWsBase)[g];
    const unsigned char *rowmap = st + kWsRowMap + 32 * g;
    auto row_of = [&](uint32_t i) { return ck(dedup ? (int)rowmap[i] : base + (int)i, 2 * kRows, p.err, kBndRow); };
    int bx, by;
    tile_pos(tile_pos0(p, first), g, bx, by);
    const uint32_t idx =
        ck((uint32_t)(by * TH + ty) * (uint32_t)p.W + (uint32_t)(bx * TW + tx), view_pixels(p), p.err, kBndPixel);
    float4 result = make_float4(0.f, 0.f, 0.f, 0.f);
    uint8_t cv = 0;
    if ((info >> 23) & 1u) {
        if ((info >> 25) & 1u) {
            const float2 s = pix_st[32 * g + lane];
            float w[4];
            bilinear_weights(s.x, s.y, w);
            float2 rg = make_float2(0.f, 0.f), ba = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 t = outrow[row_of((info >> (5 * k)) & 31u)];
                const float2 wk = make_float2(w[k], w[k]);
                rg = __ffma2_rn(wk, make_float2(t.x, t.y), rg);
                ba = __ffma2_rn(wk, make_float2(t.z, t.w), ba);
            }
            result = make_float4(rg.x, rg.y, ba.x, ba.y);
            cv = (uint8_t)((info >> 20) & 7u);
        } else {
            result = outrow[row_of(info & 31u)];
            cv = 1;
        }
    }
    __stcs(p.out + idx, result);
    if (p.evals) p.evals[idx] = cv;
}

// kDedup: group_dedup (the variant without it carries no code for it).
template <int ALG, int TW, int MD, bool kDedup>
__global__ void __launch_bounds__(kWsThreads, 4) mlp_filter_ws_kernel(const ExactParams p, const MlpDevice m,
                                                                      int *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ unsigned long long block_stats[kNumStats];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < kNumStats) block_stats[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(ws_bar(sm, kBarFull, s), kWsProducerWarps);
            tc::mbar_init(ws_bar(sm, kBarEmpty, s), 1);
            tc::mbar_init(ws_bar(sm, kBarDone, s), 1);
            tc::mbar_init(ws_bar(sm, kBarGathered, s), kWsProducerWarps);
        }
    }
    Chain ch;
    chain_setup(ch, sm, m);  // operand image, MMA barrier, TMEM (warp 0); ends in a CTA barrier
    const float *inv_a1 = reinterpret_cast<const float *>(sm + kImgA1);
    const uint32_t lt = lanemask_lt();
    Counters cnt;
#pragma unroll
    for (int i = 0; i < kNumStats; ++i) cnt.v[i] = 0;
    const long long n_groups = (p.n_tiles + kGroupTiles - 1) / kGroupTiles;
    const long long G = gridDim.x;
    constexpr bool dedup = kDedup;

    if (warp < 4) {
        // ---------------- consumer ----------------
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kWsConsumerRegs));
        const int tid = threadIdx.x;
        for (long long j = 0;; ++j) {
            const long long grp = blockIdx.x + j * G;
            if (grp >= n_groups) break;
            const int s = (int)(j & 1);
            const uint32_t par = (uint32_t)((j >> 1) & 1);
            unsigned char *st = ws_stage(sm, s);
            if (cons_or(!tc::mbar_wait(ws_bar(sm, kBarFull, s), par, kMaxTries))) {
                if (tid == 0) atomicExch(err, CTF_ERR_TIMEOUT);
                break;
            }
            // the row values and row map of this stage are free once the
            // gather of group j - 2 is done (it always is by now: each
            // producer warp gathers group j - 2 before its step 1 of group j)
            if (j >= 2 && cons_or(!tc::mbar_wait(ws_bar(sm, kBarGathered, s), par ^ 1u, kMaxTries))) {
                if (tid == 0) atomicExch(err, CTF_ERR_TIMEOUT);
                break;
            }
            const int *count = reinterpret_cast<const int *>(st + kWsCount);
            int2 *texlist = reinterpret_cast<int2 *>(st + kWsTex);
            int R = 0;
            int2 xy[2] = {make_int2(0, 0), make_int2(0, 0)};
            if (dedup) {
                // the distinct texels of the group get rows in the order their
                // first list entries win a 512-slot hash table (in H, which no
                // MMA reads between chains); the row map sends every list
                // entry to its texel's row
                unsigned long long *hkey = reinterpret_cast<unsigned long long *>(sm + kSmH);
                unsigned char *hrow = sm + kSmH + 512 * 8;
                int *nuniq = reinterpret_cast<int *>(sm + kSmH + 512 * 8 + 512);
                for (int i = tid; i < 512; i += kRows) hkey[i] = ~0ull;
                if (tid == 0) *nuniq = 0;
                cons_sync();
                int slot[2] = {0, 0};
                bool has[2] = {false, false}, won[2] = {false, false};
                int2 t2[2] = {make_int2(0, 0), make_int2(0, 0)};
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int e = tid + kRows * c, g = e >> 5;
                    int n_g = count[0];
#pragma unroll
                    for (int k = 1; k < kGroupTiles; ++k) n_g = g == k ? count[k] : n_g;
                    if ((e & 31) < n_g) {
                        has[c] = true;
                        t2[c] = texlist[e];
                        const unsigned long long key =
                            ((unsigned long long)(uint32_t)t2[c].y << 32) | (uint32_t)t2[c].x;
                        unsigned h = (((uint32_t)t2[c].x * 0x9E3779B1u) ^ ((uint32_t)t2[c].y * 0x85EBCA77u)) >> 23;
                        // at most 256 keys in 512 slots: the probe always ends
                        for (int probe = 0; probe < 512; ++probe) {
                            const unsigned long long old = atomicCAS(&hkey[h], ~0ull, key);
                            if (old == ~0ull || old == key) {
                                won[c] = old == ~0ull;
                                slot[c] = (int)h;
                                break;
                            }
                            h = (h + 1) & 511u;
                        }
                    }
                }
                cons_sync();  // every list entry is in the table; the lists have been read
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (won[c]) {
                        const int row = ck(atomicAdd(nuniq, 1), 2 * kRows, p.err, kBndRow);
                        hrow[slot[c]] = (unsigned char)row;
                        texlist[row] = t2[c];  // the distinct texels reuse the list space
                    }
                }
                cons_sync();
                unsigned char *rowmap = st + kWsRowMap;
#pragma unroll
                for (int c = 0; c < 2; ++c)
                    if (has[c]) rowmap[tid + kRows * c] = hrow[slot[c]];
                R = *nuniq;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int row = kRows * c + tid;
                    if (row < R) xy[c] = texlist[row];
                }
            } else {
                // slot g owns rows [base_g, base_g + count[g]) in slot order
                int start[kGroupTiles];
#pragma unroll
                for (int g = 0; g < kGroupTiles; ++g) {
                    start[g] = R;
                    R += count[g];
                }
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int row = kRows * c + tid;
                    if (row < R) {
                        int g = 0;
#pragma unroll
                        for (int k = 1; k < kGroupTiles; ++k) g = row >= start[k] ? k : g;
                        int b = start[0];
#pragma unroll
                        for (int k = 1; k < kGroupTiles; ++k) b = k == g ? start[k] : b;
                        xy[c] = texlist[32 * g + ck(row - b, 32, p.err, kBndTexList)];
                    }
                }
                if (tid < kGroupTiles) reinterpret_cast<int *>(st + kWsBase)[tid] = start[tid];
            }
            if (tid == 0) cnt.v[kStatTexelEvalsUnique] += R;
            cons_sync();  // every consumer thread has read the lists, counts and distinct texels
            if (tid == 0) mbar_arrive(ws_bar(sm, kBarEmpty, s));
            float4 *outrow = reinterpret_cast<float4 *>(st + kWsOut);
            const int passes = (R + kRows - 1) / kRows;
            bool ok = true;
            for (int c = 0; c < passes && ok; ++c) {
                const int row = kRows * c + tid;
                if (row < R) {
                    const int2 t = c == 0 ? xy[0] : xy[1];
                    float f[kMlpIn];
                    texel_features(m, t.x, t.y, f);
                    store_x_row(sm, tid, f, m.fp8, inv_a1);
                } else {
                    store_zero_x_row(sm, tid);
                }
                float4 v;
                ok = ws_chain(ch, m.fp8, v, err);
                if (ok) outrow[ck(row, 2 * kRows, p.err, kBndRow)] = v;
            }
            if (!ok) break;
            cons_sync();  // every row value is written
            if (tid == 0) mbar_arrive(ws_bar(sm, kBarDone, s));
        }
    } else {
        // ---------------- producers: two tile slots per warp ----------------
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kWsProducerRegs));
        const int pw = warp - 4;
        int *ranks = reinterpret_cast<int *>(sm + kWsRanks) + 32 * pw;
        for (long long j = 0;; ++j) {
            const long long grp = blockIdx.x + j * G;
            const bool have = grp < n_groups;
            if (have) {
                const int s = (int)(j & 1);
                const uint32_t par = (uint32_t)((j >> 1) & 1);
                // the stage's lists are free once the consumer has read those of group j - 2
                if (j >= 2 && !__all_sync(FULL, tc::mbar_wait(ws_bar(sm, kBarEmpty, s), par ^ 1u, kMaxTries))) {
                    if (lane == 0) atomicExch(err, CTF_ERR_TIMEOUT);
                    break;
                }
#pragma unroll 1
                for (int k = 0; k < kWsSlotsPerProducer; ++k)
                    ws_step1<ALG, TW, MD>(p, grp * kGroupTiles, kWsSlotsPerProducer * pw + k, ws_stage(sm, s), lane, lt,
                                          ranks, cnt);
                __syncwarp();
                if (lane == 0) mbar_arrive(ws_bar(sm, kBarFull, s));
            }
            if (j >= 1) {
                // gather group j - 1 once its row values are written
                const int s1 = (int)((j - 1) & 1);
                const uint32_t par1 = (uint32_t)(((j - 1) >> 1) & 1);
                if (!__all_sync(FULL, tc::mbar_wait(ws_bar(sm, kBarDone, s1), par1, kMaxTries))) {
                    if (lane == 0) atomicExch(err, CTF_ERR_TIMEOUT);
                    break;
                }
#pragma unroll 1
                for (int k = 0; k < kWsSlotsPerProducer; ++k)
                    ws_gather<TW>(p, (grp - G) * kGroupTiles, kWsSlotsPerProducer * pw + k, ws_stage(sm, s1), lane,
                                  dedup);
                __syncwarp();
                if (lane == 0) mbar_arrive(ws_bar(sm, kBarGathered, s1));
            }
            if (!have) break;
        }
    }

    if (p.stats && lane == 0) {
#pragma unroll
        for (int i = 0; i < kNumStats; ++i)
            if (cnt.v[i]) atomicAdd(&block_stats[i], (unsigned long long)cnt.v[i]);
    }
    chain_teardown(ch);  // CTA barrier, then warp 0 frees the TMEM
    if (p.stats && threadIdx.x < kNumStats && block_stats[threadIdx.x])
        atomicAdd(p.stats + threadIdx.x, block_stats[threadIdx.x]);
}

using WsFn = void (*)(const ExactParams, const MlpDevice, int *);

template <int TW, bool kDedup>
WsFn ws_pick(int alg, int md) {
    switch (alg) {
    case ALG_STF: return mlp_filter_ws_kernel<ALG_STF, TW, 16, kDedup>;
    case ALG_BOX: return mlp_filter_ws_kernel<ALG_BOX, TW, 16, kDedup>;
    case ALG_MASK:
        return md == 11 ? mlp_filter_ws_kernel<ALG_MASK, TW, 11, kDedup> : mlp_filter_ws_kernel<ALG_MASK, TW, 16, kDedup>;
    default: return nullptr;
    }
}

cudaError_t ws_prepare(WsFn fn) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(dev, reinterpret_cast<const void *>(fn));
    if (done.count(key)) return cudaSuccess;
    // setmaxnreg.inc waits until the producers have released what it asks for:
    // the split only adds up if the kernel starts with kWsLaunchRegs registers
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if (fa.numRegs != kWsLaunchRegs) return cudaErrorInvalidDeviceFunction;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kWsBytes);
    if (e == cudaSuccess) done.insert(key);
    return e;
}

// Only the group_dedup variant is launched: without the option the
// producers compute the features themselves (ctf_mlp_ws2.cu).
WsFn ws_kernel(int alg, int tile_w, int mask_dim, bool dedup) {
    if (!dedup) return nullptr;
    switch (tile_w) {
    case 8: return ws_pick<8, true>(alg, mask_dim);
    case 4: return ws_pick<4, true>(alg, mask_dim);
    case 16: return ws_pick<16, true>(alg, mask_dim);
    default: return nullptr;
    }
}

}  // namespace

bool mlp_filter_ws_applies(const ExactParams &, int alg) {
    return alg == ALG_STF || alg == ALG_BOX || alg == ALG_MASK;
}

cudaError_t prepare_mlp_filter_ws(int alg, int tile_w, int mask_dim) {
    WsFn fn = ws_kernel(alg, tile_w, mask_dim, true);
    return fn ? ws_prepare(fn) : cudaErrorInvalidValue;
}

cudaError_t launch_mlp_filter_ws(const ExactParams &p, const MlpDevice &m, int alg, int tile_w, int mask_dim,
                                 int *err, cudaStream_t stream) {
    WsFn fn = ws_kernel(alg, tile_w, mask_dim, p.group_dedup != 0);
    if (!fn) return cudaErrorInvalidValue;
    if (p.n_tiles == 0) return cudaSuccess;
    if (p.n_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;  // tile positions use 32-bit arithmetic
    cudaError_t e = ws_prepare(fn);
    if (e != cudaSuccess) return e;
    const long long groups = (p.n_tiles + kGroupTiles - 1) / kGroupTiles;
    const long long cap = (long long)device_sm_count() * 4;
    const int grid = (int)(groups < cap ? groups : cap);
    fn<<<grid, kWsThreads, kWsBytes, stream>>>(p, m, err);
    return cudaGetLastError();
}

}  // namespace ctf
