// ctf_mlp_chain.cuh -- the tcgen05 MLP chain of the learned texel decode for
// one 128-row tile (features -> three MMA layers -> RGBA per row), shared by
// the decode, filter and batched kernels.  See ctf_mlp.cu for the design.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "ctf_device.cuh"
#include "ctf_internal.h"
#include "ctf_mlp.cuh"
#include "ctf_select.cuh"
#include "tc_ops.cuh"

namespace ctf {
namespace {

constexpr int kRows = 128;
constexpr int kTmemCols = 128;
constexpr uint32_t kMaxTries = 1u << 24;  // bounded mbarrier polls (about a second)

// Dynamic shared memory of one CTA (offsets in bytes).
constexpr int kSmImg = 0;
constexpr int kSmX = 14080;              // A operand of layer 1: 128 x 32 B
constexpr int kSmH = kSmX + 4096;        // A operand of layers 2 and 3: 128 x 128 B
constexpr int kSmBar = kSmH + 16384;     // mbarrier (8 B)
constexpr int kSmTmem = kSmBar + 8;      // TMEM base address (4 B)
constexpr int kSmList = kSmBar + 64;     // List Merge tables (4 x ListTable)
constexpr int kSmRanks = kSmList + 4 * (int)sizeof(ListTable);  // Mask rank slots (4 x 32 ints)
// Packed groups of 8 tiles (collaborative algorithms and STF): per pixel the
// fractions (s, t) and a packed word, the texel value of every list row, the
// texels per tile; the texel lists themselves sit in the X buffer until the
// first chain overwrites it.
constexpr int kGroupTiles = 8;
constexpr int kSmPixST = kSmRanks + 4 * 32 * 4;       // 256 x float2
constexpr int kSmPixInfo = kSmPixST + 256 * 8;        // 256 x uint32
constexpr int kSmOut = kSmPixInfo + 256 * 4;          // 256 rows x float4
constexpr int kSmCount = kSmOut + 256 * 16;           // 8 x int
constexpr int kSmRowMap = kSmCount + kGroupTiles * 4;  // 256 x u8: list entry -> row (group_dedup)
constexpr int kSmNUnique = kSmRowMap + 256;           // int
constexpr int kSmTexList = kSmX;                      // 8 tiles x 32 x int2 (2 KB, inside X)
// group_dedup: a 512-slot hash table of texels and their rows, inside H
// (free between the chains of two groups)
constexpr int kSmHashKey = kSmH;                      // 512 x u64
constexpr int kSmHashRow = kSmH + 512 * 8;            // 512 x u8
constexpr int kSmBytes = kSmNUnique + 16;
// Reserve enough shared memory that at most 4 CTAs share an SM: 4 x 128 TMEM
// columns fill the SM's 512 (5 x 54 KB exceed the SM's 228 KB).
constexpr int kSmRequest = 54 * 1024;
static_assert(kSmBytes <= kSmRequest, "shared memory layout");
static_assert(5 * kSmRequest > 228 * 1024, "more than 4 CTAs per SM would overcommit TMEM");

// Tiles per CTA iteration of the learned filter: per-pixel 4-tap fills the
// 128 rows with one tile per warp and tap, the other algorithms pack the
// texel lists of two tiles per warp into as few 128-row chains as they need.
__host__ __device__ constexpr int mlp_group_tiles(int alg) { return alg == 0 ? 4 : kGroupTiles; }

struct Chain {
    unsigned char *sm;
    uint32_t tmem;
    uint64_t *bar;
    uint32_t phase;
};

// Position of tile first + g (0 <= g < 8) from the position of `first`: one
// 32-bit division per group instead of a 64-bit division per tile and phase
// (a view has fewer than 2^31 tiles).
struct TilePos {
    uint32_t bx0, by0, tiles_x;
};

__device__ __forceinline__ TilePos tile_pos0(const ExactParams &p, long long first) {
    TilePos t;
    t.tiles_x = (uint32_t)p.tiles_x;
    const uint32_t f = (uint32_t)first;
    t.by0 = f / t.tiles_x;
    t.bx0 = f - t.by0 * t.tiles_x;
    return t;
}

__device__ __forceinline__ void tile_pos(const TilePos &t, int g, int &bx, int &by) {
    uint32_t x = t.bx0 + (uint32_t)g, y = t.by0;
    while (x >= t.tiles_x) {
        x -= t.tiles_x;
        ++y;
    }
    bx = (int)x;
    by = (int)y;
}

// Features of texel (x, y) (inside the texture) in FP32.
__device__ __forceinline__ void texel_features(const MlpDevice &m, int x, int y, float f[kMlpIn]) {
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const float gx = __fsub_rn(__fmul_rn(__fadd_rn((float)x, 0.5f), m.sx[g]), 0.5f);
        const float gy = __fsub_rn(__fmul_rn(__fadd_rn((float)y, 0.5f), m.sy[g]), 0.5f);
        const float fx0 = floorf(gx), fy0 = floorf(gy);
        const float fx = __fsub_rn(gx, fx0), fy = __fsub_rn(gy, fy0);
        const int x0 = (int)fx0, y0 = (int)fy0;
        const int xa = min(max(x0, 0), m.gw[g] - 1), xb = min(max(x0 + 1, 0), m.gw[g] - 1);
        const int ya = min(max(y0, 0), m.gh[g] - 1), yb = min(max(y0 + 1, 0), m.gh[g] - 1);
        const uint4 *L = reinterpret_cast<const uint4 *>(m.lat[g]);
        const long long cells = (long long)m.gw[g] * m.gh[g];
        const uint4 q00 = __ldg(L + ck((size_t)ya * m.gw[g] + xa, cells, m.err, kBndLatent));
        const uint4 q10 = __ldg(L + ck((size_t)ya * m.gw[g] + xb, cells, m.err, kBndLatent));
        const uint4 q01 = __ldg(L + ck((size_t)yb * m.gw[g] + xa, cells, m.err, kBndLatent));
        const uint4 q11 = __ldg(L + ck((size_t)yb * m.gw[g] + xb, cells, m.err, kBndLatent));
        const float ofx = __fsub_rn(1.f, fx), ofy = __fsub_rn(1.f, fy);
        const float w00 = __fmul_rn(ofx, ofy), w10 = __fmul_rn(fx, ofy), w01 = __fmul_rn(ofx, fy),
                    w11 = __fmul_rn(fx, fy);
        const __half2 *h00 = reinterpret_cast<const __half2 *>(&q00);
        const __half2 *h10 = reinterpret_cast<const __half2 *>(&q10);
        const __half2 *h01 = reinterpret_cast<const __half2 *>(&q01);
        const __half2 *h11 = reinterpret_cast<const __half2 *>(&q11);
        // channels 2c and 2c+1 together: packed multiply and FMAs round each
        // component like their scalar forms
        const float2 v00 = make_float2(w00, w00), v10 = make_float2(w10, w10), v01 = make_float2(w01, w01),
                     v11 = make_float2(w11, w11);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float2 acc = __fmul2_rn(v00, __half22float2(h00[c]));
            acc = __ffma2_rn(v10, __half22float2(h10[c]), acc);
            acc = __ffma2_rn(v01, __half22float2(h01[c]), acc);
            acc = __ffma2_rn(v11, __half22float2(h11[c]), acc);
            f[g * 8 + 2 * c] = acc.x;
            f[g * 8 + 2 * c + 1] = acc.y;
        }
    }
}

__device__ __forceinline__ uint32_t pack_half2(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// relu(a), relu(b) as FP16 (a in the low half), round to nearest.
__device__ __forceinline__ uint32_t relu_half2(float a, float b) {
    uint32_t r;
    asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    return r;
}

// relu(a), relu(b) as E4M3 (a in the low byte), round to nearest, saturating.
__device__ __forceinline__ uint16_t relu_e4m3x2(float a, float b) {
    uint16_t r;
    asm("cvt.rn.satfinite.relu.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(b), "f"(a));
    return r;
}

// E4M3 pair: bytes of a (low) and b (high), round to nearest, saturating.
__device__ __forceinline__ uint16_t pack_e4m3x2(float a, float b) {
    const __nv_fp8x2_storage_t v = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    return (uint16_t)v;
}

// Row `row` of a layer-1 A operand at X (K-major core matrices, 32 bytes a
// row) from 16 features.
__device__ __forceinline__ void store_x_row_at(unsigned char *X, int row, const float f[kMlpIn], bool fp8,
                                               const float *inv_a) {
    if (!fp8) {
        uint4 c0 = make_uint4(pack_half2(f[0], f[1]), pack_half2(f[2], f[3]), pack_half2(f[4], f[5]),
                              pack_half2(f[6], f[7]));
        uint4 c1 = make_uint4(pack_half2(f[8], f[9]), pack_half2(f[10], f[11]), pack_half2(f[12], f[13]),
                              pack_half2(f[14], f[15]));
        *reinterpret_cast<uint4 *>(X + core_offset(row, 0, 16, 2)) = c0;
        *reinterpret_cast<uint4 *>(X + core_offset(row, 8, 16, 2)) = c1;
    } else {
        // K padded to 32: features 0..15 in the first 16-byte chunk, zeros after
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint16_t lo =
                pack_e4m3x2(__fmul_rn(f[4 * i], inv_a[4 * i]), __fmul_rn(f[4 * i + 1], inv_a[4 * i + 1]));
            const uint16_t hi =
                pack_e4m3x2(__fmul_rn(f[4 * i + 2], inv_a[4 * i + 2]), __fmul_rn(f[4 * i + 3], inv_a[4 * i + 3]));
            w[i] = (uint32_t)lo | ((uint32_t)hi << 16);
        }
        *reinterpret_cast<uint4 *>(X + core_offset(row, 0, 32, 1)) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4 *>(X + core_offset(row, 16, 32, 1)) = make_uint4(0u, 0u, 0u, 0u);
    }
}

// Row `row` of the layer-1 A operand of the chain area from 16 features.
__device__ __forceinline__ void store_x_row(unsigned char *sm, int row, const float f[kMlpIn], bool fp8,
                                            const float *inv_a) {
    store_x_row_at(sm + kSmX, row, f, fp8, inv_a);
}

__device__ __forceinline__ void store_zero_x_row(unsigned char *sm, int row) {
    unsigned char *X = sm + kSmX;
    *reinterpret_cast<uint4 *>(X + (row / 8) * 256 + (row % 8) * 16) = make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4 *>(X + (row / 8) * 256 + 128 + (row % 8) * 16) = make_uint4(0u, 0u, 0u, 0u);
}

// Hidden epilogue: TMEM columns [col, col+64) of this thread's row -> bias,
// ReLU -> next layer's A operand (FP16; or E4M3, with the output scale and
// the bias of an FP8 texture already multiplied on the host by the inverse
// activation scale of the next layer's input).
__device__ __forceinline__ void hidden_epilogue(unsigned char *sm, uint32_t taddr, const float *bias,
                                                const float *oscale, bool fp8, int row) {
    float d[64];
#pragma unroll
    for (int q = 0; q < 4; ++q) tc::tmem_ld16(taddr + 16 * q, d + 16 * q);
    tc::tmem_wait_ld();
    tc::regs_after_wait<64>(d);
    unsigned char *H = sm + kSmH;
    // Bias and scale in packed pairs; the ReLU is applied by the conversion
    // (the rounding of a negative value is not positive, and the positive
    // scales do not change signs).
    const float2 *b2 = reinterpret_cast<const float2 *>(bias);
    if (!fp8) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 8 * c + 2 * i;
                const float2 t = __fadd2_rn(make_float2(d[k], d[k + 1]), b2[k / 2]);
                w[i] = relu_half2(t.x, t.y);
            }
            *reinterpret_cast<uint4 *>(H + core_offset(row, 8 * c, 64, 2)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else {
        const float2 *o2 = reinterpret_cast<const float2 *>(oscale);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 16 * c + 4 * i;
                const float2 t0 = __ffma2_rn(make_float2(d[k], d[k + 1]), o2[k / 2], b2[k / 2]);
                const float2 t1 = __ffma2_rn(make_float2(d[k + 2], d[k + 3]), o2[k / 2 + 1], b2[k / 2 + 1]);
                w[i] = (uint32_t)relu_e4m3x2(t0.x, t0.y) | ((uint32_t)relu_e4m3x2(t1.x, t1.y) << 16);
            }
            *reinterpret_cast<uint4 *>(H + core_offset(row, 16 * c, 64, 1)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// The three layers for the 128 rows whose layer-1 operand is in place.
// Every thread of the CTA calls it; returns false (for every thread alike)
// if an MMA did not complete within the wait bound.
__device__ __forceinline__ bool mlp_chain(Chain &ch, bool fp8, float4 &out, int *err) {
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
    // K-major no-swizzle descriptors; one MMA covers K = 16 (FP16) or 32 (E4M3)
    const uint32_t esz = fp8 ? 1u : 2u;
    const uint32_t kstep_bytes = 256;  // two 16-byte core-matrix columns = 32 bytes of K per row group
    const uint32_t sboX = fp8 ? 256u : 256u;   // K = 32 B per row either way
    const uint32_t sboH = fp8 ? 512u : 1024u;  // 64 elements per row
    const int nk_h = fp8 ? 2 : 4;              // MMAs over K = 64
    const uint32_t id64 = fp8 ? tc::idesc_e4m3(128, 64) : tc::idesc_f16(128, 64);
    const uint32_t id16 = fp8 ? tc::idesc_e4m3(128, 16) : tc::idesc_f16(128, 16);
    (void)esz;

    bool timed_out = false;
    // ---- layer 1: D[0..64) = X * W1^T
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
        tc::fence_after_sync();
        const uint64_t a = tc::smem_desc(sX, 128, sboX), b = tc::smem_desc(sW1, 128, sboX);
        if (fp8) tc::mma_e4m3(ch.tmem, a, b, id64, false);
        else tc::mma_f16(ch.tmem, a, b, id64, false);
        tc::commit(ch.bar);
    }
    timed_out |= !tc::mbar_wait(ch.bar, ch.phase, kMaxTries);
    __syncwarp();  // the lanes may leave the wait apart; tcgen05.ld needs the whole warp
    ch.phase ^= 1u;
    tc::fence_after_sync();
    hidden_epilogue(sm, lane_base + 0, b1, s1, fp8, tid);
    // ---- layer 2: D[64..128) = H1 * W2^T
    tc::fence_proxy_async();
    tc::fence_before_sync();
    if (__syncthreads_or(timed_out)) {
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
    __syncwarp();  // the lanes may leave the wait apart; tcgen05.ld needs the whole warp
    ch.phase ^= 1u;
    tc::fence_after_sync();
    // the layer-2 MMAs have read H1, so H2 may overwrite it
    hidden_epilogue(sm, lane_base + 64, b2, s2, fp8, tid);
    // ---- layer 3: D[0..16) = H2 * W3^T
    tc::fence_proxy_async();
    tc::fence_before_sync();
    if (__syncthreads_or(timed_out)) {
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
    __syncwarp();  // the lanes may leave the wait apart; tcgen05.ld needs the whole warp
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
    if (__syncthreads_or(timed_out)) {
        if (tid == 0) atomicExch(err, CTF_ERR_TIMEOUT);
        return false;
    }
    return true;
}

// CTA set-up shared by both kernels: operand image into shared memory,
// mbarrier, 128 TMEM columns.
__device__ __forceinline__ void chain_setup(Chain &ch, unsigned char *sm, const MlpDevice &m) {
    const uint4 *src = m.img;
    uint4 *dst = reinterpret_cast<uint4 *>(sm + kSmImg);
    if (src)
        for (int i = threadIdx.x; i < kImgBytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    // every thread's part of the image, written through the generic proxy,
    // ordered before the MMAs that read it through the async proxy
    tc::fence_proxy_async();
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kSmBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + kSmTmem);
    if (threadIdx.x == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
    }
    if ((threadIdx.x >> 5) == 0) {
        tc::tmem_alloc(tslot, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    ch.sm = sm;
    ch.bar = bar;
    ch.tmem = *tslot;
    ch.phase = 0;
}

__device__ __forceinline__ void chain_teardown(const Chain &ch) {
    tc::fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        __syncwarp();  // tcgen05.dealloc needs the whole warp
        tc::fence_after_sync();
        tc::tmem_dealloc(ch.tmem, kTmemCols);
    }
}


// One iteration of the learned-decode filter for the calling warp's pixel
// tile `tile` of view p: step 1 of the collaborative flow, the warp's texels
// through the MLP chain (all 4 warps of the CTA call this together), the
// gather and filter, the store.  Returns false if the chain gave up.
template <int ALG, int TW, int MD>
__device__ __forceinline__ bool mlp_warp_tile(const ExactParams &p, const MlpDevice &m, Chain &ch, long long tile,
                                              int lane, uint32_t lt, ListTable *T, Counters &cnt,
                                              const float *inv_a1, int *err) {
    constexpr int TH = 32 / TW;
    unsigned char *sm = ch.sm;
    const int tx = lane % TW, ty = lane / TW;
    const float fW = (float)p.Wt, fH = (float)p.Ht;
    bool ok = true;
    const bool valid = tile < p.n_tiles;
    const uint32_t t32 = (uint32_t)tile, tiles_x = (uint32_t)p.tiles_x;  // fewer than 2^31 tiles
    const int by = valid ? (int)(t32 / tiles_x) : 0, bx = valid ? (int)(t32 - (uint32_t)by * tiles_x) : 0;
    const int px = bx * TW + tx, py = by * TH + ty;
    const bool inside = valid && px < p.W && py < p.H;
    const uint32_t idx = ck(inside ? (uint32_t)py * (uint32_t)p.W + (uint32_t)px : 0u, view_pixels(p), p.err,
                            kBndPixel);
    PixelSetup ps;
    float2 uv = make_float2(0.f, 0.f);
    float4 jac = make_float4(0.f, 0.f, 0.f, 0.f);
    bool covered = inside;
    if (inside) {
        uv = __ldcs(p.uv + idx);
        if (ALG >= ALG_LIST) jac = __ldcs(p.jac + idx);
        if (p.cov) covered = __ldcs(p.cov + idx) != 0;
    }
    ps.active = covered;
    setup_coords(uv, fW, fH, ps);

    float4 result = make_float4(0.f, 0.f, 0.f, 0.f);
    uint8_t count = 0;
    if (ALG == ALG_4TAP) {
        const uint32_t A = __ballot_sync(FULL, ps.active);
        if (valid) {
            cnt.v[kStatTilesTotal] += 1;
            if (A == 0) {
                cnt.v[kStatTilesEmpty] += 1;
            } else {
                cnt.v[kStatPixelsActive] += __popc(A);
                cnt.v[kStatTilesDirect] += 1;
                cnt.v[kStatTexelEvals] += 4 * __popc(A);
                cnt.v[kStatTexelEvalsUnique] += 4 * __popc(A);
            }
        }
        float4 tap[4];
#pragma unroll 1
        for (int k = 0; k < 4; ++k) {
            if (ps.active) {
                const int x = min(max(ps.ulx + (k & 1), 0), p.Wt - 1);
                const int y = min(max(ps.uly + (k >> 1), 0), p.Ht - 1);
                float f[kMlpIn];
                texel_features(m, x, y, f);
                store_x_row(sm, threadIdx.x, f, m.fp8, inv_a1);
            } else {
                store_zero_x_row(sm, threadIdx.x);
            }
            ok = mlp_chain(ch, m.fp8, tap[k], err);
            if (!ok) return false;
        }
        if (!ok) return false;
        if (ps.active) {
            float w[4];
            bilinear_weights(ps.s, ps.t, w);
            float r = 0.f, g = 0.f, b = 0.f, a = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                r = __fmaf_rn(w[k], tap[k].x, r);
                g = __fmaf_rn(w[k], tap[k].y, g);
                b = __fmaf_rn(w[k], tap[k].z, b);
                a = __fmaf_rn(w[k], tap[k].w, a);
            }
            result = make_float4(r, g, b, a);
            count = 4;
        }
    } else {
        Selection sel;
        if (valid) {
            sel = select_tile<ALG, MD, true>(p, ps, jac, px, py, lane, lt, T,
                                          reinterpret_cast<int *>(sm + kSmRanks) + 32 * (threadIdx.x >> 5), cnt);
        } else {
            sel.path = PATH_EMPTY;
            sel.produce = false;
            sel.count = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) sel.src[k] = lane;
        }
        // step 2: the lane's texel goes into the lane's own row
        if (sel.produce) {
            const int x = min(max(sel.tx, 0), p.Wt - 1), y = min(max(sel.ty, 0), p.Ht - 1);
            float f[kMlpIn];
            texel_features(m, x, y, f);
            store_x_row(sm, threadIdx.x, f, m.fp8, inv_a1);
        } else {
            store_zero_x_row(sm, threadIdx.x);
        }
        float4 val;
        ok = mlp_chain(ch, m.fp8, val, err);
        if (!ok) return false;
        if (sel.path == PATH_SUCCESS) {
            // step 3: gather the 2x2 taps from the producing lanes
            float4 tap[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                tap[k].x = __shfl_sync(FULL, val.x, sel.src[k]);
                tap[k].y = __shfl_sync(FULL, val.y, sel.src[k]);
                tap[k].z = __shfl_sync(FULL, val.z, sel.src[k]);
                tap[k].w = __shfl_sync(FULL, val.w, sel.src[k]);
            }
            if (ps.active) {
                float w[4];
                bilinear_weights(ps.s, ps.t, w);
                float r = 0.f, g = 0.f, b = 0.f, a = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    r = __fmaf_rn(w[k], tap[k].x, r);
                    g = __fmaf_rn(w[k], tap[k].y, g);
                    b = __fmaf_rn(w[k], tap[k].z, b);
                    a = __fmaf_rn(w[k], tap[k].w, a);
                }
                result = make_float4(r, g, b, a);
                count = sel.count;
            }
        } else if (ps.active) {
            result = val;
            count = 1;
        }
    }
    if (inside) {
        __stcs(p.out + idx, result);
        if (p.evals) p.evals[idx] = count;
    }
        return true;
}

// One iteration of the learned-decode filter for the collaborative
// algorithms and STF.  The CTA's 4 warps run step 1 on two pixel tiles each
// (slots g = warp and g = 4 + warp of the group of 8 tiles from `first`); the
// texel lists of the 8 tiles are packed into consecutive rows in slot order
// and decoded by as few 128-row chains as they fill (none for an empty
// group), and every pixel then gathers its taps from the rows.  Which thread
// computes a texel does not change its value: the rows of an MMA are
// independent.  Returns false (for every thread alike) if a chain gave up.
template <int ALG, int TW, int MD>
__device__ __forceinline__ bool mlp_group(const ExactParams &p, const MlpDevice &m, Chain &ch, long long first,
                                          int lane, uint32_t lt, ListTable *T, Counters &cnt, const float *inv_a1,
                                          int *err) {
    constexpr int TH = 32 / TW;
    unsigned char *sm = ch.sm;
    const int warp = threadIdx.x >> 5, tx = lane % TW, ty = lane / TW;
    const float fW = (float)p.Wt, fH = (float)p.Ht;
    float2 *pix_st = reinterpret_cast<float2 *>(sm + kSmPixST);
    uint32_t *pix_info = reinterpret_cast<uint32_t *>(sm + kSmPixInfo);
    int2 *texlist = reinterpret_cast<int2 *>(sm + kSmTexList);
    float4 *outrow = reinterpret_cast<float4 *>(sm + kSmOut);
    int *count = reinterpret_cast<int *>(sm + kSmCount);
    int *ranks = reinterpret_cast<int *>(sm + kSmRanks) + 32 * warp;

    // ---- step 1 on the warp's two tiles; the texel list of slot g goes to
    // texlist[32 g + rank], and each pixel keeps (s, t) and a packed word:
    // bits 0-19 the list indices of its 4 taps (success) or of its own texel
    // (bits 0-4, fallback), 20-22 its count, 23 active, 24 inside, 25 success.
    const TilePos tp = tile_pos0(p, first);
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        const int g = 4 * h + warp;
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
        setup_coords(uv, fW, fH, ps);
        Selection sel;
        if (valid) {
            sel = select_tile<ALG, MD, true, false>(p, ps, jac, px, py, lane, lt, T, ranks, cnt);
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
        // (inactive pixels carry arbitrary tap indices: masked to their fields)
        uint32_t info = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) info |= ((uint32_t)sel.rk[k] & 31u) << (5 * k);
        info = succ ? info : ((uint32_t)sel.my_rank & 31u);
        info |= ((uint32_t)sel.count << 20) | (ps.active ? 1u << 23 : 0u) | (inside ? 1u << 24 : 0u) |
                (succ ? 1u << 25 : 0u);
        pix_st[32 * g + lane] = make_float2(ps.s, ps.t);
        pix_info[32 * g + lane] = info;
    }
    __syncthreads();

    // ---- rows.  Without group_dedup slot g owns rows [base_g, base_g +
    // count[g]) in slot order.  With it, the distinct texels of the group
    // get rows in the order their first lists entries win a shared hash
    // table, and rowmap sends every list entry to its texel's row.  Every
    // thread then reads the texels of its rows (threadIdx.x and 128 +
    // threadIdx.x) before the first chain overwrites the X buffer that holds
    // the lists.
    int cnts[kGroupTiles];
#pragma unroll
    for (int g = 0; g < kGroupTiles; ++g) cnts[g] = count[g];
    int R = 0, my_base[2] = {0, 0};
    int2 xy[2] = {make_int2(0, 0), make_int2(0, 0)};
    unsigned char *rowmap = sm + kSmRowMap;
    if (p.group_dedup) {  // CTA-uniform
        unsigned long long *hkey = reinterpret_cast<unsigned long long *>(sm + kSmHashKey);
        unsigned char *hrow = sm + kSmHashRow;
        int *nuniq = reinterpret_cast<int *>(sm + kSmNUnique);
        for (int i = threadIdx.x; i < 512; i += kRows) hkey[i] = ~0ull;
        if (threadIdx.x == 0) *nuniq = 0;
        __syncthreads();
        int slot[2] = {0, 0};
        bool has[2] = {false, false}, won[2] = {false, false};
        int2 t2[2] = {make_int2(0, 0), make_int2(0, 0)};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int e = (int)threadIdx.x + kRows * c, g = e >> 5;
            int n_g = cnts[0];
#pragma unroll
            for (int k = 1; k < kGroupTiles; ++k) n_g = g == k ? cnts[k] : n_g;
            if ((e & 31) < n_g) {
                has[c] = true;
                t2[c] = texlist[e];
                const unsigned long long key = ((unsigned long long)(uint32_t)t2[c].y << 32) | (uint32_t)t2[c].x;
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
        __syncthreads();
        int2 *uxy = texlist;  // the lists have been read: the distinct texels reuse the space
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (won[c]) {
                const int row = ck(atomicAdd(nuniq, 1), 2 * kRows, p.err, kBndRow);
                hrow[slot[c]] = (unsigned char)row;
                uxy[row] = t2[c];
            }
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 2; ++c)
            if (has[c]) rowmap[threadIdx.x + kRows * c] = hrow[slot[c]];
        R = *nuniq;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int row = kRows * c + (int)threadIdx.x;
            if (row < R) xy[c] = uxy[row];
        }
    } else {
        int start[kGroupTiles];
#pragma unroll
        for (int g = 0; g < kGroupTiles; ++g) {
            start[g] = R;
            if (g == warp) my_base[0] = R;
            if (g == 4 + warp) my_base[1] = R;
            R += cnts[g];
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int row = kRows * c + (int)threadIdx.x;
            if (row < R) {
                int g = 0, b = 0;
#pragma unroll
                for (int k = 1; k < kGroupTiles; ++k) {
                    if (row >= start[k]) {
                        g = k;
                        b = start[k];
                    }
                }
                xy[c] = texlist[32 * g + ck(row - b, 32, p.err, kBndTexList)];
            }
        }
    }
    if (threadIdx.x == 0) cnt.v[kStatTexelEvalsUnique] += R;
    __syncthreads();

    // ---- the chains (CTA-uniform count: 0, 1 or 2)
    const int passes = (R + kRows - 1) / kRows;
#pragma unroll 1
    for (int c = 0; c < passes; ++c) {
        const int row = kRows * c + (int)threadIdx.x;
        if (row < R) {
            const int2 t = c == 0 ? xy[0] : xy[1];
            float f[kMlpIn];
            texel_features(m, t.x, t.y, f);
            store_x_row(sm, threadIdx.x, f, m.fp8, inv_a1);
        } else {
            store_zero_x_row(sm, threadIdx.x);
        }
        float4 v;
        if (!mlp_chain(ch, m.fp8, v, err)) return false;
        outrow[ck(row, 2 * kRows, p.err, kBndRow)] = v;
    }
    __syncthreads();

    // ---- step 3: gather from the rows, filter, store
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        const int g = 4 * h + warp;
        const uint32_t info = pix_info[32 * g + lane];
        if (!((info >> 24) & 1u)) continue;  // outside the frame (or no tile)
        int bx, by;
        tile_pos(tp, g, bx, by);
        const uint32_t idx =
            ck((uint32_t)(by * TH + ty) * (uint32_t)p.W + (uint32_t)(bx * TW + tx), view_pixels(p), p.err, kBndPixel);
        const int b = h == 0 ? my_base[0] : my_base[1];
        const bool dedup = p.group_dedup != 0;
        // row of list entry i of this tile
        auto row_of = [&](uint32_t i) {
            return ck(dedup ? (int)rowmap[32 * g + (int)i] : b + (int)i, 2 * kRows, p.err, kBndRow);
        };
        float4 result = make_float4(0.f, 0.f, 0.f, 0.f);
        uint8_t cv = 0;
        if ((info >> 23) & 1u) {
            if ((info >> 25) & 1u) {
                const float2 st = pix_st[32 * g + lane];
                float w[4];
                bilinear_weights(st.x, st.y, w);
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
    return true;
}

}  // namespace
}  // namespace ctf
