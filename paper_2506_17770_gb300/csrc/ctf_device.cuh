// ctf_device.cuh -- device helpers of the CUDA path: the STF random draw,
// the exact block decode, the per-pixel setup and the bijection h of Mask
// Sampling.  sm_103a only.  Every floating-point step that decides a texel or
// a weight uses explicit round-to-nearest intrinsics so that no contraction
// changes a result.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ctf_debug.cuh"

namespace ctf {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): per round two 32x32->64 products,
// the high halves xor'ed with the other two words and the round key, the key
// advanced by the Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// One-tap STF offset: counter (px, py, view, 0), key (seed lo, seed hi);
// xi = (r >> 8) * 2^-24 (exact in float); right neighbour when xi0 < s,
// lower neighbour when xi1 < t.
__device__ __forceinline__ void stf_offset(int px, int py, int view, uint32_t k0, uint32_t k1, float s,
                                           float t, int &dx, int &dy) {
    uint4 r = philox4x32_10(make_uint4((uint32_t)px, (uint32_t)py, (uint32_t)view, 0u), k0, k1);
    float xi0 = __fmul_rn((float)(r.x >> 8), 5.9604644775390625e-08f);  // 2^-24
    float xi1 = __fmul_rn((float)(r.y >> 8), 5.9604644775390625e-08f);
    dx = xi0 < s ? 1 : 0;
    dy = xi1 < t ? 1 : 0;
}

// The same draw with the third word of the Philox output as xi2 (fallback
// C+ picks its extra texel with it).
__device__ __forceinline__ void stf_draw(int px, int py, int view, uint32_t k0, uint32_t k1, float s, float t, int &dx,
                                         int &dy, float &xi2) {
    uint4 r = philox4x32_10(make_uint4((uint32_t)px, (uint32_t)py, (uint32_t)view, 0u), k0, k1);
    float xi0 = __fmul_rn((float)(r.x >> 8), 5.9604644775390625e-08f);  // 2^-24
    float xi1 = __fmul_rn((float)(r.y >> 8), 5.9604644775390625e-08f);
    xi2 = __fmul_rn((float)(r.z >> 8), 5.9604644775390625e-08f);
    dx = xi0 < s ? 1 : 0;
    dy = xi1 < t ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Block decode.  Texture = (Wt/4) x (Ht/4) blocks of 8 bytes read as one
// uint2: .x = c0 | c1 << 16, .y = 2-bit indices.  Returns RGBA8 packed
// little-endian (r in the low byte), alpha 255.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t expand_channel_pair(uint32_t e0, uint32_t e1, uint32_t sel) {
    // palette entry of one channel: e0, e1, (2e0+e1+1)/3, (e0+2e1+1)/3
    uint32_t p2 = (2u * e0 + e1 + 1u) / 3u;
    uint32_t p3 = (e0 + 2u * e1 + 1u) / 3u;
    uint32_t v = sel == 0 ? e0 : (sel == 1 ? e1 : (sel == 2 ? p2 : p3));
    return v;
}

__device__ __forceinline__ uint32_t decode_block_texel(uint2 blk, int x, int y) {
    uint32_t c0 = blk.x & 0xffffu, c1 = blk.x >> 16;
    uint32_t sel = (blk.y >> (2 * (((y & 3) << 2) | (x & 3)))) & 3u;
    uint32_t r0 = c0 >> 11, g0 = (c0 >> 5) & 63u, b0 = c0 & 31u;
    uint32_t r1 = c1 >> 11, g1 = (c1 >> 5) & 63u, b1 = c1 & 31u;
    r0 = (r0 << 3) | (r0 >> 2);
    g0 = (g0 << 2) | (g0 >> 4);
    b0 = (b0 << 3) | (b0 >> 2);
    r1 = (r1 << 3) | (r1 >> 2);
    g1 = (g1 << 2) | (g1 >> 4);
    b1 = (b1 << 3) | (b1 >> 2);
    uint32_t r = expand_channel_pair(r0, r1, sel);
    uint32_t g = expand_channel_pair(g0, g1, sel);
    uint32_t b = expand_channel_pair(b0, b1, sel);
    return r | (g << 8) | (b << 16) | 0xff000000u;
}

// Clamp-to-edge texel fetch of packed RGBA8 (err: the device error word of
// the debug build's index check, or nullptr).
__device__ __forceinline__ uint32_t fetch_block_texel(const uint2 *__restrict__ blocks, int nbx, int Wt, int Ht,
                                                      int x, int y, int *err = nullptr) {
    x = min(max(x, 0), Wt - 1);
    y = min(max(y, 0), Ht - 1);
    uint2 blk = __ldg(blocks + ck((size_t)(y >> 2) * (size_t)nbx + (x >> 2), (long long)nbx * (Ht / 4), err, kBndBlock));
    return decode_block_texel(blk, x, y);
}

// ---------------------------------------------------------------------------
// Per-pixel setup (Appendix code, first lines) and the minification vote.
// ---------------------------------------------------------------------------
struct PixelSetup {
    int ulx, uly;
    float s, t;
    bool active;
    bool minified;
};

constexpr float kCoordLimit = 4194304.0f;  // 2^22

__device__ __forceinline__ void setup_coords(float2 uv, float fW, float fH, PixelSetup &p) {
    // x - 0.5 is x + (-0.5) in IEEE arithmetic; the packed operations round
    // each component like their scalar forms
    const float2 xy = __fadd2_rn(__fmul2_rn(uv, make_float2(fW, fH)), make_float2(-0.5f, -0.5f));
    bool ok = fabsf(xy.x) < kCoordLimit && fabsf(xy.y) < kCoordLimit;  // false for NaN
    float fx = floorf(xy.x), fy = floorf(xy.y);
    p.ulx = ok ? (int)fx : 0;
    p.uly = ok ? (int)fy : 0;
    const float2 st = __fadd2_rn(xy, make_float2(-fx, -fy));  // read for active pixels only
    p.s = st.x;
    p.t = st.y;
    p.active = p.active && ok;
}

__device__ __forceinline__ bool is_minified(float4 j, float fW, float fH) {
    const float2 ab = __fmul2_rn(make_float2(j.x, j.y), make_float2(fW, fH));
    const float2 cd = __fmul2_rn(make_float2(j.z, j.w), make_float2(fW, fH));
    const float2 ab2 = __fmul2_rn(ab, ab), cd2 = __fmul2_rn(cd, cd);
    const float rx = __fadd_rn(ab2.x, ab2.y), ry = __fadd_rn(cd2.x, cd2.y);
    return !(rx <= 1.0f && ry <= 1.0f);
}

// Bilinear weights of taps k = (k%2, k/2): (1-s)(1-t), s(1-t), (1-s)t, st.
__device__ __forceinline__ void bilinear_weights(float s, float t, float w[4]) {
    const float2 o = __fadd2_rn(make_float2(1.0f, 1.0f), make_float2(-s, -t));
    const float2 w01 = __fmul2_rn(make_float2(o.x, s), make_float2(o.y, o.y));
    const float2 w23 = __fmul2_rn(make_float2(o.x, s), make_float2(t, t));
    w[0] = w01.x;
    w[1] = w01.y;
    w[2] = w23.x;
    w[3] = w23.y;
}

// h(i, A) for a 32-bit lane mask: lane of the i-th set bit.
__device__ __forceinline__ int nth_set_lane(uint32_t A, int i) { return (int)__fns(A, 0, i + 1); }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace ctf
