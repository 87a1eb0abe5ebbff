// ctf_device.cuh -- device helpers of the CUDA path: the STF random draw,
// the exact block decode, the per-pixel setup and the bijection h of Mask
// Sampling.  sm_103a only.  Every floating-point step that decides a texel or
// a weight uses explicit round-to-nearest intrinsics so that no contraction
// changes a result.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

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

// Clamp-to-edge texel fetch of packed RGBA8.
__device__ __forceinline__ uint32_t fetch_block_texel(const uint2 *__restrict__ blocks, int nbx, int Wt, int Ht,
                                                      int x, int y) {
    x = min(max(x, 0), Wt - 1);
    y = min(max(y, 0), Ht - 1);
    uint2 blk = __ldg(blocks + (size_t)(y >> 2) * (size_t)nbx + (x >> 2));
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
    float xf = __fsub_rn(__fmul_rn(uv.x, fW), 0.5f);
    float yf = __fsub_rn(__fmul_rn(uv.y, fH), 0.5f);
    bool ok = fabsf(xf) < kCoordLimit && fabsf(yf) < kCoordLimit;  // false for NaN
    float fx = floorf(xf), fy = floorf(yf);
    p.ulx = ok ? (int)fx : 0;
    p.uly = ok ? (int)fy : 0;
    p.s = __fsub_rn(xf, fx);  // read for active pixels only
    p.t = __fsub_rn(yf, fy);
    p.active = p.active && ok;
}

__device__ __forceinline__ bool is_minified(float4 j, float fW, float fH) {
    float a = __fmul_rn(j.x, fW), b = __fmul_rn(j.y, fH);
    float c = __fmul_rn(j.z, fW), d = __fmul_rn(j.w, fH);
    float rx = __fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b));
    float ry = __fadd_rn(__fmul_rn(c, c), __fmul_rn(d, d));
    return !(rx <= 1.0f && ry <= 1.0f);
}

// Bilinear weights of taps k = (k%2, k/2).
__device__ __forceinline__ void bilinear_weights(float s, float t, float w[4]) {
    float os = __fsub_rn(1.0f, s), ot = __fsub_rn(1.0f, t);
    w[0] = __fmul_rn(os, ot);
    w[1] = __fmul_rn(s, ot);
    w[2] = __fmul_rn(os, t);
    w[3] = __fmul_rn(s, t);
}

// acc = 0; acc = fma(w_k, p_k, acc) for k = 0..3, per channel; alpha of
// every block texel is 1.0.
__device__ __forceinline__ float4 filter_rgba8(const float w[4], const uint32_t p[4], const float *lut) {
    float r = 0.f, g = 0.f, b = 0.f, a = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        r = __fmaf_rn(w[k], lut[p[k] & 0xffu], r);
        g = __fmaf_rn(w[k], lut[(p[k] >> 8) & 0xffu], g);
        b = __fmaf_rn(w[k], lut[(p[k] >> 16) & 0xffu], b);
        a = __fmaf_rn(w[k], 1.0f, a);
    }
    return make_float4(r, g, b, a);
}

__device__ __forceinline__ float4 rgba8_to_float(uint32_t p, const float *lut) {
    return make_float4(lut[p & 0xffu], lut[(p >> 8) & 0xffu], lut[(p >> 16) & 0xffu], 1.0f);
}

// h(i, A) for a 32-bit lane mask: lane of the i-th set bit.
__device__ __forceinline__ int nth_set_lane(uint32_t A, int i) { return (int)__fns(A, 0, i + 1); }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace ctf
