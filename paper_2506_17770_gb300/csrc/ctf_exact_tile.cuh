// ctf_exact_tile.cuh -- one warp tile of the exact-decode filter (the
// collaborative flow of Sec. 3 with the block decode as texel evaluation),
// shared by the per-view kernel (ctf_filter.cu) and the batched persistent
// kernel (ctf_batch.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ctf_device.cuh"
#include "ctf_internal.h"
#include "ctf_select.cuh"

namespace ctf {
namespace {

struct Inputs {
    float2 uv;
    float4 jac;
    bool covered;  // inside the frame and covered
};

template <bool kJac>
__device__ __forceinline__ Inputs load_inputs(const ExactParams &p, bool inside, uint32_t idx) {
    Inputs in;
    in.uv = make_float2(0.f, 0.f);
    in.jac = make_float4(0.f, 0.f, 0.f, 0.f);
    in.covered = inside;
    if (inside) {
        in.uv = __ldcs(p.uv + idx);
        if (kJac) in.jac = __ldcs(p.jac + idx);
        if (p.cov) in.covered = __ldcs(p.cov + idx) != 0;
    }
    return in;
}

// Unpredicated variant: every lane loads, lanes outside the frame at pixel 0
// (any valid index), and their inputs count as uncovered.
template <bool kJac>
__device__ __forceinline__ Inputs load_inputs_any(const ExactParams &p, bool inside, uint32_t idx) {
    Inputs in;
    const uint32_t i = inside ? idx : 0u;
    in.uv = __ldcs(p.uv + i);
    in.jac = kJac ? __ldcs(p.jac + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    in.covered = inside && (p.cov == nullptr || __ldcs(p.cov + i) != 0);
    return in;
}

__device__ __forceinline__ void store_pixel(const ExactParams &p, uint32_t idx, float4 v, uint8_t count) {
    __stcs(p.out + idx, v);
    if (p.evals) p.evals[idx] = count;
}

// Decode tables, built in shared memory by every CTA: the two endpoints of a
// block expand to 8-bit channels laid out in 10-bit fields (r bits 0-9, g
// 10-19, b 20-29) by two lookups each, so that the palette entries 2 and 3,
// (2a+b+1)/3 with (a, b) = (c0, c1) or (c1, c0), come out of one integer
// expression for all three channels, and `val` turns a field into the
// channel value: val[v] = v/255 for v < 256, val[256 + s] = floor(s/3)/255
// for s < 768 (both correctly rounded, IEEE division); the interpolated
// entries carry the offset 256 in every field of the sum.
struct DecodeTables {
    uint32_t rg[2048];  // c >> 5 = (r5 << 6) | g6  ->  r8 | g8 << 10
    uint32_t b[32];     // c & 31 = b5              ->  b8 << 20
    float val[1024];
};

__device__ __forceinline__ void build_decode_tables(DecodeTables *t) {
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) {
        const uint32_t r5 = (uint32_t)i >> 6, g6 = (uint32_t)i & 63u;
        t->rg[i] = ((r5 << 3) | (r5 >> 2)) | (((g6 << 2) | (g6 >> 4)) << 10);
    }
    for (int i = threadIdx.x; i < 32; i += blockDim.x) t->b[i] = (((uint32_t)i << 3) | ((uint32_t)i >> 2)) << 20;
    for (int i = threadIdx.x; i < 1024; i += blockDim.x)
        t->val[i] = i < 256 ? __fdiv_rn((float)i, 255.0f) : __fdiv_rn((float)((i - 256) / 3), 255.0f);
}

// RGB of texel (x, y) of a block (alpha is 1): palette c0, c1,
// (2c0+c1+1)/3, (c0+2c1+1)/3, 2-bit index at bits 2*(4*(y&3)+(x&3)).
__device__ __forceinline__ float3 decode_texel_f(uint2 blk, int x, int y, const DecodeTables *T) {
    const uint32_t sel = (blk.y >> ((((uint32_t)y & 3u) << 3) | (((uint32_t)x & 3u) << 1))) & 3u;
    const uint32_t c0 = blk.x & 0xffffu, c1 = blk.x >> 16;
    const uint32_t e0 = T->rg[c0 >> 5] | T->b[c0 & 31u];
    const uint32_t e1 = T->rg[c1 >> 5] | T->b[c1 & 31u];
    const bool odd = (sel & 1u) != 0, mid = (sel & 2u) != 0;
    const uint32_t a = odd ? e1 : e0, b = odd ? e0 : e1;
    // per field 2a + b + 1 + 256 <= 1022: no carry between the fields
    const uint32_t v = mid ? (2u * a + b + 0x10140501u) : a;
    return make_float3(T->val[v & 0x3ffu], T->val[(v >> 10) & 0x3ffu], T->val[v >> 20]);
}

// Clamp-to-edge fetch and decode of texel (x, y).
__device__ __forceinline__ float3 fetch_decode(const ExactParams &p, int x, int y, const DecodeTables *T) {
    x = min(max(x, 0), p.Wt - 1);
    y = min(max(y, 0), p.Ht - 1);
    const uint2 blk = __ldg(p.blocks + (uint32_t)(y >> 2) * (uint32_t)p.nbx + (uint32_t)(x >> 2));
    return decode_texel_f(blk, x, y, T);
}

// acc = fma(w_k, p_k, acc) from 0, k = 0..3; alpha of every block texel is
// 1.  The channels run in pairs (r, g) and (b, a) through packed FMAs that
// round each component like fmaf.
__device__ __forceinline__ float4 filter4(const float w[4], const float3 t[4]) {
    float2 rg = make_float2(0.f, 0.f), ba = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 wk = make_float2(w[k], w[k]);
        rg = __ffma2_rn(wk, make_float2(t[k].x, t[k].y), rg);
        ba = __ffma2_rn(wk, make_float2(t[k].z, 1.0f), ba);
    }
    return make_float4(rg.x, rg.y, ba.x, ba.y);
}

// CTAs of 8 warps per SM that the exact kernels ask the compiler to fit:
// the collaborative kernels are issue-bound, and five CTAs (40 warps) hide
// more latency than the registers a looser cap would buy.
template <int ALG>
constexpr int min_blocks() {
    return ALG >= ALG_LIST ? 5 : 1;
}

template <int ALG, int TW, int MD, bool kStats>
__device__ __forceinline__ void filter_tile(const ExactParams &p, const Inputs &in, int px, int py, bool inside,
                                            uint32_t idx, int lane, uint32_t lt, const DecodeTables *tabs,
                                            ListTable *T, int *ranks, Counters &cnt) {
    PixelSetup ps;
    ps.active = in.covered;
    setup_coords(in.uv, (float)p.Wt, (float)p.Ht, ps);
    // Every path ends in one store per pixel: RGBA 0 and count 0 unless the
    // pixel is active.
    float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t count = 0;

    if (ALG == ALG_4TAP) {
        // ---------------- per-pixel 4-tap ----------------
        if (kStats) {
            const uint32_t A = __ballot_sync(FULL, ps.active);
            cnt.v[kStatTilesTotal] += 1;
            if (A == 0) {
                cnt.v[kStatTilesEmpty] += 1;
            } else {
                const int nactive = __popc(A);
                cnt.v[kStatPixelsActive] += nactive;
                cnt.v[kStatTilesDirect] += 1;
                cnt.v[kStatTexelEvals] += 4 * nactive;
                cnt.v[kStatTexelEvalsUnique] += 4 * nactive;
            }
        }
        // inactive lanes decode too (their own clamped texels): the warp
        // stays converged and the values are dropped
        float3 t[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) t[k] = fetch_decode(p, ps.ulx + (k & 1), ps.uly + (k >> 1), tabs);
        if (ps.active) {
            float w[4];
            bilinear_weights(ps.s, ps.t, w);
            res = filter4(w, t);
            count = 4;
        }
    } else {
        const Selection sel = select_tile<ALG, MD, kStats>(p, ps, in.jac, px, py, lane, lt, T, ranks, cnt);
        // step 2: exact decode of the lane's texel (clamped to the texture);
        // lanes that produce nothing decode their own upper-left texel, which
        // the warp reads anyway, and drop it
        const float3 val = fetch_decode(p, sel.tx, sel.ty, tabs);
        if (sel.path == PATH_SUCCESS) {
            // step 3: gather the 2x2 taps from their producers and filter
            float3 t[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                t[k].x = __shfl_sync(FULL, val.x, sel.src[k]);
                t[k].y = __shfl_sync(FULL, val.y, sel.src[k]);
                t[k].z = __shfl_sync(FULL, val.z, sel.src[k]);
            }
            if (ps.active) {
                float w[4];
                bilinear_weights(ps.s, ps.t, w);
                res = filter4(w, t);
                count = sel.count;
            }
        } else if (ps.active) {
            res = make_float4(val.x, val.y, val.z, 1.0f);
            count = 1;
        }
    }
    if (inside) store_pixel(p, idx, res, (uint8_t)count);
}

}  // namespace
}  // namespace ctf
