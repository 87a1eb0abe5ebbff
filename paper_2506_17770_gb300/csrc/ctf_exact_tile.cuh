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

__device__ __forceinline__ void store_pixel(const ExactParams &p, uint32_t idx, float4 v, uint8_t count) {
    __stcs(p.out + idx, v);
    if (p.evals) p.evals[idx] = count;
}

__device__ __forceinline__ float3 to_float3(uint32_t rgba8, const float *lut) {
    return make_float3(lut[rgba8 & 0xffu], lut[(rgba8 >> 8) & 0xffu], lut[(rgba8 >> 16) & 0xffu]);
}

// acc = fma(w_k, p_k, acc) from 0, k = 0..3; alpha of every block texel is 1.
__device__ __forceinline__ float4 filter4(const float w[4], const float3 t[4]) {
    float r = 0.f, g = 0.f, b = 0.f, a = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        r = __fmaf_rn(w[k], t[k].x, r);
        g = __fmaf_rn(w[k], t[k].y, g);
        b = __fmaf_rn(w[k], t[k].z, b);
        a = __fmaf_rn(w[k], 1.0f, a);
    }
    return make_float4(r, g, b, a);
}

template <int ALG, int TW, int MD>
__device__ __forceinline__ void filter_tile(const ExactParams &p, const Inputs &in, int px, int py, bool inside,
                                            uint32_t idx, int lane, uint32_t lt, const float *lut, ListTable *T,
                                            Counters &cnt) {
    PixelSetup ps;
    ps.active = in.covered;
    setup_coords(in.uv, (float)p.Wt, (float)p.Ht, ps);

    if (ALG == ALG_4TAP) {
        // ---------------- per-pixel 4-tap ----------------
        const uint32_t A = __ballot_sync(FULL, ps.active);
        cnt.v[kStatTilesTotal] += 1;
        if (A == 0) {
            cnt.v[kStatTilesEmpty] += 1;
        } else {
            const int nactive = __popc(A);
            cnt.v[kStatPixelsActive] += nactive;
            cnt.v[kStatTilesDirect] += 1;
            cnt.v[kStatTexelEvals] += 4 * nactive;
        }
        if (ps.active) {
            float3 t[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                t[k] = to_float3(fetch_block_texel(p.blocks, p.nbx, p.Wt, p.Ht, ps.ulx + (k & 1), ps.uly + (k >> 1)), lut);
            float w[4];
            bilinear_weights(ps.s, ps.t, w);
            store_pixel(p, idx, filter4(w, t), 4);
        } else if (inside) {
            store_pixel(p, idx, make_float4(0.f, 0.f, 0.f, 0.f), 0);
        }
        return;
    }

    const Selection sel = select_tile<ALG, MD>(p, ps, in.jac, px, py, lane, lt, T, cnt);
    // step 2: exact decode of the lane's texel (clamped to the texture)
    float3 val = make_float3(0.f, 0.f, 0.f);
    if (sel.produce) val = to_float3(fetch_block_texel(p.blocks, p.nbx, p.Wt, p.Ht, sel.tx, sel.ty), lut);
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
            store_pixel(p, idx, filter4(w, t), sel.count);
        } else if (inside) {
            store_pixel(p, idx, make_float4(0.f, 0.f, 0.f, 0.f), 0);
        }
    } else if (ps.active) {
        store_pixel(p, idx, make_float4(val.x, val.y, val.z, 1.0f), 1);
    } else if (inside) {
        store_pixel(p, idx, make_float4(0.f, 0.f, 0.f, 0.f), 0);
    }
}

}  // namespace
}  // namespace ctf
