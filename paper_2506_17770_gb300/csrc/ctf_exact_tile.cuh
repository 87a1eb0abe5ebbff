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
        idx = ck(idx, view_pixels(p), p.err, kBndPixel);
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
    const uint32_t i = ck(inside ? idx : 0u, view_pixels(p), p.err, kBndPixel);
    in.uv = __ldcs(p.uv + i);
    in.jac = kJac ? __ldcs(p.jac + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    in.covered = inside && (p.cov == nullptr || __ldcs(p.cov + i) != 0);
    return in;
}

__device__ __forceinline__ void store_pixel(const ExactParams &p, uint32_t idx, float4 v, uint8_t count) {
    idx = ck(idx, view_pixels(p), p.err, kBndPixel);
    __stcs(p.out + idx, v);
    if (p.evals) p.evals[idx] = count;
}

// The decode tables (DecodeTables, ctf_internal.h) into this CTA's shared
// memory, 16 bytes per thread and step; the interpolated palette entries
// carry the offset 256 in every field of the sum.
__device__ __forceinline__ void load_decode_tables(DecodeTables *t, const DecodeTables *g) {
    const uint4 *src = reinterpret_cast<const uint4 *>(g);
    uint4 *dst = reinterpret_cast<uint4 *>(t);
    for (int i = threadIdx.x; i < (int)(sizeof(DecodeTables) / 16); i += blockDim.x) dst[i] = __ldg(src + i);
}

// RGB of texel (x, y) of a block (alpha is 1): palette c0, c1,
// (2c0+c1+1)/3, (c0+2c1+1)/3, 2-bit index at bits 2*(4*(y&3)+(x&3)).
__device__ __forceinline__ float3 decode_texel_f(uint2 blk, int x, int y, const DecodeTables *T, int *err) {
    const uint32_t sel = (blk.y >> ((((uint32_t)y & 3u) << 3) | (((uint32_t)x & 3u) << 1))) & 3u;
    const uint32_t c0 = blk.x & 0xffffu, c1 = blk.x >> 16;
    const uint32_t e0 = T->rg[ck(c0 >> 5, 2048, err, kBndDecodeTable)] | T->b[ck(c0 & 31u, 32, err, kBndDecodeTable)];
    const uint32_t e1 = T->rg[ck(c1 >> 5, 2048, err, kBndDecodeTable)] | T->b[ck(c1 & 31u, 32, err, kBndDecodeTable)];
    const bool odd = (sel & 1u) != 0, mid = (sel & 2u) != 0;
    const uint32_t a = odd ? e1 : e0, b = odd ? e0 : e1;
    // per field 2a + b + 1 + 256 <= 1022: no carry between the fields
    const uint32_t v = mid ? (2u * a + b + 0x10140501u) : a;
    return make_float3(T->val[ck(v & 0x3ffu, 1024, err, kBndDecodeTable)],
                       T->val[ck((v >> 10) & 0x3ffu, 1024, err, kBndDecodeTable)],
                       T->val[ck(v >> 20, 1024, err, kBndDecodeTable)]);
}

// Clamp-to-edge fetch and decode of texel (x, y).
__device__ __forceinline__ float3 fetch_decode(const ExactParams &p, int x, int y, const DecodeTables *T) {
    x = min(max(x, 0), p.Wt - 1);
    y = min(max(y, 0), p.Ht - 1);
    const uint2 blk = __ldg(p.blocks + ck((uint32_t)(y >> 2) * (uint32_t)p.nbx + (uint32_t)(x >> 2),
                                          texture_blocks(p), p.err, kBndBlock));
    return decode_texel_f(blk, x, y, T, p.err);
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

// ---------------------------------------------------------------------------
// Fallbacks C and C+ (Sec. 3.4) for a magnified tile whose texel set does
// not fit the budget; mode 1 = C, 2 = C+.  Every active lane draws its
// one-tap STF texel.  C: every active lane produces it.  C+: the distinct
// STF texels are produced by the first n active lanes (in the order of the
// lowest lane that draws each), and remaining active lane c (index among the
// active lanes) takes the footprint of active lane
// l = round_half_up((na-1)(c-n)/(na-1-n)) (l = 0 when na-1 = n: eq. 2 with
// the na active lanes for the 32) and produces one of its nonzero-weight
// taps outside that set, drawn by weight with the third word of its own STF
// draw (nothing if there is none).  Every active pixel then blends the
// produced texels of its footprint that have nonzero weight by eq. 1:
// exact bilinear when all are present, the texel itself when one is, else
// fma(1 - S_w, S_p / N, S_wp) per channel (tap order, FP32 RN).
// The texels a lane looks for are found in a per-warp open-addressing hash
// table in shared memory (64 slots for at most 32 keys), empty between
// tiles.  Warp-collective; kept out of line so that it does not weigh on the
// registers of the common path.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long texel_key(int x, int y) {
    return ((unsigned long long)(uint32_t)y << 32) | (uint32_t)x;
}

// no texel: x = INT_MIN is never a texel coordinate (|x| < 2^22 + 2)
constexpr unsigned long long kNoTexel = 0x8000000080000000ull;

struct FbTable {
    unsigned long long key[64];  // kNoTexel = empty
    unsigned char lane[64];      // the lane that inserted the key
};

__device__ __forceinline__ unsigned fb_hash(unsigned long long k) {
    return (((uint32_t)k * 0x9E3779B1u) ^ ((uint32_t)(k >> 32) * 0x85EBCA77u)) >> 26;
}

// Insert texel key k for `lane`; a key already present keeps its lane.
__device__ __forceinline__ void fb_insert(FbTable *t, unsigned long long k, int lane) {
    unsigned h = fb_hash(k);
    for (int probe = 0; probe < 64; ++probe) {  // at most 32 keys in 64 slots: the probe ends
        const unsigned long long old = atomicCAS(&t->key[h], kNoTexel, k);
        if (old == kNoTexel) {
            t->lane[h] = (unsigned char)lane;
            return;
        }
        if (old == k) return;
        h = (h + 1) & 63u;
    }
}

// The lane that inserted texel key k, or -1.
__device__ __forceinline__ int fb_find(const FbTable *t, unsigned long long k) {
    unsigned h = fb_hash(k);
    for (int probe = 0; probe < 64; ++probe) {
        const unsigned long long v = t->key[h];
        if (v == k) return t->lane[h];
        if (v == kNoTexel) return -1;
        h = (h + 1) & 63u;
    }
    return -1;
}

// Empty the table (every lane two slots); the caller syncs the warp.
__device__ __forceinline__ void fb_clear(FbTable *t, int lane) {
    t->key[lane] = kNoTexel;
    t->key[lane + 32] = kNoTexel;
}

struct FallbackOut {
    float4 res;
    uint32_t count;
};

// The block fields and the STF key are passed by value: a kernel parameter
// handed by reference to an out-of-line function would be copied to local
// memory for the whole kernel.
struct FallbackArgs {
    const uint2 *blocks;
    int Wt, Ht, nbx;
    int view;
    int y0;  // row of the whole view at which the frame starts
    uint32_t k0, k1;
    int mode;
    int *err;  // device error word (index checks of the debug build)
};

// Which texel a lane of an over-budget tile produces under fallback C
// (mode 1) or C+ (mode 2), from its one-tap STF draw; warp-collective.
struct FbChoice {
    bool produce;
    int qx, qy;  // the texel (unclamped)
};

__device__ __forceinline__ FbChoice fb_choose(int mode, int view, int y0, uint32_t k0, uint32_t k1, int ulx, int uly,
                                              float s, float t, bool active, int px, int py, uint32_t A, int lane,
                                              uint32_t lt, FbTable *tab) {
    const int na = __popc(A);
    const int ai = __popc(A & lt);
    int dx = 0, dy = 0;
    float xi2 = 0.f;
    if (active) stf_draw(px, py + y0, view, k0, k1, s, t, dx, dy, xi2);
    const int sx = ulx + dx, sy = uly + dy;
    FbChoice c;
    c.qx = sx;
    c.qy = sy;
    c.produce = active;
    if (mode == 2) {
        // distinct STF texels: the lowest active lane of each group leads
        const unsigned long long skey = active ? texel_key(sx, sy) : texel_key(INT_MIN, lane);  // distinct when inactive
        const uint32_t grp = __match_any_sync(FULL, skey);
        const uint32_t L = __ballot_sync(FULL, active && (__ffs(grp) - 1) == lane);
        const int n = __popc(L);
        if (active) fb_insert(tab, skey, lane);
        __syncwarp();
        const int lead = nth_set_lane(L, active && ai < n ? ai : 0);
        const int ux = __shfl_sync(FULL, sx, lead), uy = __shfl_sync(FULL, sy, lead);
        // remaining lanes: the footprint of source lane h(l, A)
        const bool extra = active && ai >= n;
        int l = 0;
        if (extra) {
            const int den = na - 1 - n;
            l = den == 0 ? 0 : (2 * (na - 1) * (ai - n) + den) / (2 * den);
        }
        const int src = nth_set_lane(A, l);
        const int sux = __shfl_sync(FULL, ulx, src), suy = __shfl_sync(FULL, uly, src);
        const float ss = __shfl_sync(FULL, s, src), st = __shfl_sync(FULL, t, src);
        if (!extra) {
            c.qx = ux;
            c.qy = uy;
            c.produce = active;
        } else {
            float w[4];
            bilinear_weights(ss, st, w);
            bool cand[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool in_set = fb_find(tab, texel_key(sux + (k & 1), suy + (k >> 1))) >= 0;
                cand[k] = w[k] > 0.f && !in_set;
            }
            float wc = 0.f;
            int last = -1;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (cand[k]) {
                    wc = __fadd_rn(wc, w[k]);
                    last = k;
                }
            }
            c.produce = last >= 0;
            if (c.produce) {
                const float tsel = __fmul_rn(xi2, wc);
                float run = 0.f;
                int pick = last;
                bool done = false;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (cand[k] && !done) {
                        run = __fadd_rn(run, w[k]);
                        if (tsel < run) {
                            pick = k;
                            done = true;
                        }
                    }
                }
                c.qx = sux + (pick & 1);
                c.qy = suy + (pick >> 1);
            }
        }
        __syncwarp();
        fb_clear(tab, lane);
        __syncwarp();
    }
    return c;
}

// Eq. 1 for every active pixel of the tile, given each lane's produced
// value `val` (the texel fb_choose chose; non-producers pass anything):
// the produced texels of the pixel's footprint with nonzero weight, found in
// the warp's table.  kAlphaOne: the texels' alpha is 1 (block textures), and
// val.w is not read.  Warp-collective; leaves the table empty.
template <bool kAlphaOne>
__device__ __forceinline__ FallbackOut fb_blend(float4 val, const FbChoice &c, int ulx, int uly, float s, float t,
                                                bool active, int lane, FbTable *tab) {
    if (c.produce) fb_insert(tab, texel_key(c.qx, c.qy), lane);
    __syncwarp();
    float w[4];
    bilinear_weights(s, t, w);
    int srcl[4];
    bool pres[4];
    int nz = 0, N = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        // any lane that produced the texel holds its value
        const int found = fb_find(tab, texel_key(ulx + (k & 1), uly + (k >> 1)));
        pres[k] = active && w[k] > 0.f && found >= 0;
        srcl[k] = found >= 0 ? found : lane;
        nz += w[k] > 0.f ? 1 : 0;
        N += pres[k] ? 1 : 0;
    }
    float4 tv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        tv[k].x = __shfl_sync(FULL, val.x, srcl[k]);
        tv[k].y = __shfl_sync(FULL, val.y, srcl[k]);
        tv[k].z = __shfl_sync(FULL, val.z, srcl[k]);
        tv[k].w = kAlphaOne ? 1.0f : __shfl_sync(FULL, val.w, srcl[k]);
    }
    __syncwarp();
    fb_clear(tab, lane);  // empty for the next tile
    __syncwarp();
    FallbackOut o;
    o.res = make_float4(0.f, 0.f, 0.f, 0.f);
    o.count = c.produce ? 1u : 0u;
    if (!active) return o;
    if (N == 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (pres[k]) o.res = tv[k];
        return o;
    }
    float4 swp = make_float4(0.f, 0.f, 0.f, 0.f), sp = make_float4(0.f, 0.f, 0.f, 0.f);
    float sw = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (!pres[k]) continue;
        swp.x = __fmaf_rn(w[k], tv[k].x, swp.x);
        swp.y = __fmaf_rn(w[k], tv[k].y, swp.y);
        swp.z = __fmaf_rn(w[k], tv[k].z, swp.z);
        swp.w = __fmaf_rn(w[k], tv[k].w, swp.w);
        sw = __fadd_rn(sw, w[k]);
        sp.x = __fadd_rn(sp.x, tv[k].x);
        sp.y = __fadd_rn(sp.y, tv[k].y);
        sp.z = __fadd_rn(sp.z, tv[k].z);
        sp.w = __fadd_rn(sp.w, tv[k].w);
    }
    if (N == nz) {
        o.res = swp;
        return o;
    }
    const float r = __fsub_rn(1.0f, sw), fn = (float)N;
    o.res = make_float4(__fmaf_rn(r, __fdiv_rn(sp.x, fn), swp.x), __fmaf_rn(r, __fdiv_rn(sp.y, fn), swp.y),
                        __fmaf_rn(r, __fdiv_rn(sp.z, fn), swp.z), __fmaf_rn(r, __fdiv_rn(sp.w, fn), swp.w));
    return o;
}

__device__ __noinline__ FallbackOut fallback_blend(const FallbackArgs fa, int ulx, int uly, float s, float t,
                                                   bool active, int px, int py, uint32_t A, int lane, uint32_t lt,
                                                   const DecodeTables *tabs, FbTable *tab) {
    const FbChoice c = fb_choose(fa.mode, fa.view, fa.y0, fa.k0, fa.k1, ulx, uly, s, t, active, px, py, A, lane, lt, tab);
    // produce; every lane decodes (non-producers their own clamped texel)
    float3 val;
    {
        const int x = min(max(c.produce ? c.qx : ulx, 0), fa.Wt - 1), y = min(max(c.produce ? c.qy : uly, 0), fa.Ht - 1);
        const uint2 blk = __ldg(fa.blocks + ck((uint32_t)(y >> 2) * (uint32_t)fa.nbx + (uint32_t)(x >> 2),
                                               (long long)fa.nbx * (fa.Ht / 4), fa.err, kBndBlock));
        val = decode_texel_f(blk, x, y, tabs, fa.err);
    }
    return fb_blend<true>(make_float4(val.x, val.y, val.z, 1.0f), c, ulx, uly, s, t, active, lane, tab);
}

// CTAs of 8 warps per SM that the exact kernels ask the compiler to fit:
// the collaborative kernels are issue-bound, and five CTAs (40 warps) hide
// more latency than the registers a looser cap would buy.
template <int ALG>
constexpr int min_blocks() {
    return ALG >= ALG_LIST ? 5 : 1;
}

// kExt: the code for the optional extensions that a kernel variant carries,
// fallbacks C / C+ (kExtFallback, for p.fallback != 0) and two texels per
// lane (kExtTwo, for p.tpl == 2); the variant without either carries none.
constexpr int kExtFallback = 1, kExtTwo = 2;

template <int ALG, int TW, int MD, bool kStats, int kExt = 0>
__device__ __forceinline__ void filter_tile(const ExactParams &p, const Inputs &in, int px, int py, bool inside,
                                            uint32_t idx, int lane, uint32_t lt, const DecodeTables *tabs,
                                            ListTable *T, int *ranks, FbTable *fbtab, Counters &cnt) {
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
        const Selection sel =
            select_tile<ALG, MD, kStats, true, (kExt & kExtTwo) != 0>(p, ps, in.jac, px, py, lane, lt, T, ranks, cnt);
        if ((kExt & kExtFallback) && ALG >= ALG_LIST && p.fallback != 0 && sel.path == PATH_FALLBACK_BUDGET) {
            // fallback C or C+ in place of one-tap STF
            FallbackArgs fa;
            fa.blocks = p.blocks;
            fa.Wt = p.Wt;
            fa.Ht = p.Ht;
            fa.nbx = p.nbx;
            fa.view = p.view;
            fa.y0 = p.y0;
            fa.k0 = p.k0;
            fa.k1 = p.k1;
            fa.mode = p.fallback;
            fa.err = p.err;
            const FallbackOut fo =
                fallback_blend(fa, ps.ulx, ps.uly, ps.s, ps.t, ps.active, px, py, sel.A, lane, lt, tabs, fbtab);
            if (kStats) {  // select_tile counted one evaluation per active lane
                const int d = __popc(__ballot_sync(FULL, fo.count != 0)) - __popc(sel.A);
                cnt.v[kStatTexelEvals] += d;
                cnt.v[kStatTexelEvalsUnique] += d;
            }
            if (inside) store_pixel(p, idx, fo.res, (uint8_t)fo.count);
            return;
        }
        // step 2: exact decode of the lane's texel (clamped to the texture);
        // lanes that produce nothing decode their own upper-left texel, which
        // the warp reads anyway, and drop it
        const float3 val = fetch_decode(p, sel.tx, sel.ty, tabs);
        const bool two = (kExt & kExtTwo) && ALG >= ALG_LIST && p.tpl == 2;
        if (sel.path == PATH_SUCCESS) {
            // step 3: gather the 2x2 taps from their producers and filter
            float3 t[4];
            if (two) {
                // second texels (non-producers decode their own texel again)
                const float3 val2 = fetch_decode(p, sel.produce2 ? sel.tx2 : sel.tx, sel.produce2 ? sel.ty2 : sel.ty,
                                                 tabs);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int l = sel.src[k] & 31;
                    const bool r = sel.src[k] >= 32;
                    const float ax = __shfl_sync(FULL, val.x, l), bx = __shfl_sync(FULL, val2.x, l);
                    const float ay = __shfl_sync(FULL, val.y, l), by = __shfl_sync(FULL, val2.y, l);
                    const float az = __shfl_sync(FULL, val.z, l), bz = __shfl_sync(FULL, val2.z, l);
                    t[k] = make_float3(r ? bx : ax, r ? by : ay, r ? bz : az);
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    t[k].x = __shfl_sync(FULL, val.x, sel.src[k]);
                    t[k].y = __shfl_sync(FULL, val.y, sel.src[k]);
                    t[k].z = __shfl_sync(FULL, val.z, sel.src[k]);
                }
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
