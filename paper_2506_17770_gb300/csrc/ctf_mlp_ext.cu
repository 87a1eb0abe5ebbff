// ctf_mlp_ext.cu -- learned-decode filter with the extensions of the
// collaborative flow: fallbacks C and C+ (Sec. 3.4, eq. 1 and 2) for tiles
// over budget, and up to two texels per lane (Sec. 5), for List Merge, Box
// and Mask Sampling on single views.
//
// A CTA of 4 warps holds one 128-row tcgen05 MLP chain (ctf_mlp_chain.cuh):
// warp w takes one pixel tile per iteration and owns rows 32w..32w+31.
//   - step 1 as in the other kernels (select_tile, with the second texel of
//     a lane when texels_per_lane is 2); for a tile over budget whose
//     magnification allows it, fb_choose (shared with the exact decode)
//     picks the texel each lane produces under C or C+;
//   - step 2: each lane's texel goes into its own row, and the CTA runs the
//     chain; when any lane of the CTA has a second texel, a second chain
//     evaluates those (round 1);
//   - step 3: a success tile reads tap k from lane src mod 32 in round
//     src div 32 and filters; a C / C+ tile blends each pixel's produced
//     footprint texels by eq. 1 (fb_blend, with the texels' learned alpha);
//     one-tap STF returns the lane's own texel.
// Every texel value is the chain's value for its row, as in every learned
// kernel, so each pixel gets the texels, counts and arithmetic of the exact
// path with the learned texel values in place of the decoded ones.
#include <climits>
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

// The warps' fallback tables and rank slots reuse the packed-group buffers
// of the chain's layout (this kernel has no packed groups).  With two texels
// per lane a Mask tile may hold up to 64 texels, so each warp has 64 rank
// slots (the chain layout's own rank slots hold 32).
constexpr int kSmFb = kSmPixST;
constexpr int kSmExtRanks = kSmFb + 4 * (int)sizeof(FbTable);  // 4 warps x 64 ints
static_assert(kSmExtRanks % 16 == 0 && kSmExtRanks + 4 * 64 * 4 <= kSmCount,
              "fallback tables and rank slots inside the group buffers");

template <int ALG, int TW, int MD>
__device__ __forceinline__ bool ext_warp_tile(const ExactParams &p, const MlpDevice &m, Chain &ch, long long tile,
                                              int lane, uint32_t lt, ListTable *T, FbTable *fbt, int *ranks,
                                              Counters &cnt, const float *inv_a1, int *err) {
    constexpr int TH = 32 / TW;
    unsigned char *sm = ch.sm;
    const int tx = lane % TW, ty = lane / TW;
    const bool valid = tile < p.n_tiles;
    const uint32_t t32 = (uint32_t)tile, tiles_x = (uint32_t)p.tiles_x;  // fewer than 2^31 tiles
    const int by = valid ? (int)(t32 / tiles_x) : 0, bx = valid ? (int)(t32 - (uint32_t)by * tiles_x) : 0;
    const int px = bx * TW + tx, py = by * TH + ty;
    const bool inside = valid && px < p.W && py < p.H;
    const uint32_t idx = ck(inside ? (uint32_t)py * (uint32_t)p.W + (uint32_t)px : 0u, view_pixels(p), p.err,
                            kBndPixel);
    float2 uv = make_float2(0.f, 0.f);
    float4 jac = make_float4(0.f, 0.f, 0.f, 0.f);
    bool covered = inside;
    if (inside) {
        uv = __ldcs(p.uv + idx);
        jac = __ldcs(p.jac + idx);
        if (p.cov) covered = __ldcs(p.cov + idx) != 0;
    }
    PixelSetup ps;
    ps.active = covered;
    setup_coords(uv, (float)p.Wt, (float)p.Ht, ps);
    Selection sel;
    if (valid) {
        sel = select_tile<ALG, MD, true, true, true>(p, ps, jac, px, py, lane, lt, T, ranks, cnt);
    } else {
        sel.path = PATH_EMPTY;
        sel.A = 0;
        sel.produce = sel.produce2 = false;
        sel.tx = sel.ty = sel.tx2 = sel.ty2 = 0;
        sel.count = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) sel.src[k] = lane;
    }
    // fallback C or C+ in place of one-tap STF (warp-uniform)
    const bool fbc = p.fallback != 0 && sel.path == PATH_FALLBACK_BUDGET;
    FbChoice fc;
    fc.produce = false;
    fc.qx = fc.qy = 0;
    if (fbc) fc = fb_choose(p.fallback, p.view, p.y0, p.k0, p.k1, ps.ulx, ps.uly, ps.s, ps.t, ps.active, px, py, sel.A,
                            lane, lt, fbt);
    // step 2: the lane's texel in its own row (lanes that produce nothing
    // decode a zero row, whose value nobody reads)
    const bool prod0 = fbc ? fc.produce : sel.produce;
    const int x0 = fbc ? fc.qx : sel.tx, y0 = fbc ? fc.qy : sel.ty;
    if (prod0) {
        float f[kMlpIn];
        texel_features(m, min(max(x0, 0), p.Wt - 1), min(max(y0, 0), p.Ht - 1), f);
        store_x_row(sm, threadIdx.x, f, m.fp8, inv_a1);
    } else {
        store_zero_x_row(sm, threadIdx.x);
    }
    float4 val0, val1 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!mlp_chain(ch, m.fp8, val0, err)) return false;
    // round 1: second texels, when any lane of the CTA has one (CTA-uniform)
    if (__syncthreads_or(sel.produce2)) {
        if (sel.produce2) {
            float f[kMlpIn];
            texel_features(m, min(max(sel.tx2, 0), p.Wt - 1), min(max(sel.ty2, 0), p.Ht - 1), f);
            store_x_row(sm, threadIdx.x, f, m.fp8, inv_a1);
        } else {
            store_zero_x_row(sm, threadIdx.x);
        }
        if (!mlp_chain(ch, m.fp8, val1, err)) return false;
    }
    float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t count = 0;
    if (fbc) {
        const FallbackOut fo = fb_blend<false>(val0, fc, ps.ulx, ps.uly, ps.s, ps.t, ps.active, lane, fbt);
        // select_tile counted one evaluation per active lane
        const int d = __popc(__ballot_sync(FULL, fo.count != 0)) - __popc(sel.A);
        if (lane == 0) {
            cnt.v[kStatTexelEvals] += d;
            cnt.v[kStatTexelEvalsUnique] += d;
        }
        res = fo.res;
        count = fo.count;
    } else if (sel.path == PATH_SUCCESS) {
        // step 3: tap k from lane src mod 32 in round src div 32
        float4 tap[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int sk = sel.src[k];  // lane + 32 x round (checked in select_tile)
            const int l = sk & 31;
            const bool r = sk >= 32;
            const float ax = __shfl_sync(FULL, val0.x, l), bx1 = __shfl_sync(FULL, val1.x, l);
            const float ay = __shfl_sync(FULL, val0.y, l), by1 = __shfl_sync(FULL, val1.y, l);
            const float az = __shfl_sync(FULL, val0.z, l), bz1 = __shfl_sync(FULL, val1.z, l);
            const float aw = __shfl_sync(FULL, val0.w, l), bw1 = __shfl_sync(FULL, val1.w, l);
            tap[k] = make_float4(r ? bx1 : ax, r ? by1 : ay, r ? bz1 : az, r ? bw1 : aw);
        }
        if (ps.active) {
            float w[4];
            bilinear_weights(ps.s, ps.t, w);
            float2 rg = make_float2(0.f, 0.f), ba = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 wk = make_float2(w[k], w[k]);
                rg = __ffma2_rn(wk, make_float2(tap[k].x, tap[k].y), rg);
                ba = __ffma2_rn(wk, make_float2(tap[k].z, tap[k].w), ba);
            }
            res = make_float4(rg.x, rg.y, ba.x, ba.y);
            count = sel.count;
        }
    } else if (ps.active) {
        res = val0;  // one-tap STF (minified or fallback 0): the lane's own texel
        count = 1;
    }
    if (inside) {
        __stcs(p.out + idx, res);
        if (p.evals) p.evals[idx] = (uint8_t)count;
    }
    return true;
}

template <int ALG, int TW, int MD>
__global__ void __launch_bounds__(kRows, 3) mlp_filter_ext_kernel(const ExactParams p, const MlpDevice m, int *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ unsigned long long block_stats[kNumStats];
    Chain ch;
    chain_setup(ch, sm, m);
    const float *inv_a1 = reinterpret_cast<const float *>(sm + kImgA1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ListTable *T = reinterpret_cast<ListTable *>(sm + kSmList) + warp;
    FbTable *fbt = reinterpret_cast<FbTable *>(sm + kSmFb) + warp;
    int *ranks = reinterpret_cast<int *>(sm + kSmExtRanks) + 64 * warp;
    if (ALG == ALG_LIST) {
#pragma unroll
        for (int s = 0; s < 8; ++s) T->keys[lane * 8 + s] = kEmpty;
    }
    fb_clear(fbt, lane);  // the fallback's texel table starts empty
    if (threadIdx.x < kNumStats) block_stats[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t lt = lanemask_lt();
    Counters cnt;
#pragma unroll
    for (int i = 0; i < kNumStats; ++i) cnt.v[i] = 0;
    const long long n_iter = (p.n_tiles + 3) / 4;
    bool ok = true;
    for (long long it = blockIdx.x; it < n_iter && ok; it += gridDim.x)
        ok = ext_warp_tile<ALG, TW, MD>(p, m, ch, it * 4 + warp, lane, lt, T, fbt, ranks, cnt, inv_a1, err);
    if (p.stats && lane == 0) {
#pragma unroll
        for (int i = 0; i < kNumStats; ++i)
            if (cnt.v[i]) atomicAdd(&block_stats[i], (unsigned long long)cnt.v[i]);
    }
    chain_teardown(ch);
    if (p.stats && threadIdx.x < kNumStats && block_stats[threadIdx.x])
        atomicAdd(p.stats + threadIdx.x, block_stats[threadIdx.x]);
}

using ExtFn = void (*)(const ExactParams, const MlpDevice, int *);

template <int TW>
ExtFn ext_pick(int alg, int md) {
    switch (alg) {
    case ALG_LIST: return mlp_filter_ext_kernel<ALG_LIST, TW, 16>;
    case ALG_BOX: return mlp_filter_ext_kernel<ALG_BOX, TW, 16>;
    case ALG_MASK: return md == 11 ? mlp_filter_ext_kernel<ALG_MASK, TW, 11> : mlp_filter_ext_kernel<ALG_MASK, TW, 16>;
    default: return nullptr;
    }
}

ExtFn ext_kernel(int alg, int tile_w, int mask_dim) {
    switch (tile_w) {
    case 8: return ext_pick<8>(alg, mask_dim);
    case 4: return ext_pick<4>(alg, mask_dim);
    case 16: return ext_pick<16>(alg, mask_dim);
    default: return nullptr;
    }
}

cudaError_t ext_prepare(ExtFn fn) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(dev, reinterpret_cast<const void *>(fn));
    if (done.count(key)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmRequest);
    if (e == cudaSuccess) done.insert(key);
    return e;
}

}  // namespace

bool mlp_filter_ext_applies(const ExactParams &p, int alg) {
    return (alg == ALG_LIST || alg == ALG_BOX || alg == ALG_MASK) && (p.fallback != 0 || p.tpl == 2);
}

cudaError_t prepare_mlp_filter_ext(int alg, int tile_w, int mask_dim) {
    ExtFn fn = ext_kernel(alg, tile_w, mask_dim);
    return fn ? ext_prepare(fn) : cudaErrorInvalidValue;
}

cudaError_t launch_mlp_filter_ext(const ExactParams &p, const MlpDevice &m, int alg, int tile_w, int mask_dim, int *err,
                                  cudaStream_t stream) {
    ExtFn fn = ext_kernel(alg, tile_w, mask_dim);
    if (!fn) return cudaErrorInvalidValue;
    if (p.n_tiles == 0) return cudaSuccess;
    if (p.n_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;  // tile positions use 32-bit arithmetic
    cudaError_t e = ext_prepare(fn);
    if (e != cudaSuccess) return e;
    const long long iters = (p.n_tiles + 3) / 4;
    const long long cap = (long long)device_sm_count() * 4;
    const int grid = (int)(iters < cap ? iters : cap);
    fn<<<grid, kRows, kSmRequest, stream>>>(p, m, err);
    return cudaGetLastError();
}

}  // namespace ctf
