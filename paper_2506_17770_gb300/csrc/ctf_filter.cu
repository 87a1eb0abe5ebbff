// ctf_filter.cu -- exact-decode filter kernels (per-pixel 4-tap, one-tap STF,
// List Merge, Box Sampling, Mask Sampling) for sm_103a.
//
// One warp filters one tile_w x tile_h pixel tile at a time and walks the
// frame with a grid stride, prefetching the next tile's inputs while it works
// on the current one.  The collaborative algorithms follow the flow of Sec. 3:
// (1) the warp collects the texel set its 2x2 footprints need, (2) each needed
// texel is decoded once, by lane h(i, A) (edge remapping, supplemental
// Sec. 2), and converted to float there, (3) every pixel gathers its 4 taps
// with shuffles and filters.  Over-budget or minified warps take the one-tap
// STF fallback.
//
// Data layout in HBM: uv float2 and jac float4 per pixel, row-major; output
// float4 per pixel plus one count byte.  The texture (8-byte blocks) is read
// through L1/L2 with __ldg; the per-pixel streams use evict-first loads and
// stores so that they do not push the texture out of L2.
//
// The path is issue-bound rather than bandwidth-bound unless the instruction
// count per tile stays near 200, so the code avoids per-lane divisions, 64-bit
// index arithmetic and per-tap work that can be derived from a neighbour
// (taps (1,0) and (1,1) sit one texel after taps (0,0) and (0,1) in both the
// box raster order and the mask bit order).
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "ctf_device.cuh"
#include "ctf_internal.h"
#include "ctf_select.cuh"
#include "ctf_exact_tile.cuh"

namespace ctf {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;

template <int ALG, int TW, int MD, bool kStats, int kExt>
__global__ void __launch_bounds__(kThreads, kExt ? 4 : min_blocks<ALG>()) exact_filter_kernel(const ExactParams p) {
    constexpr int TH = 32 / TW;
    constexpr bool kJac = ALG >= ALG_LIST;
    __shared__ DecodeTables tabs;
    __shared__ int rank_slots[kWarps][64];
    __shared__ FbTable fb_tab[kWarps];  // fallback C / C+ texel lookups
    __shared__ unsigned long long block_stats[kNumStats];
    extern __shared__ __align__(16) unsigned char dyn_smem[];

    if (threadIdx.x < kNumStats) block_stats[threadIdx.x] = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ListTable *T = ALG == ALG_LIST ? reinterpret_cast<ListTable *>(dyn_smem) + warp : nullptr;
    if (ALG == ALG_LIST) {
#pragma unroll
        for (int s = 0; s < 8; ++s) T->keys[lane * 8 + s] = kEmpty;
    }
    if (kExt & kExtFallback) fb_clear(&fb_tab[warp], lane);  // the fallback's texel table starts empty

    const int tx = lane % TW, ty = lane / TW;
    const uint32_t lt = lanemask_lt();
    Counters cnt;
#pragma unroll
    for (int i = 0; i < kNumStats; ++i) cnt.v[i] = 0;

    // Warp-uniform tile walk: tile -> (bx, by) once, then advanced by the
    // grid stride without dividing again.  A pixel's index is the tile's
    // first pixel plus a per-lane offset, and the lane is inside the frame
    // while bx < lim_x and by < lim_y (per-lane bounds).  Lanes outside
    // read pixel 0, which exists whenever there is a tile, and drop it.
    const uint32_t W = (uint32_t)p.W, H = (uint32_t)p.H;
    const uint32_t ntiles = (uint32_t)p.n_tiles, tiles_x = (uint32_t)p.tiles_x;
    const uint32_t lim_x = (W - (uint32_t)tx + TW - 1) / TW, lim_y = (H - (uint32_t)ty + TH - 1) / TH;
    const uint32_t lane_off = (uint32_t)ty * W + (uint32_t)tx;
    const uint32_t stride = gridDim.x * kWarps;
    const uint32_t sbx = stride % tiles_x, sby = stride / tiles_x;
    const uint32_t tile0 = blockIdx.x * kWarps + warp;
    const uint32_t n_mine = tile0 < ntiles ? (ntiles - 1u - tile0) / stride + 1u : 0u;
    uint32_t bx = tile0 % tiles_x, by = tile0 / tiles_x;

    bool inside = n_mine > 0 && bx < lim_x && by < lim_y;
    uint32_t idx = by * (TH * W) + bx * TW + lane_off;
    Inputs cur = load_inputs_any<kJac>(p, inside, idx);
    // the decode tables come in while the first tile's inputs are in flight
    load_decode_tables(&tabs, p.tables);
    __syncthreads();

    for (uint32_t i = 0; i < n_mine; ++i) {
        // prefetch the next tile of this warp
        uint32_t nbx = bx + sbx, nby = by + sby;
        if (nbx >= tiles_x) {
            nbx -= tiles_x;
            ++nby;
        }
        const bool ninside = i + 1u < n_mine && nbx < lim_x && nby < lim_y;
        const uint32_t nidx = nby * (TH * W) + nbx * TW + lane_off;
        const Inputs nxt = load_inputs_any<kJac>(p, ninside, nidx);

        filter_tile<ALG, TW, MD, kStats, kExt>(p, cur, (int)(bx * TW) + tx, (int)(by * TH) + ty, inside, idx, lane, lt,
                                         &tabs, T, rank_slots[warp], &fb_tab[warp], cnt);

        bx = nbx;
        by = nby;
        inside = ninside;
        idx = nidx;
        cur = nxt;
    }

    if (kStats && p.stats) {  // (the extension variants always count; p.stats decides)
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < kNumStats; ++i)
                if (cnt.v[i]) atomicAdd(&block_stats[i], (unsigned long long)cnt.v[i]);
        }
        __syncthreads();
        if (threadIdx.x < kNumStats && block_stats[threadIdx.x]) atomicAdd(p.stats + threadIdx.x, block_stats[threadIdx.x]);
    }
}

using KernelFn = void (*)(const ExactParams);

// The collaborative algorithms have variants for the optional extensions
// (fallbacks C / C+, two texels per lane, both).  These are built with the
// counters only (kStats; a null stats pointer skips the final sums), which
// halves their number.
template <int ALG, int TW, int MD, bool kStats>
KernelFn pick_fb(int ext) {
    if constexpr (ALG >= ALG_LIST && kStats) {
        switch (ext) {
        case kExtFallback: return exact_filter_kernel<ALG, TW, MD, kStats, kExtFallback>;
        case kExtTwo: return exact_filter_kernel<ALG, TW, MD, kStats, kExtTwo>;
        case kExtFallback | kExtTwo: return exact_filter_kernel<ALG, TW, MD, kStats, kExtFallback | kExtTwo>;
        default: return exact_filter_kernel<ALG, TW, MD, kStats, 0>;
        }
    } else {
        return exact_filter_kernel<ALG, TW, MD, kStats, 0>;
    }
}

template <int ALG, int TW, bool kStats>
KernelFn pick_mask(int md, int fb) {
    if constexpr (ALG == ALG_MASK) {
        return md == 11 ? pick_fb<ALG, TW, 11, kStats>(fb) : pick_fb<ALG, TW, 16, kStats>(fb);
    } else {
        return pick_fb<ALG, TW, 16, kStats>(fb);
    }
}

template <int TW, bool kStats>
KernelFn pick_alg(int alg, int md, int fb) {
    switch (alg) {
    case ALG_4TAP: return pick_mask<ALG_4TAP, TW, kStats>(md, fb);
    case ALG_STF: return pick_mask<ALG_STF, TW, kStats>(md, fb);
    case ALG_LIST: return pick_mask<ALG_LIST, TW, kStats>(md, fb);
    case ALG_BOX: return pick_mask<ALG_BOX, TW, kStats>(md, fb);
    case ALG_MASK: return pick_mask<ALG_MASK, TW, kStats>(md, fb);
    default: return nullptr;
    }
}

}  // namespace

int device_sm_count() {
    static int cached_dev = -1, cached = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != cached_dev) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached = n > 0 ? n : 1;
        cached_dev = dev;
    }
    return cached;
}

cudaError_t launch_exact_filter(const ExactParams &p, int alg, int tile_w, int mask_dim, cudaStream_t stream) {
    KernelFn fn = nullptr;
    const bool st = p.stats != nullptr;
    const int fb = (p.fallback != 0 ? kExtFallback : 0) | (p.tpl == 2 ? kExtTwo : 0);
    switch (tile_w) {
    case 8: fn = st || fb ? pick_alg<8, true>(alg, mask_dim, fb) : pick_alg<8, false>(alg, mask_dim, 0); break;
    case 4: fn = st || fb ? pick_alg<4, true>(alg, mask_dim, fb) : pick_alg<4, false>(alg, mask_dim, 0); break;
    case 16: fn = st || fb ? pick_alg<16, true>(alg, mask_dim, fb) : pick_alg<16, false>(alg, mask_dim, 0); break;
    default: return cudaErrorInvalidValue;
    }
    if (!fn) return cudaErrorInvalidValue;
    if (p.n_tiles == 0) return cudaSuccess;
    if (p.n_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    const size_t smem = alg == ALG_LIST ? sizeof(ListTable) * kWarps : 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long want = (p.n_tiles + kWarps - 1) / kWarps;
    const long long cap = (long long)device_sm_count() * per_sm;
    const int grid = (int)(want < cap ? want : cap);
    fn<<<grid, kThreads, smem, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace ctf
