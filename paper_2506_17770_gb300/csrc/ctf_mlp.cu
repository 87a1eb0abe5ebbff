// ctf_mlp.cu -- learned texel decode on the 5th-generation tensor cores.
//
// The paper produces texels with a neural decompressor (Sec. 4.3.1, "inference
// on sample") and notes that collaborative filtering cuts the number of such
// evaluations per pixel; this module is that costly texel evaluation.  A texel
// (x, y) is decoded by
//   f = bilinear samples of two FP16 latent grids at the texel centre (16 ch)
//   h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), rgba = saturate(W3 h2 + b3)
// with FP16 (or FP8 E4M3) operands and FP32 accumulation.
//
// One CTA of 128 threads owns a 128-row tile: thread r computes the features
// of row r into shared memory, one elected thread issues the three layers as
// tcgen05.mma (M = 128; N = 64, 64, 16; K = 16 or 64) with the accumulators in
// tensor memory, and after each layer every thread reads its row back with
// tcgen05.ld (warp w owns TMEM lanes 32w..32w+31), adds the bias, applies the
// ReLU, converts, and writes the next layer's A operand.  MMA completion is
// tracked with an mbarrier whose waits are bounded: a wait that gives up sets
// the library's error word and every thread of the CTA leaves together.
//
// Two kernels here use the chain: a decode of an explicit list of texels, and
// the learned-decode filter for per-pixel 4-tap and List Merge.  Per-pixel
// 4-tap gives each warp one pixel tile (its lane's row per tap, four chains
// per iteration); List Merge gives each warp two tiles of a group of 8, packs
// the group's texel lists into consecutive rows (one or two chains) and
// gathers every pixel's taps from the rows (ctf_mlp_chain.cuh, mlp_group;
// the persistent batch kernel runs the same for every algorithm).  STF, Box
// and Mask Sampling on single views run in the kernel whose warps are
// specialised by role (ctf_mlp_ws.cu), which gives the same outputs.
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

// ---------------------------------------------------------------------------
// Decode an explicit list of texels.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRows) mlp_decode_kernel(const MlpDevice m, int Wt, int Ht, const int2 *xy, int n,
                                                           float4 *out, int *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    Chain ch;
    chain_setup(ch, sm, m);
    const float *inv_a1 = reinterpret_cast<const float *>(sm + kImgA1);
    const int ntiles = (n + kRows - 1) / kRows;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int row = tile * kRows + threadIdx.x;
        if (row < n) {
            const int2 c = xy[row];
            const int x = min(max(c.x, 0), Wt - 1), y = min(max(c.y, 0), Ht - 1);
            float f[kMlpIn];
            texel_features(m, x, y, f);
            store_x_row(sm, threadIdx.x, f, m.fp8, inv_a1);
        } else {
            store_zero_x_row(sm, threadIdx.x);
        }
        float4 v;
        if (!mlp_chain(ch, m.fp8, v, err)) break;
        if (row < n) out[row] = v;
    }
    chain_teardown(ch);
}

// ---------------------------------------------------------------------------
// Learned-decode filter for per-pixel 4-tap and List Merge: 4 warps; a group
// of 8 pixel tiles (4 for per-pixel 4-tap) per CTA iteration.
// ---------------------------------------------------------------------------
template <int ALG, int TW, int MD>
__global__ void __launch_bounds__(kRows, 4) mlp_filter_kernel(const ExactParams p, const MlpDevice m, int *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ unsigned long long block_stats[kNumStats];
    Chain ch;
    chain_setup(ch, sm, m);
    const float *inv_a1 = reinterpret_cast<const float *>(sm + kImgA1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ListTable *T = reinterpret_cast<ListTable *>(sm + kSmList) + warp;
    if (ALG == ALG_LIST) {
#pragma unroll
        for (int s = 0; s < 8; ++s) T->keys[lane * 8 + s] = kEmpty;
    }
    if (threadIdx.x < kNumStats) block_stats[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t lt = lanemask_lt();
    Counters cnt;
#pragma unroll
    for (int i = 0; i < kNumStats; ++i) cnt.v[i] = 0;
    constexpr int kTiles = mlp_group_tiles(ALG);
    const long long n_iter = (p.n_tiles + kTiles - 1) / kTiles;
    bool ok = true;
    for (long long it = blockIdx.x; it < n_iter && ok; it += gridDim.x) {
        if (ALG == ALG_4TAP) ok = mlp_warp_tile<ALG, TW, MD>(p, m, ch, it * kTiles + warp, lane, lt, T, cnt, inv_a1, err);
        else ok = mlp_group<ALG, TW, MD>(p, m, ch, it * kTiles, lane, lt, T, cnt, inv_a1, err);
    }
    if (p.stats) {
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < kNumStats; ++i)
                if (cnt.v[i]) atomicAdd(&block_stats[i], (unsigned long long)cnt.v[i]);
        }
    }
    chain_teardown(ch);
    if (p.stats && threadIdx.x < kNumStats && block_stats[threadIdx.x])
        atomicAdd(p.stats + threadIdx.x, block_stats[threadIdx.x]);
}

// An mbarrier that nothing arrives on: every thread's bounded wait gives up
// and the CTA records a timeout, as the chain does for an MMA that never
// completes.
__global__ void bounded_wait_selftest_kernel(uint32_t polls, int *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    const bool done = tc::mbar_wait(&bar, 0, polls);
    if (__syncthreads_or(!done) && threadIdx.x == 0) atomicExch(err, CTF_ERR_TIMEOUT);
}

using FilterFn = void (*)(const ExactParams, const MlpDevice, int *);

template <int ALG, int TW>
FilterFn pick_mask(int md) {
    if constexpr (ALG == ALG_MASK) {
        return md == 11 ? mlp_filter_kernel<ALG, TW, 11> : mlp_filter_kernel<ALG, TW, 16>;
    } else {
        return mlp_filter_kernel<ALG, TW, 16>;
    }
}

// (STF, Box and Mask Sampling run in mlp_filter_ws_kernel.)
template <int TW>
FilterFn pick_alg(int alg, int md) {
    switch (alg) {
    case ALG_4TAP: return pick_mask<ALG_4TAP, TW>(md);
    case ALG_LIST: return pick_mask<ALG_LIST, TW>(md);
    default: return nullptr;
    }
}

// Opt each kernel into its dynamic shared memory once per device.
template <typename F>
cudaError_t prepare(F fn) {
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

cudaError_t launch_mlp_decode(const MlpDevice &m, int Wt, int Ht, const int2 *xy, int n, float4 *out, int *err,
                              cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = prepare(mlp_decode_kernel);
    if (e != cudaSuccess) return e;
    const int ntiles = (n + kRows - 1) / kRows;
    const int cap = device_sm_count() * 4;
    mlp_decode_kernel<<<ntiles < cap ? ntiles : cap, kRows, kSmRequest, stream>>>(m, Wt, Ht, xy, n, out, err);
    return cudaGetLastError();
}

cudaError_t prepare_mlp_filter(int alg, int tile_w, int mask_dim) {
    if (alg == ALG_LIST) {
        cudaError_t e = prepare_mlp_filter_pf(alg, tile_w, mask_dim);
        if (e != cudaSuccess) return e;
    }
    if (alg == ALG_STF || alg == ALG_BOX || alg == ALG_MASK) {
        cudaError_t e = prepare_mlp_filter_pf(alg, tile_w, mask_dim);
        return e == cudaSuccess ? prepare_mlp_filter_ws(alg, tile_w, mask_dim) : e;
    }
    FilterFn fn = nullptr;
    switch (tile_w) {
    case 8: fn = pick_alg<8>(alg, mask_dim); break;
    case 4: fn = pick_alg<4>(alg, mask_dim); break;
    case 16: fn = pick_alg<16>(alg, mask_dim); break;
    default: return cudaErrorInvalidValue;
    }
    return fn ? prepare(fn) : cudaErrorInvalidValue;
}

cudaError_t launch_bounded_wait_selftest(uint32_t polls, int *err, cudaStream_t stream) {
    bounded_wait_selftest_kernel<<<1, kRows, 0, stream>>>(polls, err);
    return cudaGetLastError();
}

cudaError_t launch_mlp_filter(const ExactParams &p, const MlpDevice &m, int alg, int tile_w, int mask_dim, int *err,
                              cudaStream_t stream) {
    // fallbacks C / C+ with one texel per lane on Box and Mask: the packed-group kernel's fallback variant
    if (mlp_filter_pf_fallback_applies(p, alg) || mlp_filter_pf_two_applies(p, alg))
        return launch_mlp_filter_pf(p, m, alg, tile_w, mask_dim, err, stream);
    // List Merge without extensions or group_dedup: the packed-group kernel's List Merge variant
    if (alg == ALG_LIST && p.fallback == 0 && p.tpl == 1 && !p.group_dedup)
        return launch_mlp_filter_pf(p, m, alg, tile_w, mask_dim, err, stream);
    if (mlp_filter_ext_applies(p, alg)) return launch_mlp_filter_ext(p, m, alg, tile_w, mask_dim, err, stream);
    if (mlp_filter_ws_applies(p, alg))
        return p.group_dedup ? launch_mlp_filter_ws(p, m, alg, tile_w, mask_dim, err, stream)
                             : launch_mlp_filter_pf(p, m, alg, tile_w, mask_dim, err, stream);
    FilterFn fn = nullptr;
    switch (tile_w) {
    case 8: fn = pick_alg<8>(alg, mask_dim); break;
    case 4: fn = pick_alg<4>(alg, mask_dim); break;
    case 16: fn = pick_alg<16>(alg, mask_dim); break;
    default: return cudaErrorInvalidValue;
    }
    if (!fn) return cudaErrorInvalidValue;
    if (p.n_tiles == 0) return cudaSuccess;
    if (p.n_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;  // tile positions use 32-bit arithmetic
    cudaError_t e = prepare(fn);
    if (e != cudaSuccess) return e;
    const long long iters = (p.n_tiles + mlp_group_tiles(alg) - 1) / mlp_group_tiles(alg);
    const long long cap = (long long)device_sm_count() * 4;
    const int grid = (int)(iters < cap ? iters : cap);
    fn<<<grid, kRows, kSmRequest, stream>>>(p, m, err);
    return cudaGetLastError();
}

}  // namespace ctf
