// ctf_batch.cu -- many views of uneven size and magnification in two
// persistent launches (one per kind of texel evaluation), optionally captured
// together into one CUDA graph, with an autotuner over the launch shape.
// Views large enough to fill the GPU alone (solo_tiles) are launched on
// their own with the single-view kernels, which then lose nothing to the
// persistent kernels' per-item view bookkeeping.
//
// Block views: persistent CTAs of 8 warps, like the per-view exact kernel;
// every warp takes items of 32 consecutive warp tiles of one view from an
// atomic counter (lane 0 fetches the next item while the current one runs)
// and walks them with the next tile's inputs prefetched.  Learned views:
// persistent CTAs of 4 warps that hold 128 TMEM columns for the whole launch;
// the CTA takes items of 8 warp tiles (two per warp, their texel lists packed
// into shared MLP chains; 4 tiles, one per warp, for per-pixel 4-tap),
// `items_per_fetch` at a time.  A prefix over each kind's per-view item
// counts maps an item to its view; the prefixes of up to 1024 block views
// (256 learned views) are cached in shared memory.
// Fetching is a plain fetch-and-add: no thread ever waits on another CTA.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ctf.h"
#include "ctf_device.cuh"
#include "ctf_exact_tile.cuh"
#include "ctf_internal.h"
#include "ctf_mlp_chain.cuh"
#include "ctf_select.cuh"

namespace ctf {
namespace {

constexpr int kBlockWarps = 8;         // warps per CTA of the block-view kernel
constexpr int kBlockItemTiles = 32;    // warp tiles per block-view item (one warp)
constexpr int kMaxViews = 4096;
constexpr int kSmViews = 1024;         // item prefixes cached in shared memory up to this many views
constexpr int kSmViewsMlp = 256;       // the same for the learned kernel (4 CTAs of it share an SM)


// One kind of views: their indices in the view table and item prefix.
struct BatchParams {
    const BatchViewDev *views;
    const int *index;             // views of this kind
    const long long *item_begin;  // nkind + 1 prefix
    int nkind;
    int nviews;                   // entries of the view table
    long long total_items;
    int items_per_fetch;
    unsigned long long *counter;
    unsigned long long *stats;
    int *err;
    const DecodeTables *tables;  // block views: the device's decode tables
};

// Last view whose first item is <= item (views with no items are skipped
// because the next view starts at the same item).
__device__ __forceinline__ int find_view(const long long *begin, const int *sbegin, int nviews, long long item) {
    int lo = 0, hi = nviews - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const long long b = sbegin ? (long long)sbegin[mid] : __ldg(begin + mid);
        if (b <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Block views: each warp on its own.
// ---------------------------------------------------------------------------
// The view bookkeeping costs registers: four CTAs per SM, not five as for the
// per-view kernels (at five the collaborative kernels spill).
template <int ALG>
constexpr int batch_min_blocks() {
    return ALG >= ALG_LIST ? 4 : 1;
}

template <int ALG, int TW, int MD, bool kFb>
__global__ void __launch_bounds__(kBlockWarps * 32, batch_min_blocks<ALG>()) batch_block_kernel(const BatchParams b) {
    constexpr int TH = 32 / TW;
    constexpr bool kJac = ALG >= ALG_LIST;
    __shared__ DecodeTables tabs;
    __shared__ int rank_slots[kBlockWarps][64];
    __shared__ FbTable fb_tab[kBlockWarps];  // fallback C / C+ texel lookups
    __shared__ unsigned long long block_stats[kNumStats];
    __shared__ int s_begin[kSmViews];
    __shared__ __align__(16) ExactParams s_params[kBlockWarps];  // each warp's current view
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    load_decode_tables(&tabs, b.tables);
    if (threadIdx.x < kNumStats) block_stats[threadIdx.x] = 0;
    const bool cached = b.nkind <= kSmViews && b.total_items < 0x7fffffffLL;
    if (cached)
        for (int i = threadIdx.x; i < b.nkind; i += blockDim.x) s_begin[i] = (int)__ldg(b.item_begin + i);
    const int *sb = cached ? s_begin : nullptr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ListTable *T = ALG == ALG_LIST ? reinterpret_cast<ListTable *>(dyn_smem) + warp : nullptr;
    if (ALG == ALG_LIST) {
#pragma unroll
        for (int s = 0; s < 8; ++s) T->keys[lane * 8 + s] = kEmpty;
    }
    if (kFb) fb_clear(&fb_tab[warp], lane);  // the fallback's texel table starts empty
    __syncthreads();
    const int tx = lane % TW, ty = lane / TW;
    const uint32_t lt = lanemask_lt();
    Counters cnt;
#pragma unroll
    for (int i = 0; i < kNumStats; ++i) cnt.v[i] = 0;

    // the next item is fetched while the current one is filtered
    int cur_k = -1;
    long long next = 0;
    if (lane == 0) next = (long long)atomicAdd(b.counter, 1ull);
    while (true) {
        const long long item = __shfl_sync(FULL, next, 0);
        if (item >= b.total_items) break;
        if (lane == 0) next = (long long)atomicAdd(b.counter, 1ull);
        const int k = ck(find_view(b.item_begin, sb, b.nkind, item), b.nkind, b.err, kBndBatch);
        if (k != cur_k) {
            // the view's parameters into this warp's shared-memory slot
            __syncwarp();
            const uint4 *src = reinterpret_cast<const uint4 *>(&b.views[ck(__ldg(b.index + k), b.nviews, b.err, kBndBatch)].p);
            uint4 *dst = reinterpret_cast<uint4 *>(&s_params[warp]);
            if (lane < (int)(sizeof(ExactParams) / 16)) dst[lane] = __ldg(src + lane);
            __syncwarp();
            cur_k = k;
        }
        const ExactParams &p = s_params[warp];
        const long long first = (item - (sb ? (long long)sb[k] : __ldg(b.item_begin + k))) * kBlockItemTiles;
        const long long last = min(first + kBlockItemTiles, (long long)p.n_tiles);
        // walk the item's tiles, the next tile's inputs in flight meanwhile;
        // a pixel's index is the tile's first pixel plus a per-lane offset,
        // and the lane is inside the frame while bx < lim_x and by < lim_y
        const uint32_t W = (uint32_t)p.W, H = (uint32_t)p.H, tiles_x = (uint32_t)p.tiles_x;
        const uint32_t lim_x = (W - (uint32_t)tx + TW - 1) / TW, lim_y = (H - (uint32_t)ty + TH - 1) / TH;
        const uint32_t lane_off = (uint32_t)ty * W + (uint32_t)tx;
        const uint32_t n_item = (uint32_t)(last - first);
        uint32_t bx = (uint32_t)(first % tiles_x), by = (uint32_t)(first / tiles_x);
        bool inside = n_item > 0 && bx < lim_x && by < lim_y;
        uint32_t idx = by * (TH * W) + bx * TW + lane_off;
        Inputs cur = load_inputs_any<kJac>(p, inside, idx);
        for (uint32_t i = 0; i < n_item; ++i) {
            uint32_t nbx = bx + 1, nby = by;
            if (nbx >= tiles_x) {
                nbx = 0;
                ++nby;
            }
            const bool ninside = i + 1u < n_item && nbx < lim_x && nby < lim_y;
            const uint32_t nidx = nby * (TH * W) + nbx * TW + lane_off;
            const Inputs nxt = load_inputs_any<kJac>(p, ninside, nidx);
            filter_tile<ALG, TW, MD, true, kFb ? kExtFallback | kExtTwo : 0>(p, cur, (int)(bx * TW) + tx, (int)(by * TH) + ty, inside, idx, lane, lt,
                                           &tabs, T, rank_slots[warp], &fb_tab[warp], cnt);
            bx = nbx;
            by = nby;
            inside = ninside;
            idx = nidx;
            cur = nxt;
        }
    }
    if (b.stats) {
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < kNumStats; ++i)
                if (cnt.v[i]) atomicAdd(&block_stats[i], (unsigned long long)cnt.v[i]);
        }
        __syncthreads();
        if (threadIdx.x < kNumStats && block_stats[threadIdx.x]) atomicAdd(b.stats + threadIdx.x, block_stats[threadIdx.x]);
    }
}

// ---------------------------------------------------------------------------
// Learned views: the 4 warps of a CTA share an MLP chain.
// ---------------------------------------------------------------------------
template <int ALG, int TW, int MD>
__global__ void __launch_bounds__(kRows, 4) batch_mlp_kernel(const BatchParams b) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ unsigned long long block_stats[kNumStats];
    __shared__ long long s_item;
    __shared__ int s_begin[kSmViewsMlp];
    __shared__ __align__(16) BatchViewDev s_view;  // the current item's view
    __shared__ int s_view_k;
    // the first view's network goes in now; a view with another network
    // reloads the operand image when its first item comes up
    Chain ch;
    const MlpDevice m0 = b.views[__ldg(b.index)].m;
    chain_setup(ch, sm, m0);
    if (threadIdx.x < kNumStats) block_stats[threadIdx.x] = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ListTable *T = reinterpret_cast<ListTable *>(sm + kSmList) + warp;
    if (ALG == ALG_LIST) {
#pragma unroll
        for (int s = 0; s < 8; ++s) T->keys[lane * 8 + s] = kEmpty;
    }
    const float *inv_a1 = reinterpret_cast<const float *>(sm + kImgA1);
    const uint32_t lt = lanemask_lt();
    Counters cnt;
#pragma unroll
    for (int i = 0; i < kNumStats; ++i) cnt.v[i] = 0;
    const unsigned char *loaded_img = reinterpret_cast<const unsigned char *>(m0.img);
    const bool cached = b.nkind <= kSmViewsMlp && b.total_items < 0x7fffffffLL;
    if (cached)
        for (int i = threadIdx.x; i < b.nkind; i += blockDim.x) s_begin[i] = (int)__ldg(b.item_begin + i);
    const int *sb = cached ? s_begin : nullptr;
    if (threadIdx.x == 0) s_view_k = -1;
    __syncthreads();

    bool ok = true;
    while (ok) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(b.counter, (unsigned long long)b.items_per_fetch);
        __syncthreads();
        const long long first = s_item;
        __syncthreads();
        if (first >= b.total_items) break;
        for (int k = 0; k < b.items_per_fetch && ok; ++k) {
            const long long item = first + k;
            if (item >= b.total_items) break;
            const int v = ck(find_view(b.item_begin, sb, b.nkind, item), b.nkind, b.err, kBndBatch);
            if (v != s_view_k) {
                // parameters of the new view into shared memory (CTA-uniform branch)
                __syncthreads();
                const uint4 *src = reinterpret_cast<const uint4 *>(b.views + ck(__ldg(b.index + v), b.nviews, b.err, kBndBatch));
                uint4 *dst = reinterpret_cast<uint4 *>(&s_view);
                for (int i = threadIdx.x; i < (int)(sizeof(BatchViewDev) / 16); i += blockDim.x) dst[i] = __ldg(src + i);
                if (threadIdx.x == 0) s_view_k = v;
                __syncthreads();
            }
            const BatchViewDev &V = s_view;
            const long long local = item - (sb ? (long long)sb[v] : __ldg(b.item_begin + v));
            const unsigned char *img = reinterpret_cast<const unsigned char *>(V.m.img);
            if (img != loaded_img) {
                tc::fence_before_sync();
                __syncthreads();
                uint4 *dst = reinterpret_cast<uint4 *>(sm + kSmImg);
                for (int i = threadIdx.x; i < kImgBytes / 16; i += blockDim.x)
                    dst[i] = __ldg(reinterpret_cast<const uint4 *>(img) + i);
                loaded_img = img;
                __syncthreads();
            }
            if (ALG == ALG_4TAP)
                ok = mlp_warp_tile<ALG, TW, MD>(V.p, V.m, ch, local * 4 + warp, lane, lt, T, cnt, inv_a1, b.err);
            else
                ok = mlp_group<ALG, TW, MD>(V.p, V.m, ch, local * kGroupTiles, lane, lt, T, cnt, inv_a1, b.err);
        }
    }
    if (b.stats && lane == 0) {
#pragma unroll
        for (int i = 0; i < kNumStats; ++i)
            if (cnt.v[i]) atomicAdd(&block_stats[i], (unsigned long long)cnt.v[i]);
    }
    chain_teardown(ch);
    if (b.stats && threadIdx.x < kNumStats && block_stats[threadIdx.x])
        atomicAdd(b.stats + threadIdx.x, block_stats[threadIdx.x]);
}

using BatchFn = void (*)(const BatchParams);

// Learned views never take fallbacks C / C+ (the plan refuses them); block
// views of the collaborative algorithms have a variant that does.
template <bool kMlp, int ALG, int TW, int MD>
BatchFn kernel_of(bool fb) {
    if constexpr (kMlp) {
        return batch_mlp_kernel<ALG, TW, MD>;
    } else if constexpr (ALG >= ALG_LIST) {
        return fb ? batch_block_kernel<ALG, TW, MD, true> : batch_block_kernel<ALG, TW, MD, false>;
    } else {
        return batch_block_kernel<ALG, TW, MD, false>;
    }
}

template <bool kMlp, int ALG, int TW>
BatchFn pick_mask(int md, bool fb) {
    if constexpr (ALG == ALG_MASK) {
        return md == 11 ? kernel_of<kMlp, ALG, TW, 11>(fb) : kernel_of<kMlp, ALG, TW, 16>(fb);
    } else {
        return kernel_of<kMlp, ALG, TW, 16>(fb);
    }
}

template <bool kMlp, int TW>
BatchFn pick_alg(int alg, int md, bool fb) {
    switch (alg) {
    case ALG_4TAP: return pick_mask<kMlp, ALG_4TAP, TW>(md, fb);
    case ALG_STF: return pick_mask<kMlp, ALG_STF, TW>(md, fb);
    case ALG_LIST: return pick_mask<kMlp, ALG_LIST, TW>(md, fb);
    case ALG_BOX: return pick_mask<kMlp, ALG_BOX, TW>(md, fb);
    case ALG_MASK: return pick_mask<kMlp, ALG_MASK, TW>(md, fb);
    default: return nullptr;
    }
}

BatchFn pick(bool mlp, int alg, int tile_w, int md, bool fb) {
    switch (tile_w) {
    case 8: return mlp ? pick_alg<true, 8>(alg, md, fb) : pick_alg<false, 8>(alg, md, fb);
    case 4: return mlp ? pick_alg<true, 4>(alg, md, fb) : pick_alg<false, 4>(alg, md, fb);
    case 16: return mlp ? pick_alg<true, 16>(alg, md, fb) : pick_alg<false, 16>(alg, md, fb);
    default: return nullptr;
    }
}

cudaError_t prepare_batch(BatchFn fn) {
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

struct ResolvedBatch {
    int tile_w = 8, tile_h = 4, budget = 32, mask_dim = 16, edge_remap = 1, group_dedup = 0, fallback = 0;
    int tpl = 1;
    int items_per_fetch = 4, ctas_per_sm = 4;
    int solo_tiles = 16384;
};

int resolve(const ctf_batch_opts *o, ResolvedBatch *r) {
    *r = ResolvedBatch();
    if (!o) return CTF_OK;
    r->tile_w = o->filter.tile_w;
    r->tile_h = o->filter.tile_h;
    r->budget = o->filter.budget;
    r->mask_dim = o->filter.mask_dim;
    r->edge_remap = o->filter.edge_remap;
    r->group_dedup = o->filter.group_dedup;
    r->fallback = o->filter.fallback;
    r->tpl = o->filter.texels_per_lane == 0 ? 1 : o->filter.texels_per_lane;
    if (o->filter.filter != 0) return report(CTF_ERR_UNSUPPORTED, "batches take the bilinear filter only");
    r->items_per_fetch = o->items_per_fetch;
    r->ctas_per_sm = o->ctas_per_sm;
    r->solo_tiles = o->solo_tiles;
    const bool shape_ok = (r->tile_w == 8 && r->tile_h == 4) || (r->tile_w == 4 && r->tile_h == 8) ||
                          (r->tile_w == 16 && r->tile_h == 2);
    if (!shape_ok) return report(CTF_ERR_ARG, "tile %dx%d not one of 8x4, 4x8, 16x2", r->tile_w, r->tile_h);
    if (r->tpl != 1 && r->tpl != 2) return report(CTF_ERR_ARG, "texels_per_lane %d not 0, 1 or 2", r->tpl);
    if (r->budget < 1 || r->budget > 32 * r->tpl)
        return report(CTF_ERR_ARG, "budget %d outside [1, %d]", r->budget, 32 * r->tpl);
    if (r->mask_dim != 16 && r->mask_dim != 11) return report(CTF_ERR_ARG, "mask_dim %d not 16 or 11", r->mask_dim);
    if (r->edge_remap != 0 && r->edge_remap != 1) return report(CTF_ERR_ARG, "edge_remap must be 0 or 1");
    if (r->group_dedup != 0 && r->group_dedup != 1) return report(CTF_ERR_ARG, "group_dedup must be 0 or 1");
    if (r->fallback < 0 || r->fallback > 2) return report(CTF_ERR_ARG, "fallback %d not 0, 1 or 2", r->fallback);
    if (r->items_per_fetch < 1 || r->items_per_fetch > 64)
        return report(CTF_ERR_ARG, "items_per_fetch %d outside [1, 64]", r->items_per_fetch);
    if (r->ctas_per_sm < 1 || r->ctas_per_sm > 4) return report(CTF_ERR_ARG, "ctas_per_sm %d outside [1, 4]", r->ctas_per_sm);
    if (r->solo_tiles < 0) return report(CTF_ERR_ARG, "solo_tiles %d is negative", r->solo_tiles);
    return CTF_OK;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Host-side plan of a batch: the device view table, the views launched on
// their own, and, per kind, the other views' indices and item prefix.
struct Plan {
    std::vector<BatchViewDev> views;
    std::vector<int> solo;
    std::vector<int> index[2];           // [0] block views, [1] learned views
    std::vector<long long> begin[2];
    long long items[2] = {0, 0};
};

int make_plan(const ctf_view *views, int nviews, ctf_algorithm alg, uint64_t seed, const ResolvedBatch &r, Plan *plan) {
    if (!views || nviews < 1 || nviews > kMaxViews) return report(CTF_ERR_ARG, "nviews %d outside [1, %d]", nviews, kMaxViews);
    if ((int)alg < CTF_ALG_4TAP || (int)alg > CTF_ALG_MASK) return report(CTF_ERR_ARG, "unknown algorithm %d", (int)alg);
    plan->views.resize(nviews);
    for (int i = 0; i < nviews; ++i) {
        const ctf_view &v = views[i];
        if (!v.tex) return report(CTF_ERR_ARG, "view %d has no texture", i);
        if (v.width < 0 || v.height < 0 || v.width > 32768 || v.height > 32768)
            return report(CTF_ERR_ARG, "view %d is %dx%d", i, v.width, v.height);
        const size_t np = (size_t)v.width * v.height;
        if (np && (!v.uv || !v.jac || !v.out_rgba)) return report(CTF_ERR_ARG, "view %d: uv, jac and out_rgba needed", i);
        if (np && (!aligned(v.uv, 8) || !aligned(v.jac, 16) || !aligned(v.out_rgba, 16)))
            return report(CTF_ERR_ALIGN, "view %d: uv 8-byte, jac and out_rgba 16-byte alignment needed", i);
        BatchViewDev &d = plan->views[i];
        std::memset(&d, 0, sizeof(d));
        ExactParams &p = d.p;
        p.blocks = static_cast<const uint2 *>(v.tex->blocks);
        p.Wt = v.tex->width;
        p.Ht = v.tex->height;
        p.nbx = v.tex->width / 4;
        p.uv = reinterpret_cast<const float2 *>(v.uv);
        p.jac = reinterpret_cast<const float4 *>(v.jac);
        p.cov = v.coverage;
        p.W = v.width;
        p.H = v.height;
        p.tiles_x = (v.width + r.tile_w - 1) / r.tile_w;
        p.n_tiles = (long long)p.tiles_x * ((v.height + r.tile_h - 1) / r.tile_h);
        p.view = v.view_id;
        p.k0 = (uint32_t)(seed & 0xffffffffu);
        p.k1 = (uint32_t)(seed >> 32);
        p.budget = r.budget;
        p.edge_remap = r.edge_remap;
        p.group_dedup = r.group_dedup;
        p.fallback = r.fallback;
        p.tpl = r.tpl;
        p.out = reinterpret_cast<float4 *>(v.out_rgba);
        p.evals = v.out_evals;
        p.stats = nullptr;
        p.tables = v.tex->tables;
        if (int rc = device_error_word(&p.err)) return rc;
        d.learned = v.tex->mode != CTF_EVAL_BLOCK;
        if (d.learned && (r.fallback || r.tpl != 1))
            return report(CTF_ERR_UNSUPPORTED,
                          "view %d: fallbacks C and C+ and two texels per lane are built for block textures only", i);
        if (d.learned) d.m = mlp_device_view(v.tex);
        if (r.solo_tiles > 0 && p.n_tiles >= r.solo_tiles) {
            plan->solo.push_back(i);
            continue;
        }
        const int kind = d.learned ? 1 : 0;
        const long long per_item = d.learned ? mlp_group_tiles((int)alg) : kBlockItemTiles;
        plan->index[kind].push_back(i);
        plan->begin[kind].push_back(plan->items[kind]);
        plan->items[kind] += (p.n_tiles + per_item - 1) / per_item;
    }
    for (int k = 0; k < 2; ++k) plan->begin[k].push_back(plan->items[k]);
    return CTF_OK;
}

// Device copy of a plan plus its two work counters (owned by the caller).
struct DevPlan {
    void *buf = nullptr;
    size_t bytes = 0;
    BatchViewDev *views = nullptr;
    int *index[2] = {nullptr, nullptr};
    long long *begin[2] = {nullptr, nullptr};
    unsigned long long *counter = nullptr;  // [2] counters, then kNumStats stats words
};

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

cudaError_t upload_plan(const Plan &plan, DevPlan *dp, cudaStream_t s) {
    const int n = (int)plan.views.size();
    const size_t vb = up256(sizeof(BatchViewDev) * n);
    size_t ib[2], bb[2];
    for (int k = 0; k < 2; ++k) {
        ib[k] = up256(4 * (plan.index[k].size() + 1));
        bb[k] = up256(8 * plan.begin[k].size());
    }
    const size_t need = vb + ib[0] + ib[1] + bb[0] + bb[1] + 256;
    if (dp->bytes < need) {
        if (dp->buf) {
            cudaStreamSynchronize(s);
            ctf::dev_free(dp->buf);
        }
        dp->buf = nullptr;
        dp->bytes = 0;
        cudaError_t e = ctf::dev_malloc(&dp->buf, need);
        if (e != cudaSuccess) return e;
        dp->bytes = need;
    }
    char *base = static_cast<char *>(dp->buf);
    dp->views = reinterpret_cast<BatchViewDev *>(base);
    base += vb;
    for (int k = 0; k < 2; ++k) {
        dp->index[k] = reinterpret_cast<int *>(base);
        base += ib[k];
        dp->begin[k] = reinterpret_cast<long long *>(base);
        base += bb[k];
    }
    dp->counter = reinterpret_cast<unsigned long long *>(base);
    cudaError_t e = cudaMemcpyAsync(dp->views, plan.views.data(), sizeof(BatchViewDev) * n, cudaMemcpyHostToDevice, s);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        if (!plan.index[k].empty())
            e = cudaMemcpyAsync(dp->index[k], plan.index[k].data(), 4 * plan.index[k].size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dp->begin[k], plan.begin[k].data(), 8 * plan.begin[k].size(), cudaMemcpyHostToDevice, s);
    }
    return e;
}

// The solo views (the single-view kernels), the counter reset, then the
// block-view kernel, then the learned-view kernel, all on stream s (so a
// capture of s records the whole batch).
cudaError_t launch_plan(const Plan &plan, const DevPlan &dp, int alg, const ResolvedBatch &r,
                        unsigned long long *stats, int *err, cudaStream_t s) {
    for (int i : plan.solo) {
        ExactParams p = plan.views[i].p;
        p.stats = stats;
        const cudaError_t le = plan.views[i].learned
                                   ? launch_mlp_filter(p, plan.views[i].m, alg, r.tile_w, r.mask_dim, err, s)
                                   : launch_exact_filter(p, alg, r.tile_w, r.mask_dim, s);
        if (le != cudaSuccess) return le;
    }
    cudaError_t e = cudaMemsetAsync(dp.counter, 0, 16, s);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < 2; ++k) {
        if (plan.items[k] == 0) continue;
        BatchFn fn = pick(k == 1, alg, r.tile_w, r.mask_dim, r.fallback != 0 || r.tpl == 2);
        if (!fn) return cudaErrorInvalidValue;
        BatchParams b;
        b.views = dp.views;
        b.index = dp.index[k];
        b.item_begin = dp.begin[k];
        b.nkind = (int)plan.index[k].size();
        b.nviews = (int)plan.views.size();
        b.total_items = plan.items[k];
        b.items_per_fetch = r.items_per_fetch;
        b.counter = dp.counter + k;
        b.stats = stats;
        b.err = err;
        b.tables = k == 0 ? plan.views[plan.index[0][0]].p.tables : nullptr;
        if (k == 1 && mlp_batch_pf_applies(alg, r.group_dedup)) {
            // learned views on the packed-group kernel (one group per fetch)
            e = launch_mlp_batch_pf(dp.views, (int)plan.views.size(), dp.index[1], dp.begin[1], b.nkind, b.total_items,
                                    b.counter, stats, err, plan.views[plan.index[1][0]].m, alg, r.tile_w, r.mask_dim, s);
            if (e != cudaSuccess) return e;
            continue;
        }
        if (k == 1) {
            e = prepare_batch(fn);
            if (e != cudaSuccess) return e;
            long long grid = (long long)device_sm_count() * r.ctas_per_sm;
            const long long useful = (plan.items[k] + r.items_per_fetch - 1) / r.items_per_fetch;
            if (grid > useful) grid = useful;
            fn<<<(int)grid, kRows, kSmRequest, s>>>(b);
        } else {
            const size_t smem = alg == ALG_LIST ? sizeof(ListTable) * kBlockWarps : 0;
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlockWarps * 32, smem) != cudaSuccess ||
                per_sm < 1)
                per_sm = 1;
            long long grid = (long long)device_sm_count() * per_sm;
            const long long useful = (plan.items[k] + kBlockWarps - 1) / kBlockWarps;
            if (grid > useful) grid = useful;
            fn<<<(int)grid, kBlockWarps * 32, smem, s>>>(b);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

DevPlan g_plan[64];
std::mutex g_plan_mu;

}  // namespace
}  // namespace ctf

struct ctf_batch_graph_s {
    ctf::DevPlan plan;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

int ctf_filter_batch(const ctf_view *views, int nviews, ctf_algorithm alg, uint64_t seed, const ctf_batch_opts *opts,
                     ctf_stats *stats, void *stream) {
    ctf::NvtxRange nvtx_range("ctf_filter_batch");
    using namespace ctf;
    clear_error();
    ResolvedBatch r;
    int rc = resolve(opts, &r);
    if (rc) return rc;
    Plan plan;
    rc = make_plan(views, nviews, alg, seed, r, &plan);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return report(CTF_ERR_UNSUPPORTED, "device ordinal %d", dev);
    int *err = nullptr;
    rc = device_error_word(&err);
    if (rc) return rc;
    unsigned long long *dstats = nullptr;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    DevPlan &dp = g_plan[dev];
    cudaError_t e = upload_plan(plan, &dp, s);
    if (e != cudaSuccess) return report_cuda(e, "batch plan upload");
    if (stats) {
        // stats words right after the two work counters in the plan buffer
        e = cudaMemsetAsync(dp.counter + 2, 0, 8 * kNumStats, s);
        if (e != cudaSuccess) return report_cuda(e, "clearing stats");
        dstats = dp.counter + 2;
    }
    e = launch_plan(plan, dp, (int)alg, r, dstats, err, s);
    if (e != cudaSuccess) return report_cuda(e, "batch launch");
    if (stats) {
        unsigned long long h[kNumStats];
        e = cudaMemcpyAsync(h, dstats, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return report_cuda(e, "reading stats");
        int64_t *o = reinterpret_cast<int64_t *>(stats);
        for (int i = 0; i < kNumStats; ++i) o[i] = (int64_t)h[i];
    }
    return CTF_OK;
}

int ctf_batch_graph_create(const ctf_view *views, int nviews, ctf_algorithm alg, uint64_t seed,
                           const ctf_batch_opts *opts, ctf_batch_graph *out) {
    using namespace ctf;
    clear_error();
    if (!out) return report(CTF_ERR_ARG, "out is NULL");
    *out = nullptr;
    ResolvedBatch r;
    int rc = resolve(opts, &r);
    if (rc) return rc;
    Plan plan;
    rc = make_plan(views, nviews, alg, seed, r, &plan);
    if (rc) return rc;
    int *err = nullptr;
    rc = device_error_word(&err);
    if (rc) return rc;
    ctf_batch_graph g = new (std::nothrow) ctf_batch_graph_s();
    if (!g) return report(CTF_ERR_OOM, "host allocation");
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = upload_plan(plan, &g->plan, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    // the kernel attributes must be set before capture
    if (e == cudaSuccess && plan.items[1]) e = prepare_batch(pick(true, (int)alg, r.tile_w, r.mask_dim, false));
    if (e == cudaSuccess && plan.items[1] && mlp_batch_pf_applies((int)alg, r.group_dedup))
        e = prepare_mlp_batch_pf((int)alg, r.tile_w, r.mask_dim);
    for (int i : plan.solo)
        if (e == cudaSuccess && plan.views[i].learned) e = prepare_mlp_filter((int)alg, r.tile_w, r.mask_dim);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = launch_plan(plan, g->plan, (int)alg, r, nullptr, err, s);
        e = cudaStreamEndCapture(s, &g->graph);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        if (g->plan.buf) ctf::dev_free(g->plan.buf);
        delete g;
        return report_cuda(e, "batch graph capture");
    }
    *out = g;
    return CTF_OK;
}

int ctf_batch_graph_launch(ctf_batch_graph g, void *stream) {
    ctf::NvtxRange nvtx_range("ctf_batch_graph_launch");
    using namespace ctf;
    clear_error();
    if (!g) return report(CTF_ERR_ARG, "graph is NULL");
    cudaError_t e = cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return report_cuda(e, "graph launch");
    return CTF_OK;
}

int ctf_batch_graph_destroy(ctf_batch_graph g) {
    ctf::clear_error();
    if (!g) return CTF_OK;
    cudaDeviceSynchronize();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->plan.buf) ctf::dev_free(g->plan.buf);
    delete g;
    return CTF_OK;
}

int ctf_batch_autotune(const ctf_view *views, int nviews, ctf_algorithm alg, uint64_t seed, const ctf_batch_opts *base,
                       ctf_batch_opts *best, double *best_ms, void *stream) {
    ctf::NvtxRange nvtx_range("ctf_batch_autotune");
    using namespace ctf;
    clear_error();
    if (!best) return report(CTF_ERR_ARG, "best is NULL");
    ctf_batch_opts b0;
    if (base) {
        b0 = *base;
    } else {
        b0.filter.tile_w = 8;
        b0.filter.tile_h = 4;
        b0.filter.budget = 32;
        b0.filter.mask_dim = 16;
        b0.filter.edge_remap = 1;
        b0.filter.group_dedup = 0;
        b0.filter.fallback = 0;
        b0.filter.texels_per_lane = 1;
        b0.filter.filter = 0;
        b0.items_per_fetch = 4;
        b0.ctas_per_sm = 4;
        b0.solo_tiles = 16384;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return report(CTF_ERR_CUDA, "event creation");
    const int shapes[3][2] = {{8, 4}, {4, 8}, {16, 2}};
    const int fetches[4] = {1, 2, 4, 8};
    const int ctas[2] = {2, 4};
    const int solos[4] = {0, 4096, 16384, 65536};
    double bestt = 1e30;
    ctf_batch_opts bestc = b0;
    int rc = CTF_OK;
    auto time_config = [&](const ctf_batch_opts &c) {
        rc = ctf_filter_batch(views, nviews, alg, seed, &c, nullptr, stream);  // warm-up
        float best_run = 1e30f;
        for (int rep = 0; rep < 3 && !rc; ++rep) {
            cudaEventRecord(e0, s);
            rc = ctf_filter_batch(views, nviews, alg, seed, &c, nullptr, stream);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best_run = std::min(best_run, ms);
        }
        if (!rc && best_run < bestt) {
            bestt = best_run;
            bestc = c;
        }
    };
    for (int si = 0; si < 3 && !rc; ++si)
        for (int fi = 0; fi < 4 && !rc; ++fi)
            for (int ci = 0; ci < 2 && !rc; ++ci) {
                ctf_batch_opts c = b0;
                c.filter.tile_w = shapes[si][0];
                c.filter.tile_h = shapes[si][1];
                c.items_per_fetch = fetches[fi];
                c.ctas_per_sm = ctas[ci];
                time_config(c);
            }
    const ctf_batch_opts shaped = bestc;
    for (int k = 0; k < 4 && !rc; ++k) {
        if (solos[k] == shaped.solo_tiles) continue;
        ctf_batch_opts c = shaped;
        c.solo_tiles = solos[k];
        time_config(c);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *best = bestc;
    if (best_ms) *best_ms = bestt;
    return CTF_OK;
}

}  // extern "C"
