// ctf_batch.cu -- many views of uneven size and magnification in one
// persistent launch, optionally captured into a CUDA graph, with an
// autotuner over the launch shape.
//
// Work is cut into items: 4 warp tiles of one view for a learned-decode view
// (one tile per warp, the 4 warps share an MLP chain), 16 warp tiles for a
// block view (4 consecutive tiles per warp, the next one's inputs prefetched).
// A prefix over the views' item counts maps a global item number to its view.
// Persistent CTAs of 128 threads take `items_per_fetch` items at a time from
// an atomic counter (a plain fetch-and-add: no thread ever waits on another
// CTA) until the items run out.  Every CTA allocates its 128 TMEM columns up
// front so that any item can use the tensor cores; the shared-memory request
// keeps at most 4 CTAs on an SM, so the 512 columns always suffice.
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

constexpr int kBlockTilesPerWarp = 4;
constexpr int kMaxViews = 4096;

struct BatchViewDev {
    ExactParams p;
    MlpDevice m;
    int learned;
    long long items;
};

struct BatchParams {
    const BatchViewDev *views;
    const long long *item_begin;  // nviews + 1 prefix
    int nviews;
    long long total_items;
    int items_per_fetch;
    unsigned long long *counter;
    unsigned long long *stats;
    int *err;
};

__device__ __forceinline__ int find_view(const long long *begin, int nviews, long long item) {
    int lo = 0, hi = nviews - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(begin + mid) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int ALG, int TW, int MD>
__global__ void __launch_bounds__(kRows) batch_kernel(const BatchParams b) {
    constexpr int TH = 32 / TW;
    constexpr bool kJac = ALG >= ALG_LIST;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ float lut[256];
    __shared__ unsigned long long block_stats[kNumStats];
    __shared__ long long s_item;
    // The operand image of the learned views is loaded per item (views may
    // use different networks); chain_setup only needs some image to start.
    Chain ch;
    const MlpDevice m0 = b.views[0].m;
    if (m0.img) {
        chain_setup(ch, sm, m0);
    } else {
        // no learned view in this batch: still allocate TMEM so that the code
        // path is the same; the image copy is skipped
        MlpDevice none = m0;
        none.img = nullptr;
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
        (void)none;
    }
    for (int i = threadIdx.x; i < 256; i += blockDim.x) lut[i] = __fdiv_rn((float)i, 255.0f);
    if (threadIdx.x < kNumStats) block_stats[threadIdx.x] = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ListTable *T = reinterpret_cast<ListTable *>(sm + kSmList) + warp;
    if (ALG == ALG_LIST) {
#pragma unroll
        for (int s = 0; s < 8; ++s) T->keys[lane * 8 + s] = kEmpty;
    }
    const float *inv_a1 = reinterpret_cast<const float *>(sm + kImgA1);
    const uint32_t lt = lanemask_lt();
    const int tx = lane % TW, ty = lane / TW;
    Counters cnt;
#pragma unroll
    for (int i = 0; i < kNumStats; ++i) cnt.v[i] = 0;
    const unsigned char *loaded_img = m0.img ? reinterpret_cast<const unsigned char *>(m0.img) : nullptr;
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
            const int v = find_view(b.item_begin, b.nviews, item);
            const BatchViewDev &V = b.views[v];
            const long long local = item - __ldg(b.item_begin + v);
            if (V.learned) {
                // this view's network into shared memory if it is not there yet
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
                ok = mlp_warp_tile<ALG, TW, MD>(V.p, V.m, ch, local * 4 + warp, lane, lt, T, cnt, inv_a1, b.err);
            } else {
                const ExactParams &p = V.p;
                for (int r = 0; r < kBlockTilesPerWarp; ++r) {
                    const long long tile = (local * 4 + warp) * kBlockTilesPerWarp + r;
                    if (tile >= p.n_tiles) break;
                    const int bx = (int)(tile % p.tiles_x), by = (int)(tile / p.tiles_x);
                    const int px = bx * TW + tx, py = by * TH + ty;
                    const bool inside = px < p.W && py < p.H;
                    const uint32_t idx = inside ? (uint32_t)py * (uint32_t)p.W + (uint32_t)px : 0u;
                    const Inputs in = load_inputs<kJac>(p, inside, idx);
                    filter_tile<ALG, TW, MD>(p, in, px, py, inside, idx, lane, lt, lut, T, cnt);
                }
            }
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

template <int ALG, int TW>
BatchFn pick_mask(int md) {
    if constexpr (ALG == ALG_MASK) {
        return md == 11 ? batch_kernel<ALG, TW, 11> : batch_kernel<ALG, TW, 16>;
    } else {
        return batch_kernel<ALG, TW, 16>;
    }
}

template <int TW>
BatchFn pick_alg(int alg, int md) {
    switch (alg) {
    case ALG_4TAP: return pick_mask<ALG_4TAP, TW>(md);
    case ALG_STF: return pick_mask<ALG_STF, TW>(md);
    case ALG_LIST: return pick_mask<ALG_LIST, TW>(md);
    case ALG_BOX: return pick_mask<ALG_BOX, TW>(md);
    case ALG_MASK: return pick_mask<ALG_MASK, TW>(md);
    default: return nullptr;
    }
}

BatchFn pick(int alg, int tile_w, int md) {
    switch (tile_w) {
    case 8: return pick_alg<8>(alg, md);
    case 4: return pick_alg<4>(alg, md);
    case 16: return pick_alg<16>(alg, md);
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
    int tile_w = 8, tile_h = 4, budget = 32, mask_dim = 16, edge_remap = 1;
    int items_per_fetch = 4, ctas_per_sm = 4;
};

int resolve(const ctf_batch_opts *o, ResolvedBatch *r) {
    *r = ResolvedBatch();
    if (!o) return CTF_OK;
    r->tile_w = o->filter.tile_w;
    r->tile_h = o->filter.tile_h;
    r->budget = o->filter.budget;
    r->mask_dim = o->filter.mask_dim;
    r->edge_remap = o->filter.edge_remap;
    r->items_per_fetch = o->items_per_fetch;
    r->ctas_per_sm = o->ctas_per_sm;
    const bool shape_ok = (r->tile_w == 8 && r->tile_h == 4) || (r->tile_w == 4 && r->tile_h == 8) ||
                          (r->tile_w == 16 && r->tile_h == 2);
    if (!shape_ok) return report(CTF_ERR_ARG, "tile %dx%d not one of 8x4, 4x8, 16x2", r->tile_w, r->tile_h);
    if (r->budget < 1 || r->budget > 32) return report(CTF_ERR_ARG, "budget %d outside [1, 32]", r->budget);
    if (r->mask_dim != 16 && r->mask_dim != 11) return report(CTF_ERR_ARG, "mask_dim %d not 16 or 11", r->mask_dim);
    if (r->edge_remap != 0 && r->edge_remap != 1) return report(CTF_ERR_ARG, "edge_remap must be 0 or 1");
    if (r->items_per_fetch < 1 || r->items_per_fetch > 64)
        return report(CTF_ERR_ARG, "items_per_fetch %d outside [1, 64]", r->items_per_fetch);
    if (r->ctas_per_sm < 1 || r->ctas_per_sm > 4) return report(CTF_ERR_ARG, "ctas_per_sm %d outside [1, 4]", r->ctas_per_sm);
    return CTF_OK;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Host-side plan of a batch: the device view table and item prefix.
struct Plan {
    std::vector<BatchViewDev> views;
    std::vector<long long> begin;
    long long total_items = 0;
};

int make_plan(const ctf_view *views, int nviews, ctf_algorithm alg, uint64_t seed, const ResolvedBatch &r, Plan *plan) {
    if (!views || nviews < 1 || nviews > kMaxViews) return report(CTF_ERR_ARG, "nviews %d outside [1, %d]", nviews, kMaxViews);
    if ((int)alg < CTF_ALG_4TAP || (int)alg > CTF_ALG_MASK) return report(CTF_ERR_ARG, "unknown algorithm %d", (int)alg);
    plan->views.resize(nviews);
    plan->begin.resize(nviews + 1);
    long long acc = 0;
    const void *img0 = nullptr;
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
        p.out = reinterpret_cast<float4 *>(v.out_rgba);
        p.evals = v.out_evals;
        p.stats = nullptr;
        d.learned = v.tex->mode != CTF_EVAL_BLOCK;
        if (d.learned) {
            d.m = mlp_device_view(v.tex);
            if (!img0) img0 = v.tex->img;
        }
        const long long per_item = d.learned ? 4 : 4 * kBlockTilesPerWarp;
        d.items = (p.n_tiles + per_item - 1) / per_item;
        plan->begin[i] = acc;
        acc += d.items;
    }
    plan->begin[nviews] = acc;
    plan->total_items = acc;
    // view 0's image doubles as the first one a CTA loads
    if (img0 && !plan->views[0].learned) plan->views[0].m.img = static_cast<const uint4 *>(img0);
    return CTF_OK;
}

// Device copy of a plan plus its work counter (owned by the caller).
struct DevPlan {
    void *buf = nullptr;
    size_t bytes = 0;
    BatchViewDev *views = nullptr;
    long long *begin = nullptr;
    unsigned long long *counter = nullptr;
};

size_t plan_bytes(int nviews) {
    return ((sizeof(BatchViewDev) * nviews + 255) & ~(size_t)255) + ((8 * (size_t)(nviews + 1) + 255) & ~(size_t)255) + 256;
}

cudaError_t upload_plan(const Plan &plan, DevPlan *dp, cudaStream_t s) {
    const int n = (int)plan.views.size();
    const size_t need = plan_bytes(n);
    if (dp->bytes < need) {
        if (dp->buf) {
            cudaStreamSynchronize(s);
            cudaFree(dp->buf);
        }
        dp->buf = nullptr;
        dp->bytes = 0;
        cudaError_t e = cudaMalloc(&dp->buf, need);
        if (e != cudaSuccess) return e;
        dp->bytes = need;
    }
    char *base = static_cast<char *>(dp->buf);
    const size_t vb = (sizeof(BatchViewDev) * n + 255) & ~(size_t)255;
    const size_t bb = (8 * (size_t)(n + 1) + 255) & ~(size_t)255;
    dp->views = reinterpret_cast<BatchViewDev *>(base);
    dp->begin = reinterpret_cast<long long *>(base + vb);
    dp->counter = reinterpret_cast<unsigned long long *>(base + vb + bb);
    cudaError_t e = cudaMemcpyAsync(dp->views, plan.views.data(), sizeof(BatchViewDev) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp->begin, plan.begin.data(), 8 * (size_t)(n + 1), cudaMemcpyHostToDevice, s);
    return e;
}

cudaError_t launch_plan(const Plan &plan, const DevPlan &dp, int alg, const ResolvedBatch &r,
                        unsigned long long *stats, int *err, cudaStream_t s) {
    BatchFn fn = pick(alg, r.tile_w, r.mask_dim);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = prepare_batch(fn);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(dp.counter, 0, 8, s);
    if (e != cudaSuccess) return e;
    if (plan.total_items == 0) return cudaSuccess;
    BatchParams b;
    b.views = dp.views;
    b.item_begin = dp.begin;
    b.nviews = (int)plan.views.size();
    b.total_items = plan.total_items;
    b.items_per_fetch = r.items_per_fetch;
    b.counter = dp.counter;
    b.stats = stats;
    b.err = err;
    long long grid = (long long)device_sm_count() * r.ctas_per_sm;
    const long long useful = (plan.total_items + r.items_per_fetch - 1) / r.items_per_fetch;
    if (grid > useful) grid = useful;
    fn<<<(int)grid, kRows, kSmRequest, s>>>(b);
    return cudaGetLastError();
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
        // counters right after the work counter in the plan buffer
        e = cudaMemsetAsync(dp.counter + 1, 0, 8 * kNumStats, s);
        if (e != cudaSuccess) return report_cuda(e, "clearing stats");
        dstats = dp.counter + 1;
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
    // the kernel attribute must be set before capture
    if (e == cudaSuccess) e = prepare_batch(pick((int)alg, r.tile_w, r.mask_dim));
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
        if (g->plan.buf) cudaFree(g->plan.buf);
        delete g;
        return report_cuda(e, "batch graph capture");
    }
    *out = g;
    return CTF_OK;
}

int ctf_batch_graph_launch(ctf_batch_graph g, void *stream) {
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
    if (g->plan.buf) cudaFree(g->plan.buf);
    delete g;
    return CTF_OK;
}

int ctf_batch_autotune(const ctf_view *views, int nviews, ctf_algorithm alg, uint64_t seed, const ctf_batch_opts *base,
                       ctf_batch_opts *best, double *best_ms, void *stream) {
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
        b0.items_per_fetch = 4;
        b0.ctas_per_sm = 4;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return report(CTF_ERR_CUDA, "event creation");
    const int shapes[3][2] = {{8, 4}, {4, 8}, {16, 2}};
    const int fetches[4] = {1, 2, 4, 8};
    const int ctas[2] = {2, 4};
    double bestt = 1e30;
    ctf_batch_opts bestc = b0;
    int rc = CTF_OK;
    for (int si = 0; si < 3 && !rc; ++si)
        for (int fi = 0; fi < 4 && !rc; ++fi)
            for (int ci = 0; ci < 2 && !rc; ++ci) {
                ctf_batch_opts c = b0;
                c.filter.tile_w = shapes[si][0];
                c.filter.tile_h = shapes[si][1];
                c.items_per_fetch = fetches[fi];
                c.ctas_per_sm = ctas[ci];
                rc = ctf_filter_batch(views, nviews, alg, seed, &c, nullptr, stream);  // warm-up
                if (rc) break;
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
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *best = bestc;
    if (best_ms) *best_ms = bestt;
    return CTF_OK;
}

}  // extern "C"
