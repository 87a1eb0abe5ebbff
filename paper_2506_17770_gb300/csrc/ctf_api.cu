// ctf_api.cu -- the C ABI (include/ctf.h): argument validation, texture
// objects, per-device scratch, error reporting.  No exception crosses the ABI.
#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>

#include <cuda_runtime.h>

#include "../../include/ctf.h"
#include "ctf_internal.h"
#include "ctf_debug.cuh"

namespace {

thread_local std::string g_last_error;

int fail(int status, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

int cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) return fail(CTF_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(CTF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Per-device scratch owned by the library: the stats counters and the
// staging buffers of ctf_filter_host.  Grown on demand, kept until exit.
struct DeviceScratch {
    unsigned long long *stats = nullptr;
    void *stage = nullptr;
    size_t stage_bytes = 0;
    int *err = nullptr;  // set by bounded device waits that gave up
};
constexpr int kMaxDevices = 64;
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mutex;

int current_device(int *dev) {
    cudaError_t e = cudaGetDevice(dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (*dev < 0 || *dev >= kMaxDevices) return fail(CTF_ERR_UNSUPPORTED, "device ordinal %d too large", *dev);
    return CTF_OK;
}

int scratch_stats(unsigned long long **out) {
    int dev = 0;
    int rc = current_device(&dev);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_scratch_mutex);
    DeviceScratch &s = g_scratch[dev];
    if (!s.stats) {
        cudaError_t e = ctf::dev_malloc(&s.stats, sizeof(unsigned long long) * ctf::kNumStats);
        if (e != cudaSuccess) {
            s.stats = nullptr;
            return cuda_fail(e, "cudaMalloc(stats)");
        }
    }
    *out = s.stats;
    return CTF_OK;
}

// Copy streams and events of the banded host path, per device (created on
// first use, guarded by g_scratch_mutex).
constexpr int kMaxBands = 4;
struct HostPipe {
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t ev[2 * kMaxBands + 2] = {};
    bool ready = false;
};
HostPipe g_pipe[kMaxDevices];

int host_pipe(HostPipe **out) {
    int dev = 0;
    int rc = current_device(&dev);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_scratch_mutex);
    HostPipe &h = g_pipe[dev];
    if (!h.ready) {
        cudaError_t e = cudaStreamCreateWithFlags(&h.in, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h.out, cudaStreamNonBlocking);
        for (int i = 0; i < 2 * kMaxBands + 2 && e == cudaSuccess; ++i)
            e = cudaEventCreateWithFlags(&h.ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "host copy streams");
        h.ready = true;
    }
    *out = &h;
    return CTF_OK;
}

int scratch_stage(size_t bytes, void **out) {
    int dev = 0;
    int rc = current_device(&dev);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_scratch_mutex);
    DeviceScratch &s = g_scratch[dev];
    if (s.stage_bytes < bytes) {
        if (s.stage) {
            cudaDeviceSynchronize();
            ctf::dev_free(s.stage);
        }
        s.stage = nullptr;
        s.stage_bytes = 0;
        cudaError_t e = ctf::dev_malloc(&s.stage, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(stage)");
        s.stage_bytes = bytes;
    }
    *out = s.stage;
    return CTF_OK;
}

struct ResolvedOpts {
    int tile_w = 8, tile_h = 4, budget = 32, mask_dim = 16, edge_remap = 1, group_dedup = 0, fallback = 0;
    int tpl = 1;
    int filter = 0;
};

int resolve_opts(const ctf_filter_opts *o, ResolvedOpts *r) {
    *r = ResolvedOpts();
    if (!o) return CTF_OK;
    r->tile_w = o->tile_w;
    r->tile_h = o->tile_h;
    r->budget = o->budget;
    r->mask_dim = o->mask_dim;
    r->edge_remap = o->edge_remap;
    r->group_dedup = o->group_dedup;
    r->fallback = o->fallback;
    r->tpl = o->texels_per_lane == 0 ? 1 : o->texels_per_lane;
    r->filter = o->filter;
    const bool shape_ok = (r->tile_w == 8 && r->tile_h == 4) || (r->tile_w == 4 && r->tile_h == 8) ||
                          (r->tile_w == 16 && r->tile_h == 2);
    if (!shape_ok) return fail(CTF_ERR_ARG, "tile %dx%d not one of 8x4, 4x8, 16x2", r->tile_w, r->tile_h);
    if (r->group_dedup != 0 && r->group_dedup != 1) return fail(CTF_ERR_ARG, "group_dedup must be 0 or 1");
    if (r->fallback < 0 || r->fallback > 2) return fail(CTF_ERR_ARG, "fallback %d not 0 (STF), 1 (C) or 2 (C+)", r->fallback);
    if (r->tpl != 1 && r->tpl != 2) return fail(CTF_ERR_ARG, "texels_per_lane %d not 0, 1 or 2", r->tpl);
    if (r->filter < 0 || r->filter > 2) return fail(CTF_ERR_ARG, "filter %d not 0, 1 or 2", r->filter);
    if (r->filter != 0 && (r->tpl != 1 || r->fallback != 0))
        return fail(CTF_ERR_UNSUPPORTED, "the bicubic filters take one texel per lane and the STF fallback");
    if (r->budget < 1 || r->budget > 32 * r->tpl)
        return fail(CTF_ERR_ARG, "budget %d outside [1, %d]", r->budget, 32 * r->tpl);
    if (r->mask_dim != 16 && r->mask_dim != 11) return fail(CTF_ERR_ARG, "mask_dim %d not 16 or 11", r->mask_dim);
    if (r->edge_remap != 0 && r->edge_remap != 1) return fail(CTF_ERR_ARG, "edge_remap must be 0 or 1");
    return CTF_OK;
}

int check_frame(int width, int height) {
    if (width < 0 || height < 0 || width > 32768 || height > 32768)
        return fail(CTF_ERR_ARG, "frame %dx%d outside [0, 32768]^2", width, height);
    return CTF_OK;
}

int validate_filter_args(ctf_texture tex, const float *uv, const float *jac, int width, int height,
                         ctf_algorithm alg, float *out, ResolvedOpts *ro, const ctf_filter_opts *opts) {
    if (!tex) return fail(CTF_ERR_ARG, "texture is NULL");
    int rc = check_frame(width, height);
    if (rc) return rc;
    if ((int)alg < CTF_ALG_4TAP || (int)alg > CTF_ALG_MASK) return fail(CTF_ERR_ARG, "unknown algorithm %d", (int)alg);
    rc = resolve_opts(opts, ro);
    if (rc) return rc;
    if (ro->filter != 0 && tex->mode != CTF_EVAL_BLOCK)
        return fail(CTF_ERR_UNSUPPORTED, "the bicubic filters are built for block textures only");
    if ((ro->fallback != 0 || ro->tpl != 1) && ro->group_dedup && tex->mode != CTF_EVAL_BLOCK)
        return fail(CTF_ERR_UNSUPPORTED,
                    "group_dedup does not combine with fallbacks C and C+ or two texels per lane on learned textures");
    if ((size_t)width * (size_t)height == 0) return CTF_OK;
    if (!uv || !jac || !out) return fail(CTF_ERR_ARG, "uv, jac and out_rgba must not be NULL");
    if (!aligned(uv, 8)) return fail(CTF_ERR_ALIGN, "uv must be 8-byte aligned");
    if (!aligned(jac, 16)) return fail(CTF_ERR_ALIGN, "jac must be 16-byte aligned");
    if (!aligned(out, 16)) return fail(CTF_ERR_ALIGN, "out_rgba must be 16-byte aligned");
    return CTF_OK;
}

// y0: the frame is the band of a view that starts at this row (whole tile
// rows); it enters only the STF counters, so a view filtered band by band
// gives the image of one call on the whole view.
int run_filter(ctf_texture tex, const float *uv, const float *jac, const uint8_t *coverage, int width, int height,
               int view_id, ctf_algorithm alg, uint64_t seed, const ResolvedOpts &ro, float *out,
               uint8_t *evals, unsigned long long *dstats, cudaStream_t stream, int y0 = 0) {
    ctf::ExactParams p;
    p.y0 = y0;
    p.blocks = static_cast<const uint2 *>(tex->blocks);
    p.Wt = tex->width;
    p.Ht = tex->height;
    p.nbx = tex->width / 4;
    p.uv = reinterpret_cast<const float2 *>(uv);
    p.jac = reinterpret_cast<const float4 *>(jac);
    p.cov = coverage;
    p.W = width;
    p.H = height;
    p.tiles_x = (width + ro.tile_w - 1) / ro.tile_w;
    const int tiles_y = (height + ro.tile_h - 1) / ro.tile_h;
    p.n_tiles = (long long)p.tiles_x * tiles_y;
    p.view = view_id;
    p.k0 = (uint32_t)(seed & 0xffffffffu);
    p.k1 = (uint32_t)(seed >> 32);
    p.budget = ro.budget;
    p.edge_remap = ro.edge_remap;
    p.group_dedup = ro.group_dedup;
    p.fallback = ro.fallback;
    p.tpl = ro.tpl;
    p.tables = tex->tables;
    p.out = reinterpret_cast<float4 *>(out);
    p.evals = evals;
    p.stats = dstats;
    int *err = nullptr;
    int rc = ctf::device_error_word(&err);
    if (rc) return rc;
    p.err = err;
    cudaError_t e;
    if (tex->mode == CTF_EVAL_BLOCK && ro.filter != 0) {
        e = ctf::launch_bicubic_filter(p, (int)alg, ro.tile_w, ro.mask_dim, ro.filter, stream);
    } else if (tex->mode == CTF_EVAL_BLOCK) {
        e = ctf::launch_exact_filter(p, (int)alg, ro.tile_w, ro.mask_dim, stream);
    } else {
        e = ctf::launch_mlp_filter(p, ctf::mlp_device_view(tex), (int)alg, ro.tile_w, ro.mask_dim, err, stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "filter launch");
    return CTF_OK;
}

int read_stats(unsigned long long *dstats, ctf_stats *stats, cudaStream_t stream) {
    unsigned long long h[ctf::kNumStats];
    cudaError_t e = cudaMemcpyAsync(h, dstats, sizeof(h), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading stats");
    stats->tiles_total = (int64_t)h[ctf::kStatTilesTotal];
    stats->tiles_empty = (int64_t)h[ctf::kStatTilesEmpty];
    stats->tiles_direct = (int64_t)h[ctf::kStatTilesDirect];
    stats->tiles_success = (int64_t)h[ctf::kStatTilesSuccess];
    stats->tiles_fallback_budget = (int64_t)h[ctf::kStatTilesFallbackBudget];
    stats->tiles_fallback_minified = (int64_t)h[ctf::kStatTilesFallbackMinified];
    stats->pixels_active = (int64_t)h[ctf::kStatPixelsActive];
    stats->texel_evals = (int64_t)h[ctf::kStatTexelEvals];
    stats->texel_evals_unique = (int64_t)h[ctf::kStatTexelEvalsUnique];
    return CTF_OK;
}

}  // namespace

// Decode tables of the exact path, made once per device: rg and b by bit
// replication of the RGB565 fields, val by IEEE single-precision division
// (correctly rounded on the host as on the device).
namespace ctf {

const DecodeTables *device_decode_tables() {
    static std::mutex mu;
    static std::map<int, DecodeTables *> made;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = made.find(dev);
    if (it != made.end()) return it->second;
    std::vector<DecodeTables> host(1);
    DecodeTables &t = host[0];
    for (uint32_t i = 0; i < 2048; ++i) {
        const uint32_t r5 = i >> 6, g6 = i & 63u;
        t.rg[i] = ((r5 << 3) | (r5 >> 2)) | (((g6 << 2) | (g6 >> 4)) << 10);
    }
    for (uint32_t i = 0; i < 32; ++i) t.b[i] = ((i << 3) | (i >> 2)) << 20;
    for (int i = 0; i < 1024; ++i) {
        volatile float num = (float)(i < 256 ? i : (i - 256) / 3);  // no contraction or reassociation
        t.val[i] = num / 255.0f;
    }
    DecodeTables *d = nullptr;
    cudaError_t e = ctf::dev_malloc(&d, sizeof(DecodeTables));
    if (e == cudaSuccess) e = cudaMemcpy(d, &t, sizeof(DecodeTables), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (d) ctf::dev_free(d);
        report_cuda(e, "decode tables");
        return nullptr;
    }
    made[dev] = d;
    return d;
}

}  // namespace ctf

// Error reporting and the per-device error word, shared with the other
// translation units of the library.
namespace ctf {

int report(int status, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

int report_cuda(cudaError_t e, const char *what) { return cuda_fail(e, what); }

void clear_error() { g_last_error.clear(); }

// The error word lives in the module's own device memory (zero at load), so
// no call that needs it allocates.  Host code only holds the symbol's
// host-side stand-in; its device address is looked up once per device.
// Word 0 is the status a kernel recorded; a CTF_ERR_BOUNDS record of the
// debug build adds the site, the index and the bound in words 1-3.
static __device__ int g_device_error_word[4];

int device_error_word(int **out) {
    int dev = 0;
    int rc = current_device(&dev);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_scratch_mutex);
    DeviceScratch &s = g_scratch[dev];
    if (!s.err) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_device_error_word);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(error word)");
        s.err = static_cast<int *>(p);
    }
    *out = s.err;
    return CTF_OK;
}

const char *bounds_site_name(int site) {
    switch (site) {
    case kBndPixel: return "the view's pixels";
    case kBndBlock: return "the texture's blocks";
    case kBndDecodeTable: return "the decode tables";
    case kBndRanks: return "a warp's rank slots";
    case kBndListTable: return "a warp's List Merge table";
    case kBndFbTable: return "a warp's fallback table";
    case kBndLatent: return "a latent grid";
    case kBndTexList: return "a group's texel lists";
    case kBndRow: return "a chain's rows";
    case kBndPixSlot: return "a group's per-pixel words";
    case kBndLane: return "a shuffle's source lane";
    case kBndBatch: return "a batch plan";
    case kBndTrain: return "the trainer's buffers";
    case kBndSelfTest: return "the self-test";
    default: return "an unknown site";
    }
}

namespace {
// One thread reads element `index` of a 32-int shared array through ck().
__global__ void bounds_selftest_kernel(int index, int *err) {
    __shared__ volatile int a[32];
    a[threadIdx.x] = (int)threadIdx.x;
    __syncwarp();
    if (threadIdx.x == 0) (void)a[ck(index, 32, err, kBndSelfTest)];
}
}  // namespace

cudaError_t launch_bounds_selftest(int index, int *err, cudaStream_t stream) {
    bounds_selftest_kernel<<<1, 32, 0, stream>>>(index, err);
    return cudaGetLastError();
}

std::mutex g_alloc_mutex;
long long g_alloc_calls = 0, g_alloc_live = 0;
int g_alloc_skip = 0, g_alloc_fail = 0;  // let `skip` through, then fail `fail`

cudaError_t dev_malloc(void **p, size_t bytes) {
    bool fail_now = false;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mutex);
        ++g_alloc_calls;
        if (g_alloc_fail > 0) {
            if (g_alloc_skip > 0) {
                --g_alloc_skip;
            } else {
                --g_alloc_fail;
                fail_now = true;
            }
        }
    }
    if (fail_now) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_alloc_mutex);
        ++g_alloc_live;
    }
    return e;
}

void dev_free(void *p) {
    if (!p) return;
    cudaFree(p);
    std::lock_guard<std::mutex> lk(g_alloc_mutex);
    --g_alloc_live;
}

}  // namespace ctf

// Helpers for the no-allocation entry point (ctf_noalloc.cu), which keeps its
// scratch in a static device array instead of the buffers above.
namespace ctf {

int noalloc_validate(ctf_texture tex, const float *uv, const float *jac, int width, int height, ctf_algorithm alg,
                     const ctf_filter_opts *opts, float *out) {
    g_last_error.clear();
    ResolvedOpts ro;
    return validate_filter_args(tex, uv, jac, width, height, alg, out, &ro, opts);
}

int noalloc_fail(int status, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

int noalloc_cuda_fail(cudaError_t e, const char *what) { return cuda_fail(e, what); }

int noalloc_run(ctf_texture tex, const float *uv, const float *jac, const uint8_t *coverage, int width, int height,
                int view_id, ctf_algorithm alg, uint64_t seed, const ctf_filter_opts *opts, float *out,
                uint8_t *evals, unsigned long long *dstats, cudaStream_t stream) {
    ResolvedOpts ro;
    int rc = resolve_opts(opts, &ro);
    if (rc) return rc;
    return run_filter(tex, uv, jac, coverage, width, height, view_id, alg, seed, ro, out, evals, dstats, stream);
}

int noalloc_read_stats(unsigned long long *dstats, ctf_stats *stats, cudaStream_t stream) {
    return read_stats(dstats, stats, stream);
}

}  // namespace ctf

extern "C" {

const char *ctf_version(void) { return "ctf-gb300 0.1 (sm_103a)"; }

const char *ctf_status_string(int status) {
    switch (status) {
    case CTF_OK: return "CTF_OK";
    case CTF_ERR_ARG: return "CTF_ERR_ARG";
    case CTF_ERR_ALIGN: return "CTF_ERR_ALIGN";
    case CTF_ERR_UNSUPPORTED: return "CTF_ERR_UNSUPPORTED";
    case CTF_ERR_OOM: return "CTF_ERR_OOM";
    case CTF_ERR_CUDA: return "CTF_ERR_CUDA";
    case CTF_ERR_TIMEOUT: return "CTF_ERR_TIMEOUT";
    case CTF_ERR_CORRUPT: return "CTF_ERR_CORRUPT";
    case CTF_ERR_BOUNDS: return "CTF_ERR_BOUNDS";
    default: return "CTF_ERR_UNKNOWN";
    }
}

const char *ctf_last_error(void) { return g_last_error.c_str(); }

int ctf_sync_check(void *stream) {
    g_last_error.clear();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronise");
    int *err = nullptr;
    int rc = ctf::device_error_word(&err);
    if (rc) return rc;
    int h[4] = {0, 0, 0, 0};
    e = cudaMemcpy(h, err, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the error word");
    if (h[0] != 0) {
        cudaMemset(err, 0, sizeof(h));
        if (h[0] == CTF_ERR_BOUNDS)
            return fail(h[0], "index %d outside [0, %d) at %s (site %d), recorded by a kernel of the debug build",
                        h[2], h[3], ctf::bounds_site_name(h[1]), h[1]);
        return fail(h[0], "a device wait gave up (status %d recorded by a kernel)", h[0]);
    }
    return CTF_OK;
}

int ctf_debug_build(void) { return ctf::kDebugBuild ? 1 : 0; }

int ctf_debug_selftest_bounds(int index, void *stream) {
    g_last_error.clear();
    if (!ctf::kDebugBuild)
        return fail(CTF_ERR_UNSUPPORTED, "the release library has no index checks (load libctf_debug.so)");
    int *err = nullptr;
    int rc = ctf::device_error_word(&err);
    if (rc) return rc;
    cudaError_t e = ctf::launch_bounds_selftest(index, err, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "self-test launch");
    return CTF_OK;
}

int64_t ctf_debug_device_allocations(void) {
    std::lock_guard<std::mutex> lk(ctf::g_alloc_mutex);
    return (int64_t)ctf::g_alloc_calls;
}

int64_t ctf_debug_live_allocations(void) {
    std::lock_guard<std::mutex> lk(ctf::g_alloc_mutex);
    return (int64_t)ctf::g_alloc_live;
}

int ctf_debug_fail_allocations(int skip, int n) {
    g_last_error.clear();
    if (skip < 0 || n < 0) return fail(CTF_ERR_ARG, "skip = %d and n = %d must not be negative", skip, n);
    std::lock_guard<std::mutex> lk(ctf::g_alloc_mutex);
    ctf::g_alloc_skip = skip;
    ctf::g_alloc_fail = n;
    return CTF_OK;
}

int ctf_selftest_bounded_wait(uint32_t polls, void *stream) {
    g_last_error.clear();
    if (polls < 1 || polls > (1u << 24)) return fail(CTF_ERR_ARG, "polls %u outside [1, 2^24]", polls);
    int *err = nullptr;
    int rc = ctf::device_error_word(&err);
    if (rc) return rc;
    cudaError_t e = ctf::launch_bounded_wait_selftest(polls, err, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "self-test launch");
    return CTF_OK;
}

int ctf_texture_create(const ctf_texture_desc *desc, ctf_texture *out) {
    ctf::NvtxRange nvtx_range("ctf_texture_create");
    g_last_error.clear();
    if (!desc || !out) return fail(CTF_ERR_ARG, "desc and out must not be NULL");
    *out = nullptr;
    if (desc->mode != CTF_EVAL_BLOCK)
        return fail(CTF_ERR_UNSUPPORTED, "mode %d needs ctf_texture_create_mlp", (int)desc->mode);
    const int W = desc->width, H = desc->height;
    if (W < 4 || H < 4 || W > 65536 || H > 65536 || W % 4 || H % 4)
        return fail(CTF_ERR_ARG, "texture %dx%d: sides must be multiples of 4 in [4, 65536]", W, H);
    if (!desc->blocks) return fail(CTF_ERR_ARG, "blocks must not be NULL");
    ctf_texture t = new (std::nothrow) ctf_texture_s();
    if (!t) return fail(CTF_ERR_OOM, "host allocation");
    t->width = W;
    t->height = H;
    t->mode = CTF_EVAL_BLOCK;
    cudaGetDevice(&t->device);
    const size_t bytes = (size_t)(W / 4) * (size_t)(H / 4) * 8;
    cudaError_t e = ctf::dev_malloc(&t->blocks, bytes);
    if (e != cudaSuccess) {
        delete t;
        return cuda_fail(e, "cudaMalloc(blocks)");
    }
    e = cudaMemcpy(t->blocks, desc->blocks, bytes, cudaMemcpyDefault);
    if (e != cudaSuccess) {
        ctf::dev_free(t->blocks);
        delete t;
        return cuda_fail(e, "copying blocks");
    }
    t->tables = ctf::device_decode_tables();
    if (!t->tables) {
        ctf::dev_free(t->blocks);
        delete t;
        return CTF_ERR_CUDA;
    }
    *out = t;
    return CTF_OK;
}

int ctf_texture_destroy(ctf_texture tex) {
    g_last_error.clear();
    if (!tex) return CTF_OK;
    cudaDeviceSynchronize();
    if (tex->blocks) ctf::dev_free(tex->blocks);
    for (int g = 0; g < 2; ++g)
        if (tex->lat[g]) ctf::dev_free(tex->lat[g]);
    if (tex->img) ctf::dev_free(tex->img);
    delete tex;
    return CTF_OK;
}

int ctf_filter(ctf_texture tex, const float *uv, const float *jac, const uint8_t *coverage, int width, int height,
               int view_id, ctf_algorithm alg, uint64_t seed, const ctf_filter_opts *opts, float *out_rgba,
               uint8_t *out_evals, ctf_stats *stats, void *stream) {
    ctf::NvtxRange nvtx_range("ctf_filter");
    g_last_error.clear();
    ResolvedOpts ro;
    int rc = validate_filter_args(tex, uv, jac, width, height, alg, out_rgba, &ro, opts);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long *dstats = nullptr;
    if (stats) {
        rc = scratch_stats(&dstats);
        if (rc) return rc;
        cudaError_t e = cudaMemsetAsync(dstats, 0, sizeof(unsigned long long) * ctf::kNumStats, s);
        if (e != cudaSuccess) return cuda_fail(e, "clearing stats");
    }
    if ((size_t)width * (size_t)height > 0) {
        rc = run_filter(tex, uv, jac, coverage, width, height, view_id, alg, seed, ro, out_rgba, out_evals, dstats, s);
        if (rc) return rc;
    }
    if (stats) return read_stats(dstats, stats, s);
    return CTF_OK;
}

}  // extern "C"

namespace {

// The device address of page-locked host memory that the GPU can read and
// write in place (mapped into the unified address space), or nullptr for
// pageable memory.
void *mapped_host(const void *h) {
    if (!h) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();  // an unknown pointer is pageable memory here
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

}  // namespace

extern "C" {

int ctf_filter_host(ctf_texture tex, const float *uv_host, const float *jac_host, const uint8_t *coverage_host,
                    int width, int height, int view_id, ctf_algorithm alg, uint64_t seed,
                    const ctf_filter_opts *opts, float *out_rgba_host, uint8_t *out_evals_host, ctf_stats *stats,
                    void *stream) {
    ctf::NvtxRange nvtx_range("ctf_filter_host");
    g_last_error.clear();
    ResolvedOpts ro;
    int rc = validate_filter_args(tex, uv_host, jac_host, width, height, alg, out_rgba_host, &ro, opts);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t np = (size_t)width * (size_t)height;
    if (np == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return CTF_OK;
    }
    const bool need_jac = alg != CTF_ALG_4TAP && alg != CTF_ALG_STF;
    // Page-locked buffers: the kernel reads the inputs and writes the image
    // in host memory itself (over NVLink-C2C on a Grace-Blackwell node), with
    // no staging copies.  The counts, one byte per pixel, go to device memory
    // and come back in one copy after the kernel: written in place they would
    // cross the link as 8-byte pieces of 128-byte lines, which took longer
    // than the copy.
    {
        void *m_uv = mapped_host(uv_host), *m_jac = need_jac ? mapped_host(jac_host) : nullptr;
        void *m_cov = mapped_host(coverage_host), *m_out = mapped_host(out_rgba_host);
        if (m_uv && (m_jac || !need_jac) && (m_cov || !coverage_host) && m_out) {
            uint8_t *d_ev = nullptr;
            if (out_evals_host) {
                void *stage = nullptr;
                rc = scratch_stage(np, &stage);
                if (rc) return rc;
                d_ev = static_cast<uint8_t *>(stage);
            }
            unsigned long long *dstats = nullptr;
            if (stats) {
                rc = scratch_stats(&dstats);
                if (rc) return rc;
                cudaError_t e = cudaMemsetAsync(dstats, 0, sizeof(unsigned long long) * ctf::kNumStats, s);
                if (e != cudaSuccess) return cuda_fail(e, "clearing stats");
            }
            rc = run_filter(tex, static_cast<const float *>(m_uv), static_cast<const float *>(m_jac),
                            static_cast<const uint8_t *>(m_cov), width, height, view_id, alg, seed, ro,
                            static_cast<float *>(m_out), d_ev, dstats, s);
            if (rc) return rc;
            if (d_ev) {
                cudaError_t e = cudaMemcpyAsync(out_evals_host, d_ev, np, cudaMemcpyDeviceToHost, s);
                if (e != cudaSuccess) return cuda_fail(e, "copying counts");
            }
            if (stats) return read_stats(dstats, stats, s);
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "stream synchronise");
            return CTF_OK;
        }
    }
    // staging layout: uv | jac | out | coverage | evals, each 256-byte aligned
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_uv = up(np * 8), b_jac = up(np * 16), b_out = up(np * 16), b_cov = up(np), b_ev = up(np);
    void *stage = nullptr;
    rc = scratch_stage(b_uv + b_jac + b_out + b_cov + b_ev, &stage);
    if (rc) return rc;
    char *base = static_cast<char *>(stage);
    float *d_uv = reinterpret_cast<float *>(base);
    float *d_jac = reinterpret_cast<float *>(base + b_uv);
    float *d_out = reinterpret_cast<float *>(base + b_uv + b_jac);
    uint8_t *d_cov = reinterpret_cast<uint8_t *>(base + b_uv + b_jac + b_out);
    uint8_t *d_ev = reinterpret_cast<uint8_t *>(base + b_uv + b_jac + b_out + b_cov);
    unsigned long long *dstats = nullptr;
    if (stats) {
        rc = scratch_stats(&dstats);
        if (rc) return rc;
        cudaError_t e = cudaMemsetAsync(dstats, 0, sizeof(unsigned long long) * ctf::kNumStats, s);
        if (e != cudaSuccess) return cuda_fail(e, "clearing stats");
    }
    // Bands of whole tile rows (a multiple of 8 rows fits every tile shape):
    // the copy-in of band b + 1, the filter of band b and the copy-out of
    // band b - 1 run at once (copy streams and the caller's stream, ordered
    // by events).  Each band is filtered as a frame that starts at its row
    // of the view, which gives the image and counts of one call on the whole
    // view; group_dedup views stay whole (their distinct-texel count depends
    // on the groups).
    HostPipe *hp = nullptr;
    rc = host_pipe(&hp);
    if (rc) return rc;
    const int nb = (ro.group_dedup || np < ((size_t)1 << 20)) ? 1 : kMaxBands;
    const int rows = ((height + nb - 1) / nb + 7) & ~7;
    const size_t W = (size_t)width;
    cudaEvent_t ev_start = hp->ev[0], ev_done = hp->ev[2 * kMaxBands + 1];
    cudaError_t e = cudaEventRecord(ev_start, s);  // the caller's earlier work on s comes first
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp->in, ev_start, 0);
    for (int b = 0; b < nb && e == cudaSuccess; ++b) {
        const int r0 = b * rows, r1 = std::min(height, r0 + rows);
        if (r0 >= r1) break;
        const size_t o = (size_t)r0 * W, n = (size_t)(r1 - r0) * W;
        e = cudaMemcpyAsync(d_uv + 2 * o, uv_host + 2 * o, n * 8, cudaMemcpyHostToDevice, hp->in);
        if (e == cudaSuccess && need_jac)
            e = cudaMemcpyAsync(d_jac + 4 * o, jac_host + 4 * o, n * 16, cudaMemcpyHostToDevice, hp->in);
        if (e == cudaSuccess && coverage_host)
            e = cudaMemcpyAsync(d_cov + o, coverage_host + o, n, cudaMemcpyHostToDevice, hp->in);
        if (e == cudaSuccess) e = cudaEventRecord(hp->ev[1 + b], hp->in);
    }
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    for (int b = 0; b < nb; ++b) {
        const int r0 = b * rows, r1 = std::min(height, r0 + rows);
        if (r0 >= r1) break;
        const size_t o = (size_t)r0 * W, n = (size_t)(r1 - r0) * W;
        e = cudaStreamWaitEvent(s, hp->ev[1 + b], 0);
        if (e != cudaSuccess) return cuda_fail(e, "band ordering");
        rc = run_filter(tex, d_uv + 2 * o, d_jac + 4 * o, coverage_host ? d_cov + o : nullptr, width, r1 - r0,
                        view_id, alg, seed, ro, d_out + 4 * o, out_evals_host ? d_ev + o : nullptr, dstats, s, r0);
        if (rc) return rc;
        e = cudaEventRecord(hp->ev[1 + kMaxBands + b], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(hp->out, hp->ev[1 + kMaxBands + b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out_rgba_host + 4 * o, d_out + 4 * o, n * 16, cudaMemcpyDeviceToHost, hp->out);
        if (e == cudaSuccess && out_evals_host)
            e = cudaMemcpyAsync(out_evals_host + o, d_ev + o, n, cudaMemcpyDeviceToHost, hp->out);
        if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    }
    e = cudaEventRecord(ev_done, hp->out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_done, 0);
    if (e != cudaSuccess) return cuda_fail(e, "band ordering");
    if (stats) return read_stats(dstats, stats, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronise");
    return CTF_OK;
}

}  // extern "C"
