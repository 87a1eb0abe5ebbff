// ctf_internal.h -- host-side declarations shared by the translation units of
// the CUDA library (not part of the public ABI).
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ctf.h"
#include "ctf_mlp.cuh"

namespace ctf {
// A named range on the host timeline around one entry point's work (NVTX:
// a profiler attached to the process shows the range and can filter the
// kernels queued inside it, e.g. ncu --nvtx --nvtx-include "ctf_filter/";
// with no tool attached it costs a pointer test).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Decode tables of the exact block decode, one copy per device in global
// memory (made on the host, ctf_api.cu) and copied into shared memory by
// every CTA: the two endpoints of a block expand to 8-bit channels laid out
// in 10-bit fields (r bits 0-9, g 10-19, b 20-29) by two lookups each, so
// that the palette entries 2 and 3, (2a+b+1)/3 with (a, b) = (c0, c1) or
// (c1, c0), come out of one integer expression for all three channels, and
// `val` turns a field into the channel value: val[v] = v/255 for v < 256,
// val[256 + s] = floor(s/3)/255 for s < 768 (both correctly rounded).
struct DecodeTables {
    uint32_t rg[2048];  // c >> 5 = (r5 << 6) | g6  ->  r8 | g8 << 10
    uint32_t b[32];     // c & 31 = b5              ->  b8 << 20
    float val[1024];
};
static_assert(sizeof(DecodeTables) % 16 == 0, "copied in 16-byte pieces");
}  // namespace ctf

// Texture object behind the opaque ctf_texture handle.
struct ctf_texture_s {
    int width = 0, height = 0;
    ctf_eval_mode mode = CTF_EVAL_BLOCK;
    int device = 0;
    void *blocks = nullptr;  // BLOCK: device copy of the blocks
    const ctf::DecodeTables *tables = nullptr;  // BLOCK: the device's decode tables (shared, not owned)
    // learned decode
    __half *lat[2] = {nullptr, nullptr};  // device latent grids [gh][gw][8]
    int gw[2] = {0, 0}, gh[2] = {0, 0};
    void *img = nullptr;                  // device operand image (kImgBytes)
    // stored (quantised) parameters as floats, for ctf_mlp_export
    std::vector<float> s_lat[2], s_w1, s_b1, s_w2, s_b2, s_w3, s_b3, s_wscale[3], s_ascale[3];
};

namespace ctf {

// Per-tile outcome counters, in the order of ctf_stats.
enum StatIndex {
    kStatTilesTotal = 0,
    kStatTilesEmpty,
    kStatTilesDirect,
    kStatTilesSuccess,
    kStatTilesFallbackBudget,
    kStatTilesFallbackMinified,
    kStatPixelsActive,
    kStatTexelEvals,
    kStatTexelEvalsUnique,
    kNumStats
};

struct __align__(16) ExactParams {
    const uint2 *blocks;  // (Wt/4)*(Ht/4) blocks
    int Wt, Ht, nbx;
    int y0;               // row of the whole view at which this frame starts (a band of it): STF counters use y0 + py
    const float2 *uv;
    const float4 *jac;
    const uint8_t *cov;   // nullable
    int W, H;
    int tiles_x;
    long long n_tiles;
    int view;
    uint32_t k0, k1;      // STF key
    int budget;
    int edge_remap;
    int group_dedup;      // learned decode: one evaluation per distinct texel of a tile group
    int fallback;         // over-budget tiles: 0 one-tap STF, 1 fallback C, 2 fallback C+
    int tpl;              // texels a lane may evaluate: 1, or 2 (budget up to 64)
    const DecodeTables *tables;  // block decode tables in global memory (block textures)
    float4 *out;
    uint8_t *evals;       // nullable
    unsigned long long *stats;  // kNumStats counters or nullptr
    int *err;             // device error word (index checks of the debug build)
};

// Pixels of the view and blocks of the texture: the bounds of the debug
// build's index checks.
__host__ __device__ inline long long view_pixels(const ExactParams &p) { return (long long)p.W * p.H; }
__host__ __device__ inline long long texture_blocks(const ExactParams &p) { return (long long)p.nbx * (p.Ht / 4); }

// Launch the exact-decode filter.  alg: ctf_algorithm; tile_w in {4, 8, 16};
// mask_dim in {11, 16}.  Returns cudaSuccess or the launch error.
cudaError_t launch_exact_filter(const ExactParams &p, int alg, int tile_w, int mask_dim, cudaStream_t stream);

// The same with a bicubic filter: filter 1 = cubic B-spline, 2 = Catmull-Rom
// (ctf_bicubic.cu).
cudaError_t launch_bicubic_filter(const ExactParams &p, int alg, int tile_w, int mask_dim, int filter,
                                  cudaStream_t stream);

// Number of SMs of the current device (cached).
int device_sm_count();

// The current device's decode tables (made once per device; nullptr and a
// recorded error if that failed).
const DecodeTables *device_decode_tables();

// Learned decode (ctf_mlp.cu).
cudaError_t launch_mlp_decode(const MlpDevice &m, int Wt, int Ht, const int2 *xy, int n, float4 *out, int *err,
                              cudaStream_t stream);
// Sets the learned filter kernel's attributes without launching it (needed
// before a stream capture records a launch of it).
cudaError_t prepare_mlp_filter(int alg, int tile_w, int mask_dim);

// One CTA whose bounded mbarrier wait runs out and records CTF_ERR_TIMEOUT.
cudaError_t launch_bounded_wait_selftest(uint32_t polls, int *err, cudaStream_t stream);
// One thread reads element `index` of a 32-int shared array through the
// debug build's index check (ctf_api.cu).
cudaError_t launch_bounds_selftest(int index, int *err, cudaStream_t stream);
// Name of a BoundsSite (ctf_debug.cuh) for error messages.
const char *bounds_site_name(int site);
cudaError_t launch_mlp_filter(const ExactParams &p, const MlpDevice &m, int alg, int tile_w, int mask_dim, int *err,
                              cudaStream_t stream);
MlpDevice mlp_device_view(const ctf_texture_s *t);
// Uploads a learned texture's stored (already quantised) parameters: the
// FP16 latent grids and the operand image (ctf_mlp_host.cu).  On failure the
// caller frees what was allocated.
int upload_mlp_texture(ctf_texture_s *t);

// 64-bit FNV-1a over n bytes, continuing from h (checkpoint checksums).
inline uint64_t fnv1a(const void *data, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char *b = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}
// The learned filters with warps specialised by role, which
// launch_mlp_filter uses for STF, Box and Mask Sampling: the features
// computed by the selecting warps (ctf_mlp_ws2.cu), and with group_dedup the
// consumer merging the group's lists (ctf_mlp_ws.cu).
bool mlp_filter_ws_applies(const ExactParams &p, int alg);
// Box and Mask with fallback C / C+ and one texel per lane run the
// fallback variant of the packed-group kernel (ctf_mlp_ws2.cu).
bool mlp_filter_pf_fallback_applies(const ExactParams &p, int alg);
// List Merge, Box and Mask with two texels per lane and no fallback: its
// variant with groups of 4 tiles.
bool mlp_filter_pf_two_applies(const ExactParams &p, int alg);
cudaError_t prepare_mlp_filter_pf(int alg, int tile_w, int mask_dim);
// The learned filter with fallbacks C / C+ or two texels per lane
// (ctf_mlp_ext.cu), for List Merge, Box and Mask Sampling.
bool mlp_filter_ext_applies(const ExactParams &p, int alg);
cudaError_t prepare_mlp_filter_ext(int alg, int tile_w, int mask_dim);
cudaError_t launch_mlp_filter_ext(const ExactParams &p, const MlpDevice &m, int alg, int tile_w, int mask_dim,
                                  int *err, cudaStream_t stream);
cudaError_t launch_mlp_filter_pf(const ExactParams &p, const MlpDevice &m, int alg, int tile_w, int mask_dim,
                                 int *err, cudaStream_t stream);
cudaError_t prepare_mlp_filter_ws(int alg, int tile_w, int mask_dim);
cudaError_t launch_mlp_filter_ws(const ExactParams &p, const MlpDevice &m, int alg, int tile_w, int mask_dim,
                                 int *err, cudaStream_t stream);

// One view of a batch plan on the device (ctf_batch.cu).
struct __align__(16) BatchViewDev {
    ExactParams p;
    MlpDevice m;
    int learned;
};
static_assert(sizeof(BatchViewDev) % 16 == 0, "copied in 16-byte pieces");
static_assert(sizeof(ExactParams) % 16 == 0 && sizeof(ExactParams) <= 32 * 16, "copied in 16-byte pieces");

// The learned views of a batch (other than per-pixel 4-tap and group_dedup)
// on the packed-group kernel (ctf_mlp_ws2.cu): the views index[0..nkind)
// of the table of nviews views, whose items (groups of 8 tiles) are numbered from
// item_begin[k]; the CTAs take items from *counter (zero at launch).  m0 is
// the first view's network, which the CTAs load first.
bool mlp_batch_pf_applies(int alg, int group_dedup);
cudaError_t prepare_mlp_batch_pf(int alg, int tile_w, int mask_dim);
cudaError_t launch_mlp_batch_pf(const BatchViewDev *views, int nviews, const int *index, const long long *item_begin,
                                int nkind, long long total_items, unsigned long long *counter, unsigned long long *stats,
                                int *err, const MlpDevice &m0, int alg, int tile_w, int mask_dim, cudaStream_t s);

// Error reporting shared by the C ABI translation units (ctf_api.cu).
int report(int status, const char *fmt, ...);
int report_cuda(cudaError_t e, const char *what);
void clear_error();
// Per-device error word that bounded device waits set (ctf_api.cu).  It is a
// file-scope __device__ int looked up once per device, so obtaining it never
// allocates.
int device_error_word(int **out);

// Every device allocation of the library goes through here (ctf_api.cu): it
// counts the calls and, when ctf_debug_fail_allocations armed it, fails
// without calling cudaMalloc (cudaErrorMemoryAllocation, no sticky error).
cudaError_t dev_malloc(void **p, size_t bytes);
template <typename T> inline cudaError_t dev_malloc(T **p, size_t bytes) {
    return dev_malloc(reinterpret_cast<void **>(p), bytes);
}
// Frees what dev_malloc gave (NULL is ignored) and keeps the count of live
// allocations that the test hooks report.
void dev_free(void *p);

}  // namespace ctf

#include "../../include/ctf.h"

namespace ctf {

// Used by ctf_filter_host_noalloc (ctf_noalloc.cu); defined in ctf_api.cu.
int noalloc_validate(ctf_texture tex, const float *uv, const float *jac, int width, int height, ctf_algorithm alg,
                     const ctf_filter_opts *opts, float *out);
int noalloc_fail(int status, const char *fmt, ...);
int noalloc_cuda_fail(cudaError_t e, const char *what);
int noalloc_run(ctf_texture tex, const float *uv, const float *jac, const uint8_t *coverage, int width, int height,
                int view_id, ctf_algorithm alg, uint64_t seed, const ctf_filter_opts *opts, float *out,
                uint8_t *evals, unsigned long long *dstats, cudaStream_t stream);
int noalloc_read_stats(unsigned long long *dstats, ctf_stats *stats, cudaStream_t stream);

}  // namespace ctf
