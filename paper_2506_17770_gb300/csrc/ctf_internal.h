// ctf_internal.h -- host-side declarations shared by the translation units of
// the CUDA library (not part of the public ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

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
    kNumStats
};

struct ExactParams {
    const uint2 *blocks;  // (Wt/4)*(Ht/4) blocks
    int Wt, Ht, nbx;
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
    float4 *out;
    uint8_t *evals;       // nullable
    unsigned long long *stats;  // kNumStats counters or nullptr
};

// Launch the exact-decode filter.  alg: ctf_algorithm; tile_w in {4, 8, 16};
// mask_dim in {11, 16}.  Returns cudaSuccess or the launch error.
cudaError_t launch_exact_filter(const ExactParams &p, int alg, int tile_w, int mask_dim, cudaStream_t stream);

// Number of SMs of the current device (cached).
int device_sm_count();

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
