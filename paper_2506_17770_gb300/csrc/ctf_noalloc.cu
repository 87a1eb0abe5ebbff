// ctf_noalloc.cu -- ctf_filter_host_noalloc: the host-buffer filter without
// any device allocation.
//
// ctf_filter_host stages the caller's host arrays in device memory that the
// library allocates with cudaMalloc on first use (and frees and re-allocates
// when a larger view arrives).  Some callers cannot allow that: a renderer or
// plug-in host whose video memory is pre-reserved by its own allocator and
// budgeted per frame, or a frame loop that must not stall, since cudaMalloc
// and cudaFree may synchronise the whole device.  For them this entry point
// keeps every byte of scratch (the staging of inputs and outputs and the
// stats counters) in one file-scope __device__ array of fixed size, created
// with the module and held by every GPU that loads the library until the
// process exits.  It calls no cudaMalloc, cudaFree or other allocating
// routine.
//
// Limits and sharing rules:
//  - the array is CTF_NOALLOC_SCRATCH_BYTES (32 MiB); a view needs 256 bytes
//    of counters plus, each rounded up to 256 bytes, 8 (uv) + 16 (jac) +
//    16 (image) + 1 (coverage) + 1 (counts) bytes per pixel: about 798,000
//    pixels at most (1024x768 fits).  Larger views are rejected with
//    CTF_ERR_ARG before anything is queued;
//  - every call on a device uses the same array and leaves its contents
//    there; the stats counters are cleared on the stream at the start of
//    each call.  Calls whose GPU work overlaps (two streams, or two host
//    threads) race on the array: serialise them;
//  - the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it; make
//    that first call before any stream capture.
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/ctf.h"
#include "ctf_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[CTF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDev = 64;
void *g_scratch_addr[kMaxDev] = {};
std::mutex g_addr_mutex;

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device (host code may
// not use the symbol itself as a pointer).
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_addr_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int ctf_filter_host_noalloc(ctf_texture tex, const float *uv_host, const float *jac_host,
                                       const uint8_t *coverage_host, int width, int height, int view_id,
                                       ctf_algorithm alg, uint64_t seed, const ctf_filter_opts *opts,
                                       float *out_rgba_host, uint8_t *out_evals_host, ctf_stats *stats,
                                       void *stream) {
    ctf::NvtxRange nvtx_range("ctf_filter_host_noalloc");
    using namespace ctf;
    // Argument checks first (they queue nothing and touch no device memory).
    int rc = noalloc_validate(tex, uv_host, jac_host, width, height, alg, opts, out_rgba_host);
    if (rc) return rc;
    const size_t np = (size_t)width * (size_t)height;
    if (np == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return CTF_OK;
    }
    const size_t b_stats = 256, b_uv = up256(np * 8), b_jac = up256(np * 16), b_out = up256(np * 16),
                 b_cov = up256(np), b_ev = up256(np);
    const size_t need = b_stats + b_uv + b_jac + b_out + b_cov + b_ev;
    if (need > (size_t)CTF_NOALLOC_SCRATCH_BYTES)
        return noalloc_fail(CTF_ERR_ARG,
                            "view of %zu pixels needs %zu bytes of scratch; ctf_filter_host_noalloc holds at most "
                            "%u bytes (about 798,000 pixels)",
                            np, need, (unsigned)CTF_NOALLOC_SCRATCH_BYTES);
    void *base_v = nullptr;
    cudaError_t e = scratch_address(&base_v);
    if (e != cudaSuccess) return noalloc_cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    char *base = static_cast<char *>(base_v);
    unsigned long long *d_stats = reinterpret_cast<unsigned long long *>(base);
    float *d_uv = reinterpret_cast<float *>(base + b_stats);
    float *d_jac = reinterpret_cast<float *>(base + b_stats + b_uv);
    float *d_out = reinterpret_cast<float *>(base + b_stats + b_uv + b_jac);
    uint8_t *d_cov = reinterpret_cast<uint8_t *>(base + b_stats + b_uv + b_jac + b_out);
    uint8_t *d_ev = reinterpret_cast<uint8_t *>(base + b_stats + b_uv + b_jac + b_out + b_cov);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool need_jac = alg != CTF_ALG_4TAP && alg != CTF_ALG_STF;
    e = cudaMemcpyAsync(d_uv, uv_host, np * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && need_jac) e = cudaMemcpyAsync(d_jac, jac_host, np * 16, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && coverage_host) e = cudaMemcpyAsync(d_cov, coverage_host, np, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return noalloc_cuda_fail(e, "host-to-device copy");
    if (stats) {
        // the counters must start at zero; the array keeps the previous call's values
        e = cudaMemsetAsync(d_stats, 0, sizeof(unsigned long long) * kNumStats, s);
        if (e != cudaSuccess) return noalloc_cuda_fail(e, "clearing stats");
    }
    rc = noalloc_run(tex, d_uv, d_jac, coverage_host ? d_cov : nullptr, width, height, view_id, alg, seed, opts,
                     d_out, out_evals_host ? d_ev : nullptr, stats ? d_stats : nullptr, s);
    if (rc) return rc;
    e = cudaMemcpyAsync(out_rgba_host, d_out, np * 16, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && out_evals_host) e = cudaMemcpyAsync(out_evals_host, d_ev, np, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return noalloc_cuda_fail(e, "device-to-host copy");
    if (stats) return noalloc_read_stats(d_stats, stats, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_cuda_fail(e, "stream synchronise");
    return CTF_OK;
}
