// ctf_filter.cu -- exact-decode filter kernels (per-pixel 4-tap, one-tap STF,
// List Merge, Box Sampling, Mask Sampling) for sm_103a.
//
// One warp filters one tile_w x tile_h pixel tile at a time and walks the
// frame with a grid stride.  The collaborative algorithms follow the flow of
// Sec. 3: (1) the warp collects the texel set its 2x2 footprints need,
// (2) each needed texel is decoded once, by lane h(i, A) (edge remapping,
// supplemental Sec. 2), (3) every pixel gathers its 4 taps with shuffles and
// filters.  Over-budget or minified warps take the one-tap STF fallback.
//
// Data layout in HBM: uv float2 and jac float4 per pixel, row-major; output
// float4 per pixel plus one count byte.  The texture (8-byte blocks) is read
// through L1/L2 with __ldg; the per-pixel streams use evict-first loads and
// stores so that they do not push the texture out of L2.
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "ctf_device.cuh"
#include "ctf_internal.h"

namespace ctf {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;

enum { ALG_4TAP = 0, ALG_STF = 1, ALG_LIST = 2, ALG_BOX = 3, ALG_MASK = 4 };

// List Merge table of one warp: open addressing over 256 slots (at most 128
// distinct keys are ever inserted, so probing always ends).
struct ListTable {
    unsigned long long keys[256];
    unsigned char index[256];
    unsigned long long list[32];
};
constexpr unsigned long long kEmpty = ~0ull;

__device__ __forceinline__ unsigned hash_key(unsigned long long k) {
    unsigned lo = (unsigned)k, hi = (unsigned)(k >> 32);
    return ((lo * 0x9E3779B1u) ^ (hi * 0x85EBCA77u)) >> 24;
}

struct WarpCounters {
    unsigned long long v[kNumStats];
};

__device__ __forceinline__ void zero_pixel(const ExactParams &p, bool inside, size_t idx) {
    if (inside) {
        __stcs(p.out + idx, make_float4(0.f, 0.f, 0.f, 0.f));
        if (p.evals) p.evals[idx] = 0;
    }
}

template <int ALG, int TW, int MD>
__global__ void __launch_bounds__(kThreads) exact_filter_kernel(const ExactParams p) {
    constexpr int TH = 32 / TW;
    constexpr bool kCollab = ALG >= ALG_LIST;
    constexpr int NW = (MD * MD + 31) / 32;
    __shared__ float lut[256];
    __shared__ unsigned long long block_stats[kNumStats];
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    ListTable *tables = reinterpret_cast<ListTable *>(dyn_smem);

    for (int i = threadIdx.x; i < 256; i += blockDim.x) lut[i] = __fdiv_rn((float)i, 255.0f);
    if (threadIdx.x < kNumStats) block_stats[threadIdx.x] = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ListTable *T = ALG == ALG_LIST ? tables + warp : nullptr;
    if (ALG == ALG_LIST) {
#pragma unroll
        for (int s = 0; s < 8; ++s) T->keys[lane * 8 + s] = kEmpty;
    }
    __syncthreads();

    const int tx = lane % TW, ty = lane / TW;
    const float fW = (float)p.Wt, fH = (float)p.Ht;
    const uint32_t lt = lanemask_lt();
    WarpCounters cnt;
#pragma unroll
    for (int i = 0; i < kNumStats; ++i) cnt.v[i] = 0;

    for (long long tile = (long long)blockIdx.x * kWarps + warp; tile < p.n_tiles;
         tile += (long long)gridDim.x * kWarps) {
        const int bx = (int)(tile % p.tiles_x), by = (int)(tile / p.tiles_x);
        const int px = bx * TW + tx, py = by * TH + ty;
        const bool inside = px < p.W && py < p.H;
        const size_t idx = inside ? (size_t)py * (size_t)p.W + (size_t)px : 0;

        PixelSetup ps;
        float2 uv = make_float2(0.f, 0.f);
        float4 jc = make_float4(0.f, 0.f, 0.f, 0.f);
        bool covered = inside;
        if (inside) {
            uv = __ldcs(p.uv + idx);
            if (kCollab) jc = __ldcs(p.jac + idx);
            if (p.cov) covered = p.cov[idx] != 0;
        }
        ps.active = covered;
        setup_coords(uv, fW, fH, ps);
        const uint32_t A = __ballot_sync(FULL, ps.active);
        cnt.v[kStatTilesTotal] += 1;
        if (A == 0) {
            cnt.v[kStatTilesEmpty] += 1;
            zero_pixel(p, inside, idx);
            continue;
        }
        const int nactive = __popc(A);
        cnt.v[kStatPixelsActive] += nactive;

        if (!kCollab) {
            // ---------------- per-pixel 4-tap or one-tap STF ----------------
            cnt.v[kStatTilesDirect] += 1;
            if (ps.active) {
                if (ALG == ALG_4TAP) {
                    uint32_t v[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        v[k] = fetch_block_texel(p.blocks, p.nbx, p.Wt, p.Ht, ps.ulx + (k & 1), ps.uly + (k >> 1));
                    float w[4];
                    bilinear_weights(ps.s, ps.t, w);
                    __stcs(p.out + idx, filter_rgba8(w, v, lut));
                    if (p.evals) p.evals[idx] = 4;
                } else {
                    int dx, dy;
                    stf_offset(px, py, p.view, p.k0, p.k1, ps.s, ps.t, dx, dy);
                    uint32_t v = fetch_block_texel(p.blocks, p.nbx, p.Wt, p.Ht, ps.ulx + dx, ps.uly + dy);
                    __stcs(p.out + idx, rgba8_to_float(v, lut));
                    if (p.evals) p.evals[idx] = 1;
                }
            } else {
                zero_pixel(p, inside, idx);
            }
            cnt.v[kStatTexelEvals] += (ALG == ALG_4TAP ? 4 : 1) * nactive;
            continue;
        }

        // ---------------- collaborative: step 1, collect ----------------
        const bool mini = __any_sync(FULL, ps.active && is_minified(jc, fW, fH));
        bool fits = false;
        int n = 0;
        int minx = 0, miny = 0, bw = 0;
        uint32_t Bw[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) Bw[w] = 0;
        if (!mini) {
            minx = __reduce_min_sync(FULL, ps.active ? ps.ulx : INT_MAX);
            miny = __reduce_min_sync(FULL, ps.active ? ps.uly : INT_MAX);
            const int maxx = __reduce_max_sync(FULL, ps.active ? ps.ulx + 1 : INT_MIN);
            const int maxy = __reduce_max_sync(FULL, ps.active ? ps.uly + 1 : INT_MIN);
            bw = maxx - minx + 1;
            const int bh = maxy - miny + 1;
            if (ALG == ALG_BOX) {
                if (bw <= p.budget && bh <= p.budget && bw * bh <= p.budget) {
                    n = bw * bh;
                    fits = true;
                }
            } else if (ALG == ALG_MASK) {
                if (bw <= MD && bh <= MD) {
                    const int t00 = (ps.uly - miny) * MD + (ps.ulx - minx);
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        uint32_t m = 0;
                        if (ps.active) {
                            const int q[4] = {t00, t00 + 1, t00 + MD, t00 + MD + 1};
#pragma unroll
                            for (int k = 0; k < 4; ++k) m |= ((q[k] >> 5) == w) ? (1u << (q[k] & 31)) : 0u;
                        }
                        Bw[w] = __reduce_or_sync(FULL, m);
                        n += __popc(Bw[w]);
                    }
                    fits = n <= p.budget;
                }
            } else {  // List Merge: exact union through the warp's hash table
                int base = 0;
                bool over = false;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const unsigned long long key =
                        ps.active ? (((unsigned long long)(uint32_t)(ps.uly + (k >> 1) - miny) << 32) |
                                     (uint32_t)(ps.ulx + (k & 1) - minx))
                                  : (kEmpty - 1ull - (unsigned long long)lane);
                    const uint32_t grp = __match_any_sync(FULL, key);
                    const bool leader = ps.active && (__ffs(grp) - 1) == lane;
                    bool inserted = false;
                    unsigned slot = 0;
                    if (leader) {
                        unsigned h = hash_key(key) & 255u;
                        for (int probe = 0; probe < 256; ++probe) {
                            const unsigned long long old = atomicCAS(&T->keys[h], kEmpty, key);
                            if (old == kEmpty) {
                                inserted = true;
                                slot = h;
                                break;
                            }
                            if (old == key) break;
                            h = (h + 1) & 255u;
                        }
                    }
                    const uint32_t newm = __ballot_sync(FULL, inserted);
                    if (inserted) {
                        const int index = base + __popc(newm & lt);
                        T->index[slot] = (unsigned char)index;
                        if (index < 32) T->list[index] = key;
                    }
                    base += __popc(newm);
                    __syncwarp();
                    if (base > p.budget) {
                        over = true;
                        break;
                    }
                }
                n = base;
                fits = !over;
            }
            if (fits) {
                if (p.edge_remap) {
                    fits = n <= nactive;
                } else {
                    const uint32_t need = n >= 32 ? FULL : ((1u << n) - 1u);
                    fits = (A & need) == need;
                }
            }
        }

        if (!fits) {
            // ---------------- fallback: one-tap STF for every active lane ----------------
            cnt.v[kStatTilesFallbackMinified] += mini ? 1 : 0;
            cnt.v[kStatTilesFallbackBudget] += mini ? 0 : 1;
            cnt.v[kStatTexelEvals] += nactive;
            if (ps.active) {
                int dx, dy;
                stf_offset(px, py, p.view, p.k0, p.k1, ps.s, ps.t, dx, dy);
                uint32_t v = fetch_block_texel(p.blocks, p.nbx, p.Wt, p.Ht, ps.ulx + dx, ps.uly + dy);
                __stcs(p.out + idx, rgba8_to_float(v, lut));
                if (p.evals) p.evals[idx] = 1;
            } else {
                zero_pixel(p, inside, idx);
            }
        } else {
            cnt.v[kStatTilesSuccess] += 1;
            cnt.v[kStatTexelEvals] += n;
            // ---------------- step 2: produce texel i on lane h(i, A) ----------------
            const int my_i = p.edge_remap ? (((A >> lane) & 1u) ? __popc(A & lt) : 32) : lane;
            uint32_t val = 0;
            if (my_i < n) {
                int x, y;
                if (ALG == ALG_BOX) {
                    x = minx + my_i % bw;
                    y = miny + my_i / bw;
                } else if (ALG == ALG_MASK) {
                    int acc = 0, t = 0;
                    bool found = false;
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        const int c = __popc(Bw[w]);
                        if (!found && my_i < acc + c) {
                            t = 32 * w + (int)__fns(Bw[w], 0, my_i - acc + 1);
                            found = true;
                        }
                        acc += c;
                    }
                    x = minx + t % MD;
                    y = miny + t / MD;
                } else {
                    const unsigned long long key = T->list[my_i];
                    x = minx + (int)(uint32_t)key;
                    y = miny + (int)(uint32_t)(key >> 32);
                }
                val = fetch_block_texel(p.blocks, p.nbx, p.Wt, p.Ht, x, y);
            }
            // ---------------- step 3: gather the 2x2 taps and filter ----------------
            uint32_t v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int dxk = ps.ulx + (k & 1) - minx, dyk = ps.uly + (k >> 1) - miny;
                int j;
                if (ALG == ALG_BOX) {
                    j = dxk + dyk * bw;
                } else if (ALG == ALG_MASK) {
                    const int q = dyk * MD + dxk;
                    const int qw = q >> 5;
                    const uint32_t below = (1u << (q & 31)) - 1u;
                    j = 0;
#pragma unroll
                    for (int w = 0; w < NW; ++w)
                        j += w < qw ? __popc(Bw[w]) : (w == qw ? __popc(Bw[w] & below) : 0);
                } else {
                    j = 0;
                    if (ps.active) {
                        const unsigned long long key =
                            ((unsigned long long)(uint32_t)dyk << 32) | (uint32_t)dxk;
                        unsigned h = hash_key(key) & 255u;
                        for (int probe = 0; probe < 256; ++probe) {
                            const unsigned long long kk = T->keys[h];
                            if (kk == key) {
                                j = T->index[h];
                                break;
                            }
                            if (kk == kEmpty) break;
                            h = (h + 1) & 255u;
                        }
                    }
                }
                const int src = p.edge_remap ? nth_set_lane(A, j) : j;
                v[k] = __shfl_sync(FULL, val, src & 31);
            }
            if (ps.active) {
                float w[4];
                bilinear_weights(ps.s, ps.t, w);
                __stcs(p.out + idx, filter_rgba8(w, v, lut));
                if (p.evals) p.evals[idx] = my_i < n ? 1 : 0;
            } else {
                zero_pixel(p, inside, idx);
            }
        }
        if (ALG == ALG_LIST) {
            __syncwarp();
#pragma unroll
            for (int s = 0; s < 8; ++s) T->keys[lane * 8 + s] = kEmpty;
            __syncwarp();
        }
    }

    if (p.stats) {
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < kNumStats; ++i)
                if (cnt.v[i]) atomicAdd(&block_stats[i], cnt.v[i]);
        }
        __syncthreads();
        if (threadIdx.x < kNumStats && block_stats[threadIdx.x]) atomicAdd(p.stats + threadIdx.x, block_stats[threadIdx.x]);
    }
}

using KernelFn = void (*)(const ExactParams);

template <int ALG, int TW>
KernelFn pick_mask(int md) {
    if constexpr (ALG == ALG_MASK) {
        return md == 11 ? exact_filter_kernel<ALG, TW, 11> : exact_filter_kernel<ALG, TW, 16>;
    } else {
        return exact_filter_kernel<ALG, TW, 16>;
    }
}

template <int TW>
KernelFn pick_alg(int alg, int md) {
    switch (alg) {
    case ALG_4TAP: return pick_mask<ALG_4TAP, TW>(md);
    case ALG_STF: return pick_mask<ALG_STF, TW>(md);
    case ALG_LIST: return pick_mask<ALG_LIST, TW>(md);
    case ALG_BOX: return pick_mask<ALG_BOX, TW>(md);
    case ALG_MASK: return pick_mask<ALG_MASK, TW>(md);
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
    switch (tile_w) {
    case 8: fn = pick_alg<8>(alg, mask_dim); break;
    case 4: fn = pick_alg<4>(alg, mask_dim); break;
    case 16: fn = pick_alg<16>(alg, mask_dim); break;
    default: return cudaErrorInvalidValue;
    }
    if (!fn) return cudaErrorInvalidValue;
    if (p.n_tiles == 0) return cudaSuccess;
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
