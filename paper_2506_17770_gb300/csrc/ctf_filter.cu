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

// ceil(4096 / w) for w = 0..32: t / w == (t * kDiv[w]) >> 12 for every
// t < 32 and w <= 32, and for every t < 256 and w <= 16 (checked
// exhaustively when the table was made).
__constant__ unsigned short kDiv[33] = {0,   4096, 2048, 1366, 1024, 820, 683, 586, 512, 456, 410,
                                        373, 342,  316,  293,  274,  256, 241, 228, 216, 205, 196,
                                        187, 179,  171,  164,  158,  152, 147, 142, 137, 133, 128};

__device__ __forceinline__ int div_small(int t, int w) { return (t * (int)kDiv[w]) >> 12; }

struct Inputs {
    float2 uv;
    float4 jac;
    bool covered;  // inside the frame and covered
};

struct Counters {
    uint32_t v[kNumStats];
};

template <bool kJac>
__device__ __forceinline__ Inputs load_inputs(const ExactParams &p, bool inside, uint32_t idx) {
    Inputs in;
    in.uv = make_float2(0.f, 0.f);
    in.jac = make_float4(0.f, 0.f, 0.f, 0.f);
    in.covered = inside;
    if (inside) {
        in.uv = __ldcs(p.uv + idx);
        if (kJac) in.jac = __ldcs(p.jac + idx);
        if (p.cov) in.covered = __ldcs(p.cov + idx) != 0;
    }
    return in;
}

__device__ __forceinline__ void store_pixel(const ExactParams &p, uint32_t idx, float4 v, uint8_t count) {
    __stcs(p.out + idx, v);
    if (p.evals) p.evals[idx] = count;
}

__device__ __forceinline__ float3 to_float3(uint32_t rgba8, const float *lut) {
    return make_float3(lut[rgba8 & 0xffu], lut[(rgba8 >> 8) & 0xffu], lut[(rgba8 >> 16) & 0xffu]);
}

// acc = fma(w_k, p_k, acc) from 0, k = 0..3; alpha of every block texel is 1.
__device__ __forceinline__ float4 filter4(const float w[4], const float3 t[4]) {
    float r = 0.f, g = 0.f, b = 0.f, a = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        r = __fmaf_rn(w[k], t[k].x, r);
        g = __fmaf_rn(w[k], t[k].y, g);
        b = __fmaf_rn(w[k], t[k].z, b);
        a = __fmaf_rn(w[k], 1.0f, a);
    }
    return make_float4(r, g, b, a);
}

// Mask Sampling words: lane bits at t00, t00+1 (row dy) and t00+S, t00+S+1
// (row dy+1) for row stride S, OR-reduced over the warp one 32-bit word at a
// time.
template <int NW>
__device__ __forceinline__ void mask_words(bool active, int t00, int S, uint32_t Bw[NW]) {
    const int tA = t00, tB = t00 + S;
    const uint32_t sA = (uint32_t)tA & 31u, sB = (uint32_t)tB & 31u;
    const uint32_t loA = 3u << sA, hiA = sA == 31u ? 1u : 0u;
    const uint32_t loB = 3u << sB, hiB = sB == 31u ? 1u : 0u;
    const int wA = tA >> 5, wB = tB >> 5;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        uint32_t m = 0;
        if (active) {
            m = (w == wA ? loA : 0u) | (w == wA + 1 ? hiA : 0u) | (w == wB ? loB : 0u) | (w == wB + 1 ? hiB : 0u);
        }
        Bw[w] = __reduce_or_sync(FULL, m);
    }
}

// h^{-1}(q, B): set bits of B below bit q.
template <int NW>
__device__ __forceinline__ int mask_rank(const uint32_t Bw[NW], const int pre[NW], int q) {
    const int qw = q >> 5;
    uint32_t word = Bw[0];
    int base = 0;
#pragma unroll
    for (int w = 1; w < NW; ++w) {
        word = qw == w ? Bw[w] : word;
        base = qw == w ? pre[w] : base;
    }
    return base + __popc(word & ((1u << (q & 31)) - 1u));
}

// h(i, B): position of the i-th set bit of B (i < popcount(B)).
template <int NW>
__device__ __forceinline__ int mask_select(const uint32_t Bw[NW], const int pre[NW], int i) {
    uint32_t word = Bw[0];
    int base = 0, wsel = 0;
#pragma unroll
    for (int w = 1; w < NW; ++w) {
        const bool ge = i >= pre[w];
        word = ge ? Bw[w] : word;
        base = ge ? pre[w] : base;
        wsel = ge ? w : wsel;
    }
    return 32 * wsel + (int)__fns(word, 0, i - base + 1);
}

template <int ALG, int TW, int MD>
__device__ __forceinline__ void filter_tile(const ExactParams &p, const Inputs &in, int px, int py, bool inside,
                                            uint32_t idx, int lane, uint32_t lt, const float *lut, ListTable *T,
                                            Counters &cnt) {
    constexpr bool kCollab = ALG >= ALG_LIST;
    constexpr int NW = (MD * MD + 31) / 32;
    const float fW = (float)p.Wt, fH = (float)p.Ht;

    PixelSetup ps;
    ps.active = in.covered;
    setup_coords(in.uv, fW, fH, ps);
    const uint32_t A = __ballot_sync(FULL, ps.active);
    cnt.v[kStatTilesTotal] += 1;
    if (A == 0) {
        cnt.v[kStatTilesEmpty] += 1;
        if (inside) store_pixel(p, idx, make_float4(0.f, 0.f, 0.f, 0.f), 0);
        return;
    }
    const int nactive = __popc(A);
    cnt.v[kStatPixelsActive] += nactive;

    if (!kCollab) {
        // ---------------- per-pixel 4-tap or one-tap STF ----------------
        cnt.v[kStatTilesDirect] += 1;
        cnt.v[kStatTexelEvals] += (ALG == ALG_4TAP ? 4 : 1) * nactive;
        if (ps.active) {
            if (ALG == ALG_4TAP) {
                float3 t[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    t[k] = to_float3(fetch_block_texel(p.blocks, p.nbx, p.Wt, p.Ht, ps.ulx + (k & 1), ps.uly + (k >> 1)),
                                     lut);
                float w[4];
                bilinear_weights(ps.s, ps.t, w);
                store_pixel(p, idx, filter4(w, t), 4);
            } else {
                int dx, dy;
                stf_offset(px, py, p.view, p.k0, p.k1, ps.s, ps.t, dx, dy);
                const float3 v = to_float3(fetch_block_texel(p.blocks, p.nbx, p.Wt, p.Ht, ps.ulx + dx, ps.uly + dy), lut);
                store_pixel(p, idx, make_float4(v.x, v.y, v.z, 1.0f), 1);
            }
        } else if (inside) {
            store_pixel(p, idx, make_float4(0.f, 0.f, 0.f, 0.f), 0);
        }
        return;
    }

    // ---------------- collaborative: step 1, collect ----------------
    const bool mini = __any_sync(FULL, ps.active && is_minified(in.jac, fW, fH));
    bool fits = false;
    int n = 0, minx = 0, miny = 0, bw = 0, mcls = 0;
    uint32_t Bw[NW];
    int pre[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        Bw[w] = 0;
        pre[w] = 0;
    }
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
            // The mask covers the M x M square of Sec. 3.3; its bits are laid
            // out with the bounding-box width bw as row stride, so that the
            // common small boxes need one or two words.  The set, hence n and
            // every output, is the same as with row stride M.
            if (bw <= MD && bh <= MD) {
                const int area = bw * bh;
                const int t00 = (ps.uly - miny) * bw + (ps.ulx - minx);
                if (area <= 32) {
                    mcls = 1;
                    const uint32_t m = ps.active ? ((3u << t00) | (3u << (t00 + bw))) : 0u;
                    Bw[0] = __reduce_or_sync(FULL, m);
                    n = __popc(Bw[0]);
                } else if (area <= 64) {
                    mcls = 2;
                    const unsigned long long m = ps.active ? ((3ull << t00) | (3ull << (t00 + bw))) : 0ull;
                    Bw[0] = __reduce_or_sync(FULL, (uint32_t)m);
                    Bw[1] = __reduce_or_sync(FULL, (uint32_t)(m >> 32));
                    pre[1] = __popc(Bw[0]);
                    n = pre[1] + __popc(Bw[1]);
                } else {
                    mcls = 3;
                    mask_words<NW>(ps.active, t00, bw, Bw);
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        pre[w] = n;
                        n += __popc(Bw[w]);
                    }
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
            const float3 v = to_float3(fetch_block_texel(p.blocks, p.nbx, p.Wt, p.Ht, ps.ulx + dx, ps.uly + dy), lut);
            store_pixel(p, idx, make_float4(v.x, v.y, v.z, 1.0f), 1);
        } else if (inside) {
            store_pixel(p, idx, make_float4(0.f, 0.f, 0.f, 0.f), 0);
        }
    } else {
        cnt.v[kStatTilesSuccess] += 1;
        cnt.v[kStatTexelEvals] += n;
        // ---------------- step 2: produce texel i on lane h(i, A) ----------------
        const bool full = A == FULL;
        const int my_i = (full || !p.edge_remap) ? lane : (((A >> lane) & 1u) ? __popc(A & lt) : 32);
        float3 val = make_float3(0.f, 0.f, 0.f);
        if (my_i < n) {
            int x, y;
            if (ALG == ALG_BOX) {
                const int q = div_small(my_i, bw);
                x = minx + (my_i - q * bw);
                y = miny + q;
            } else if (ALG == ALG_MASK) {
                int t;
                if (mcls == 1) {
                    t = (int)__fns(Bw[0], 0, my_i + 1);
                } else if (mcls == 2) {
                    t = my_i < pre[1] ? (int)__fns(Bw[0], 0, my_i + 1) : 32 + (int)__fns(Bw[1], 0, my_i - pre[1] + 1);
                } else {
                    t = mask_select<NW>(Bw, pre, my_i);
                }
                const int q = div_small(t, bw);
                x = minx + (t - q * bw);
                y = miny + q;
            } else {
                const unsigned long long key = T->list[my_i];
                x = minx + (int)(uint32_t)key;
                y = miny + (int)(uint32_t)(key >> 32);
            }
            val = to_float3(fetch_block_texel(p.blocks, p.nbx, p.Wt, p.Ht, x, y), lut);
        }
        // ---------------- step 3: gather the 2x2 taps and filter ----------------
        int j[4];
        const int dx0 = ps.ulx - minx, dy0 = ps.uly - miny;
        if (ALG == ALG_BOX) {
            j[0] = dx0 + dy0 * bw;
            j[1] = j[0] + 1;
            j[2] = j[0] + bw;
            j[3] = j[2] + 1;
        } else if (ALG == ALG_MASK) {
            const int t00 = dy0 * bw + dx0, t01 = t00 + bw;
            if (mcls == 1) {
                j[0] = __popc(Bw[0] & ((1u << t00) - 1u));
                j[2] = __popc(Bw[0] & ((1u << t01) - 1u));
            } else if (mcls == 2) {
                const unsigned long long B = ((unsigned long long)Bw[1] << 32) | Bw[0];
                j[0] = __popcll(B & ((1ull << t00) - 1ull));
                j[2] = __popcll(B & ((1ull << t01) - 1ull));
            } else {
                j[0] = mask_rank<NW>(Bw, pre, t00);
                j[2] = mask_rank<NW>(Bw, pre, t01);
            }
            j[1] = j[0] + 1;
            j[3] = j[2] + 1;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                j[k] = 0;
                if (ps.active) {
                    const unsigned long long key =
                        ((unsigned long long)(uint32_t)(dy0 + (k >> 1)) << 32) | (uint32_t)(dx0 + (k & 1));
                    unsigned h = hash_key(key) & 255u;
                    for (int probe = 0; probe < 256; ++probe) {
                        const unsigned long long kk = T->keys[h];
                        if (kk == key) {
                            j[k] = T->index[h];
                            break;
                        }
                        if (kk == kEmpty) break;
                        h = (h + 1) & 255u;
                    }
                }
            }
        }
        if (!full && p.edge_remap) {
#pragma unroll
            for (int k = 0; k < 4; ++k) j[k] = nth_set_lane(A, j[k]);
        }
        float3 t[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int src = j[k] & 31;
            t[k].x = __shfl_sync(FULL, val.x, src);
            t[k].y = __shfl_sync(FULL, val.y, src);
            t[k].z = __shfl_sync(FULL, val.z, src);
        }
        if (ps.active) {
            float w[4];
            bilinear_weights(ps.s, ps.t, w);
            store_pixel(p, idx, filter4(w, t), my_i < n ? 1 : 0);
        } else if (inside) {
            store_pixel(p, idx, make_float4(0.f, 0.f, 0.f, 0.f), 0);
        }
    }
    if (ALG == ALG_LIST) {
        __syncwarp();
#pragma unroll
        for (int s = 0; s < 8; ++s) T->keys[lane * 8 + s] = kEmpty;
        __syncwarp();
    }
}

template <int ALG, int TW, int MD>
__global__ void __launch_bounds__(kThreads) exact_filter_kernel(const ExactParams p) {
    constexpr int TH = 32 / TW;
    constexpr bool kJac = ALG >= ALG_LIST;
    __shared__ float lut[256];
    __shared__ unsigned long long block_stats[kNumStats];
    extern __shared__ __align__(16) unsigned char dyn_smem[];

    for (int i = threadIdx.x; i < 256; i += blockDim.x) lut[i] = __fdiv_rn((float)i, 255.0f);
    if (threadIdx.x < kNumStats) block_stats[threadIdx.x] = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ListTable *T = ALG == ALG_LIST ? reinterpret_cast<ListTable *>(dyn_smem) + warp : nullptr;
    if (ALG == ALG_LIST) {
#pragma unroll
        for (int s = 0; s < 8; ++s) T->keys[lane * 8 + s] = kEmpty;
    }
    __syncthreads();

    const int tx = lane % TW, ty = lane / TW;
    const uint32_t lt = lanemask_lt();
    Counters cnt;
#pragma unroll
    for (int i = 0; i < kNumStats; ++i) cnt.v[i] = 0;

    // Warp-uniform tile walk: tile -> (bx, by) once, then advanced by the
    // grid stride without dividing again.
    const uint32_t ntiles = (uint32_t)p.n_tiles, tiles_x = (uint32_t)p.tiles_x;
    const uint32_t stride = gridDim.x * kWarps;
    const uint32_t sbx = stride % tiles_x, sby = stride / tiles_x;
    uint32_t tile = blockIdx.x * kWarps + warp;
    uint32_t bx = tile % tiles_x, by = tile / tiles_x;

    int px = (int)(bx * TW) + tx, py = (int)(by * TH) + ty;
    bool inside = tile < ntiles && px < p.W && py < p.H;
    uint32_t idx = inside ? (uint32_t)py * (uint32_t)p.W + (uint32_t)px : 0u;
    Inputs cur = load_inputs<kJac>(p, inside, idx);

    while (tile < ntiles) {
        // prefetch the next tile of this warp
        uint32_t nbx = bx + sbx, nby = by + sby;
        if (nbx >= tiles_x) {
            nbx -= tiles_x;
            ++nby;
        }
        const uint32_t ntile = tile + stride;
        const int npx = (int)(nbx * TW) + tx, npy = (int)(nby * TH) + ty;
        const bool ninside = ntile < ntiles && npx < p.W && npy < p.H;
        const uint32_t nidx = ninside ? (uint32_t)npy * (uint32_t)p.W + (uint32_t)npx : 0u;
        const Inputs nxt = load_inputs<kJac>(p, ninside, nidx);

        filter_tile<ALG, TW, MD>(p, cur, px, py, inside, idx, lane, lt, lut, T, cnt);

        tile = ntile;
        bx = nbx;
        by = nby;
        px = npx;
        py = npy;
        inside = ninside;
        idx = nidx;
        cur = nxt;
    }

    if (p.stats) {
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
