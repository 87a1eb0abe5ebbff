// ctf_bicubic.cu -- the exact-decode filter with the bicubic filters of
// Sec. 4.2 (cubic B-spline and Catmull-Rom over a 4x4 footprint): per-pixel
// 16-tap, one-tap STF, List Merge, Box Sampling and Mask Sampling.
//
// The paper notes that the algorithms serve any discrete filter, with only
// the footprint corners, the weights, the bits each pixel sets and the final
// loop changed (Sec. 4.2, Appendix).  So this kernel is the bilinear one of
// ctf_filter.cu with a 4x4 footprint: the texels from one left of and above
// the upper-left texel of the bilinear footprint, separable weights
// w_x(s) w_y(t), a 4x4 block of bits per pixel in the mask, 16 taps gathered
// by shuffles and summed as acc = fma(w_k, p_k, acc) in tap order
// k = 4 j + i.  Minified and over-budget warps take one-tap STF, which draws
// a tap per axis with probability |w| / sum |w|; Catmull-Rom's negative
// lobes scale the texel by the signed sums.  One texel per lane, block
// textures only.
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

// 1-D cubic weights of the taps at -1, 0, 1, 2 from the upper-left texel,
// f in [0, 1); every term one round-to-nearest operation in the order
// written.  B-spline: ((1-f)^3, 3f^3 - 6f^2 + 4, -3f^3 + 3f^2 + 3f + 1,
// f^3) / 6; Catmull-Rom: (2f^2 - f^3 - f, 3f^3 - 5f^2 + 2,
// -3f^3 + 4f^2 + f, f^3 - f^2) / 2.
template <int FILT>
__device__ __forceinline__ void cubic_weights(float f, float w[4]) {
    const float f2 = __fmul_rn(f, f), f3 = __fmul_rn(f2, f);
    if (FILT == 1) {
        const float u = __fsub_rn(1.0f, f);
        w[0] = __fdiv_rn(__fmul_rn(__fmul_rn(u, u), u), 6.0f);
        w[1] = __fdiv_rn(__fadd_rn(__fsub_rn(__fmul_rn(3.0f, f3), __fmul_rn(6.0f, f2)), 4.0f), 6.0f);
        w[2] = __fdiv_rn(
            __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(-3.0f, f3), __fmul_rn(3.0f, f2)), __fmul_rn(3.0f, f)), 1.0f),
            6.0f);
        w[3] = __fdiv_rn(f3, 6.0f);
    } else {
        w[0] = __fmul_rn(0.5f, __fsub_rn(__fsub_rn(__fmul_rn(2.0f, f2), f3), f));
        w[1] = __fmul_rn(0.5f, __fadd_rn(__fsub_rn(__fmul_rn(3.0f, f3), __fmul_rn(5.0f, f2)), 2.0f));
        w[2] = __fmul_rn(0.5f, __fadd_rn(__fadd_rn(__fmul_rn(-3.0f, f3), __fmul_rn(4.0f, f2)), f));
        w[3] = __fmul_rn(0.5f, __fsub_rn(f3, f2));
    }
}

// One of 4 taps drawn with probability |w_i| / sum |w|: cumulative sums in
// tap order, the first i with xi S < c_i; g = S with the sign of w_i.
__device__ __forceinline__ int pick_tap(const float w[4], float xi, float &g) {
    const float a0 = fabsf(w[0]), a1 = fabsf(w[1]), a2 = fabsf(w[2]), a3 = fabsf(w[3]);
    const float c0 = a0, c1 = __fadd_rn(c0, a1), c2 = __fadd_rn(c1, a2), S = __fadd_rn(c2, a3);
    const float t = __fmul_rn(xi, S);
    const int i = t < c0 ? 0 : (t < c1 ? 1 : (t < c2 ? 2 : 3));
    g = w[i] < 0.f ? -S : S;
    return i;
}

// Bits of a pixel's 4x4 block (rows r at position t00 + r * bw, 4 bits
// each) that fall in 32-bit word w of the mask.
__device__ __forceinline__ uint32_t block_bits(int t00, int bw, int w) {
    uint32_t m = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int pos = t00 + r * bw, wd = pos >> 5, sh = pos & 31;
        if (wd == w) m |= 0xFu << sh;
        if (wd + 1 == w && sh > 28) m |= 0xFu >> (32 - sh);
    }
    return m;
}

template <int ALG, int TW, int MD, int FILT, bool kStats>
__global__ void __launch_bounds__(kThreads) bicubic_filter_kernel(const ExactParams p) {
    constexpr int TH = 32 / TW;
    constexpr bool kJac = ALG >= ALG_LIST;
    constexpr int NW = (MD * MD + 31) / 32;
    __shared__ DecodeTables tabs;
    __shared__ int rank_slots[kWarps][32];
    __shared__ unsigned long long block_stats[kNumStats];
    extern __shared__ __align__(16) unsigned char dyn_smem[];

    if (threadIdx.x < kNumStats) block_stats[threadIdx.x] = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ListTable *T = ALG == ALG_LIST ? reinterpret_cast<ListTable *>(dyn_smem) + warp : nullptr;
    if (ALG == ALG_LIST) {
#pragma unroll
        for (int s = 0; s < 8; ++s) T->keys[lane * 8 + s] = kEmpty;
    }
    load_decode_tables(&tabs, p.tables);
    __syncthreads();
    int *ranks = rank_slots[warp];
    const int tx = lane % TW, ty = lane / TW;
    const uint32_t lt = lanemask_lt();
    Counters cnt;
#pragma unroll
    for (int i = 0; i < kNumStats; ++i) cnt.v[i] = 0;
    const float fW = (float)p.Wt, fH = (float)p.Ht;

    const long long stride = (long long)gridDim.x * kWarps;
    for (long long tile = (long long)blockIdx.x * kWarps + warp; tile < p.n_tiles; tile += stride) {
        const int bx = (int)(tile % p.tiles_x), by = (int)(tile / p.tiles_x);
        const int px = bx * TW + tx, py = by * TH + ty;
        const bool inside = px < p.W && py < p.H;
        const uint32_t idx = inside ? (uint32_t)py * (uint32_t)p.W + (uint32_t)px : 0u;
        const Inputs in = load_inputs_any<kJac>(p, inside, idx);
        PixelSetup ps;
        ps.active = in.covered;
        setup_coords(in.uv, fW, fH, ps);
        const int ox = ps.ulx - 1, oy = ps.uly - 1;  // the 4x4 footprint's corner
        float wx[4], wy[4];
        cubic_weights<FILT>(ps.s, wx);
        cubic_weights<FILT>(ps.t, wy);

        const uint32_t A = __ballot_sync(FULL, ps.active);
        const int nactive = __popc(A);
        if (kStats) {
            cnt.v[kStatTilesTotal] += 1;
            cnt.v[kStatPixelsActive] += nactive;
            if (A == 0) cnt.v[kStatTilesEmpty] += 1;
        }
        float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
        uint32_t count = 0;
        if (A == 0) {
            if (inside) store_pixel(p, idx, res, 0);
            continue;
        }

        if (ALG == ALG_4TAP) {  // per pixel: all 16 taps
            if (kStats) {
                cnt.v[kStatTilesDirect] += 1;
                cnt.v[kStatTexelEvals] += 16 * nactive;
                cnt.v[kStatTexelEvalsUnique] += 16 * nactive;
            }
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
            for (int k = 0; k < 16; ++k) {
                const float w = __fmul_rn(wx[k & 3], wy[k >> 2]);
                const float3 v = fetch_decode(p, ox + (k & 3), oy + (k >> 2), &tabs);
                acc.x = __fmaf_rn(w, v.x, acc.x);
                acc.y = __fmaf_rn(w, v.y, acc.y);
                acc.z = __fmaf_rn(w, v.z, acc.z);
                acc.w = __fmaf_rn(w, 1.0f, acc.w);
            }
            if (ps.active) {
                res = acc;
                count = 16;
            }
            if (inside) store_pixel(p, idx, res, (uint8_t)count);
            continue;
        }

        // ---- step 1: minification vote, the texel set, the success test
        bool fits = false, mini = false;
        int n = 0, minx = 0, miny = 0, bw = 0, mcls = 0;
        uint32_t Bw[NW];
        int pre[NW];
        if (ALG >= ALG_LIST) {
            mini = __any_sync(FULL, ps.active && is_minified(in.jac, fW, fH));
            if (!mini) {
                minx = __reduce_min_sync(FULL, ps.active ? ox : INT_MAX);
                miny = __reduce_min_sync(FULL, ps.active ? oy : INT_MAX);
                const int maxx = __reduce_max_sync(FULL, ps.active ? ox : INT_MIN) + 3;
                const int maxy = __reduce_max_sync(FULL, ps.active ? oy : INT_MIN) + 3;
                bw = maxx - minx + 1;
                const int bh = maxy - miny + 1;
                const int t00 = (oy - miny) * bw + (ox - minx);
                if (ALG == ALG_BOX) {
                    if (bw <= p.budget && bh <= p.budget && bw * bh <= p.budget) {
                        n = bw * bh;
                        fits = true;
                    }
                } else if (ALG == ALG_MASK) {
                    if (bw <= MD && bh <= MD) {
                        const int area = bw * bh;
                        mcls = area <= 32 ? 1 : 3;
                        if (mcls == 1) {
                            const uint32_t m = ps.active ? block_bits(t00, bw, 0) : 0u;
                            Bw[0] = __reduce_or_sync(FULL, m);
                            n = __popc(Bw[0]);
                        } else {
#pragma unroll
                            for (int w = 0; w < NW; ++w) {
                                Bw[w] = __reduce_or_sync(FULL, ps.active ? block_bits(t00, bw, w) : 0u);
                                pre[w] = n;
                                n += __popc(Bw[w]);
                            }
                        }
                        fits = n <= p.budget;
                    }
                } else {  // List Merge: the 16 taps of every pixel into the warp's hash table
                    int base = 0;
                    bool over = false;
#pragma unroll 1
                    for (int k = 0; k < 16; ++k) {
                        const unsigned long long key =
                            ps.active ? (((unsigned long long)(uint32_t)(oy + (k >> 2) - miny) << 32) |
                                         (uint32_t)(ox + (k & 3) - minx))
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
                            T->index[ck(slot, 256, p.err, kBndListTable)] = (unsigned char)index;
                            if (index < 64) T->list[ck(index, 64, p.err, kBndListTable)] = key;
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
        }

        if (!fits) {
            // ---- one-tap STF (minified, over budget, or the STF algorithm)
            if (kStats) {
                if (ALG >= ALG_LIST) {
                    cnt.v[kStatTilesFallbackMinified] += mini ? 1 : 0;
                    cnt.v[kStatTilesFallbackBudget] += mini ? 0 : 1;
                } else {
                    cnt.v[kStatTilesDirect] += 1;
                }
                cnt.v[kStatTexelEvals] += nactive;
                cnt.v[kStatTexelEvalsUnique] += nactive;
            }
            uint4 r = philox4x32_10(make_uint4((uint32_t)px, (uint32_t)(py + p.y0), (uint32_t)p.view, 0u), p.k0, p.k1);
            float gx, gy;
            const int i = pick_tap(wx, __fmul_rn((float)(r.x >> 8), 5.9604644775390625e-08f), gx);
            const int j = pick_tap(wy, __fmul_rn((float)(r.y >> 8), 5.9604644775390625e-08f), gy);
            const float3 v = fetch_decode(p, ox + i, oy + j, &tabs);
            if (ps.active) {
                res = FILT == 2 ? make_float4(__fmul_rn(__fmul_rn(v.x, gx), gy), __fmul_rn(__fmul_rn(v.y, gx), gy),
                                              __fmul_rn(__fmul_rn(v.z, gx), gy), __fmul_rn(__fmul_rn(1.0f, gx), gy))
                                : make_float4(v.x, v.y, v.z, 1.0f);
                count = 1;
            }
            if (inside) store_pixel(p, idx, res, (uint8_t)count);
            if (ALG == ALG_LIST) {
                __syncwarp();
#pragma unroll
                for (int s = 0; s < 8; ++s) T->keys[lane * 8 + s] = kEmpty;
                __syncwarp();
            }
            continue;
        }

        // ---- success: texel i by lane h(i, A) (or lane i); the counts follow that
        if (kStats) {
            cnt.v[kStatTilesSuccess] += 1;
            cnt.v[kStatTexelEvals] += n;
            cnt.v[kStatTexelEvalsUnique] += n;
        }
        const bool full = A == FULL;
        const int my_i = (full || !p.edge_remap) ? lane : (((A >> lane) & 1u) ? __popc(A & lt) : 32);
        count = my_i < n ? 1u : 0u;
        const int dx0 = ox - minx, dy0 = oy - miny, t00 = dy0 * bw + dx0;
        int qx = ps.ulx, qy = ps.uly;  // the texel this lane decodes
        int src[16];                   // lane holding tap k
        if (ALG == ALG_BOX || (ALG == ALG_MASK && mcls == 1)) {
            // a box of at most 32 texels: lane L decodes box position L
            const bool in_set = ALG == ALG_BOX ? lane < n : ((Bw[0] >> lane) & 1u) != 0;
            if (in_set) {
                const int q = div_small(lane, bw);
                qx = minx + (lane - q * bw);
                qy = miny + q;
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) src[k] = t00 + (k >> 2) * bw + (k & 3);
        } else {
            if (ALG == ALG_MASK) {
                // ranks of the 16 taps; the pixels file each rank's position
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int t = t00 + (k >> 2) * bw + (k & 3);
                    src[k] = mask_rank<NW>(Bw, pre, t);
                    if (ps.active) ranks[ck(src[k], 32, p.err, kBndRanks)] = t;
                }
                __syncwarp();
                if (my_i < n) {
                    const int t = ranks[ck(my_i, 32, p.err, kBndRanks)];
                    const int q = div_small(t, bw);
                    qx = minx + (t - q * bw);
                    qy = miny + q;
                }
                __syncwarp();
            } else {
#pragma unroll 1
                for (int k = 0; k < 16; ++k) {
                    int jk = 0;
                    if (ps.active) {
                        const unsigned long long key =
                            ((unsigned long long)(uint32_t)(dy0 + (k >> 2)) << 32) | (uint32_t)(dx0 + (k & 3));
                        unsigned h = hash_key(key) & 255u;
                        for (int probe = 0; probe < 256; ++probe) {
                            const unsigned long long kk = T->keys[h];
                            if (kk == key) {
                                jk = ck((int)T->index[h], 64, p.err, kBndListTable);
                                break;
                            }
                            if (kk == kEmpty) break;
                            h = (h + 1) & 255u;
                        }
                    }
                    src[k] = jk;
                }
                if (my_i < n) {
                    const unsigned long long key = T->list[ck(my_i, 64, p.err, kBndListTable)];
                    qx = minx + (int)(uint32_t)key;
                    qy = miny + (int)(uint32_t)(key >> 32);
                }
            }
            if (!full && p.edge_remap) {
#pragma unroll
                for (int k = 0; k < 16; ++k) src[k] = nth_set_lane(A, src[k]);
            }
        }
        // ---- decode, gather the 16 taps, filter in tap order
        const float3 val = fetch_decode(p, qx, qy, &tabs);
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float w = __fmul_rn(wx[k & 3], wy[k >> 2]);
            const float vx = __shfl_sync(FULL, val.x, src[k]);
            const float vy = __shfl_sync(FULL, val.y, src[k]);
            const float vz = __shfl_sync(FULL, val.z, src[k]);
            acc.x = __fmaf_rn(w, vx, acc.x);
            acc.y = __fmaf_rn(w, vy, acc.y);
            acc.z = __fmaf_rn(w, vz, acc.z);
            acc.w = __fmaf_rn(w, 1.0f, acc.w);
        }
        if (ps.active) res = acc;
        else count = 0;
        if (inside) store_pixel(p, idx, res, (uint8_t)count);
        if (ALG == ALG_LIST) {
            __syncwarp();
#pragma unroll
            for (int s = 0; s < 8; ++s) T->keys[lane * 8 + s] = kEmpty;
            __syncwarp();
        }
    }

    if (kStats) {
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

template <int ALG, int TW, int FILT, bool kStats>
KernelFn pick_mask(int md) {
    if constexpr (ALG == ALG_MASK) {
        return md == 11 ? bicubic_filter_kernel<ALG, TW, 11, FILT, kStats>
                        : bicubic_filter_kernel<ALG, TW, 16, FILT, kStats>;
    } else {
        return bicubic_filter_kernel<ALG, TW, 16, FILT, kStats>;
    }
}

template <int TW, int FILT, bool kStats>
KernelFn pick_alg(int alg, int md) {
    switch (alg) {
    case ALG_4TAP: return pick_mask<ALG_4TAP, TW, FILT, kStats>(md);
    case ALG_STF: return pick_mask<ALG_STF, TW, FILT, kStats>(md);
    case ALG_LIST: return pick_mask<ALG_LIST, TW, FILT, kStats>(md);
    case ALG_BOX: return pick_mask<ALG_BOX, TW, FILT, kStats>(md);
    case ALG_MASK: return pick_mask<ALG_MASK, TW, FILT, kStats>(md);
    default: return nullptr;
    }
}

template <int FILT, bool kStats>
KernelFn pick_tile(int alg, int tile_w, int md) {
    switch (tile_w) {
    case 8: return pick_alg<8, FILT, kStats>(alg, md);
    case 4: return pick_alg<4, FILT, kStats>(alg, md);
    case 16: return pick_alg<16, FILT, kStats>(alg, md);
    default: return nullptr;
    }
}

}  // namespace

cudaError_t launch_bicubic_filter(const ExactParams &p, int alg, int tile_w, int mask_dim, int filter,
                                  cudaStream_t stream) {
    const bool st = p.stats != nullptr;
    KernelFn fn = nullptr;
    if (filter == 1) fn = st ? pick_tile<1, true>(alg, tile_w, mask_dim) : pick_tile<1, false>(alg, tile_w, mask_dim);
    else if (filter == 2) fn = st ? pick_tile<2, true>(alg, tile_w, mask_dim) : pick_tile<2, false>(alg, tile_w, mask_dim);
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
