// ctf_select.cuh -- step 1 of the collaborative flow (Sec. 3) for one warp
// tile, shared by the exact-decode and the learned-decode kernels: the
// minification vote, the texel set of List Merge (Sec. 3.1), Box Sampling
// (Sec. 3.2) or Mask Sampling (Sec. 3.3), the success test with edge
// remapping (supplemental Sec. 2), and for the success path the texel each
// producing lane evaluates and the lanes each pixel gathers its 4 taps from.
// STF fallback and direct algorithms leave each lane its own texel.
#pragma once
#include <climits>
#include <cstdint>

#include "ctf_device.cuh"
#include "ctf_internal.h"

namespace ctf {

enum { ALG_4TAP = 0, ALG_STF = 1, ALG_LIST = 2, ALG_BOX = 3, ALG_MASK = 4 };
enum { PATH_EMPTY = 0, PATH_SUCCESS = 1, PATH_FALLBACK_BUDGET = 2, PATH_FALLBACK_MINIFIED = 3, PATH_DIRECT = 4 };

// List Merge table of one warp: open addressing over 256 slots (at most 128
// distinct keys are ever inserted, so probing always ends).
struct ListTable {
    unsigned long long keys[256];
    unsigned char index[256];
    unsigned long long list[64];
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

struct Counters {
    uint32_t v[kNumStats];
};

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

// Outcome of step 1 for one lane.
struct Selection {
    int path;        // PATH_*
    uint32_t A;      // active-lane mask
    int n;           // texels the warp evaluates (success path)
    bool produce;    // this lane evaluates a texel
    int tx, ty;      // that texel (unclamped)
    int src[4];      // success path: lane holding tap k = (k%2, k/2); with two
                     // texels per lane, lane + 32 * round
    bool produce2;   // two texels per lane: this lane evaluates a second texel
    int tx2, ty2;    // that texel (unclamped)
    int rk[4];       // success path: index of tap k in the warp's texel list
    int my_rank;     // index of this lane's texel in that list (when produce)
    int my_rank2;    // two texels per lane: index of this lane's second texel (when produce2)
    uint8_t count;   // texel evaluations of this lane
};

// Step 1 for the collaborative algorithms (ALG >= ALG_LIST) and the STF
// algorithm.  `ps` holds the lane's setup (ps.active already decided).
// `ranks` is a per-warp array of 32 ints in shared memory (Mask Sampling
// passes texel coordinates through it); counters are kept when kStats.
// kTwo: the variant that may evaluate two texels per lane (p.tpl == 2); the
// other carries no code for it.
template <int ALG, int MD, bool kStats, bool kUnique = true, bool kTwo = false>
__device__ __forceinline__ Selection select_tile(const ExactParams &p, const PixelSetup &ps, const float4 jac,
                                                 int px, int py, int lane, uint32_t lt, ListTable *T, int *ranks,
                                                 Counters &cnt) {
    constexpr int NW = (MD * MD + 31) / 32;
    constexpr int kRanksN = kTwo ? 64 : 32;  // rank slots the caller provides
    const float fW = (float)p.Wt, fH = (float)p.Ht;
    Selection sel;
    sel.A = __ballot_sync(FULL, ps.active);
    sel.n = 0;
    sel.produce = false;
    sel.tx = ps.ulx;  // lanes that produce nothing keep their own upper-left texel
    sel.ty = ps.uly;
    sel.count = 0;  // sel.src and sel.rk are set on the success path only
    sel.my_rank = 0;
    sel.my_rank2 = 0;
    sel.produce2 = false;
    sel.tx2 = sel.ty2 = 0;
    if (kStats) cnt.v[kStatTilesTotal] += 1;
    if (sel.A == 0) {
        sel.path = PATH_EMPTY;
        if (kStats) cnt.v[kStatTilesEmpty] += 1;
        return sel;
    }
    const uint32_t A = sel.A;
    const int nactive = __popc(A);
    if (kStats) cnt.v[kStatPixelsActive] += nactive;

    bool mini = false, fits = false;
    int n = 0, minx = 0, miny = 0, bw = 0, mcls = 0;
    uint32_t Bw[NW];  // mask words and their prefix popcounts, set (and read) per size class
    int pre[NW];
    if (ALG >= ALG_LIST) {
        mini = __any_sync(FULL, ps.active && is_minified(jac, fW, fH));
        if (!mini) {
            minx = __reduce_min_sync(FULL, ps.active ? ps.ulx : INT_MAX);
            miny = __reduce_min_sync(FULL, ps.active ? ps.uly : INT_MAX);
            const int maxx = __reduce_max_sync(FULL, ps.active ? ps.ulx : INT_MIN) + 1;
            const int maxy = __reduce_max_sync(FULL, ps.active ? ps.uly : INT_MIN) + 1;
            bw = maxx - minx + 1;
            const int bh = maxy - miny + 1;
            if (ALG == ALG_BOX) {
                if (bw <= p.budget && bh <= p.budget && bw * bh <= p.budget) {
                    n = bw * bh;
                    fits = true;
                }
            } else if (ALG == ALG_MASK) {
                // The mask covers the M x M square of Sec. 3.3; its bits are
                // laid out with the bounding-box width bw as row stride, so
                // that the common small boxes need one or two words.  The set,
                // hence n and every output, is the same as with row stride M.
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
                const int tpl = kTwo ? p.tpl : 1;
                if (p.edge_remap) {
                    fits = n <= tpl * nactive;
                } else {
                    const uint32_t need = n >= 32 ? FULL : ((1u << n) - 1u);
                    fits = (A & need) == need;
                }
            }
        }
    }

    if (!fits) {
        // one-tap STF: every active lane evaluates its own stochastic texel
        if (ALG >= ALG_LIST) {
            sel.path = mini ? PATH_FALLBACK_MINIFIED : PATH_FALLBACK_BUDGET;
            if (kStats) cnt.v[kStatTilesFallbackMinified] += mini ? 1 : 0;
            if (kStats) cnt.v[kStatTilesFallbackBudget] += mini ? 0 : 1;
        } else {
            sel.path = PATH_DIRECT;
            if (kStats) cnt.v[kStatTilesDirect] += 1;
        }
        if (kStats) cnt.v[kStatTexelEvals] += nactive;
        if (kStats && kUnique) cnt.v[kStatTexelEvalsUnique] += nactive;
        if (ps.active) {
            int dx, dy;
            stf_offset(px, py + p.y0, p.view, p.k0, p.k1, ps.s, ps.t, dx, dy);
            sel.produce = true;
            sel.my_rank = __popc(A & lt);  // producers are the active lanes
            sel.tx = ps.ulx + dx;
            sel.ty = ps.uly + dy;
            sel.count = 1;
        }
    } else {
        sel.path = PATH_SUCCESS;
        sel.n = n;
        if (kStats) cnt.v[kStatTilesSuccess] += 1;
        if (kStats) cnt.v[kStatTexelEvals] += n;
        if (kStats && kUnique) cnt.v[kStatTexelEvalsUnique] += n;
        const bool full = A == FULL;
        // Evaluation counts follow the paper's assignment of texel i to lane
        // h(i, A) (edge remapping) or to lane i, whichever lane of the warp
        // does the arithmetic.
        const int my_i = (full || !p.edge_remap) ? lane : (((A >> lane) & 1u) ? __popc(A & lt) : 32);
        sel.count = my_i < n ? 1 : 0;
        const int dx0 = ps.ulx - minx, dy0 = ps.uly - miny;
        const int t00 = dy0 * bw + dx0, t01 = t00 + bw;  // box positions of taps (0,0) and (0,1)
        int j[4];  // lanes that hold taps k = (k%2, k/2)
        if (kTwo && p.tpl == 2) {
            // Up to two texels per lane (Sec. 5).  The counts follow the
            // paper's assignment extended round-robin: texel i by active
            // lane i mod na (edge remapping) or lane i mod 32, so lane a
            // counts [a < n] + [a + na < n].  The arithmetic: index i (a box
            // position, or a rank for the larger masks and List Merge) is
            // evaluated by lane i mod 32 in round i div 32, and each tap is
            // read from that lane and round.
            const int na = p.edge_remap ? nactive : 32;
            const int a = p.edge_remap ? (((A >> lane) & 1u) ? __popc(A & lt) : 64) : lane;
            sel.count = (uint8_t)((a < n ? 1 : 0) + (a + na < n ? 1 : 0));
            int pos0 = -1, pos1 = -1;  // box positions of this lane's texels (direct)
            if (ALG == ALG_BOX || (ALG == ALG_MASK && mcls <= 2)) {
                // a box of at most 64 texels: positions lane and lane + 32
                j[0] = t00;
                j[1] = t00 + 1;
                j[2] = t01;
                j[3] = t01 + 1;
                if (ALG == ALG_BOX) {
                    pos0 = lane < n ? lane : -1;
                    pos1 = lane + 32 < n ? lane + 32 : -1;
                } else {
                    pos0 = ((Bw[0] >> lane) & 1u) ? lane : -1;
                    pos1 = (mcls == 2 && ((Bw[1] >> lane) & 1u)) ? lane + 32 : -1;
                }
            } else if (ALG == ALG_MASK) {
                // ranks: the pixels file the box position of each tap's rank
                j[0] = mask_rank<NW>(Bw, pre, t00);
                j[2] = mask_rank<NW>(Bw, pre, t01);
                j[1] = j[0] + 1;
                j[3] = j[2] + 1;
                if (ps.active) {
                    ranks[ck(j[0], kRanksN, p.err, kBndRanks)] = t00;
                    ranks[ck(j[1], kRanksN, p.err, kBndRanks)] = t00 + 1;
                    ranks[ck(j[2], kRanksN, p.err, kBndRanks)] = t01;
                    ranks[ck(j[3], kRanksN, p.err, kBndRanks)] = t01 + 1;
                }
                __syncwarp();
                pos0 = lane < n ? ranks[ck(lane, kRanksN, p.err, kBndRanks)] : -1;
                pos1 = lane + 32 < n ? ranks[ck(lane + 32, kRanksN, p.err, kBndRanks)] : -1;
                __syncwarp();
            } else {  // List Merge: list indices of the taps, list order
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
                                j[k] = ck((int)T->index[h], 64, p.err, kBndListTable);
                                break;
                            }
                            if (kk == kEmpty) break;
                            h = (h + 1) & 255u;
                        }
                    }
                }
                if (lane < n) {
                    const unsigned long long key = T->list[ck(lane, 64, p.err, kBndListTable)];
                    sel.produce = true;
                    sel.tx = minx + (int)(uint32_t)key;
                    sel.ty = miny + (int)(uint32_t)(key >> 32);
                }
                if (lane + 32 < n) {
                    const unsigned long long key = T->list[ck(lane + 32, 64, p.err, kBndListTable)];
                    sel.produce2 = true;
                    sel.tx2 = minx + (int)(uint32_t)key;
                    sel.ty2 = miny + (int)(uint32_t)(key >> 32);
                }
            }
            if (ALG != ALG_LIST) {
                // box position -> texel (bw <= 16 for the masks: div_small
                // holds; a Box row may be wider)
                if (pos0 >= 0) {
                    const int q = ALG == ALG_BOX ? pos0 / bw : div_small(pos0, bw);
                    sel.produce = true;
                    sel.tx = minx + (pos0 - q * bw);
                    sel.ty = miny + q;
                }
                if (pos1 >= 0) {
                    const int q = ALG == ALG_BOX ? pos1 / bw : div_small(pos1, bw);
                    sel.produce2 = true;
                    sel.tx2 = minx + (pos1 - q * bw);
                    sel.ty2 = miny + q;
                }
            }
            // the dense ranks of the taps and of this lane's texels in the
            // tile's texel list (what the learned decode packs): the index
            // itself but for the small masks, whose indices are box positions
            if (ALG == ALG_MASK && mcls <= 2) {
                const unsigned long long B = ((unsigned long long)(mcls == 2 ? Bw[1] : 0u) << 32) | Bw[0];
#pragma unroll
                for (int k = 0; k < 4; ++k) sel.rk[k] = __popcll(B & ((1ull << (j[k] & 63)) - 1ull));
                sel.my_rank = __popcll(B & ((1ull << lane) - 1ull));
                sel.my_rank2 = __popcll(B & ((1ull << (lane + 32)) - 1ull));
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) sel.rk[k] = j[k];
                sel.my_rank = lane;
                sel.my_rank2 = lane + 32;
            }
            // lane + 32 x round; inactive pixels carry arbitrary indices, whose
            // shuffled values they drop
#pragma unroll
            for (int k = 0; k < 4; ++k) sel.src[k] = ps.active ? ck(j[k], 64, p.err, kBndLane) : j[k];
            if (ALG == ALG_LIST) {
                __syncwarp();
#pragma unroll
                for (int s = 0; s < 8; ++s) T->keys[lane * 8 + s] = kEmpty;
                __syncwarp();
            }
            return sel;
        }
        if (ALG == ALG_BOX || (ALG == ALG_MASK && mcls == 1)) {
            // A box of at most 32 texels: lane L evaluates box position L
            // when it is in the set, so each tap is read from the lane of its
            // box position and no compaction is needed.  The texels, hence
            // every output, are those of the paper's lane assignment.
            j[0] = t00;
            j[1] = t00 + 1;
            j[2] = t01;
            j[3] = t01 + 1;
            const bool in_set = ALG == ALG_BOX ? lane < n : ((Bw[0] >> lane) & 1u) != 0;
            // the texel list in rank order (what the learned decode packs)
            if (ALG == ALG_BOX) {
#pragma unroll
                for (int k = 0; k < 4; ++k) sel.rk[k] = j[k];
                sel.my_rank = lane;
            } else {
                sel.rk[0] = __popc(Bw[0] & ((1u << t00) - 1u));
                sel.rk[1] = sel.rk[0] + 1;
                sel.rk[2] = __popc(Bw[0] & ((1u << t01) - 1u));
                sel.rk[3] = sel.rk[2] + 1;
                sel.my_rank = __popc(Bw[0] & lt);
            }
            if (in_set) {
                const int q = div_small(lane, bw);
                sel.produce = true;
                sel.tx = minx + (lane - q * bw);
                sel.ty = miny + q;
            }
        } else {
            // Larger masks and List Merge: texel i is evaluated by lane
            // h(i, A); each tap is read from the lane of its rank.
            if (ALG == ALG_MASK) {
                if (mcls == 2) {
                    const unsigned long long B = ((unsigned long long)Bw[1] << 32) | Bw[0];
                    j[0] = __popcll(B & ((1ull << t00) - 1ull));
                    j[2] = __popcll(B & ((1ull << t01) - 1ull));
                } else {
                    j[0] = mask_rank<NW>(Bw, pre, t00);
                    j[2] = mask_rank<NW>(Bw, pre, t01);
                }
                j[1] = j[0] + 1;
                j[3] = j[2] + 1;
                // The texel of rank i (the i-th set bit, h(i, B)) reaches its
                // producer through the warp's rank slots, so no bit search is
                // needed.  Up to 64 bits, lane L stands for bit positions L
                // and L + 32, and the rank of a set bit is a masked popcount;
                // larger masks are filled by the pixels, each at the ranks of
                // its taps.
                if (mcls == 2) {
                    if ((Bw[0] >> lane) & 1u) ranks[ck(__popc(Bw[0] & lt), kRanksN, p.err, kBndRanks)] = lane;
                    if ((Bw[1] >> lane) & 1u)
                        ranks[ck(pre[1] + __popc(Bw[1] & lt), kRanksN, p.err, kBndRanks)] = lane + 32;
                } else if (ps.active) {
                    ranks[ck(j[0], kRanksN, p.err, kBndRanks)] = t00;
                    ranks[ck(j[1], kRanksN, p.err, kBndRanks)] = t00 + 1;
                    ranks[ck(j[2], kRanksN, p.err, kBndRanks)] = t01;
                    ranks[ck(j[3], kRanksN, p.err, kBndRanks)] = t01 + 1;
                }
                __syncwarp();
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
                                j[k] = ck((int)T->index[h], 64, p.err, kBndListTable);
                                break;
                            }
                            if (kk == kEmpty) break;
                            h = (h + 1) & 255u;
                        }
                    }
                }
            }
            if (my_i < n) {
                int x, y;
                if (ALG == ALG_MASK) {
                    const int t = ranks[ck(my_i, kRanksN, p.err, kBndRanks)];  // bit position dy * bw + dx
                    const int q = div_small(t, bw);
                    x = minx + (t - q * bw);
                    y = miny + q;
                } else {
                    const unsigned long long key = T->list[ck(my_i, 64, p.err, kBndListTable)];
                    x = minx + (int)(uint32_t)key;
                    y = miny + (int)(uint32_t)(key >> 32);
                }
                sel.produce = true;
                sel.tx = x;
                sel.ty = y;
            }
            if (ALG == ALG_MASK) __syncwarp();  // rank slots free for the next tile
#pragma unroll
            for (int k = 0; k < 4; ++k) sel.rk[k] = j[k];
            sel.my_rank = my_i;
            if (!full && p.edge_remap) {
#pragma unroll
                for (int k = 0; k < 4; ++k) j[k] = nth_set_lane(A, j[k]);
            }
        }
        // (inactive pixels carry arbitrary lanes, whose shuffled values they drop)
#pragma unroll
        for (int k = 0; k < 4; ++k) sel.src[k] = ps.active ? ck(j[k], 32, p.err, kBndLane) : j[k];
    }
    if (ALG == ALG_LIST) {
        __syncwarp();
#pragma unroll
        for (int s = 0; s < 8; ++s) T->keys[lane * 8 + s] = kEmpty;
        __syncwarp();
    }
    return sel;
}

}  // namespace ctf
