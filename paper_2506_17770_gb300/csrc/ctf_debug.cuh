// ctf_debug.cuh -- index checks of the debug build.
//
// Built with -DCTF_DEBUG (libctf_debug.so), every data-dependent index the
// kernels use to reach a texel, a pixel or an entry of a shared-memory table
// goes through ck(i, n, err, site): an index outside [0, n) is recorded in
// the device error word (status CTF_ERR_BOUNDS; the first record wins and
// keeps the site, the index and the bound in the three words after the
// status) and replaced by 0, so the access stays inside its buffer and the
// kernel runs on to its end.  ctf_sync_check then reports the record.  In
// the release build ck() is the index itself and no code is added.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ctf.h"

namespace ctf {

// Where a checked index is used (the site word of a CTF_ERR_BOUNDS record).
enum BoundsSite {
    kBndPixel = 1,     // pixel inputs and outputs of a view (n = W x H)
    kBndBlock,         // 8-byte block of a block texture (n = Wt/4 x Ht/4)
    kBndDecodeTable,   // the block decode tables in shared memory
    kBndRanks,         // a warp's rank slots (Mask Sampling)
    kBndListTable,     // a warp's List Merge table and texel list
    kBndFbTable,       // a warp's fallback C / C+ texel table
    kBndLatent,        // a cell of a latent grid (n = gw x gh)
    kBndTexList,       // a group's texel lists (8 tiles x 32 entries)
    kBndRow,           // a chain row of the learned filters (operand and value rows)
    kBndPixSlot,       // a group's per-pixel words (8 tiles x 32 pixels)
    kBndLane,          // a source lane of a shuffle (n = 32)
    kBndBatch,         // a view or tile of a batch plan
    kBndTrain,         // a texel, cell or partial sum of the trainer
    kBndSelfTest,      // ctf_debug_selftest_bounds
    kBndNumSites
};

#ifdef CTF_DEBUG
constexpr bool kDebugBuild = true;

__device__ __forceinline__ void bounds_fail(int *err, int site, long long i, long long n) {
    if (err && atomicCAS(err, 0, (int)CTF_ERR_BOUNDS) == 0) {
        err[1] = site;
        err[2] = (int)(i < INT32_MIN ? INT32_MIN : (i > INT32_MAX ? INT32_MAX : i));
        err[3] = (int)(n > INT32_MAX ? INT32_MAX : n);
        __threadfence();
    }
}

template <typename I>
__device__ __forceinline__ I ck(I i, long long n, int *err, int site) {
    if ((long long)i >= 0 && (long long)i < n) return i;
    bounds_fail(err, site, (long long)i, n);
    return I(0);
}
#else
constexpr bool kDebugBuild = false;

template <typename I>
__device__ __forceinline__ I ck(I i, long long, int *, int) {
    return i;
}
#endif

}  // namespace ctf
