// ctf_train.cu -- training of the learned texel decode on the GPU.
//
// The network of ctf_mlp.cu (two 8-channel latent grids sampled bilinearly,
// 16 -> 64 -> 64 -> 4 with ReLU) is fitted to the exact decode of a block
// texture.  FP32 master parameters live in one device buffer:
//   [w1 1024 | b1 64 | w2 4096 | b2 64 | w3 256 | b3 4 | pad 4 | latent0 | latent1]
// A step samples a batch of texels with Philox4x32-10.  A CTA of 128
// threads takes up to 128 texels per round and runs the forward and
// backward pass as tcgen05 MMAs over them (FP16 operands in shared memory,
// FP32 accumulation in TMEM; bias, ReLU and the loss in FP32): the layer
// products, the input-side gradients and the weight gradients, which it
// sums over its rounds in TMEM.  It adds those sums, like the latent-grid
// gradient scatter, to 64-bit fixed-point accumulators (integer atomics are
// order-independent, so a step is deterministic).  An Adam kernel converts
// the sums back, updates parameters and moments, and clears the
// accumulators.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/ctf.h"
#include "ctf_device.cuh"
#include "ctf_internal.h"

namespace ctf {
namespace {

constexpr int kOffW1 = 0, kOffB1 = 1024, kOffW2 = 1088, kOffB2 = 5184, kOffW3 = 5248, kOffB3 = 5504;
constexpr int kWeights = 5508;
constexpr int kOffLat = 5512;
constexpr double kFix = 17592186044416.0;  // 2^44: gradient fixed point
constexpr double kLossFix = 4294967296.0;  // 2^32: loss fixed point
constexpr int kThreads = 128;              // threads of the activation-statistics kernel
constexpr int kT = 128;                    // rows of a round of the gradient kernel (one per thread)
constexpr int kMaxRounds = 4;              // rounds per CTA, at most (unless the batch needs more)
constexpr int kMaxGradCtas = 1024;         // CTAs of the gradient kernel, at most (their partial sums)

struct GradParams {
    const float *params;
    const uint2 *blocks;
    int Wt, Ht, nbx;
    int gw[2], gh[2];
    float sx[2], sy[2];
    const int2 *xy;        // explicit texels, or nullptr: Philox sampling
    int n;                 // texels in this call
    int rounds;            // rounds per CTA
    int per_round;         // texels per round (at most kT; the other rows of the round are empty)
    uint32_t step;         // Philox counter word
    uint32_t k0, k1;       // Philox key
    float dscale;          // 2 / batch
    long long *grad;       // fixed-point gradient accumulators (same layout as params)
    uint32_t *touched;     // one bit per latent cell (grid 0 cells, then grid 1) whose gradient a texel reached
    long long *loss;       // fixed-point sum of squared errors
    int *err;              // device error word: a wait that gave up records CTF_ERR_TIMEOUT
    unsigned char *wimg;   // the weight image of the gradient kernel (pack_kernel)
    float *partial;        // per-CTA weight-gradient sums [CTA][kWeights] (reduce_kernel adds them up)
};

// v * 2^44 is exact in FP32 (a power-of-two scale), so this rounds the same
// value as the FP64 product would, without FP64 arithmetic.
__device__ __forceinline__ long long to_fix(float v) { return __float2ll_rn(v * 0x1p44f); }

// Shared memory of the gradient kernel (bytes).  Every matrix is an MMA
// operand in FP16, stored K-major in 8-row x 16-byte core matrices (element
// (r, k) at (r/8) * (K/8) * 128 + (k/8) * 128 + (r%8) * 16 + (k%8) * 2):
//   weights as the B operands of the forward and backward products:
//   W1 [64 x 16], W2 [64 x 64], W3 [16 x 64] (rows 4..15 zero), W3^T
//   [64 x 16] (columns 4..15 zero), W2^T [64 x 64], W1^T [16 x 64];
//   AH, one row per texel of the round, 176 channels: H2 (0..63), a ones
//   block (64..79: channel 64 is 1, the rest 0), H1 (80..143), the
//   features F (144..159) and a second ones block (160..175);
//   DH, one row per texel, 128 channels: dH2 (0..63), dH1 (64..127);
//   DE, one row per texel, 16 channels: the output errors (0..3), zeros.
// The weight gradients are products over the round's texels with the
// texel as the reduction index: the same AH and DH buffers, read
// MN-major (channels along MN, texels along K), give
//   [dH2; dH1]^T [H1 | F | 1] -> dW2, dW1 and the bias sums db2, db1 (one
//   MMA chain, M = 128 channels, N = 96), and
//   [H2 | 1 | ...]^T DE -> dW3^T and db3 (M = 128, N = 16),
// accumulated in TMEM over the CTA's rounds.
constexpr int kGW1 = 0;
constexpr int kGW2 = kGW1 + 2048;
constexpr int kGW3 = kGW2 + 8192;
constexpr int kGW3T = kGW3 + 2048;
constexpr int kGW2T = kGW3T + 2048;
constexpr int kGW1T = kGW2T + 8192;
constexpr int kGBias = kGW1T + 2048;              // b1[64], b2[64], b3[4] (FP32)
constexpr int kAHK = 176, kAHGroup = kAHK / 8 * 128;  // channels, bytes per 8-row group
constexpr int kChH2 = 0, kChOnes = 64, kChH1 = 80, kChF = 144, kChOnes2 = 160;
constexpr int kGAH = kGBias + 640;
constexpr int kDHGroup = 128 / 8 * 128;
constexpr int kGDH = kGAH + 16 * kAHGroup;
constexpr int kGDE = kGDH + 16 * kDHGroup;
constexpr int kGXY = kGDE + 16 * 256;             // int2 [128] texel coordinates
constexpr int kGBar = kGXY + 128 * 8;             // MMA barrier (8 B), TMEM base (4 B)
constexpr int kGSlot = kGBar + 8;
constexpr int kGLoss = kGBar + 16;                // float [128] per-thread squared errors
constexpr int kGradSmemBytes = kGLoss + 128 * 4;
static_assert(kGAH % 16 == 0 && kGDH % 16 == 0 && kGDE % 16 == 0, "16-byte operand buffers");
static_assert(2 * (kGradSmemBytes + 1024) <= 228 * 1024 && 3 * (kGradSmemBytes + 1024) > 228 * 1024,
              "exactly two CTAs (2 x 256 TMEM columns) per SM");
constexpr size_t kGradSmem = kGradSmemBytes;
// TMEM columns (FP32, lane = row): forward D1 / backward dE W3^T [0, 64),
// D2 / dH2 W2^T [64, 128), D3 / dH1 W1^T [128, 144), the weight-gradient
// sums [144, 240) and [240, 256).
constexpr uint32_t kTcCols = 256, kColA = 0, kColB = 64, kColC = 128, kColWG1 = 144, kColWG2 = 240;
constexpr uint32_t kGradTries = 1u << 24;

__host__ __device__ constexpr uint32_t idesc_f16_t(int M, int N, int ta, int tb) {
    return (1u << 4) | ((uint32_t)ta << 15) | ((uint32_t)tb << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t h2pack(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ uint32_t relu_h2(float a, float b) {
    uint32_t r;
    asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    return r;
}

// Offset of element (r, k) in a K-major FP16 operand with K channels.
__device__ __forceinline__ int kofs(int r, int k, int K) { return (r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

// One MMA (FP16 operands, FP32 accumulation), issued by one thread.
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, bool acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)acc)
        : "memory");
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ uint32_t saddr_of(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// The MMAs issued since the last commit: thread 0 commits them to the
// barrier and polls it; every thread learns the outcome at a CTA barrier.
// Returns false (for all threads alike) if they did not complete within
// the bound.
__device__ __forceinline__ bool tc_sync(uint64_t *bar, uint32_t &phase) {
    bool ok = true;
    if (threadIdx.x == 0) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr_of(bar))
                     : "memory");
        ok = false;
        const uint32_t a = saddr_of(bar);
        for (uint32_t i = 0; i < kGradTries && !ok; ++i) {
            uint32_t done;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(a), "r"(phase)
                : "memory");
            ok = done != 0;
        }
    }
    phase ^= 1u;
    __syncwarp();
    const bool bad = __syncthreads_or(!ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return !bad;
}

// Generic-proxy shared-memory writes of every thread made visible to the
// MMAs that thread 0 issues next.
__device__ __forceinline__ void tc_publish() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    // the loaded registers pass through an empty asm after the wait, so that
    // no use of them can be scheduled before it
#pragma unroll
    for (int i = 0; i < 16; ++i) asm volatile("" : "+r"(r[i]));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void bilinear_taps(const GradParams &g, int grid, int x, int y, int idx[4], float w[4]) {
    // grid is 0 or 1; selecting by value keeps the parameter block out of local memory
    const float sx = grid ? g.sx[1] : g.sx[0], sy = grid ? g.sy[1] : g.sy[0];
    const int gw = grid ? g.gw[1] : g.gw[0], gh = grid ? g.gh[1] : g.gh[0];
    const float gx = __fsub_rn(__fmul_rn(__fadd_rn((float)x, 0.5f), sx), 0.5f);
    const float gy = __fsub_rn(__fmul_rn(__fadd_rn((float)y, 0.5f), sy), 0.5f);
    const float fx0 = floorf(gx), fy0 = floorf(gy);
    const float fx = __fsub_rn(gx, fx0), fy = __fsub_rn(gy, fy0);
    const int x0 = (int)fx0, y0 = (int)fy0;
    const int xa = min(max(x0, 0), gw - 1), xb = min(max(x0 + 1, 0), gw - 1);
    const int ya = min(max(y0, 0), gh - 1), yb = min(max(y0 + 1, 0), gh - 1);
    const long long cells = (long long)gw * gh;
    idx[0] = ck(ya * gw + xa, cells, g.err, kBndLatent);
    idx[1] = ck(ya * gw + xb, cells, g.err, kBndLatent);
    idx[2] = ck(yb * gw + xa, cells, g.err, kBndLatent);
    idx[3] = ck(yb * gw + xb, cells, g.err, kBndLatent);
    const float ofx = __fsub_rn(1.f, fx), ofy = __fsub_rn(1.f, fy);
    w[0] = __fmul_rn(ofx, ofy);
    w[1] = __fmul_rn(fx, ofy);
    w[2] = __fmul_rn(ofx, fy);
    w[3] = __fmul_rn(fx, fy);
}


// The gradient kernel's weight image (the first kGAH bytes of its shared
// memory): W1, W2, W3 (padded) and their transposes as FP16 operands, the
// biases in FP32, from the current FP32 master parameters.  One thread per
// parameter of the network.
__global__ void pack_kernel(const float *params, unsigned char *img) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 1024) {
        const int o = i >> 4, k = i & 15;
        const __half w = __float2half_rn(params[kOffW1 + i]);
        *reinterpret_cast<__half *>(img + kGW1 + kofs(o, k, 16)) = w;
        *reinterpret_cast<__half *>(img + kGW1T + kofs(k, o, 64)) = w;
    } else if (i < 1024 + 4096) {
        const int j = i - 1024, o = j >> 6, k = j & 63;
        const __half w = __float2half_rn(params[kOffW2 + j]);
        *reinterpret_cast<__half *>(img + kGW2 + kofs(o, k, 64)) = w;
        *reinterpret_cast<__half *>(img + kGW2T + kofs(k, o, 64)) = w;
    } else if (i < 1024 + 4096 + 1024) {
        const int j = i - 5120, c = j >> 6, k = j & 63;
        const __half w = __float2half_rn(c < 4 ? params[kOffW3 + j] : 0.f);
        *reinterpret_cast<__half *>(img + kGW3 + kofs(c, k, 64)) = w;   // rows 4..15 zero
        *reinterpret_cast<__half *>(img + kGW3T + kofs(k, c, 16)) = w;  // columns 4..15 zero
    } else if (i < 6144 + 160) {
        const int j = i - 6144;  // biases b1 (64), b2 (64), b3 (4), zero padding
        float v = 0.f;
        if (j < 64) v = params[kOffB1 + j];
        else if (j < 128) v = params[kOffB2 + j - 64];
        else if (j < 132) v = params[kOffB3 + j - 128];
        reinterpret_cast<float *>(img + kGBias)[j] = v;
    }
}
constexpr int kPackThreads = 6144 + 160;
static_assert(kGBias + 160 * 4 == kGAH, "the image ends where the activations begin");

// Forward and backward pass of kT texels per round on the tensor cores:
// thread t owns texel row t of every per-texel operand and TMEM lane t.
// Per round: features (FP32, from the FP32 master latents) and targets;
// H1 = relu(F W1^T + b1), H2 = relu(H1 W2^T + b2), Y = H2 W3^T + b3 (FP16
// operands, FP32 accumulation, bias and ReLU in FP32); e = Y - target;
// dH2 = (e W3) masked by H2 > 0, dH1 = (dH2 W2) masked by H1 > 0,
// dF = dH1 W1; the weight gradients accumulate in TMEM; dF, times the
// bilinear tap weights and 2 / batch, goes to the latent cells.  The CTA's
// weight-gradient sums (times 2 / batch) and its squared errors go to the
// 64-bit fixed-point accumulators at the end.  Rows past the batch carry
// e = 0 and so contribute nothing.
__global__ void __launch_bounds__(kT, 2) grad_kernel(const GradParams g) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kGBar);
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + kGSlot);
    float *sloss = reinterpret_cast<float *>(sm + kGLoss);
    unsigned char *AH = sm + kGAH, *DH = sm + kGDH, *DE = sm + kGDE;
    const float *P = g.params;  // latents (FP32 master values)
    // ---- the weights as FP16 operands and the biases (the image that
    // pack_kernel made from the current parameters), the constant ones blocks
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(g.wimg);
        uint4 *dst = reinterpret_cast<uint4 *>(sm);
        for (int i = tid; i < kGAH / 16; i += kT) dst[i] = __ldg(src + i);
    }
    const float *B = reinterpret_cast<const float *>(sm + kGBias);
    {
        // the ones blocks of every row: channels 64 and 160 are 1, the rest of
        // their 16-channel blocks 0 (never written again)
        const uint4 one = make_uint4(0x3C00u, 0u, 0u, 0u), zero = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(AH + kofs(tid, kChOnes, kAHK)) = one;
        *reinterpret_cast<uint4 *>(AH + kofs(tid, kChOnes + 8, kAHK)) = zero;
        *reinterpret_cast<uint4 *>(AH + kofs(tid, kChOnes2, kAHK)) = one;
        *reinterpret_cast<uint4 *>(AH + kofs(tid, kChOnes2 + 8, kAHK)) = zero;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr_of(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr_of(slot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot;
    const uint32_t lane_t = tmem + ((uint32_t)(32 * (tid >> 5)) << 16);  // this thread's TMEM lane
    uint32_t phase = 0;
    bool ok = true;
    const size_t lat1 = (size_t)g.gw[0] * g.gh[0] * 8;  // start of the second grid
    const uint32_t sAH = saddr_of(AH), sDH = saddr_of(DH), sDE = saddr_of(DE);
    const uint32_t id64 = idesc_f16_t(128, 64, 0, 0), id16 = idesc_f16_t(128, 16, 0, 0);
    const uint32_t idW1 = idesc_f16_t(128, 96, 1, 1), idW2 = idesc_f16_t(128, 16, 1, 1);
    float loss = 0.f;

#pragma unroll 1
    for (int r = 0; r < g.rounds && ok; ++r) {
        const int i0 = (blockIdx.x * g.rounds + r) * g.per_round;
        const int i = i0 + tid;
        const bool valid = tid < g.per_round && i < g.n;
        // ---- the texel of row tid, its features and its target
        int x, y;
        if (g.xy) {
            const int2 c = valid ? g.xy[ck(i, g.n, g.err, kBndTrain)] : make_int2(0, 0);
            x = min(max(c.x, 0), g.Wt - 1);
            y = min(max(c.y, 0), g.Ht - 1);
        } else {
            const uint4 rr = philox4x32_10(make_uint4((uint32_t)i, g.step, 0x5A4Du, 0u), g.k0, g.k1);
            x = (int)(((unsigned long long)rr.x * (unsigned)g.Wt) >> 32);
            y = (int)(((unsigned long long)rr.y * (unsigned)g.Ht) >> 32);
        }
        {
            float f[16];
#pragma unroll
            for (int gi = 0; gi < 2; ++gi) {
                int tap[4];
                float tw[4];
                bilinear_taps(g, gi, x, y, tap, tw);
                const float *lg = P + kOffLat + (gi ? lat1 : 0);
                float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float4 v0 = __ldg(reinterpret_cast<const float4 *>(lg + (size_t)tap[k] * 8));
                    const float4 v1 = __ldg(reinterpret_cast<const float4 *>(lg + (size_t)tap[k] * 8 + 4));
                    acc[0] = __fmaf_rn(tw[k], v0.x, acc[0]);
                    acc[1] = __fmaf_rn(tw[k], v0.y, acc[1]);
                    acc[2] = __fmaf_rn(tw[k], v0.z, acc[2]);
                    acc[3] = __fmaf_rn(tw[k], v0.w, acc[3]);
                    acc[4] = __fmaf_rn(tw[k], v1.x, acc[4]);
                    acc[5] = __fmaf_rn(tw[k], v1.y, acc[5]);
                    acc[6] = __fmaf_rn(tw[k], v1.z, acc[6]);
                    acc[7] = __fmaf_rn(tw[k], v1.w, acc[7]);
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) f[gi * 8 + c] = acc[c];
            }
            *reinterpret_cast<uint4 *>(AH + kofs(tid, kChF, kAHK)) =
                make_uint4(h2pack(f[0], f[1]), h2pack(f[2], f[3]), h2pack(f[4], f[5]), h2pack(f[6], f[7]));
            *reinterpret_cast<uint4 *>(AH + kofs(tid, kChF + 8, kAHK)) =
                make_uint4(h2pack(f[8], f[9]), h2pack(f[10], f[11]), h2pack(f[12], f[13]), h2pack(f[14], f[15]));
        }
        float tgt[4];
        {
            const uint32_t px = fetch_block_texel(g.blocks, g.nbx, g.Wt, g.Ht, x, y, g.err);
#pragma unroll
            for (int c = 0; c < 4; ++c) tgt[c] = __fdiv_rn((float)((px >> (8 * c)) & 0xffu), 255.f);
        }
        tc_publish();
        // ---- H1 = relu(F W1^T + b1)
        if (tid == 0)
            tc_mma(tmem + kColA, sdesc(sAH + kChF / 8 * 128, 128, kAHGroup), sdesc(saddr_of(sm + kGW1), 128, 256), id64,
                   false);
        if (!(ok = tc_sync(bar, phase))) break;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float d[16];
            tld16(lane_t + kColA + 16 * q, d);
            uint32_t w[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                w[j] = relu_h2(__fadd_rn(d[2 * j], B[16 * q + 2 * j]), __fadd_rn(d[2 * j + 1], B[16 * q + 2 * j + 1]));
            *reinterpret_cast<uint4 *>(AH + kofs(tid, kChH1 + 16 * q, kAHK)) = make_uint4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<uint4 *>(AH + kofs(tid, kChH1 + 16 * q + 8, kAHK)) = make_uint4(w[4], w[5], w[6], w[7]);
        }
        tc_publish();
        // ---- H2 = relu(H1 W2^T + b2)
        if (tid == 0)
            for (int j = 0; j < 4; ++j)
                tc_mma(tmem + kColB, sdesc(sAH + kChH1 / 8 * 128 + 256 * j, 128, kAHGroup),
                       sdesc(saddr_of(sm + kGW2) + 256 * j, 128, 1024), id64, j > 0);
        if (!(ok = tc_sync(bar, phase))) break;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float d[16];
            tld16(lane_t + kColB + 16 * q, d);
            uint32_t w[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                w[j] = relu_h2(__fadd_rn(d[2 * j], B[64 + 16 * q + 2 * j]),
                               __fadd_rn(d[2 * j + 1], B[64 + 16 * q + 2 * j + 1]));
            *reinterpret_cast<uint4 *>(AH + kofs(tid, kChH2 + 16 * q, kAHK)) = make_uint4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<uint4 *>(AH + kofs(tid, kChH2 + 16 * q + 8, kAHK)) = make_uint4(w[4], w[5], w[6], w[7]);
        }
        tc_publish();
        // ---- Y = H2 W3^T + b3, e = Y - target (0 past the batch)
        if (tid == 0)
            for (int j = 0; j < 4; ++j)
                tc_mma(tmem + kColC, sdesc(sAH + kChH2 / 8 * 128 + 256 * j, 128, kAHGroup),
                       sdesc(saddr_of(sm + kGW3) + 256 * j, 128, 1024), id16, j > 0);
        if (!(ok = tc_sync(bar, phase))) break;
        {
            float d[16];
            tld16(lane_t + kColC, d);
            float e[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                e[c] = valid ? __fsub_rn(__fadd_rn(d[c], B[128 + c]), tgt[c]) : 0.f;
                loss = __fmaf_rn(e[c], e[c], loss);
            }
            *reinterpret_cast<uint4 *>(DE + kofs(tid, 0, 16)) = make_uint4(h2pack(e[0], e[1]), h2pack(e[2], e[3]), 0u, 0u);
            *reinterpret_cast<uint4 *>(DE + kofs(tid, 8, 16)) = make_uint4(0u, 0u, 0u, 0u);
        }
        tc_publish();
        // ---- dH2 = (e W3) masked by H2 > 0
        if (tid == 0)
            tc_mma(tmem + kColA, sdesc(sDE, 128, 256), sdesc(saddr_of(sm + kGW3T), 128, 256), id64, false);
        if (!(ok = tc_sync(bar, phase))) break;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float d[16];
            tld16(lane_t + kColA + 16 * q, d);
            const uint4 h0 = *reinterpret_cast<const uint4 *>(AH + kofs(tid, kChH2 + 16 * q, kAHK));
            const uint4 h1 = *reinterpret_cast<const uint4 *>(AH + kofs(tid, kChH2 + 16 * q + 8, kAHK));
            const __half *hh0 = reinterpret_cast<const __half *>(&h0), *hh1 = reinterpret_cast<const __half *>(&h1);
            uint32_t w[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const __half a = j < 4 ? hh0[2 * j] : hh1[2 * j - 8], b = j < 4 ? hh0[2 * j + 1] : hh1[2 * j - 7];
                w[j] = h2pack(__half2float(a) > 0.f ? d[2 * j] : 0.f, __half2float(b) > 0.f ? d[2 * j + 1] : 0.f);
            }
            *reinterpret_cast<uint4 *>(DH + kofs(tid, 16 * q, 128)) = make_uint4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<uint4 *>(DH + kofs(tid, 16 * q + 8, 128)) = make_uint4(w[4], w[5], w[6], w[7]);
        }
        tc_publish();
        // ---- dH1 = (dH2 W2) masked by H1 > 0
        if (tid == 0)
            for (int j = 0; j < 4; ++j)
                tc_mma(tmem + kColB, sdesc(sDH + 256 * j, 128, kDHGroup), sdesc(saddr_of(sm + kGW2T) + 256 * j, 128, 1024),
                       id64, j > 0);
        if (!(ok = tc_sync(bar, phase))) break;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float d[16];
            tld16(lane_t + kColB + 16 * q, d);
            const uint4 h0 = *reinterpret_cast<const uint4 *>(AH + kofs(tid, kChH1 + 16 * q, kAHK));
            const uint4 h1 = *reinterpret_cast<const uint4 *>(AH + kofs(tid, kChH1 + 16 * q + 8, kAHK));
            const __half *hh0 = reinterpret_cast<const __half *>(&h0), *hh1 = reinterpret_cast<const __half *>(&h1);
            uint32_t w[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const __half a = j < 4 ? hh0[2 * j] : hh1[2 * j - 8], b = j < 4 ? hh0[2 * j + 1] : hh1[2 * j - 7];
                w[j] = h2pack(__half2float(a) > 0.f ? d[2 * j] : 0.f, __half2float(b) > 0.f ? d[2 * j + 1] : 0.f);
            }
            *reinterpret_cast<uint4 *>(DH + kofs(tid, 64 + 16 * q, 128)) = make_uint4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<uint4 *>(DH + kofs(tid, 64 + 16 * q + 8, 128)) = make_uint4(w[4], w[5], w[6], w[7]);
        }
        tc_publish();
        // ---- dF = dH1 W1; the weight gradients of the round (texels as the
        // reduction index, both operands read MN-major)
        if (tid == 0) {
            for (int j = 0; j < 4; ++j)
                tc_mma(tmem + kColC, sdesc(sDH + 64 / 8 * 128 + 256 * j, 128, kDHGroup),
                       sdesc(saddr_of(sm + kGW1T) + 256 * j, 128, 1024), id16, j > 0);
            for (int s = 0; s < kT / 16; ++s) {
                const bool acc = r > 0 || s > 0;
                // [dH2 dH1]^T [H1 F 1]: A = DH (channels along MN), B = AH channels 80..175
                tc_mma(tmem + kColWG1, sdesc(sDH + 2 * kDHGroup * s, kDHGroup, 128),
                       sdesc(sAH + kChH1 / 8 * 128 + 2 * kAHGroup * s, kAHGroup, 128), idW1, acc);
                // [H2 1 H1]^T e: A = AH channels 0..127, B = DE
                tc_mma(tmem + kColWG2, sdesc(sAH + 2 * kAHGroup * s, kAHGroup, 128), sdesc(sDE + 512 * s, 256, 128),
                       idW2, acc);
            }
        }
        if (!(ok = tc_sync(bar, phase))) break;
        // ---- the latent-grid gradient of texel row tid
        float df[16];
        tld16(lane_t + kColC, df);  // warp-collective: every lane takes it
        if (valid) {
#pragma unroll
            for (int gi = 0; gi < 2; ++gi) {
                int tap[4];
                float tw[4];
                bilinear_taps(g, gi, x, y, tap, tw);
                unsigned long long *gl = reinterpret_cast<unsigned long long *>(g.grad + kOffLat + (gi ? lat1 : 0));
                const uint32_t cell0 = gi ? (uint32_t)(lat1 / 8) : 0u;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t cell = cell0 + (uint32_t)tap[k];
                    atomicOr(g.touched + (cell >> 5), 1u << (cell & 31u));
                    const float wk = __fmul_rn(tw[k], g.dscale);
#pragma unroll
                    for (int ch = 0; ch < 8; ++ch) {
                        const long long v = to_fix(__fmul_rn(wk, df[gi * 8 + ch]));
                        if (v) atomicAdd(gl + (size_t)tap[k] * 8 + ch, (unsigned long long)v);
                    }
                }
            }
        }
    }
    // ---- the CTA's weight-gradient sums, row m = tid of the two products,
    // stored as this CTA's partial sums (reduce_kernel adds the CTAs' up in
    // CTA order: no atomics on the few thousand weight entries)
    if (ok) {
        float *W = g.partial + (size_t)ck((int)blockIdx.x, kMaxGradCtas, g.err, kBndTrain) * kWeights;
        const int m = tid;
#pragma unroll 1
        for (int q = 0; q < 6; ++q) {
            float d[16];
            tld16(lane_t + kColWG1 + 16 * q, d);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int n = 16 * q + j;
                if (m < 64 && n < 64) W[kOffW2 + m * 64 + n] = d[j];                          // dW2
                else if (m >= 64 && n >= 64 && n < 80) W[kOffW1 + (m - 64) * 16 + (n - 64)] = d[j];  // dW1
                else if (n == 80) W[m < 64 ? kOffB2 + m : kOffB1 + (m - 64)] = d[j];           // db2, db1
            }
        }
        {
            float d[16];
            tld16(lane_t + kColWG2, d);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (m < 64) W[kOffW3 + c * 64 + m] = d[c];
                else if (m == 64) W[kOffB3 + c] = d[c];
            }
        }
        sloss[tid] = loss;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (ok && tid == 0) {
        float tot = 0.f;
        for (int s = 0; s < kT; ++s) tot = __fadd_rn(tot, sloss[s]);
        atomicAdd(reinterpret_cast<unsigned long long *>(g.loss), (unsigned long long)__double2ll_rn((double)tot * kLossFix));
    }
    if (!ok && tid == 0 && g.err) atomicExch(g.err, CTF_ERR_TIMEOUT);
    if (tid < 32) {
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
    }
}

// The weight gradients: the CTAs' partial sums added up in CTA order (FP64),
// times 2 / batch, into the fixed-point accumulators.  A block takes 16
// entries; its 16 thread rows each add every 16th CTA in order (loads
// issued 8 at a time), and the 16 row sums are added in row order, so the
// result does not depend on timing.
constexpr int kRedEntries = 16, kRedRows = 16;
__global__ void __launch_bounds__(kRedEntries * kRedRows) reduce_kernel(const float *partial, int ctas, double dscale,
                                                                       long long *grad) {
    __shared__ double part[kRedRows][kRedEntries];
    const int e = blockIdx.x * kRedEntries + (threadIdx.x % kRedEntries), row = threadIdx.x / kRedEntries;
    double acc = 0.0;
    if (e < kWeights) {
        for (int c0 = row; c0 < ctas; c0 += 8 * kRedRows) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = c0 + j * kRedRows;
                v[j] = c < ctas ? __ldg(partial + (size_t)c * kWeights + e) : 0.f;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) acc += (double)v[j];
        }
    }
    part[row][threadIdx.x % kRedEntries] = acc;
    __syncthreads();
    if (row == 0 && e < kWeights) {
        double tot = 0.0;
        for (int r = 0; r < kRedRows; ++r) tot += part[r][threadIdx.x];
        grad[e] = __double2ll_rn(tot * dscale * kFix);
    }
}

struct AdamParams {
    float *params, *m, *v;
    long long *grad;
    const uint32_t *touched;  // latent cells with a gradient this step (the others' gradients are zero)
    size_t n;
    float beta1, beta2, eps;
    float step_w, step_lat;  // learning rate / (1 - beta1^t), weights and latents
    float inv_bc2;           // 1 / (1 - beta2^t)
};

__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// p -= step * m / (sqrt(v / (1 - beta2^t)) + eps) after the moment updates
// (bias corrections folded into step and inv_bc2; approximate square root
// and division, as an optimiser needs no correctly rounded update).
__device__ __forceinline__ void adam_update(const AdamParams &a, long long gi, float step, float &p, float &m,
                                            float &v) {
    const float gr = __ll2float_rn(gi) * 0x1p-44f;  // fixed point back to FP32 (exact scale)
    m = __fmaf_rn(a.beta1, m, (1.f - a.beta1) * gr);
    v = __fmaf_rn(a.beta2, v, (1.f - a.beta2) * (gr * gr));
    p = __fmaf_rn(-step, __fdividef(m, sqrt_approx(v * a.inv_bc2) + a.eps), p);
}

__device__ __forceinline__ void adam_quad(const AdamParams &a, float step, float4 &p, float4 &m, float4 &v,
                                          longlong2 g01, longlong2 g23) {
    adam_update(a, g01.x, step, p.x, m.x, v.x);
    adam_update(a, g01.y, step, p.y, m.y, v.y);
    adam_update(a, g23.x, step, p.z, m.z, v.z);
    adam_update(a, g23.y, step, p.w, m.w, v.w);
}

// Whether quad q has a gradient to read: the weights always, a latent quad
// (half of a cell's 8 channels) when a texel of the step reached its cell.
// The gradient of any other latent is exactly zero, so skipping its read and
// its clearing leaves every update bit for bit the same.
__device__ __forceinline__ bool quad_has_grad(const AdamParams &a, size_t q) {
    if (q < (size_t)kOffLat / 4) return true;
    const size_t cell = (4 * q - kOffLat) >> 3;
    return (__ldg(a.touched + (cell >> 5)) >> (cell & 31)) & 1u;
}

// Four parameters per quad, two quads per iteration so that both sets of
// loads are in flight together.  The buffer length and the start of the
// latents are multiples of 4; the padding quad (parameters, moments and
// gradients all zero) stays zero.
__global__ void adam_kernel(const AdamParams a) {
    static_assert(kWeights % 4 == 0 && kOffLat == kWeights + 4, "one padding quad");
    const size_t n4 = a.n / 4, stride = (size_t)gridDim.x * blockDim.x;
    float4 *__restrict__ P = reinterpret_cast<float4 *>(a.params);
    float4 *__restrict__ M = reinterpret_cast<float4 *>(a.m);
    float4 *__restrict__ V = reinterpret_cast<float4 *>(a.v);
    longlong2 *__restrict__ G = reinterpret_cast<longlong2 *>(a.grad);
    const longlong2 z = make_longlong2(0, 0);
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n4; q += 2 * stride) {
        const size_t q2 = q + stride;
        const bool two = q2 < n4;
        const bool gq = quad_has_grad(a, q), gq2 = two && quad_has_grad(a, q2);
        const longlong2 g0 = gq ? G[2 * q] : z, g1 = gq ? G[2 * q + 1] : z;
        float4 p = P[q], m = M[q], v = V[q];
        longlong2 h0 = z, h1 = z;
        float4 p2 = make_float4(0.f, 0.f, 0.f, 0.f), m2 = p2, v2 = p2;
        if (two) {
            if (gq2) {
                h0 = G[2 * q2];
                h1 = G[2 * q2 + 1];
            }
            p2 = P[q2];
            m2 = M[q2];
            v2 = V[q2];
        }
        adam_quad(a, q < (size_t)kWeights / 4 ? a.step_w : a.step_lat, p, m, v, g0, g1);
        if (gq) {
            G[2 * q] = z;
            G[2 * q + 1] = z;
        }
        P[q] = p;
        M[q] = m;
        V[q] = v;
        if (two) {
            adam_quad(a, q2 < (size_t)kWeights / 4 ? a.step_w : a.step_lat, p2, m2, v2, h0, h1);
            if (gq2) {
                G[2 * q2] = z;
                G[2 * q2 + 1] = z;
            }
            P[q2] = p2;
            M[q2] = m2;
            V[q2] = v2;
        }
    }
}

__global__ void init_kernel(float *params, size_t n, uint32_t k0, uint32_t k1) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0x1A17u, 0u), k0, k1);
        const float u0 = ((float)(r.x >> 8) + 0.5f) * 5.9604644775390625e-08f;
        const float u1 = ((float)(r.y >> 8) + 0.5f) * 5.9604644775390625e-08f;
        float v = 0.f;
        if (i < (size_t)kOffB1) v = (2.f * u0 - 1.f) * sqrtf(6.f / 16.f);
        else if (i >= (size_t)kOffW2 && i < (size_t)kOffB2) v = (2.f * u0 - 1.f) * sqrtf(6.f / 64.f);
        else if (i >= (size_t)kOffW3 && i < (size_t)kOffB3) v = (2.f * u0 - 1.f) * sqrtf(6.f / 64.f);
        else if (i >= (size_t)kOffB3 && i < (size_t)kWeights) v = 0.5f;
        else if (i >= (size_t)kOffLat) v = 0.5f * sqrtf(-2.f * logf(u0)) * cospif(2.f * u1);
        params[i] = v;
    }
}

// Largest |input| of each layer per input channel over every texel (FP8
// scales).  Values are non-negative, so their bit patterns order like ints.
__global__ void __launch_bounds__(kThreads) actstats_kernel(const GradParams g, unsigned *amax) {
    __shared__ float W[kWeights];
    __shared__ unsigned smax[144];
    for (int i = threadIdx.x; i < kWeights; i += kThreads) W[i] = g.params[i];
    for (int i = threadIdx.x; i < 144; i += kThreads) smax[i] = 0u;
    __syncthreads();
    const float *lat[2] = {g.params + kOffLat, g.params + kOffLat + (size_t)g.gw[0] * g.gh[0] * 8};
    const long long total = (long long)g.Wt * g.Ht;
    for (long long t = blockIdx.x * (long long)kThreads + threadIdx.x; t < total; t += (long long)gridDim.x * kThreads) {
        const int x = (int)(t % g.Wt), y = (int)(t / g.Wt);
        float f[16];
#pragma unroll
        for (int gi = 0; gi < 2; ++gi) {
            int tap[4];
            float tw[4];
            bilinear_taps(g, gi, x, y, tap, tw);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) acc = __fmaf_rn(tw[k], __ldg(lat[gi] + (size_t)tap[k] * 8 + c), acc);
                f[gi * 8 + c] = acc;
            }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) atomicMax(&smax[k], __float_as_uint(fabsf(f[k])));
        float h1[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) {
            float a = W[kOffB1 + j];
#pragma unroll
            for (int k = 0; k < 16; ++k) a = __fmaf_rn(W[kOffW1 + j * 16 + k], f[k], a);
            h1[j] = fmaxf(a, 0.f);
            atomicMax(&smax[16 + j], __float_as_uint(h1[j]));
        }
        for (int j = 0; j < 64; ++j) {
            float a = W[kOffB2 + j];
#pragma unroll
            for (int k = 0; k < 64; ++k) a = __fmaf_rn(W[kOffW2 + j * 64 + k], h1[k], a);
            atomicMax(&smax[80 + j], __float_as_uint(fmaxf(a, 0.f)));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 144; i += kThreads) atomicMax(amax + i, smax[i]);
}

// Squared RGB error and largest channel error of a learned texture's decoded
// texels against the exact decode, for texels [start, start + n).
__global__ void compare_kernel(const uint2 *blocks, int nbx, int Wt, int Ht, const float4 *dec, long long start, int n,
                               double *sse, unsigned *maxabs) {
    double acc = 0.0;
    float mx = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const long long t = start + i;
        const int x = (int)(t % Wt), y = (int)(t / Wt);
        const uint32_t px = fetch_block_texel(blocks, nbx, Wt, Ht, x, y);
        const float4 d = dec[i];
        const float e0 = d.x - __fdiv_rn((float)(px & 0xffu), 255.f);
        const float e1 = d.y - __fdiv_rn((float)((px >> 8) & 0xffu), 255.f);
        const float e2 = d.z - __fdiv_rn((float)((px >> 16) & 0xffu), 255.f);
        const float e3 = d.w - __fdiv_rn((float)(px >> 24), 255.f);
        acc += (double)e0 * e0 + (double)e1 * e1 + (double)e2 * e2;
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(e0), fabsf(e1)), fmaxf(fabsf(e2), fabsf(e3))));
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(FULL, acc, o);
        mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(sse, acc);
        atomicMax(maxabs, __float_as_uint(mx));
    }
}

__global__ void linear_xy_kernel(int2 *xy, long long start, int n, int Wt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const long long t = start + i;
        xy[i] = make_int2((int)(t % Wt), (int)(t / Wt));
    }
}

}  // namespace
}  // namespace ctf

struct ctf_trainer_s {
    ctf_texture src = nullptr;
    ctf_train_desc desc{};
    int Wt = 0, Ht = 0;
    size_t n_lat[2] = {0, 0};
    size_t nparams = 0;
    float *params = nullptr, *m = nullptr, *v = nullptr;
    long long *grad = nullptr, *loss = nullptr;
    uint32_t *touched = nullptr;  // latent cells a step's texels reached (zero between steps)
    unsigned char *wimg = nullptr;  // FP16 weight operands of the gradient kernel
    float *partial = nullptr;       // per-CTA weight-gradient sums of the gradient kernel
    size_t touched_words = 0;
    int64_t step = 0;
};

namespace ctf {
namespace {

GradParams grad_params(const ctf_trainer_s *t) {
    GradParams g;
    g.params = t->params;
    g.blocks = static_cast<const uint2 *>(t->src->blocks);
    g.Wt = t->Wt;
    g.Ht = t->Ht;
    g.nbx = t->Wt / 4;
    for (int i = 0; i < 2; ++i) {
        g.gw[i] = t->desc.latent_w[i];
        g.gh[i] = t->desc.latent_h[i];
        g.sx[i] = (float)g.gw[i] / (float)t->Wt;
        g.sy[i] = (float)g.gh[i] / (float)t->Ht;
    }
    g.xy = nullptr;
    g.n = 0;
    g.rounds = 1;
    g.step = 0;
    g.k0 = (uint32_t)(t->desc.seed & 0xffffffffu);
    g.k1 = (uint32_t)(t->desc.seed >> 32);
    g.dscale = 0.f;
    g.grad = t->grad;
    g.touched = t->touched;
    g.loss = t->loss;
    g.per_round = kT;
    g.wimg = t->wimg;
    g.partial = t->partial;
    g.err = nullptr;
    device_error_word(&g.err);  // a static device word: no allocation; nullptr if it cannot be had
    return g;
}

cudaError_t launch_grad(const GradParams &g, cudaStream_t s) {
    static std::mutex mu;
    static bool attr[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (!attr[dev]) {
            cudaError_t e = cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem);
            if (e != cudaSuccess) return e;
            attr[dev] = true;
        }
    }
    // Two CTAs fit on an SM (TMEM and shared memory).  Small batches take 64
    // texels per round (the other 64 rows of the MMAs stay empty) so that
    // more SMs have work; a CTA's fixed costs (weights in, sums out) favour a
    // few rounds each once there are 256 CTAs, and at most kMaxGradCtas CTAs
    // hold partial sums.  The split depends on the batch alone, so a step
    // gives the same sums on any device.
    GradParams gp = g;
    gp.per_round = g.n >= 32768 ? kT : kT / 2;
    int rounds = g.n / (gp.per_round * 256);
    rounds = rounds < 1 ? 1 : (rounds > kMaxRounds ? kMaxRounds : rounds);
    const int need = (g.n + gp.per_round * kMaxGradCtas - 1) / (gp.per_round * kMaxGradCtas);
    gp.rounds = rounds > need ? rounds : need;
    const int ctas = (g.n + gp.per_round * gp.rounds - 1) / (gp.per_round * gp.rounds);
    if (ctas == 0) return cudaSuccess;
    pack_kernel<<<(kPackThreads + 255) / 256, 256, 0, s>>>(g.params, g.wimg);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    grad_kernel<<<ctas, kT, kGradSmem, s>>>(gp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_kernel<<<(kWeights + kRedEntries - 1) / kRedEntries, kRedEntries * kRedRows, 0, s>>>(
        g.partial, ctas, (double)g.dscale, g.grad);
    return cudaGetLastError();
}

int check_desc(const ctf_train_desc *d) {
    if (!d) return report(CTF_ERR_ARG, "desc is NULL");
    for (int g = 0; g < 2; ++g)
        if (d->latent_w[g] < 1 || d->latent_h[g] < 1 || d->latent_w[g] > 16384 || d->latent_h[g] > 16384)
            return report(CTF_ERR_ARG, "latent grid %d is %dx%d", g, d->latent_w[g], d->latent_h[g]);
    if (d->batch < 1 || d->batch > 4194304) return report(CTF_ERR_ARG, "batch %d outside [1, 4194304]", d->batch);
    if (d->total_steps < 1) return report(CTF_ERR_ARG, "total_steps must be positive");
    if (!(d->lr_weights > 0.f) || !(d->lr_latents > 0.f) || !(d->lr_final_frac >= 0.f) || !(d->beta1 >= 0.f) ||
        !(d->beta1 < 1.f) || !(d->beta2 >= 0.f) || !(d->beta2 < 1.f) || !(d->eps > 0.f))
        return report(CTF_ERR_ARG, "learning rates / Adam constants out of range");
    return CTF_OK;
}

void free_trainer(ctf_trainer_s *t) {
    if (!t) return;
    ctf::dev_free(t->params);
    ctf::dev_free(t->m);
    ctf::dev_free(t->v);
    ctf::dev_free(t->grad);
    ctf::dev_free(t->touched);
    ctf::dev_free(t->loss);
    ctf::dev_free(t->wimg);
    ctf::dev_free(t->partial);
    delete t;
}

int alloc_trainer(ctf_texture src, const ctf_train_desc *d, ctf_trainer_s **out) {
    if (!src || src->mode != CTF_EVAL_BLOCK) return report(CTF_ERR_ARG, "the source must be an exact block texture");
    int rc = check_desc(d);
    if (rc) return rc;
    ctf_trainer_s *t = new (std::nothrow) ctf_trainer_s();
    if (!t) return report(CTF_ERR_OOM, "host allocation");
    t->src = src;
    t->desc = *d;
    t->Wt = src->width;
    t->Ht = src->height;
    for (int g = 0; g < 2; ++g) t->n_lat[g] = (size_t)d->latent_w[g] * d->latent_h[g] * 8;
    t->nparams = kOffLat + t->n_lat[0] + t->n_lat[1];
    t->touched_words = ((t->n_lat[0] + t->n_lat[1]) / 8 + 31) / 32;
    cudaError_t e = ctf::dev_malloc(&t->params, t->nparams * 4);
    if (e == cudaSuccess) e = ctf::dev_malloc(&t->touched, t->touched_words * 4);
    if (e == cudaSuccess) e = cudaMemset(t->touched, 0, t->touched_words * 4);
    if (e == cudaSuccess) e = ctf::dev_malloc(&t->m, t->nparams * 4);
    if (e == cudaSuccess) e = ctf::dev_malloc(&t->v, t->nparams * 4);
    if (e == cudaSuccess) e = ctf::dev_malloc(&t->grad, t->nparams * 8);
    if (e == cudaSuccess) e = ctf::dev_malloc(&t->loss, 8);
    if (e == cudaSuccess) e = ctf::dev_malloc(&t->wimg, kGAH);
    if (e == cudaSuccess) e = ctf::dev_malloc(&t->partial, (size_t)kMaxGradCtas * kWeights * 4);
    if (e == cudaSuccess) e = cudaMemset(t->m, 0, t->nparams * 4);
    if (e == cudaSuccess) e = cudaMemset(t->v, 0, t->nparams * 4);
    if (e == cudaSuccess) e = cudaMemset(t->grad, 0, t->nparams * 8);
    if (e == cudaSuccess) e = cudaMemset(t->params, 0, t->nparams * 4);
    if (e == cudaSuccess) e = cudaMemset(t->loss, 0, 8);
    if (e != cudaSuccess) {
        free_trainer(t);
        return report_cuda(e, "trainer allocation");
    }
    *out = t;
    return CTF_OK;
}

// Array order of ctf_mlp_arrays and their offsets / sizes in the parameter buffer.
void layout(const ctf_trainer_s *t, size_t off[8], size_t cnt[8]) {
    const size_t o[8] = {kOffLat, kOffLat + t->n_lat[0], kOffW1, kOffB1, kOffW2, kOffB2, kOffW3, kOffB3};
    const size_t c[8] = {t->n_lat[0], t->n_lat[1], 1024, 64, 4096, 64, 256, 4};
    for (int i = 0; i < 8; ++i) {
        off[i] = o[i];
        cnt[i] = c[i];
    }
}

void arrays_of(const ctf_mlp_arrays *a, float *p[8]) {
    p[0] = a->latent[0];
    p[1] = a->latent[1];
    p[2] = a->w1;
    p[3] = a->b1;
    p[4] = a->w2;
    p[5] = a->b2;
    p[6] = a->w3;
    p[7] = a->b3;
}

constexpr char kMagic[8] = {'C', 'T', 'F', 'T', 'R', 'N', '0', '1'};
constexpr uint32_t kVersion = 1;

}  // namespace
}  // namespace ctf

extern "C" {

int ctf_trainer_create(ctf_texture exact_src, const ctf_train_desc *desc, ctf_trainer *out) {
    using namespace ctf;
    clear_error();
    if (!out) return report(CTF_ERR_ARG, "out is NULL");
    *out = nullptr;
    ctf_trainer_s *t = nullptr;
    int rc = alloc_trainer(exact_src, desc, &t);
    if (rc) return rc;
    init_kernel<<<1024, 256>>>(t->params, t->nparams, (uint32_t)(desc->seed & 0xffffffffu), (uint32_t)(desc->seed >> 32));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_trainer(t);
        return report_cuda(e, "parameter initialisation");
    }
    *out = t;
    return CTF_OK;
}

int ctf_trainer_destroy(ctf_trainer t) {
    ctf::clear_error();
    if (!t) return CTF_OK;
    cudaDeviceSynchronize();
    ctf::free_trainer(t);
    return CTF_OK;
}

int64_t ctf_trainer_steps_done(ctf_trainer t) { return t ? t->step : -1; }

int ctf_trainer_step(ctf_trainer t, int64_t steps, void *stream) {
    ctf::NvtxRange nvtx_range("ctf_trainer_step");
    using namespace ctf;
    clear_error();
    if (!t) return report(CTF_ERR_ARG, "trainer is NULL");
    if (steps < 0) return report(CTF_ERR_ARG, "negative step count");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GradParams g = grad_params(t);
    g.n = t->desc.batch;
    g.dscale = 2.0f / (float)t->desc.batch;
    AdamParams a;
    a.params = t->params;
    a.m = t->m;
    a.v = t->v;
    a.grad = t->grad;
    a.touched = t->touched;
    a.n = t->nparams;
    a.beta1 = t->desc.beta1;
    a.beta2 = t->desc.beta2;
    a.eps = t->desc.eps;
    for (int64_t k = 0; k < steps; ++k) {
        const int64_t st = t->step;
        g.step = (uint32_t)st;
        cudaError_t e = cudaMemsetAsync(t->loss, 0, 8, s);
        if (e == cudaSuccess) e = launch_grad(g, s);
        const double frac = std::fmin(1.0, (double)st / (double)t->desc.total_steps);
        const double sched = 1.0 - (1.0 - t->desc.lr_final_frac) * frac;
        const double bc1 = 1.0 - std::pow((double)t->desc.beta1, (double)(st + 1));
        const double bc2 = 1.0 - std::pow((double)t->desc.beta2, (double)(st + 1));
        a.step_w = (float)(t->desc.lr_weights * sched / bc1);
        a.step_lat = (float)(t->desc.lr_latents * sched / bc1);
        a.inv_bc2 = (float)(1.0 / bc2);
        if (e == cudaSuccess) {
            adam_kernel<<<device_sm_count() * 8, 256, 0, s>>>(a);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(t->touched, 0, t->touched_words * 4, s);
        if (e != cudaSuccess) return report_cuda(e, "training step");
        t->step = st + 1;
    }
    return CTF_OK;
}

int ctf_trainer_gradients(ctf_trainer t, const int32_t *xy, int n, double *loss, const ctf_mlp_arrays *grads,
                          void *stream) {
    using namespace ctf;
    clear_error();
    if (!t) return report(CTF_ERR_ARG, "trainer is NULL");
    if (n < 1 || !xy) return report(CTF_ERR_ARG, "need n >= 1 texels");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GradParams g = grad_params(t);
    g.xy = reinterpret_cast<const int2 *>(xy);
    g.n = n;
    g.dscale = 2.0f / (float)n;
    // the accumulators are zero between steps; use them and clear them again
    cudaError_t e = cudaMemsetAsync(t->loss, 0, 8, s);
    if (e == cudaSuccess) e = launch_grad(g, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return report_cuda(e, "gradient kernel");
    std::vector<long long> h(t->nparams);
    long long hl = 0;
    e = cudaMemcpy(h.data(), t->grad, t->nparams * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&hl, t->loss, 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(t->grad, 0, t->nparams * 8);
    if (e == cudaSuccess) e = cudaMemset(t->touched, 0, t->touched_words * 4);
    if (e != cudaSuccess) return report_cuda(e, "reading gradients");
    if (loss) *loss = (double)hl / kLossFix / (double)n;
    if (grads) {
        size_t off[8], cnt[8];
        float *p[8];
        layout(t, off, cnt);
        arrays_of(grads, p);
        for (int i = 0; i < 8; ++i)
            if (p[i])
                for (size_t k = 0; k < cnt[i]; ++k) p[i][k] = (float)((double)h[off[i] + k] / kFix);
    }
    return CTF_OK;
}

int ctf_trainer_get_params(ctf_trainer t, const ctf_mlp_arrays *out) {
    using namespace ctf;
    clear_error();
    if (!t || !out) return report(CTF_ERR_ARG, "trainer and out must not be NULL");
    size_t off[8], cnt[8];
    float *p[8];
    layout(t, off, cnt);
    arrays_of(out, p);
    cudaDeviceSynchronize();
    for (int i = 0; i < 8; ++i)
        if (p[i]) {
            cudaError_t e = cudaMemcpy(p[i], t->params + off[i], cnt[i] * 4, cudaMemcpyDefault);
            if (e != cudaSuccess) return report_cuda(e, "copying parameters out");
        }
    return CTF_OK;
}

int ctf_trainer_set_params(ctf_trainer t, const ctf_mlp_arrays *in) {
    using namespace ctf;
    clear_error();
    if (!t || !in) return report(CTF_ERR_ARG, "trainer and in must not be NULL");
    size_t off[8], cnt[8];
    float *p[8];
    layout(t, off, cnt);
    arrays_of(in, p);
    cudaDeviceSynchronize();
    for (int i = 0; i < 8; ++i)
        if (p[i]) {
            cudaError_t e = cudaMemcpy(t->params + off[i], p[i], cnt[i] * 4, cudaMemcpyDefault);
            if (e != cudaSuccess) return report_cuda(e, "copying parameters in");
        }
    return CTF_OK;
}

int ctf_trainer_export(ctf_trainer t, ctf_eval_mode mode, ctf_texture *out) {
    using namespace ctf;
    clear_error();
    if (!t || !out) return report(CTF_ERR_ARG, "trainer and out must not be NULL");
    ctf_mlp_desc d;
    std::memset(&d, 0, sizeof(d));
    d.width = t->Wt;
    d.height = t->Ht;
    d.mode = mode;
    for (int g = 0; g < 2; ++g) {
        d.latent_w[g] = t->desc.latent_w[g];
        d.latent_h[g] = t->desc.latent_h[g];
    }
    d.latent[0] = t->params + kOffLat;
    d.latent[1] = t->params + kOffLat + t->n_lat[0];
    d.w1 = t->params + kOffW1;
    d.b1 = t->params + kOffB1;
    d.w2 = t->params + kOffW2;
    d.b2 = t->params + kOffB2;
    d.w3 = t->params + kOffW3;
    d.b3 = t->params + kOffB3;
    std::vector<float> amax(144, 0.f);
    if (mode == CTF_EVAL_MLP_FP8) {
        unsigned *dmax = nullptr;
        cudaError_t e = ctf::dev_malloc(&dmax, 144 * 4);
        if (e == cudaSuccess) e = cudaMemset(dmax, 0, 144 * 4);
        if (e == cudaSuccess) {
            GradParams g = grad_params(t);
            actstats_kernel<<<device_sm_count() * 4, kThreads>>>(g, dmax);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpy(amax.data(), dmax, 144 * 4, cudaMemcpyDeviceToHost);
        ctf::dev_free(dmax);
        if (e != cudaSuccess) return report_cuda(e, "activation statistics");
        d.act_absmax[0] = amax.data();
        d.act_absmax[1] = amax.data() + 16;
        d.act_absmax[2] = amax.data() + 80;
    } else {
        cudaDeviceSynchronize();
    }
    return ctf_texture_create_mlp(&d, out);
}

int ctf_trainer_save(ctf_trainer t, const char *path) {
    using namespace ctf;
    clear_error();
    if (!t || !path) return report(CTF_ERR_ARG, "trainer and path must not be NULL");
    cudaDeviceSynchronize();
    std::vector<float> buf(3 * t->nparams);
    cudaError_t e = cudaMemcpy(buf.data(), t->params, t->nparams * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(buf.data() + t->nparams, t->m, t->nparams * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(buf.data() + 2 * t->nparams, t->v, t->nparams * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return report_cuda(e, "reading the training state");
    FILE *f = std::fopen(path, "wb");
    if (!f) return report(CTF_ERR_ARG, "cannot open %s for writing", path);
    uint64_t h = 1469598103934665603ull;
    const uint32_t ver = kVersion;
    const int32_t dims[6] = {t->Wt, t->Ht, t->desc.latent_w[0], t->desc.latent_h[0], t->desc.latent_w[1],
                             t->desc.latent_h[1]};
    const uint64_t np = t->nparams;
    const int64_t step = t->step;
    bool ok = true;
    auto put = [&](const void *p, size_t n) {
        ok = ok && std::fwrite(p, 1, n, f) == n;
        h = fnv1a(p, n, h);
    };
    put(kMagic, 8);
    put(&ver, 4);
    put(dims, sizeof(dims));
    put(&np, 8);
    put(&step, 8);
    put(&t->desc, sizeof(t->desc));
    put(buf.data(), buf.size() * 4);
    ok = ok && std::fwrite(&h, 1, 8, f) == 8;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return report(CTF_ERR_ARG, "writing %s failed", path);
    return CTF_OK;
}

int ctf_trainer_load(ctf_texture exact_src, const char *path, ctf_trainer *out) {
    using namespace ctf;
    clear_error();
    if (!out || !path) return report(CTF_ERR_ARG, "path and out must not be NULL");
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) return report(CTF_ERR_ARG, "cannot open %s", path);
    std::vector<unsigned char> all;
    unsigned char tmp[65536];
    size_t k;
    while ((k = std::fread(tmp, 1, sizeof(tmp), f)) > 0) all.insert(all.end(), tmp, tmp + k);
    std::fclose(f);
    const size_t head = 8 + 4 + 24 + 8 + 8 + sizeof(ctf_train_desc);
    if (all.size() < head + 8 || std::memcmp(all.data(), kMagic, 8) != 0)
        return report(CTF_ERR_CORRUPT, "%s is not a training checkpoint", path);
    uint64_t stored = 0;
    std::memcpy(&stored, all.data() + all.size() - 8, 8);
    if (fnv1a(all.data(), all.size() - 8, 1469598103934665603ull) != stored)
        return report(CTF_ERR_CORRUPT, "checksum mismatch in %s", path);
    uint32_t ver;
    int32_t dims[6];
    uint64_t np;
    int64_t step;
    ctf_train_desc d;
    const unsigned char *p = all.data() + 8;
    std::memcpy(&ver, p, 4);
    p += 4;
    std::memcpy(dims, p, 24);
    p += 24;
    std::memcpy(&np, p, 8);
    p += 8;
    std::memcpy(&step, p, 8);
    p += 8;
    std::memcpy(&d, p, sizeof(d));
    p += sizeof(d);
    if (ver != kVersion) return report(CTF_ERR_CORRUPT, "checkpoint version %u, expected %u", ver, kVersion);
    if (!exact_src || exact_src->width != dims[0] || exact_src->height != dims[1])
        return report(CTF_ERR_CORRUPT, "checkpoint is for a %dx%d texture", dims[0], dims[1]);
    ctf_trainer_s *t = nullptr;
    int rc = alloc_trainer(exact_src, &d, &t);
    if (rc) return rc;
    if (t->nparams != np || all.size() != head + 12 * np + 8) {
        free_trainer(t);
        return report(CTF_ERR_CORRUPT, "checkpoint sizes do not match its description");
    }
    const float *fp = reinterpret_cast<const float *>(p);
    cudaError_t e = cudaMemcpy(t->params, fp, np * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t->m, fp + np, np * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t->v, fp + 2 * np, np * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_trainer(t);
        return report_cuda(e, "uploading the training state");
    }
    t->step = step;
    *out = t;
    return CTF_OK;
}

int ctf_texture_compare(ctf_texture ref, ctf_texture learned, double *mse_rgb, double *max_abs, void *stream) {
    using namespace ctf;
    clear_error();
    if (!ref || !learned || ref->mode != CTF_EVAL_BLOCK || learned->mode == CTF_EVAL_BLOCK)
        return report(CTF_ERR_ARG, "need an exact block texture and a learned-decode texture");
    if (ref->width != learned->width || ref->height != learned->height)
        return report(CTF_ERR_ARG, "texture sizes differ");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int *err = nullptr;
    int rc = device_error_word(&err);
    if (rc) return rc;
    const long long total = (long long)ref->width * ref->height;
    const int chunk = 1 << 22;
    int2 *xy = nullptr;
    float4 *dec = nullptr;
    double *sse = nullptr;
    unsigned *mx = nullptr;
    cudaError_t e = ctf::dev_malloc(&xy, (size_t)chunk * 8);
    if (e == cudaSuccess) e = ctf::dev_malloc(&dec, (size_t)chunk * 16);
    if (e == cudaSuccess) e = ctf::dev_malloc(&sse, 8);
    if (e == cudaSuccess) e = ctf::dev_malloc(&mx, 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(sse, 0, 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(mx, 0, 4, s);
    const MlpDevice m = mlp_device_view(learned);
    for (long long st = 0; st < total && e == cudaSuccess; st += chunk) {
        const int n = (int)std::min<long long>(chunk, total - st);
        linear_xy_kernel<<<1024, 256, 0, s>>>(xy, st, n, ref->width);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_mlp_decode(m, learned->width, learned->height, xy, n, dec, err, s);
        if (e == cudaSuccess) {
            compare_kernel<<<1024, 256, 0, s>>>(static_cast<const uint2 *>(ref->blocks), ref->width / 4, ref->width,
                                                ref->height, dec, st, n, sse, mx);
            e = cudaGetLastError();
        }
    }
    double h_sse = 0.0;
    unsigned h_mx = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_sse, sse, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_mx, mx, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    ctf::dev_free(xy);
    ctf::dev_free(dec);
    ctf::dev_free(sse);
    ctf::dev_free(mx);
    if (e != cudaSuccess) return report_cuda(e, "texture comparison");
    if (mse_rgb) *mse_rgb = h_sse / (3.0 * (double)total);
    if (max_abs) {
        float f;
        std::memcpy(&f, &h_mx, 4);
        *max_abs = f;
    }
    return CTF_OK;
}

}  // extern "C"
