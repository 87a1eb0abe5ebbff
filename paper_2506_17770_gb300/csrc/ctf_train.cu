// ctf_train.cu -- training of the learned texel decode on the GPU.
//
// The network of ctf_mlp.cu (two 8-channel latent grids sampled bilinearly,
// 16 -> 64 -> 64 -> 4 with ReLU) is fitted to the exact decode of a block
// texture.  FP32 master parameters live in one device buffer:
//   [w1 1024 | b1 64 | w2 4096 | b2 64 | w3 256 | b3 4 | pad 4 | latent0 | latent1]
// A step samples a batch of texels with Philox4x32-10.  A CTA of 512 threads
// takes 128 texels per round and runs the forward and backward pass in FP32
// as register-tiled products over them (weights and feature-major
// activations in shared memory).  It sums the weight gradients of its
// texels in texel order, and adds them, like the latent-grid gradient
// scatter, to 64-bit fixed-point accumulators (integer atomics are
// order-independent, so a step is deterministic).  An Adam kernel converts
// the sums back, updates parameters and moments, and clears the
// accumulators.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

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
constexpr int kGradThreads = 512;          // threads of the gradient kernel
constexpr int kT = 128;                    // texels per round of the gradient kernel
constexpr int kMaxRounds = 4;              // rounds per CTA, at most
constexpr int kLd = kT + 4;                // row stride of the feature-major activation rows (floats)

struct GradParams {
    const float *params;
    const uint2 *blocks;
    int Wt, Ht, nbx;
    int gw[2], gh[2];
    float sx[2], sy[2];
    const int2 *xy;        // explicit texels, or nullptr: Philox sampling
    int n;                 // texels in this call
    int rounds;            // rounds of kT texels per CTA
    uint32_t step;         // Philox counter word
    uint32_t k0, k1;       // Philox key
    float dscale;          // 2 / batch
    long long *grad;       // fixed-point gradient accumulators (same layout as params)
    uint32_t *touched;     // one bit per latent cell (grid 0 cells, then grid 1) whose gradient a texel reached
    long long *loss;       // fixed-point sum of squared errors
};

// v * 2^44 is exact in FP32 (a power-of-two scale), so this rounds the same
// value as the FP64 product would, without FP64 arithmetic.
__device__ __forceinline__ long long to_fix(float v) { return __float2ll_rn(v * 0x1p44f); }

// Shared memory of the gradient kernel (floats).  The weights are held as
// stored ([out][in]) and transposed; activations are feature-major rows of
// kLd floats (one column per texel), so that every product below reads
// 16-byte vectors along a contiguous index.  kLd = 132 puts consecutive rows
// 4 banks apart.
constexpr int kSW1 = 0;                    // W1 [64][16]
constexpr int kSW1t = 1024;                // W1^T [16][64]
constexpr int kSW2 = 2048;                 // W2 [64][64]
constexpr int kSW2t = 6144;                // W2^T [64][64]
constexpr int kSW3 = 10240;                // W3 [4][64]
constexpr int kSB1 = 10496, kSB2 = 10560, kSB3 = 10624;
constexpr int kSF = 10628;                 // F^T  [16][kLd]  features
constexpr int kSH1 = kSF + 16 * kLd;       // H1^T [64][kLd]
constexpr int kSH2 = kSH1 + 64 * kLd;      // H2^T [64][kLd]
constexpr int kSD2 = kSH2 + 64 * kLd;      // dH2^T [64][kLd] (masked)
constexpr int kSD1 = kSD2 + 64 * kLd;      // dH1^T [64][kLd] (masked)
constexpr int kSDY = kSD1 + 64 * kLd;      // dY^T [4][kLd]
constexpr int kSDF = kSDY + 4 * kLd;       // dF^T [16][kLd]
constexpr int kSE = kSDF + 16 * kLd;       // output errors [4][kT]
constexpr int kSXY = kSE + 4 * kT;         // texel coordinates, int2 [kT]
constexpr int kSmFloats = kSXY + 2 * kT;
constexpr size_t kGradSmem = (size_t)kSmFloats * 4;
static_assert(kSF % 4 == 0 && kSH1 % 4 == 0 && kSD2 % 4 == 0 && kSDY % 4 == 0 && kSE % 4 == 0 && kLd % 4 == 0,
              "16-byte rows");
static_assert(kGradSmem <= 227 * 1024, "shared memory");

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// acc[i][j] += sum over k < K of A[k][m0 + i] * B[k][n0 + j]: A rows of lda
// floats (contiguous in m), B rows of kLd floats (contiguous in n), k
// ascending, one fused multiply-add per term.
template <int K>
__device__ __forceinline__ void mm44(const float *A, int lda, const float *B, int m0, int n0, float (&acc)[4][4]) {
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        const float4 a = ld4(A + k * lda + m0), b = ld4(B + k * kLd + n0);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = __fmaf_rn(av[i], bv[j], acc[i][j]);
    }
}

// Block of one thread in a 64 x 128 product: warps tile 4 x 4 blocks of
// 16 x 32, lanes 4 x 8 blocks of 4 x 4.
__device__ __forceinline__ void tile_64x128(int tid, int &m0, int &n0) {
    const int w = tid >> 5, l = tid & 31;
    m0 = (w & 3) * 16 + (l >> 3) * 4;
    n0 = (w >> 2) * 32 + (l & 7) * 4;
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
    idx[0] = ya * gw + xa;
    idx[1] = ya * gw + xb;
    idx[2] = yb * gw + xa;
    idx[3] = yb * gw + xb;
    const float ofx = __fsub_rn(1.f, fx), ofy = __fsub_rn(1.f, fy);
    w[0] = __fmul_rn(ofx, ofy);
    w[1] = __fmul_rn(fx, ofy);
    w[2] = __fmul_rn(ofx, fy);
    w[3] = __fmul_rn(fx, fy);
}

// Forward and backward pass of kT texels per round, as products over the
// round's texels.  Every texel's activations and input-side gradients come
// out of the same operations in the same order as a per-texel evaluation;
// the weight gradients are summed over the CTA's texels in texel order.
__global__ void __launch_bounds__(kGradThreads, 1) grad_kernel(const GradParams g) {
    extern __shared__ __align__(16) float sm[];
    const int tid = threadIdx.x;
    // transposed copies are read transposed from global (L2) and written in
    // order, which keeps the shared-memory stores free of bank conflicts
    for (int i = tid; i < 1024; i += kGradThreads) {
        sm[kSW1 + i] = g.params[kOffW1 + i];
        sm[kSW1t + i] = g.params[kOffW1 + (i & 63) * 16 + (i >> 6)];
    }
    for (int i = tid; i < 4096; i += kGradThreads) {
        sm[kSW2 + i] = g.params[kOffW2 + i];
        sm[kSW2t + i] = g.params[kOffW2 + (i & 63) * 64 + (i >> 6)];
    }
    for (int i = tid; i < 256; i += kGradThreads) sm[kSW3 + i] = g.params[kOffW3 + i];
    if (tid < 64) {
        sm[kSB1 + tid] = g.params[kOffB1 + tid];
        sm[kSB2 + tid] = g.params[kOffB2 + tid];
    }
    if (tid < 4) sm[kSB3 + tid] = g.params[kOffB3 + tid];
    const float *W1 = sm + kSW1, *W1t = sm + kSW1t, *W2 = sm + kSW2, *W2t = sm + kSW2t, *W3 = sm + kSW3;
    const float *B1 = sm + kSB1, *B2 = sm + kSB2, *B3 = sm + kSB3;
    float *F = sm + kSF, *H1 = sm + kSH1, *H2 = sm + kSH2, *D2 = sm + kSD2, *D1 = sm + kSD1, *DY = sm + kSDY,
          *DF = sm + kSDF, *E = sm + kSE;
    int2 *XY = reinterpret_cast<int2 *>(sm + kSXY);
    const size_t lat1 = (size_t)g.gw[0] * g.gh[0] * 8;  // start of the second grid
    const int w = tid >> 5, l = tid & 31;
    int m0, n0;
    tile_64x128(tid, m0, n0);
    // persistent weight-gradient sums of this thread:
    //   dW2 rows m2 + {0, 4}, columns n2 + {0, 8, 16, 24}; dW1 row tid/8,
    //   columns (tid%8) + {0, 8}; dW3 (tid < 256) row tid/64, column tid%64;
    //   db2 (tid < 64), db1 (64 <= tid < 128), db3 (128 <= tid < 132)
    const int m2 = (w & 7) * 8 + (l >> 3), n2 = (w >> 3) * 32 + (l & 7);
    const int m1 = tid >> 3, n1 = tid & 7;
    float aW2[2][4] = {}, aW1[2] = {}, aW3 = 0.f, aB = 0.f, loss = 0.f;
    __syncthreads();

#pragma unroll 1
    for (int r = 0; r < g.rounds; ++r) {
        const int i0 = (blockIdx.x * g.rounds + r) * kT;
        // ---- texels of the round
        if (tid < kT) {
            const int i = i0 + tid;
            int x, y;
            if (g.xy) {
                const int2 c = i < g.n ? g.xy[i] : make_int2(0, 0);
                x = min(max(c.x, 0), g.Wt - 1);
                y = min(max(c.y, 0), g.Ht - 1);
            } else {
                const uint4 rr = philox4x32_10(make_uint4((uint32_t)i, g.step, 0x5A4Du, 0u), g.k0, g.k1);
                x = (int)(((unsigned long long)rr.x * (unsigned)g.Wt) >> 32);
                y = (int)(((unsigned long long)rr.y * (unsigned)g.Ht) >> 32);
            }
            XY[tid] = make_int2(x, y);
        }
        __syncthreads();
        // ---- features: texel t, grid q/2, channels 4(q%2) .. +3
        {
            const int t = tid & (kT - 1), q = tid >> 7, gi = q >> 1, c0 = (q & 1) * 4;
            const int2 c = XY[t];
            int tap[4];
            float tw[4];
            bilinear_taps(g, gi, c.x, c.y, tap, tw);
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            const float *lg = g.params + kOffLat + (gi ? lat1 : 0);
            for (int k = 0; k < 4; ++k) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(lg + (size_t)tap[k] * 8 + c0));
                acc[0] = __fmaf_rn(tw[k], v.x, acc[0]);
                acc[1] = __fmaf_rn(tw[k], v.y, acc[1]);
                acc[2] = __fmaf_rn(tw[k], v.z, acc[2]);
                acc[3] = __fmaf_rn(tw[k], v.w, acc[3]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) F[(gi * 8 + c0 + j) * kLd + t] = acc[j];
        }
        __syncthreads();
        // ---- H1 = relu(W1 F + b1), H2 = relu(W2 H1 + b2)
        {
            float acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = B1[m0 + i];
            mm44<16>(W1t, 64, F, m0, n0, acc);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                st4(H1 + (m0 + i) * kLd + n0, make_float4(fmaxf(acc[i][0], 0.f), fmaxf(acc[i][1], 0.f),
                                                          fmaxf(acc[i][2], 0.f), fmaxf(acc[i][3], 0.f)));
        }
        __syncthreads();
        {
            float acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = B2[m0 + i];
            mm44<64>(W2t, 64, H1, m0, n0, acc);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                st4(H2 + (m0 + i) * kLd + n0, make_float4(fmaxf(acc[i][0], 0.f), fmaxf(acc[i][1], 0.f),
                                                          fmaxf(acc[i][2], 0.f), fmaxf(acc[i][3], 0.f)));
        }
        __syncthreads();
        // ---- output channel c of texel t, its error and dY = 2 e / batch
        {
            const int t = tid & (kT - 1), c = tid >> 7;
            const bool valid = i0 + t < g.n;
            float a = B3[c];
#pragma unroll 4
            for (int k = 0; k < 64; k += 4) {
                const float4 wv = ld4(W3 + c * 64 + k);
                a = __fmaf_rn(wv.x, H2[k * kLd + t], a);
                a = __fmaf_rn(wv.y, H2[(k + 1) * kLd + t], a);
                a = __fmaf_rn(wv.z, H2[(k + 2) * kLd + t], a);
                a = __fmaf_rn(wv.w, H2[(k + 3) * kLd + t], a);
            }
            const int2 xy = XY[t];
            const uint32_t px = fetch_block_texel(g.blocks, g.nbx, g.Wt, g.Ht, xy.x, xy.y);
            const float tgt = __fdiv_rn((float)((px >> (8 * c)) & 0xffu), 255.f);
            const float e = __fsub_rn(a, tgt);
            E[c * kT + t] = e;
            DY[c * kLd + t] = valid ? __fmul_rn(e, g.dscale) : 0.f;
        }
        __syncthreads();
        // ---- loss (texel order, channels in order); dW3 += dY H2^T; dH2 = (W3^T dY) masked by H2 > 0
        if (tid < kT && i0 + tid < g.n) {
#pragma unroll
            for (int c = 0; c < 4; ++c) loss = __fmaf_rn(E[c * kT + tid], E[c * kT + tid], loss);
        }
        if (tid < 256) {
            const float *dy = DY + (tid >> 6) * kLd, *h = H2 + (tid & 63) * kLd;
#pragma unroll 4
            for (int t = 0; t < kT; t += 4) {
                const float4 a = ld4(dy + t), b = ld4(h + t);
                aW3 = __fmaf_rn(a.x, b.x, aW3);
                aW3 = __fmaf_rn(a.y, b.y, aW3);
                aW3 = __fmaf_rn(a.z, b.z, aW3);
                aW3 = __fmaf_rn(a.w, b.w, aW3);
            }
        }
        {
            float acc[4][4] = {};
            mm44<4>(W3, 64, DY, m0, n0, acc);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 h = ld4(H2 + (m0 + i) * kLd + n0);
                st4(D2 + (m0 + i) * kLd + n0, make_float4(h.x > 0.f ? acc[i][0] : 0.f, h.y > 0.f ? acc[i][1] : 0.f,
                                                          h.z > 0.f ? acc[i][2] : 0.f, h.w > 0.f ? acc[i][3] : 0.f));
            }
        }
        __syncthreads();
        // ---- dW2 += dH2 H1^T; dH1 = (W2^T dH2) masked by H1 > 0
        {
            const float *a0 = D2 + m2 * kLd, *a1 = D2 + (m2 + 4) * kLd;
            const float *b0 = H1 + n2 * kLd;
#pragma unroll 2
            for (int t = 0; t < kT; t += 4) {
                const float4 x0 = ld4(a0 + t), x1 = ld4(a1 + t);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float4 y = ld4(b0 + 8 * j * kLd + t);
                    aW2[0][j] = __fmaf_rn(x0.x, y.x, aW2[0][j]);
                    aW2[0][j] = __fmaf_rn(x0.y, y.y, aW2[0][j]);
                    aW2[0][j] = __fmaf_rn(x0.z, y.z, aW2[0][j]);
                    aW2[0][j] = __fmaf_rn(x0.w, y.w, aW2[0][j]);
                    aW2[1][j] = __fmaf_rn(x1.x, y.x, aW2[1][j]);
                    aW2[1][j] = __fmaf_rn(x1.y, y.y, aW2[1][j]);
                    aW2[1][j] = __fmaf_rn(x1.z, y.z, aW2[1][j]);
                    aW2[1][j] = __fmaf_rn(x1.w, y.w, aW2[1][j]);
                }
            }
        }
        {
            float acc[4][4] = {};
            mm44<64>(W2, 64, D2, m0, n0, acc);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 h = ld4(H1 + (m0 + i) * kLd + n0);
                st4(D1 + (m0 + i) * kLd + n0, make_float4(h.x > 0.f ? acc[i][0] : 0.f, h.y > 0.f ? acc[i][1] : 0.f,
                                                          h.z > 0.f ? acc[i][2] : 0.f, h.w > 0.f ? acc[i][3] : 0.f));
            }
        }
        __syncthreads();
        // ---- dW1 += dH1 F^T; bias sums; dF = W1^T dH1 (warps 0-3)
        {
            const float *a = D1 + m1 * kLd, *b0 = F + n1 * kLd, *b1 = F + (n1 + 8) * kLd;
#pragma unroll 4
            for (int t = 0; t < kT; t += 4) {
                const float4 x = ld4(a + t), y0 = ld4(b0 + t), y1 = ld4(b1 + t);
                aW1[0] = __fmaf_rn(x.x, y0.x, aW1[0]);
                aW1[0] = __fmaf_rn(x.y, y0.y, aW1[0]);
                aW1[0] = __fmaf_rn(x.z, y0.z, aW1[0]);
                aW1[0] = __fmaf_rn(x.w, y0.w, aW1[0]);
                aW1[1] = __fmaf_rn(x.x, y1.x, aW1[1]);
                aW1[1] = __fmaf_rn(x.y, y1.y, aW1[1]);
                aW1[1] = __fmaf_rn(x.z, y1.z, aW1[1]);
                aW1[1] = __fmaf_rn(x.w, y1.w, aW1[1]);
            }
        }
        if (tid < 132) {
            const float *row = tid < 64 ? D2 + tid * kLd : (tid < 128 ? D1 + (tid - 64) * kLd : DY + (tid - 128) * kLd);
#pragma unroll 4
            for (int t = 0; t < kT; t += 4) {
                const float4 v = ld4(row + t);
                aB = __fadd_rn(aB, v.x);
                aB = __fadd_rn(aB, v.y);
                aB = __fadd_rn(aB, v.z);
                aB = __fadd_rn(aB, v.w);
            }
        }
        if (w < 4) {
            float acc[4][4] = {};
            const int fm = (l >> 3) * 4, fn = w * 32 + (l & 7) * 4;
            mm44<64>(W1, 16, D1, fm, fn, acc);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                st4(DF + (fm + i) * kLd + fn, make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]));
        }
        __syncthreads();
        // ---- latent-grid gradient: texel t, grid q/2, taps 2(q%2), 2(q%2) + 1
        {
            const int t = tid & (kT - 1), q = tid >> 7, gi = q >> 1, hi = q & 1;
            if (i0 + t < g.n) {
                const int2 c = XY[t];
                int tap[4];
                float tw[4];
                bilinear_taps(g, gi, c.x, c.y, tap, tw);
                unsigned long long *gl = reinterpret_cast<unsigned long long *>(g.grad + kOffLat + (gi ? lat1 : 0));
                const int ta[2] = {hi ? tap[2] : tap[0], hi ? tap[3] : tap[1]};
                const float wa[2] = {hi ? tw[2] : tw[0], hi ? tw[3] : tw[1]};
                const uint32_t cell0 = gi ? (uint32_t)(lat1 / 8) : 0u;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const uint32_t cell = cell0 + (uint32_t)ta[k];
                    atomicOr(g.touched + (cell >> 5), 1u << (cell & 31u));
#pragma unroll
                    for (int ch = 0; ch < 8; ++ch) {
                        const long long v = to_fix(__fmul_rn(wa[k], DF[(gi * 8 + ch) * kLd + t]));
                        if (v) atomicAdd(gl + (size_t)ta[k] * 8 + ch, (unsigned long long)v);
                    }
                }
            }
        }
        __syncthreads();
    }
    // ---- flush the CTA's sums
    unsigned long long *G = reinterpret_cast<unsigned long long *>(g.grad);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            atomicAdd(G + kOffW2 + (m2 + 4 * i) * 64 + n2 + 8 * j, (unsigned long long)to_fix(aW2[i][j]));
    atomicAdd(G + kOffW1 + m1 * 16 + n1, (unsigned long long)to_fix(aW1[0]));
    atomicAdd(G + kOffW1 + m1 * 16 + n1 + 8, (unsigned long long)to_fix(aW1[1]));
    if (tid < 256) atomicAdd(G + kOffW3 + tid, (unsigned long long)to_fix(aW3));
    if (tid < 132)
        atomicAdd(G + (tid < 64 ? kOffB2 + tid : (tid < 128 ? kOffB1 + tid - 64 : kOffB3 + tid - 128)),
                  (unsigned long long)to_fix(aB));
    E[tid] = loss;
    __syncthreads();
    if (tid == 0) {
        float tot = 0.f;
        for (int s = 0; s < kT; ++s) tot = __fadd_rn(tot, E[s]);
        atomicAdd(reinterpret_cast<unsigned long long *>(g.loss), (unsigned long long)__double2ll_rn((double)tot * kLossFix));
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
    return g;
}

cudaError_t launch_grad(const GradParams &g, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    // One CTA per SM fits (shared memory and registers).  A CTA's fixed
    // costs (weights in, sums out) favour a few rounds each: kMaxRounds once
    // there are 128 CTAs of them, fewer below.  The split depends on the
    // batch alone, so a step gives the same sums on any device.
    GradParams gp = g;
    gp.rounds = g.n / (kT * 128);
    gp.rounds = gp.rounds < 1 ? 1 : (gp.rounds > kMaxRounds ? kMaxRounds : gp.rounds);
    const int ctas = (g.n + kT * gp.rounds - 1) / (kT * gp.rounds);
    if (ctas == 0) return cudaSuccess;
    grad_kernel<<<ctas, kGradThreads, kGradSmem, s>>>(gp);
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
