// ctf_train.cu -- training of the learned texel decode on the GPU.
//
// The network of ctf_mlp.cu (two 8-channel latent grids sampled bilinearly,
// 16 -> 64 -> 64 -> 4 with ReLU) is fitted to the exact decode of a block
// texture.  FP32 master parameters live in one device buffer:
//   [w1 1024 | b1 64 | w2 4096 | b2 64 | w3 256 | b3 4 | pad 4 | latent0 | latent1]
// A step samples a batch of texels with Philox4x32-10, and for every texel
// one thread runs the forward and backward pass in FP32 (weights in shared
// memory, per-texel activations in shared-memory rows).  The CTA then sums
// the weight gradients of its 128 texels in a fixed order, and adds them,
// like the latent-grid gradient scatter, to 64-bit fixed-point accumulators
// (integer atomics are order-independent, so a step is deterministic).  An
// Adam kernel converts the sums back, updates parameters and moments, and
// clears the accumulators.
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
constexpr int kThreads = 128;
constexpr int kRounds = 4;                 // rounds of 128 texels per CTA
constexpr int kRow = 68;                   // row length of the per-texel activation rows

struct GradParams {
    const float *params;
    const uint2 *blocks;
    int Wt, Ht, nbx;
    int gw[2], gh[2];
    float sx[2], sy[2];
    const int2 *xy;        // explicit texels, or nullptr: Philox sampling
    int n;                 // texels in this call
    uint32_t step;         // Philox counter word
    uint32_t k0, k1;       // Philox key
    float dscale;          // 2 / batch
    long long *grad;       // fixed-point gradient accumulators (same layout as params)
    long long *loss;       // fixed-point sum of squared errors
};

__device__ __forceinline__ long long to_fix(float v) { return __double2ll_rn((double)v * kFix); }

// Shared memory of the gradient kernel (floats).  Per-texel rows have a
// stride of 68 floats: 16-byte aligned, and 8 threads reading 16 bytes each
// from their own rows touch all 32 banks once.
constexpr int kRowF = 20;                     // features (16 used)
constexpr int kSmF = 5512;                    // [128][20]
constexpr int kSmH1 = kSmF + 128 * kRowF;     // [128][68]
constexpr int kSmH2 = kSmH1 + 128 * kRow;
constexpr int kSmD1 = kSmH2 + 128 * kRow;
constexpr int kSmD2 = kSmD1 + 128 * kRow;
constexpr int kSmDY = kSmD2 + 128 * kRow;     // [128][4]
constexpr int kSmLoss = kSmDY + 128 * 4;      // [128]
constexpr int kSmAcc = kSmLoss + 128;         // [44][128] per-thread gradient sums
constexpr int kNAcc = 44;
constexpr int kSmFloats = kSmAcc + kNAcc * 128;
constexpr size_t kGradSmem = (size_t)kSmFloats * 4;

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// y = W x + b over own rows: W [OUT][IN] and b in shared memory, x and y
// rows of this thread; 8 outputs at a time, 4 inputs per step.
template <int IN, int OUT>
__device__ __forceinline__ void dense_fwd(const float *W, const float *b, const float *x, float *y) {
#pragma unroll 1
    for (int j = 0; j < OUT; j += 8) {
        float acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = b[j + q];
#pragma unroll 4
        for (int k = 0; k < IN; k += 4) {
            const float4 xv = ld4(x + k);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 w = ld4(W + (j + q) * IN + k);
                acc[q] = __fmaf_rn(w.x, xv.x, acc[q]);
                acc[q] = __fmaf_rn(w.y, xv.y, acc[q]);
                acc[q] = __fmaf_rn(w.z, xv.z, acc[q]);
                acc[q] = __fmaf_rn(w.w, xv.w, acc[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < 8; q += 4)
            st4(y + j + q, make_float4(fmaxf(acc[q], 0.f), fmaxf(acc[q + 1], 0.f), fmaxf(acc[q + 2], 0.f),
                                       fmaxf(acc[q + 3], 0.f)));
    }
}

// dx = W^T dy over own rows, masked by (h > 0): W [OUT][IN]; 8 inputs at a
// time, one output per step.
template <int IN, int OUT>
__device__ __forceinline__ void dense_bwd(const float *W, const float *dy, const float *h, float *dx) {
#pragma unroll 1
    for (int k = 0; k < IN; k += 8) {
        float acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = 0.f;
#pragma unroll 4
        for (int j = 0; j < OUT; ++j) {
            const float d = dy[j];
            const float4 w0 = ld4(W + j * IN + k), w1 = ld4(W + j * IN + k + 4);
            acc[0] = __fmaf_rn(w0.x, d, acc[0]);
            acc[1] = __fmaf_rn(w0.y, d, acc[1]);
            acc[2] = __fmaf_rn(w0.z, d, acc[2]);
            acc[3] = __fmaf_rn(w0.w, d, acc[3]);
            acc[4] = __fmaf_rn(w1.x, d, acc[4]);
            acc[5] = __fmaf_rn(w1.y, d, acc[5]);
            acc[6] = __fmaf_rn(w1.z, d, acc[6]);
            acc[7] = __fmaf_rn(w1.w, d, acc[7]);
        }
        const float4 h0 = ld4(h + k), h1 = ld4(h + k + 4);
        st4(dx + k, make_float4(h0.x > 0.f ? acc[0] : 0.f, h0.y > 0.f ? acc[1] : 0.f, h0.z > 0.f ? acc[2] : 0.f,
                                h0.w > 0.f ? acc[3] : 0.f));
        st4(dx + k + 4, make_float4(h1.x > 0.f ? acc[4] : 0.f, h1.y > 0.f ? acc[5] : 0.f,
                                    h1.z > 0.f ? acc[6] : 0.f, h1.w > 0.f ? acc[7] : 0.f));
    }
}

__device__ __forceinline__ void bilinear_taps(const GradParams &g, int grid, int x, int y, int idx[4], float w[4]) {
    const float gx = __fsub_rn(__fmul_rn(__fadd_rn((float)x, 0.5f), g.sx[grid]), 0.5f);
    const float gy = __fsub_rn(__fmul_rn(__fadd_rn((float)y, 0.5f), g.sy[grid]), 0.5f);
    const float fx0 = floorf(gx), fy0 = floorf(gy);
    const float fx = __fsub_rn(gx, fx0), fy = __fsub_rn(gy, fy0);
    const int x0 = (int)fx0, y0 = (int)fy0;
    const int xa = min(max(x0, 0), g.gw[grid] - 1), xb = min(max(x0 + 1, 0), g.gw[grid] - 1);
    const int ya = min(max(y0, 0), g.gh[grid] - 1), yb = min(max(y0 + 1, 0), g.gh[grid] - 1);
    idx[0] = ya * g.gw[grid] + xa;
    idx[1] = ya * g.gw[grid] + xb;
    idx[2] = yb * g.gw[grid] + xa;
    idx[3] = yb * g.gw[grid] + xb;
    const float ofx = __fsub_rn(1.f, fx), ofy = __fsub_rn(1.f, fy);
    w[0] = __fmul_rn(ofx, ofy);
    w[1] = __fmul_rn(fx, ofy);
    w[2] = __fmul_rn(ofx, fy);
    w[3] = __fmul_rn(fx, fy);
}

__global__ void __launch_bounds__(kThreads) grad_kernel(const GradParams g) {
    extern __shared__ __align__(16) float sm[];
    const int tid = threadIdx.x;
    for (int i = tid; i < kWeights; i += kThreads) sm[i] = g.params[i];
    static_assert(kSmF % 4 == 0 && kSmH1 % 4 == 0 && kSmD2 % 4 == 0 && kSmDY % 4 == 0, "16-byte rows");
    float *W1 = sm + kOffW1, *B1 = sm + kOffB1, *W2 = sm + kOffW2, *B2 = sm + kOffB2, *W3 = sm + kOffW3,
          *B3 = sm + kOffB3;
    float *F = sm + kSmF, *H1 = sm + kSmH1, *H2 = sm + kSmH2, *D1 = sm + kSmD1, *D2 = sm + kSmD2, *DY = sm + kSmDY,
          *LS = sm + kSmLoss;
    const float *lat[2] = {g.params + kOffLat, g.params + kOffLat + (size_t)g.gw[0] * g.gh[0] * 8};
    long long *glat[2] = {g.grad + kOffLat, g.grad + kOffLat + (size_t)g.gw[0] * g.gh[0] * 8};
    // reduction ownership: dW2 (j2, i2..i2+31), dW1 (j2, k1..k1+7), dW3 (c3, i3, i3+1)
    const int j2 = tid >> 1, i2 = (tid & 1) * 32, k1 = (tid & 1) * 8;
    const int c3 = tid >> 5, i3 = (tid & 31) * 2;
    // per-thread sums: [0,32) dW2, [32,40) dW1, [40,42) dW3, 42 db1/db2, 43 db3
    float *ACC = sm + kSmAcc;
#pragma unroll
    for (int q = 0; q < kNAcc; ++q) ACC[q * 128 + tid] = 0.f;
    float loss = 0.f;
    __syncthreads();

#pragma unroll 1
    for (int r = 0; r < kRounds; ++r) {
        const int i = (blockIdx.x * kRounds + r) * kThreads + tid;
        const bool valid = i < g.n;
        // ---- texel and target
        int x, y;
        if (g.xy) {
            const int2 c = valid ? g.xy[i] : make_int2(0, 0);
            x = min(max(c.x, 0), g.Wt - 1);
            y = min(max(c.y, 0), g.Ht - 1);
        } else {
            const uint4 rr = philox4x32_10(make_uint4((uint32_t)i, g.step, 0x5A4Du, 0u), g.k0, g.k1);
            x = (int)(((unsigned long long)rr.x * (unsigned)g.Wt) >> 32);
            y = (int)(((unsigned long long)rr.y * (unsigned)g.Ht) >> 32);
        }
        const uint32_t px = fetch_block_texel(g.blocks, g.nbx, g.Wt, g.Ht, x, y);
        float tgt[4];
        tgt[0] = __fdiv_rn((float)(px & 0xffu), 255.f);
        tgt[1] = __fdiv_rn((float)((px >> 8) & 0xffu), 255.f);
        tgt[2] = __fdiv_rn((float)((px >> 16) & 0xffu), 255.f);
        tgt[3] = __fdiv_rn((float)(px >> 24), 255.f);
        // ---- features
        int tap[2][4];
        float tw[2][4];
        float f[16];
#pragma unroll
        for (int gi = 0; gi < 2; ++gi) {
            bilinear_taps(g, gi, x, y, tap[gi], tw[gi]);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) acc = __fmaf_rn(tw[gi][k], __ldg(lat[gi] + (size_t)tap[gi][k] * 8 + c), acc);
                f[gi * 8 + c] = acc;
            }
        }
        float *Fr = F + tid * kRowF, *H1r = H1 + tid * kRow, *H2r = H2 + tid * kRow;
        float *D1r = D1 + tid * kRow, *D2r = D2 + tid * kRow, *DYr = DY + tid * 4;
#pragma unroll
        for (int k = 0; k < 16; k += 4)
            st4(Fr + k, valid ? make_float4(f[k], f[k + 1], f[k + 2], f[k + 3]) : make_float4(0.f, 0.f, 0.f, 0.f));
        // ---- forward (features are valid for every texel; rows of invalid ones are masked below)
#pragma unroll
        for (int k = 0; k < 16; k += 4) st4(D1r + k, make_float4(f[k], f[k + 1], f[k + 2], f[k + 3]));
        dense_fwd<16, 64>(W1, B1, D1r, H1r);
        dense_fwd<64, 64>(W2, B2, H1r, H2r);
        float dy[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float a = B3[c];
#pragma unroll 4
            for (int k = 0; k < 64; k += 4) {
                const float4 hv = ld4(H2r + k), w = ld4(W3 + c * 64 + k);
                a = __fmaf_rn(w.x, hv.x, a);
                a = __fmaf_rn(w.y, hv.y, a);
                a = __fmaf_rn(w.z, hv.z, a);
                a = __fmaf_rn(w.w, hv.w, a);
            }
            const float e = __fsub_rn(a, tgt[c]);
            if (valid) loss = __fmaf_rn(e, e, loss);
            dy[c] = valid ? __fmul_rn(e, g.dscale) : 0.f;
        }
        st4(DYr, make_float4(dy[0], dy[1], dy[2], dy[3]));
        // ---- backward: dh2 = W3^T dy (masked), dh1 = W2^T dh2 (masked), df = W1^T dh1
        dense_bwd<64, 4>(W3, DYr, H2r, D2r);
        dense_bwd<64, 64>(W2, D2r, H1r, D1r);
        float df[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) df[k] = 0.f;
#pragma unroll 4
        for (int j = 0; j < 64; ++j) {
            const float d = D1r[j];
#pragma unroll
            for (int k = 0; k < 16; k += 4) {
                const float4 w = ld4(W1 + j * 16 + k);
                df[k] = __fmaf_rn(w.x, d, df[k]);
                df[k + 1] = __fmaf_rn(w.y, d, df[k + 1]);
                df[k + 2] = __fmaf_rn(w.z, d, df[k + 2]);
                df[k + 3] = __fmaf_rn(w.w, d, df[k + 3]);
            }
        }
        // ---- latent-grid gradient: each feature is a bilinear blend of 4 taps
        if (valid) {
#pragma unroll
            for (int gi = 0; gi < 2; ++gi)
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const long long v = to_fix(__fmul_rn(tw[gi][k], df[gi * 8 + c]));
                        if (v) atomicAdd(reinterpret_cast<unsigned long long *>(glat[gi] + (size_t)tap[gi][k] * 8 + c),
                                         (unsigned long long)v);
                    }
        }
        __syncthreads();
        // ---- weight gradients of the 128 texels, summed in a fixed order
        {
            float aW2[32], aW1[8], aW3[2], aB, aB3;
#pragma unroll
            for (int q = 0; q < 32; ++q) aW2[q] = ACC[q * 128 + tid];
#pragma unroll
            for (int q = 0; q < 8; ++q) aW1[q] = ACC[(32 + q) * 128 + tid];
            aW3[0] = ACC[40 * 128 + tid];
            aW3[1] = ACC[41 * 128 + tid];
            aB = ACC[42 * 128 + tid];
            aB3 = ACC[43 * 128 + tid];
#pragma unroll 1
            for (int s = 0; s < kThreads; ++s) {
                const float d2 = D2[s * kRow + j2], d1 = D1[s * kRow + j2];
#pragma unroll
                for (int q = 0; q < 32; ++q) aW2[q] = __fmaf_rn(d2, H1[s * kRow + i2 + q], aW2[q]);
#pragma unroll
                for (int q = 0; q < 8; ++q) aW1[q] = __fmaf_rn(d1, F[s * kRowF + k1 + q], aW1[q]);
                const float dyc = DY[s * 4 + c3];
                aW3[0] = __fmaf_rn(dyc, H2[s * kRow + i3], aW3[0]);
                aW3[1] = __fmaf_rn(dyc, H2[s * kRow + i3 + 1], aW3[1]);
                aB = __fadd_rn(aB, tid < 64 ? D1[s * kRow + tid] : D2[s * kRow + tid - 64]);
                if (tid < 4) aB3 = __fadd_rn(aB3, DY[s * 4 + tid]);
            }
#pragma unroll
            for (int q = 0; q < 32; ++q) ACC[q * 128 + tid] = aW2[q];
#pragma unroll
            for (int q = 0; q < 8; ++q) ACC[(32 + q) * 128 + tid] = aW1[q];
            ACC[40 * 128 + tid] = aW3[0];
            ACC[41 * 128 + tid] = aW3[1];
            ACC[42 * 128 + tid] = aB;
            ACC[43 * 128 + tid] = aB3;
        }
        __syncthreads();
    }
    // ---- flush the CTA's sums
    unsigned long long *G = reinterpret_cast<unsigned long long *>(g.grad);
#pragma unroll 4
    for (int q = 0; q < 32; ++q) atomicAdd(G + kOffW2 + j2 * 64 + i2 + q, (unsigned long long)to_fix(ACC[q * 128 + tid]));
#pragma unroll
    for (int q = 0; q < 8; ++q)
        atomicAdd(G + kOffW1 + j2 * 16 + k1 + q, (unsigned long long)to_fix(ACC[(32 + q) * 128 + tid]));
    atomicAdd(G + kOffW3 + c3 * 64 + i3, (unsigned long long)to_fix(ACC[40 * 128 + tid]));
    atomicAdd(G + kOffW3 + c3 * 64 + i3 + 1, (unsigned long long)to_fix(ACC[41 * 128 + tid]));
    atomicAdd(G + (tid < 64 ? kOffB1 + tid : kOffB2 + tid - 64), (unsigned long long)to_fix(ACC[42 * 128 + tid]));
    if (tid < 4) atomicAdd(G + kOffB3 + tid, (unsigned long long)to_fix(ACC[43 * 128 + tid]));
    LS[tid] = loss;
    __syncthreads();
    if (tid == 0) {
        float tot = 0.f;
        for (int s = 0; s < kThreads; ++s) tot = __fadd_rn(tot, LS[s]);
        atomicAdd(reinterpret_cast<unsigned long long *>(g.loss), (unsigned long long)__double2ll_rn((double)tot * kLossFix));
    }
}

struct AdamParams {
    float *params, *m, *v;
    long long *grad;
    size_t n;
    float lr_w, lr_lat, beta1, beta2, eps;
    float bc1, bc2;  // 1 - beta^t
};

__global__ void adam_kernel(const AdamParams a) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < a.n; i += (size_t)gridDim.x * blockDim.x) {
        if (i >= (size_t)kWeights && i < (size_t)kOffLat) continue;
        const long long gi = a.grad[i];
        a.grad[i] = 0;
        const float gr = (float)((double)gi / kFix);
        const float m = __fmaf_rn(a.beta1, a.m[i], __fmul_rn(1.f - a.beta1, gr));
        const float v = __fmaf_rn(a.beta2, a.v[i], __fmul_rn(1.f - a.beta2, __fmul_rn(gr, gr)));
        a.m[i] = m;
        a.v[i] = v;
        const float mh = __fdiv_rn(m, a.bc1), vh = __fdiv_rn(v, a.bc2);
        const float lr = i < (size_t)kWeights ? a.lr_w : a.lr_lat;
        a.params[i] = __fsub_rn(a.params[i], __fdiv_rn(__fmul_rn(lr, mh), __fadd_rn(__fsqrt_rn(vh), a.eps)));
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
    g.step = 0;
    g.k0 = (uint32_t)(t->desc.seed & 0xffffffffu);
    g.k1 = (uint32_t)(t->desc.seed >> 32);
    g.dscale = 0.f;
    g.grad = t->grad;
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
    const int ctas = (g.n + kThreads * kRounds - 1) / (kThreads * kRounds);
    if (ctas == 0) return cudaSuccess;
    grad_kernel<<<ctas, kThreads, kGradSmem, s>>>(g);
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
    cudaFree(t->params);
    cudaFree(t->m);
    cudaFree(t->v);
    cudaFree(t->grad);
    cudaFree(t->loss);
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
    cudaError_t e = cudaMalloc(&t->params, t->nparams * 4);
    if (e == cudaSuccess) e = cudaMalloc(&t->m, t->nparams * 4);
    if (e == cudaSuccess) e = cudaMalloc(&t->v, t->nparams * 4);
    if (e == cudaSuccess) e = cudaMalloc(&t->grad, t->nparams * 8);
    if (e == cudaSuccess) e = cudaMalloc(&t->loss, 8);
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

uint64_t fnv1a(const void *data, size_t n, uint64_t h) {
    const unsigned char *b = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
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
        a.lr_w = (float)(t->desc.lr_weights * sched);
        a.lr_lat = (float)(t->desc.lr_latents * sched);
        a.bc1 = (float)(1.0 - std::pow((double)t->desc.beta1, (double)(st + 1)));
        a.bc2 = (float)(1.0 - std::pow((double)t->desc.beta2, (double)(st + 1)));
        if (e == cudaSuccess) {
            adam_kernel<<<2048, 256, 0, s>>>(a);
            e = cudaGetLastError();
        }
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
        cudaError_t e = cudaMalloc(&dmax, 144 * 4);
        if (e == cudaSuccess) e = cudaMemset(dmax, 0, 144 * 4);
        if (e == cudaSuccess) {
            GradParams g = grad_params(t);
            actstats_kernel<<<device_sm_count() * 4, kThreads>>>(g, dmax);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpy(amax.data(), dmax, 144 * 4, cudaMemcpyDeviceToHost);
        cudaFree(dmax);
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
    cudaError_t e = cudaMalloc(&xy, (size_t)chunk * 8);
    if (e == cudaSuccess) e = cudaMalloc(&dec, (size_t)chunk * 16);
    if (e == cudaSuccess) e = cudaMalloc(&sse, 8);
    if (e == cudaSuccess) e = cudaMalloc(&mx, 4);
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
    cudaFree(xy);
    cudaFree(dec);
    cudaFree(sse);
    cudaFree(mx);
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
