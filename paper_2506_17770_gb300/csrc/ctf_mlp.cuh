// ctf_mlp.cuh -- shared-memory layout and device parameters of the learned
// texel decode: a 16 -> 64 -> 64 -> 4 MLP (ReLU between layers) over the
// bilinear samples of two latent grids of 8 FP16 channels.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace ctf {

constexpr int kMlpCh = 8;       // channels per latent grid
constexpr int kMlpIn = 16;      // features = 2 grids x 8 channels
constexpr int kMlpHidden = 64;  // hidden width
constexpr int kMlpOut = 4;      // RGBA
constexpr int kMlpOut16 = 16;   // layer 3 padded to the smallest MMA width

// Operand image (the same bytes in global memory and in shared memory).
// Every matrix is stored K-major in 8-row x 16-byte core matrices:
// element (row r, k) at (r/8)*SBO + (k/8)*128 + (r%8)*16 + (k%8)*esize with
// SBO = (K/8)*128.  For FP16: W1 [64 x 16], W2 [64 x 64], W3 [16 x 64] (rows
// 4..15 zero); biases FP32.  For FP8 (E4M3, one byte per element, 16
// elements per core-matrix row): W1 [64 x 32] (K padded from 16), W2 and W3
// [.. x 64]; plus per-output-channel weight scales and per-input-channel
// activation scales.
constexpr int kImgW1 = 0;
constexpr int kImgW2 = 2048;
constexpr int kImgW3 = 2048 + 8192;
constexpr int kImgB1 = 12288;
constexpr int kImgB2 = kImgB1 + 256;
constexpr int kImgB3 = kImgB2 + 256;
// FP8 extras: output scales of layers 1..3 (64, 64, 16 floats) and the
// inverse activation scales of the inputs of layers 1..3 (32, 64, 64
// floats).  The output scales and biases of layers 1 and 2 are stored
// multiplied by the inverse activation scale of the next layer's input,
// which the hidden epilogues then need no more (layer 1's inputs, the
// features, are scaled by A1).
constexpr int kImgS1 = kImgB3 + 64;
constexpr int kImgS2 = kImgS1 + 256;
constexpr int kImgS3 = kImgS2 + 256;
constexpr int kImgA1 = kImgS3 + 64;
constexpr int kImgA2 = kImgA1 + 128;
constexpr int kImgA3 = kImgA2 + 256;
constexpr int kImgBytes = kImgA3 + 256;  // 14080

__host__ __device__ constexpr int core_offset(int r, int k, int K, int esize) {
    // 16-byte core-matrix rows hold 16/esize elements
    return (r / 8) * ((K * esize / 16) * 128) + (k * esize / 16) * 128 + (r % 8) * 16 + (k % (16 / esize)) * esize;
}

struct MlpDevice {
    const __half *lat[2];  // [gh][gw][8] FP16
    int gw[2], gh[2];
    float sx[2], sy[2];    // grid texels per texture texel
    const uint4 *img;      // operand image (kImgBytes)
    int fp8;               // 0: FP16 operands, 1: E4M3 operands
    int *err;              // device error word (index checks of the debug build)
};

}  // namespace ctf
