// Shapes and packed layouts of the learned initial guess (4-layer periodic CNN, 3 x 3 kernels,
// channels 2 -> 32 -> 32 -> 32 -> 1), shared by the inference and training kernels.
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"

namespace acp {
namespace cnn {

constexpr int kC = 32;  // hidden channels

// packed FP32 weights (the host layout of acp_cnn_set_weights): W1 (32,2,3,3), b1 (32),
// W2 (32,32,3,3), b2, W3 (32,32,3,3), b3, W4 (1,32,3,3), b4 (1), each row-major (output channel,
// input channel, dy + 1, dx + 1)
constexpr int kW1 = 0, kB1 = kW1 + kC * 2 * 9, kW2 = kB1 + kC, kB2 = kW2 + kC * kC * 9, kW3 = kB2 + kC,
              kB3 = kW3 + kC * kC * 9, kW4 = kB3 + kC, kB4 = kW4 + kC * 9, kNumWeights = kB4 + 1;
static_assert(kNumWeights == ACP_CNN_WEIGHTS, "weight count of the header");

// bfloat16 copies for inference: per layer [input channel][tap][output channel] (output channel
// fastest, so a thread reads the 32 weights of one tap with four 16-byte loads)
constexpr int kO1 = 0, kO2 = kO1 + 2 * 9 * kC, kO3 = kO2 + kC * 9 * kC, kO4 = kO3 + kC * 9 * kC,
              kNumBf16 = kO4 + kC * 9;
constexpr int kNumBias = 3 * kC + 1;

// layer l (0-based): input channels, output channels, offset of W and b in the packed layout
__host__ __device__ constexpr int cin_of(int l) { return l == 0 ? 2 : kC; }
__host__ __device__ constexpr int cout_of(int l) { return l == 3 ? 1 : kC; }
__host__ __device__ constexpr int w_off(int l) { return l == 0 ? kW1 : l == 1 ? kW2 : l == 2 ? kW3 : kW4; }
__host__ __device__ constexpr int b_off(int l) { return l == 0 ? kB1 : l == 1 ? kB2 : l == 2 ? kB3 : kB4; }

}  // namespace cnn

// cnn.cu: rebuild the bfloat16 copies from the FP32 master weights; per-column RMS of an N-row
// block
acp_status cnn_repack(acp_ctx* ctx);
acp_status cnn_col_rms(acp_ctx* ctx, int N, const double* R, int ldr, int ncol, double* rms);

}  // namespace acp
