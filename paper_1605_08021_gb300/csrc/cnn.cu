// Learned initial guess for the 2D Sternheimer solves (Eq. eqncompressU and Alg. 1 solve
// Q(H - s)Q x = Q b; the Krylov iteration may start from any x0 in range(Q) and is refined to the
// same tolerance, so x0 changes iteration counts, not results).
//
// The guess is x0 = rms(r) net(r / rms(r), V_eff - s) for a right-hand side r and shift s, with
// a 4-layer periodic CNN: 3 x 3 cross-correlations with periodic wrap, channels 2 -> 32 -> 32 ->
// 32 -> 1, tanh after layers 1-3.  Weights are bfloat16 copies of an FP32 master set; activations
// and accumulation are FP32.
//
// Kernel: a persistent CTA per SM loads all weights into shared memory once, then walks over
// work items (16 x 16 output tile, column).  An item reads its 24 x 24 input tile (halo 4 = one
// point per layer, periodic), and runs the four layers on shared-memory tiles of 22^2, 20^2,
// 18^2 and 16^2 points, so the network is evaluated without any intermediate in device memory.
#include <cuda_bf16.h>

#include <mutex>

#include "cnn.cuh"

namespace acp {

namespace {

using namespace cnn;

constexpr int kT = 16;               // output tile edge
constexpr int kHalo = 4;             // one point per 3 x 3 layer
constexpr int kIn = kT + 2 * kHalo;  // 24
constexpr int kThreads = 256;

// shared memory: weights, biases, the input tile and two activation tiles
constexpr size_t kSmWeights = (size_t)kNumBf16 * 2;         // 38592 bytes
constexpr size_t kSmBias = 512;
constexpr size_t kSmIn = (size_t)2 * kIn * kIn * 4;         // 4608
constexpr size_t kSmA = (size_t)kC * 22 * 22 * 4;           // 61952 (layer 1 and 3 outputs)
constexpr size_t kSmB = (size_t)kC * 20 * 20 * 4;           // 51200 (layer 2 output)
constexpr size_t kSmemBytes = kSmWeights + kSmBias + kSmIn + kSmA + kSmB;
static_assert(kSmWeights % 16 == 0, "16-byte alignment of the bias block");

__global__ void cnn_pack_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb,
                                float* __restrict__ bias) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kNumWeights; e += gridDim.x * blockDim.x) {
    // decode e into (layer, o, c, tap) of the host layout, or a bias
    int base, cin, cout, off;
    if (e < kB1) { base = kW1; cin = 2; cout = kC; off = kO1; }
    else if (e < kW2) { bias[e - kB1] = w[e]; continue; }
    else if (e < kB2) { base = kW2; cin = kC; cout = kC; off = kO2; }
    else if (e < kW3) { bias[kC + e - kB2] = w[e]; continue; }
    else if (e < kB3) { base = kW3; cin = kC; cout = kC; off = kO3; }
    else if (e < kW4) { bias[2 * kC + e - kB3] = w[e]; continue; }
    else if (e < kB4) { base = kW4; cin = kC; cout = 1; off = kO4; }
    else { bias[3 * kC] = w[e]; continue; }
    const int r = e - base;
    const int tap = r % 9, c = (r / 9) % cin, o = r / (9 * cin);
    wb[off + (c * 9 + tap) * cout + o] = __float2bfloat16_rn(w[e]);
  }
}

// rms[j] = sqrt(mean_a R[a, j]^2), one CTA per column
__global__ void col_rms_kernel(int N, const double* __restrict__ R, int ldr, double* __restrict__ rms) {
  __shared__ double red[32];
  const double* r = R + (size_t)blockIdx.x * ldr;
  double s = 0.0;
  for (int a = threadIdx.x; a < N; a += blockDim.x) s += r[a] * r[a];
  s = block_sum(s, red);
  if (threadIdx.x == 0) rms[blockIdx.x] = sqrt(s / N);
}

__device__ __forceinline__ float bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }

// One 3 x 3 layer on shared-memory tiles: in [CIN][win][win] -> out [32][win-2][win-2].
template <int CIN>
__device__ __forceinline__ void conv_layer32(const float* __restrict__ in, int win, float* __restrict__ out,
                                             const __nv_bfloat16* __restrict__ w, const float* __restrict__ b) {
  const int wout = win - 2, npts = wout * wout;
  for (int pt = threadIdx.x; pt < npts; pt += blockDim.x) {
    const int y = pt / wout, x = pt - y * wout;
    float acc[kC];
#pragma unroll
    for (int o = 0; o < kC; ++o) acc[o] = b[o];
    for (int c = 0; c < CIN; ++c) {
      const float* ic = in + c * win * win + y * win + x;
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const float a = ic[(tap / 3) * win + (tap % 3)];
        const uint4* w4 = reinterpret_cast<const uint4*>(w + (c * 9 + tap) * kC);
#pragma unroll
        for (int v = 0; v < kC / 8; ++v) {
          const uint4 u = w4[v];
          acc[8 * v + 0] = fmaf(bf16_lo(u.x), a, acc[8 * v + 0]);
          acc[8 * v + 1] = fmaf(bf16_hi(u.x), a, acc[8 * v + 1]);
          acc[8 * v + 2] = fmaf(bf16_lo(u.y), a, acc[8 * v + 2]);
          acc[8 * v + 3] = fmaf(bf16_hi(u.y), a, acc[8 * v + 3]);
          acc[8 * v + 4] = fmaf(bf16_lo(u.z), a, acc[8 * v + 4]);
          acc[8 * v + 5] = fmaf(bf16_hi(u.z), a, acc[8 * v + 5]);
          acc[8 * v + 6] = fmaf(bf16_lo(u.w), a, acc[8 * v + 6]);
          acc[8 * v + 7] = fmaf(bf16_hi(u.w), a, acc[8 * v + 7]);
        }
      }
    }
#pragma unroll
    for (int o = 0; o < kC; ++o) out[o * npts + pt] = tanhf(acc[o]);
  }
}

__global__ void __launch_bounds__(kThreads, 1)
    cnn_x0_kernel(int nx, int ny, int ncol, const double* __restrict__ R, int ldr, const double* __restrict__ V,
                  const double* __restrict__ shift, const double* __restrict__ rms,
                  const __nv_bfloat16* __restrict__ wb, const float* __restrict__ bias, double* __restrict__ X0,
                  int ldx) {
  extern __shared__ __align__(16) uint8_t cnn_smem[];
  __nv_bfloat16* wsm = reinterpret_cast<__nv_bfloat16*>(cnn_smem);
  float* bsm = reinterpret_cast<float*>(cnn_smem + kSmWeights);
  float* tin = reinterpret_cast<float*>(cnn_smem + kSmWeights + kSmBias);
  float* A = reinterpret_cast<float*>(cnn_smem + kSmWeights + kSmBias + kSmIn);
  float* B = reinterpret_cast<float*>(cnn_smem + kSmWeights + kSmBias + kSmIn + kSmA);
  {
    const uint4* src = reinterpret_cast<const uint4*>(wb);
    uint4* dst = reinterpret_cast<uint4*>(wsm);
    for (int e = threadIdx.x; e < (int)(kSmWeights / 16); e += blockDim.x) dst[e] = src[e];
    for (int e = threadIdx.x; e < kNumBias; e += blockDim.x) bsm[e] = bias[e];
  }
  __syncthreads();
  const int tiles_x = (nx + kT - 1) / kT, tiles_y = (ny + kT - 1) / kT;
  const long long per_col = (long long)tiles_x * tiles_y;
  const long long total = per_col * ncol;
  for (long long item = blockIdx.x; item < total; item += gridDim.x) {
    const int col = (int)(item / per_col);
    const int t = (int)(item - (long long)col * per_col);
    const int ty = t / tiles_x, tx = t - ty * tiles_x;
    const double s = rms[col];
    double* xo = X0 + (size_t)col * ldx;
    if (!(s > 0.0)) {  // zero right-hand side (uniform over the CTA): x0 = 0
      for (int pt = threadIdx.x; pt < kT * kT; pt += blockDim.x) {
        const int gy = ty * kT + pt / kT, gx = tx * kT + pt % kT;
        if (gy < ny && gx < nx) xo[(size_t)gy * nx + gx] = 0.0;
      }
      continue;
    }
    const double sh = shift[col];
    const double* r = R + (size_t)col * ldr;
    for (int e = threadIdx.x; e < kIn * kIn; e += blockDim.x) {
      const int yy = e / kIn, xx = e - yy * kIn;
      int gy = (ty * kT - kHalo + yy) % ny;
      int gx = (tx * kT - kHalo + xx) % nx;
      if (gy < 0) gy += ny;
      if (gx < 0) gx += nx;
      const size_t g = (size_t)gy * nx + gx;
      tin[e] = (float)(r[g] / s);
      tin[kIn * kIn + e] = (float)(V[g] - sh);
    }
    __syncthreads();
    conv_layer32<2>(tin, kIn, A, wsm + kO1, bsm);
    __syncthreads();
    conv_layer32<kC>(A, kIn - 2, B, wsm + kO2, bsm + kC);
    __syncthreads();
    conv_layer32<kC>(B, kIn - 4, A, wsm + kO3, bsm + 2 * kC);
    __syncthreads();
    // layer 4 (one output channel, no activation) straight to device memory
    {
      const int win = kIn - 6;  // 18
      for (int pt = threadIdx.x; pt < kT * kT; pt += blockDim.x) {
        const int y = pt / kT, x = pt - y * kT;
        float acc = bsm[3 * kC];
        for (int c = 0; c < kC; ++c) {
          const float* ic = A + c * win * win + y * win + x;
#pragma unroll
          for (int tap = 0; tap < 9; ++tap)
            acc = fmaf(__bfloat162float(wsm[kO4 + c * 9 + tap]), ic[(tap / 3) * win + (tap % 3)], acc);
        }
        const int gy = ty * kT + y, gx = tx * kT + x;
        if (gy < ny && gx < nx) xo[(size_t)gy * nx + gx] = s * (double)acc;
      }
    }
    __syncthreads();
  }
}

}  // namespace

// bfloat16 copies and FP32 biases from the FP32 master weights in the workspace
acp_status cnn_repack(acp_ctx* ctx) {
  float* w32 = nullptr;
  __nv_bfloat16* wb = nullptr;
  float* bias = nullptr;
  ACP_TRY(ws(ctx, "cnn_w32", (size_t)kNumWeights, &w32));
  ACP_TRY(ws(ctx, "cnn_bf16", (size_t)kNumBf16, &wb));
  ACP_TRY(ws(ctx, "cnn_bias", (size_t)kNumBias, &bias));
  ::acp::note_launch(ctx);
  cnn_pack_kernel<<<(kNumWeights + 255) / 256, 256, 0, ctx->stream>>>(w32, wb, bias);
  ACP_LAUNCH(ctx);
  return ACP_OK;
}

acp_status cnn_col_rms(acp_ctx* ctx, int N, const double* R, int ldr, int ncol, double* rms) {
  if (ncol <= 0) return ACP_OK;
  ::acp::note_launch(ctx);
  col_rms_kernel<<<ncol, 256, 0, ctx->stream>>>(N, R, ldr, rms);
  ACP_LAUNCH(ctx);
  return ACP_OK;
}

acp_status cnn_set_weights(acp_ctx* ctx, const float* w_h) {
  float *w32 = nullptr, *m = nullptr, *v = nullptr;
  ACP_TRY(ws(ctx, "cnn_w32", (size_t)kNumWeights, &w32));
  ACP_TRY(ws(ctx, "cnn_adam_m", (size_t)kNumWeights, &m));
  ACP_TRY(ws(ctx, "cnn_adam_v", (size_t)kNumWeights, &v));
  ACP_CUDA(ctx, cudaMemcpyAsync(w32, w_h, sizeof(float) * kNumWeights, cudaMemcpyHostToDevice, ctx->stream));
  ACP_CUDA(ctx, cudaMemsetAsync(m, 0, sizeof(float) * kNumWeights, ctx->stream));
  ACP_CUDA(ctx, cudaMemsetAsync(v, 0, sizeof(float) * kNumWeights, ctx->stream));
  ACP_TRY(cnn_repack(ctx));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // the host buffer may go away
  ctx->cnn_ready = true;
  ctx->cnn_steps = 0;
  return ACP_OK;
}

acp_status cnn_initial_guess(acp_ctx* ctx, const double* R, int ldr, int ncol, const double* shift_d, double* X0,
                             int ldx) {
  if (ncol <= 0) return ACP_OK;
  if (ctx->dim != 2) return set_error(ctx, ACP_E_ARG, "the learned initial guess is defined on 2D grids");
  if (!ctx->cnn_ready) return set_error(ctx, ACP_E_ARG, "no network weights (acp_cnn_set_weights)");
  __nv_bfloat16* wb = nullptr;
  float* bias = nullptr;
  double* rms = nullptr;
  ACP_TRY(ws(ctx, "cnn_bf16", (size_t)kNumBf16, &wb));
  ACP_TRY(ws(ctx, "cnn_bias", (size_t)kNumBias, &bias));
  ACP_TRY(ws(ctx, "cnn_rms", (size_t)ncol, &rms));
  static int sm_count[64] = {};
  {
    // the kernel's dynamic shared memory (157 KB) is set once per device, as is the SM count
    std::lock_guard<std::mutex> lock(device_mutex());
    if (ctx->device < 0 || ctx->device >= 64) return set_error(ctx, ACP_E_ARG, "device ordinal out of range");
    if (sm_count[ctx->device] == 0) {
      if ((size_t)ctx->smem_optin < kSmemBytes)
        return set_error(ctx, ACP_E_ARG, "the device allows %zu bytes of shared memory per CTA, the network needs %zu",
                         (size_t)ctx->smem_optin, kSmemBytes);
      ACP_CUDA(ctx, cudaFuncSetAttribute(cnn_x0_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
      int n = 0;
      ACP_CUDA(ctx, cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, ctx->device));
      sm_count[ctx->device] = n > 0 ? n : 1;
    }
  }
  ACP_TRY(cnn_col_rms(ctx, ctx->N, R, ldr, ncol, rms));
  const long long items = (long long)((ctx->nx + kT - 1) / kT) * ((ctx->ny + kT - 1) / kT) * ncol;
  const int blocks = (int)std::min<long long>(items, sm_count[ctx->device]);
  ::acp::note_launch(ctx);
  cnn_x0_kernel<<<blocks, kThreads, kSmemBytes, ctx->stream>>>(ctx->nx, ctx->ny, ncol, R, ldr, ctx->d_V, shift_d,
                                                               rms, wb, bias, X0, ldx);
  ACP_LAUNCH(ctx);
  return ACP_OK;
}

}  // namespace acp
