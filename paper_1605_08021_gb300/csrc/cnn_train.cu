// Training of the learned initial guess: forward pass with stored activations, the loss
// mean_s ||x0_s - x*_s||^2 / ||x*_s||^2 over solved samples, the backward pass of the 4-layer
// periodic CNN, and one Adam step (Kingma and Ba, 2015) on the FP32 master weights, after which
// the bfloat16 inference copies are rebuilt.
//
// Training computes with the FP32 master weights (inference convolves with their bfloat16
// roundings).  A batch lives on its own nx x ny grid and carries its shifted potentials V - s per
// sample, so one context (weights and Adam state) trains on systems of any grid.  Activations
// are stored per layer as [sample][channel][grid point] in FP32; every kernel indexes the
// periodic 3 x 3 neighbourhood of its grid point directly (no tiling constraints on the grid).
//
// Layer l: z = b + sum_c W[o, c, p+1, q+1] a[c, y+p, x+q] (periodic), a_next = tanh(z) for l < 3.
//   dL/da[c, y, x] = sum_{o,p,q} W[o, c, p+1, q+1] g[o, y-p, x-q]
//   dL/dW[o, c, p+1, q+1] = sum_{s,y,x} g[s, o, y, x] a[s, c, y+p, x+q],  dL/db[o] = sum g[s, o, y, x]
// with g = dL/dz, and dL/dz = dL/da (1 - a^2) through tanh.
#include "cnn.cuh"

namespace acp {

namespace {

using namespace cnn;

constexpr int kThreads = 256;

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// a0[s] = (R_s / rms_s, VS_s) as FP32 (channel 0 is zero for a zero sample)
__global__ void train_inputs_kernel(int N, const double* __restrict__ R, const double* __restrict__ VS,
                                    const double* __restrict__ rms, float* __restrict__ a0) {
  const int s = blockIdx.y;
  const double rs = rms[s];
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    a0[((size_t)s * 2 + 0) * N + a] = rs > 0.0 ? (float)(R[(size_t)s * N + a] / rs) : 0.f;
    a0[((size_t)s * 2 + 1) * N + a] = (float)VS[(size_t)s * N + a];
  }
}

// out[s][o][pt] = act(b[o] + sum_c sum_tap W[o, c, tap] in[s][c][pt + offset(tap)])
template <int COUT, bool ACT>
__global__ void __launch_bounds__(kThreads) train_fwd_kernel(int nx, int ny, int cin, const float* __restrict__ W,
                                                             const float* __restrict__ b, const float* __restrict__ in,
                                                             float* __restrict__ out) {
  const int N = nx * ny, s = blockIdx.y;
  const int pt = blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= N) return;
  const int y = pt / nx, x = pt - y * nx;
  int nb[9];
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) nb[tap] = wrap(y + tap / 3 - 1, ny) * nx + wrap(x + tap % 3 - 1, nx);
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = b[o];
  for (int c = 0; c < cin; ++c) {
    const float* ic = in + ((size_t)s * cin + c) * N;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const float a = ic[nb[tap]];
#pragma unroll
      for (int o = 0; o < COUT; ++o) acc[o] = fmaf(W[(o * cin + c) * 9 + tap], a, acc[o]);
    }
  }
#pragma unroll
  for (int o = 0; o < COUT; ++o) out[((size_t)s * COUT + o) * N + pt] = ACT ? tanhf(acc[o]) : acc[o];
}

// loss_s = ||rms_s z4_s - x*_s||^2 / ||x*_s||^2 / S and g4_s = rms_s * 2 (rms_s z4_s - x*_s) /
// (||x*_s||^2 S); one CTA per sample (a zero sample has x0 = 0 and no gradient)
__global__ void train_loss_kernel(int N, int S, const float* __restrict__ z4, const double* __restrict__ rms,
                                  const double* __restrict__ Xs, double* __restrict__ loss, float* __restrict__ g4) {
  __shared__ double red[32];
  const int s = blockIdx.x;
  const double rs = rms[s];
  const double* xs = Xs + (size_t)s * N;
  const float* z = z4 + (size_t)s * N;
  double d2 = 0.0, n2 = 0.0;
  for (int a = threadIdx.x; a < N; a += blockDim.x) {
    const double x0 = rs > 0.0 ? rs * (double)z[a] : 0.0;
    const double d = x0 - xs[a];
    d2 += d * d;
    n2 += xs[a] * xs[a];
  }
  d2 = block_sum(d2, red);
  n2 = block_sum(n2, red);
  const double sc = n2 > 0.0 ? 1.0 / (n2 * S) : 0.0;
  if (threadIdx.x == 0) loss[s] = d2 * sc;
  for (int a = threadIdx.x; a < N; a += blockDim.x) {
    const double x0 = rs > 0.0 ? rs * (double)z[a] : 0.0;
    g4[(size_t)s * N + a] = rs > 0.0 ? (float)(rs * 2.0 * (x0 - xs[a]) * sc) : 0.f;
  }
}

// gin[s][c][pt] = (sum_o sum_tap W[o, c, tap] g[s][o][pt - offset(tap)]) (1 - ain[s][c][pt]^2)
template <int COUT>
__global__ void __launch_bounds__(kThreads) train_bwd_data_kernel(int nx, int ny, const float* __restrict__ W,
                                                                  const float* __restrict__ g,
                                                                  const float* __restrict__ ain,
                                                                  float* __restrict__ gin) {
  constexpr int CIN = kC;
  const int N = nx * ny, s = blockIdx.y;
  const int pt = blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= N) return;
  const int y = pt / nx, x = pt - y * nx;
  int nb[9];  // the point that reads this one through tap (y - p, x - q)
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) nb[tap] = wrap(y - (tap / 3 - 1), ny) * nx + wrap(x - (tap % 3 - 1), nx);
  float acc[CIN];
#pragma unroll
  for (int c = 0; c < CIN; ++c) acc[c] = 0.f;
  for (int o = 0; o < COUT; ++o) {
    const float* go = g + ((size_t)s * COUT + o) * N;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const float gv = go[nb[tap]];
#pragma unroll
      for (int c = 0; c < CIN; ++c) acc[c] = fmaf(W[(o * CIN + c) * 9 + tap], gv, acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < CIN; ++c) {
    const float a = ain[((size_t)s * CIN + c) * N + pt];
    gin[((size_t)s * CIN + c) * N + pt] = acc[c] * (1.f - a * a);
  }
}

// one CTA per (input channel c, output channel o): dW[o, c, 0..8] over all samples and points,
// and db[o] in the CTAs of c = 0 (FP64 sums)
__global__ void __launch_bounds__(kThreads) train_bwd_weight_kernel(int nx, int ny, int S, int cin, int cout,
                                                                    const float* __restrict__ g,
                                                                    const float* __restrict__ ain,
                                                                    float* __restrict__ dW, float* __restrict__ db) {
  __shared__ double red[32];
  const int c = blockIdx.x, o = blockIdx.y;
  const int N = nx * ny;
  double acc[9], accb = 0.0;
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) acc[tap] = 0.0;
  const long long total = (long long)S * N;
  for (long long e = threadIdx.x; e < total; e += blockDim.x) {
    const int s = (int)(e / N), pt = (int)(e - (long long)s * N);
    const int y = pt / nx, x = pt - y * nx;
    const double gv = g[((size_t)s * cout + o) * N + pt];
    const float* ac = ain + ((size_t)s * cin + c) * N;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap)
      acc[tap] += gv * (double)ac[wrap(y + tap / 3 - 1, ny) * nx + wrap(x + tap % 3 - 1, nx)];
    accb += gv;
  }
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const double t = block_sum(acc[tap], red);
    if (threadIdx.x == 0) dW[(o * cin + c) * 9 + tap] = (float)t;
  }
  if (c == 0) {
    const double t = block_sum(accb, red);
    if (threadIdx.x == 0) db[o] = (float)t;
  }
}

__global__ void adam_kernel(int n, float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace

acp_status cnn_train_step(acp_ctx* ctx, int nx, int ny, const double* R, const double* VS, const double* Xs, int S,
                          float lr, double* loss_h, float* grad_h) {
  if (!ctx->cnn_ready) return set_error(ctx, ACP_E_ARG, "no network weights (acp_cnn_set_weights)");
  if (S < 1 || S > 65535) return set_error(ctx, ACP_E_ARG, "nsamp %d outside [1, 65535]", S);
  if (nx < 3 || ny < 3 || (long long)nx * ny > (1LL << 26))
    return set_error(ctx, ACP_E_ARG, "training grid %d x %d outside [3, ...] with nx ny <= 2^26", nx, ny);
  const int N = nx * ny;
  const size_t hid = (size_t)S * kC * N;
  float *w = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  float *a0 = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *z4 = nullptr, *gA = nullptr, *gB = nullptr;
  double *rms = nullptr, *loss = nullptr;
  ACP_TRY(ws(ctx, "cnn_w32", (size_t)kNumWeights, &w));
  ACP_TRY(ws(ctx, "cnn_adam_m", (size_t)kNumWeights, &m));
  ACP_TRY(ws(ctx, "cnn_adam_v", (size_t)kNumWeights, &v));
  ACP_TRY(ws(ctx, "cnn_grad", (size_t)kNumWeights, &grad));
  ACP_TRY(ws(ctx, "cnn_a0", (size_t)S * 2 * N, &a0));
  ACP_TRY(ws(ctx, "cnn_a1", hid, &a1));
  ACP_TRY(ws(ctx, "cnn_a2", hid, &a2));
  ACP_TRY(ws(ctx, "cnn_a3", hid, &a3));
  ACP_TRY(ws(ctx, "cnn_z4", (size_t)S * N, &z4));
  ACP_TRY(ws(ctx, "cnn_gA", hid, &gA));
  ACP_TRY(ws(ctx, "cnn_gB", hid, &gB));
  ACP_TRY(ws(ctx, "cnn_trms", (size_t)S, &rms));
  ACP_TRY(ws(ctx, "cnn_loss", (size_t)S, &loss));
  cudaStream_t st = ctx->stream;
  const dim3 pts((N + kThreads - 1) / kThreads, S);
  ACP_TRY(cnn_col_rms(ctx, N, R, N, S, rms));
  ::acp::note_launch(ctx);
  train_inputs_kernel<<<dim3((N + 255) / 256, S), 256, 0, st>>>(N, R, VS, rms, a0);
  ACP_LAUNCH(ctx);
  // forward
  ::acp::note_launch(ctx);
  train_fwd_kernel<kC, true><<<pts, kThreads, 0, st>>>(nx, ny, 2, w + kW1, w + kB1, a0, a1);
  ACP_LAUNCH(ctx);
  ::acp::note_launch(ctx);
  train_fwd_kernel<kC, true><<<pts, kThreads, 0, st>>>(nx, ny, kC, w + kW2, w + kB2, a1, a2);
  ACP_LAUNCH(ctx);
  ::acp::note_launch(ctx);
  train_fwd_kernel<kC, true><<<pts, kThreads, 0, st>>>(nx, ny, kC, w + kW3, w + kB3, a2, a3);
  ACP_LAUNCH(ctx);
  ::acp::note_launch(ctx);
  train_fwd_kernel<1, false><<<pts, kThreads, 0, st>>>(nx, ny, kC, w + kW4, w + kB4, a3, z4);
  ACP_LAUNCH(ctx);
  // loss and dL/dz4
  ::acp::note_launch(ctx);
  train_loss_kernel<<<S, 256, 0, st>>>(N, S, z4, rms, Xs, loss, gB);
  ACP_LAUNCH(ctx);
  // layer 4: weights from (g4, a3); g3 = (W4^T g4) (1 - a3^2)
  ::acp::note_launch(ctx);
  train_bwd_weight_kernel<<<dim3(kC, 1), kThreads, 0, st>>>(nx, ny, S, kC, 1, gB, a3, grad + kW4, grad + kB4);
  ACP_LAUNCH(ctx);
  ::acp::note_launch(ctx);
  train_bwd_data_kernel<1><<<pts, kThreads, 0, st>>>(nx, ny, w + kW4, gB, a3, gA);
  ACP_LAUNCH(ctx);
  // layer 3: weights from (g3, a2); g2 = (W3^T g3) (1 - a2^2)
  ::acp::note_launch(ctx);
  train_bwd_weight_kernel<<<dim3(kC, kC), kThreads, 0, st>>>(nx, ny, S, kC, kC, gA, a2, grad + kW3, grad + kB3);
  ACP_LAUNCH(ctx);
  ::acp::note_launch(ctx);
  train_bwd_data_kernel<kC><<<pts, kThreads, 0, st>>>(nx, ny, w + kW3, gA, a2, gB);
  ACP_LAUNCH(ctx);
  // layer 2: weights from (g2, a1); g1 = (W2^T g2) (1 - a1^2)
  ::acp::note_launch(ctx);
  train_bwd_weight_kernel<<<dim3(kC, kC), kThreads, 0, st>>>(nx, ny, S, kC, kC, gB, a1, grad + kW2, grad + kB2);
  ACP_LAUNCH(ctx);
  ::acp::note_launch(ctx);
  train_bwd_data_kernel<kC><<<pts, kThreads, 0, st>>>(nx, ny, w + kW2, gB, a1, gA);
  ACP_LAUNCH(ctx);
  // layer 1: weights from (g1, a0)
  ::acp::note_launch(ctx);
  train_bwd_weight_kernel<<<dim3(2, kC), kThreads, 0, st>>>(nx, ny, S, 2, kC, gA, a0, grad + kW1, grad + kB1);
  ACP_LAUNCH(ctx);
  // loss before the step, gradient (optional)
  std::vector<double> lh(S);
  ACP_CUDA(ctx, cudaMemcpyAsync(lh.data(), loss, sizeof(double) * S, cudaMemcpyDeviceToHost, st));
  if (grad_h) ACP_CUDA(ctx, cudaMemcpyAsync(grad_h, grad, sizeof(float) * kNumWeights, cudaMemcpyDeviceToHost, st));
  // Adam with the published defaults, bias corrections from the step count
  // (the bias corrections use the same FP32 betas as the moment updates)
  const float b1 = 0.9f, b2 = 0.999f;
  const long long t = ++ctx->cnn_steps;
  const float c1 = (float)(1.0 - std::pow((double)b1, (double)t)), c2 = (float)(1.0 - std::pow((double)b2, (double)t));
  ::acp::note_launch(ctx);
  adam_kernel<<<(kNumWeights + 255) / 256, 256, 0, st>>>(kNumWeights, w, m, v, grad, lr, b1, b2, 1e-8f, c1, c2);
  ACP_LAUNCH(ctx);
  ACP_TRY(cnn_repack(ctx));
  ACP_CUDA(ctx, cudaStreamSynchronize(st));
  double sum = 0.0;
  for (double x : lh) sum += x;
  if (loss_h) *loss_h = sum;
  return ACP_OK;
}

}  // namespace acp
