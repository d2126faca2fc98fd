// FP32 form of the spectral Hamiltonian for the mixed-precision Sternheimer solves: the kinetic
// term of H (Eq. Hamil) by a shared-memory Stockham FFT in single precision, the local potential
// and the shift, fused with the Lanczos three-term recurrence.
//
// Layout: FP32 blocks of grid functions with leading dimension ld (>= N, a multiple of 32, the
// padding stays zero).  One CTA owns a pair of columns packed as z = x0 + i x1 (the kinetic
// symbol is real and even, so the two halves stay separate), which lets the CTA finish the
// Lanczos coefficient alpha = v . (H - s) v itself.
#include "internal.cuh"

namespace acp {

namespace {

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 caddf(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csubf(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscalef(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cimulf(float2 a, float s) { return make_float2(-a.y * s, a.x * s); }

template <int R>
__device__ __forceinline__ void dftf(float2 (&a)[R], float dir);

template <>
__device__ __forceinline__ void dftf<2>(float2 (&a)[2], float) {
  const float2 t = a[0];
  a[0] = caddf(t, a[1]);
  a[1] = csubf(t, a[1]);
}

template <>
__device__ __forceinline__ void dftf<4>(float2 (&a)[4], float dir) {
  const float2 s02 = caddf(a[0], a[2]), d02 = csubf(a[0], a[2]);
  const float2 s13 = caddf(a[1], a[3]), d13 = cimulf(csubf(a[1], a[3]), dir);
  a[0] = caddf(s02, s13);
  a[2] = csubf(s02, s13);
  a[1] = caddf(d02, d13);
  a[3] = csubf(d02, d13);
}

template <>
__device__ __forceinline__ void dftf<3>(float2 (&a)[3], float dir) {
  const float c = -0.5f, s = 0.866025403784438647f;
  const float2 t1 = caddf(a[1], a[2]), t2 = cimulf(csubf(a[1], a[2]), dir * s);
  const float2 m = caddf(a[0], cscalef(t1, c));
  a[0] = caddf(a[0], t1);
  a[1] = caddf(m, t2);
  a[2] = csubf(m, t2);
}

template <>
__device__ __forceinline__ void dftf<5>(float2 (&a)[5], float dir) {
  const float c1 = 0.309016994374947424f, s1 = 0.951056516295153572f;
  const float c2 = -0.809016994374947424f, s2 = 0.587785252292473129f;
  const float2 t1 = caddf(a[1], a[4]), t2 = caddf(a[2], a[3]);
  const float2 d1 = csubf(a[1], a[4]), d2 = csubf(a[2], a[3]);
  const float2 m1 = caddf(a[0], caddf(cscalef(t1, c1), cscalef(t2, c2)));
  const float2 m2 = caddf(a[0], caddf(cscalef(t1, c2), cscalef(t2, c1)));
  const float2 e1 = cimulf(caddf(cscalef(d1, s1), cscalef(d2, s2)), dir);
  const float2 e2 = cimulf(csubf(cscalef(d1, s2), cscalef(d2, s1)), dir);
  a[0] = caddf(a[0], caddf(t1, t2));
  a[1] = caddf(m1, e1);
  a[4] = csubf(m1, e1);
  a[2] = caddf(m2, e2);
  a[3] = csubf(m2, e2);
}

template <int R, bool Wide> struct MaxBf;
template <bool W> struct MaxBf<2, W> { static constexpr int v = W ? 5 : 4; };
template <bool W> struct MaxBf<3, W> { static constexpr int v = 4; };
template <bool W> struct MaxBf<4, W> { static constexpr int v = 3; };
template <bool W> struct MaxBf<5, W> { static constexpr int v = 2; };

template <int R, bool Wide>
__device__ __forceinline__ void fft_stage_f(float2* s, int N, int Ns, const float2* __restrict__ tw, float dir) {
  constexpr int B = MaxBf<R, Wide>::v;
  const int nb = N / R;
  const int stride = N / (Ns * R);
  float2 a[B][R];
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = threadIdx.x + b * blockDim.x;
    if (j < nb) {
#pragma unroll
      for (int r = 0; r < R; ++r) a[b][r] = s[j + r * nb];
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = threadIdx.x + b * blockDim.x;
    if (j < nb) {
      const int k = j % Ns;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = __ldg(&tw[r * k * stride]);
        if (dir > 0) w.y = -w.y;
        a[b][r] = cmulf(a[b][r], w);
      }
      dftf<R>(a[b], dir);
      const int base = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) s[base + r * Ns] = a[b][r];
    }
  }
  __syncthreads();
}

struct PlanArgF {
  int n, nst;
  int rad[24];
};

template <bool Wide>
__device__ void fft_f(float2* s, const PlanArgF& p, const float2* __restrict__ tw, float dir) {
  int Ns = 1;
  for (int st = 0; st < p.nst; ++st) {
    switch (p.rad[st]) {
      case 4: fft_stage_f<4, Wide>(s, p.n, Ns, tw, dir); break;
      case 2: fft_stage_f<2, Wide>(s, p.n, Ns, tw, dir); break;
      case 3: fft_stage_f<3, Wide>(s, p.n, Ns, tw, dir); break;
      default: fft_stage_f<5, Wide>(s, p.n, Ns, tw, dir); break;
    }
    Ns *= p.rad[st];
  }
}

__device__ __forceinline__ float block_sum_f(float v, float* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  float t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.f;
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[0] = t;
  }
  __syncthreads();
  const float r = red[0];
  __syncthreads();
  return r;
}

constexpr int kMaxThreads = 512;
constexpr int kMaxThreadsWide = 1024;  // grids beyond the 512-thread plan (see the FP64 kernels)

// P = (H - s_j) x_j - alpha_j x_j - beta_j xp_j with alpha_j = x_j . (H - s_j) x_j (Lanczos form,
// xp != nullptr), or Y = (H - s_j) x_j.  shift (nullable) per column; active (nullable) masks
// columns; alpha (nullable) receives the coefficients.
// Two CTAs per SM (64 registers per thread, a few spilled): the FFT stages wait on shared and L1
// loads behind CTA barriers, and a second resident CTA hides them (33% faster than one CTA of
// 120 registers on the 64-atom chain).  The wide form runs one CTA of up to 1024 threads per SM,
// with the same 64 registers per thread.
template <bool Wide>
__global__ void __launch_bounds__(Wide ? kMaxThreadsWide : kMaxThreads, Wide ? 1 : 2)
    spectral32_kernel(const float* __restrict__ X, int ldx, int ncol, PlanArgF plan, const float2* __restrict__ tw,
                      const float* __restrict__ kin, const float* __restrict__ V, const float* __restrict__ shift,
                      float* __restrict__ Y, int ldy, float* __restrict__ alpha, const int* __restrict__ active,
                      const float* __restrict__ Xp, int ldp, const float* __restrict__ beta,
                      const int* __restrict__ kdev, long long kstride) {
  extern __shared__ float2 sbuf32[];
  __shared__ float red[32];
  if (kdev) {
    // stored Lanczos basis: x = slot k, x_prev = slot k - 1, with k read from device memory so
    // that a captured sequence of steps can be replayed
    const long long k = *kdev;
    X += k * kstride;
    Xp += (k - 1) * kstride;
  }
  const int c0 = 2 * blockIdx.x, c1 = c0 + 1;
  const bool act0 = (active == nullptr) || active[c0] != 0;
  const bool act1 = (c1 < ncol) && ((active == nullptr) || active[c1] != 0);
  if (!act0 && !act1) return;
  const int N = plan.n;
  const float* x0 = X + (size_t)c0 * ldx;
  const float* x1 = X + (size_t)c1 * ldx;
  for (int a = threadIdx.x; a < N; a += blockDim.x)
    sbuf32[a] = make_float2(act0 ? x0[a] : 0.f, act1 ? x1[a] : 0.f);
  __syncthreads();
  fft_f<Wide>(sbuf32, plan, tw, -1.f);
  for (int a = threadIdx.x; a < N; a += blockDim.x) sbuf32[a] = cscalef(sbuf32[a], __ldg(&kin[a]));
  __syncthreads();
  fft_f<Wide>(sbuf32, plan, tw, 1.f);
  const float invN = 1.f / N;
  const float sh0 = (shift && act0) ? shift[c0] : 0.f;
  const float sh1 = (shift && act1) ? shift[c1] : 0.f;
  float dot0 = 0.f, dot1 = 0.f;
  const bool lanczos = (Xp != nullptr);
  float* y0 = Y + (size_t)c0 * ldy;
  float* y1 = Y + (size_t)c1 * ldy;
  for (int a = threadIdx.x; a < N; a += blockDim.x) {
    const float2 z = sbuf32[a];
    const float v = __ldg(&V[a]);
    const float xa0 = act0 ? x0[a] : 0.f, xa1 = act1 ? x1[a] : 0.f;
    const float ya0 = fmaf(z.x, invN, (v - sh0) * xa0);
    const float ya1 = fmaf(z.y, invN, (v - sh1) * xa1);
    dot0 = fmaf(xa0, ya0, dot0);
    dot1 = fmaf(xa1, ya1, dot1);
    if (lanczos) {
      sbuf32[a] = make_float2(ya0, ya1);
    } else {
      if (act0) y0[a] = ya0;
      if (act1) y1[a] = ya1;
    }
  }
  if (alpha || lanczos) {
    dot0 = block_sum_f(dot0, red);
    dot1 = block_sum_f(dot1, red);
    if (alpha && threadIdx.x == 0) {
      if (act0) alpha[c0] = dot0;
      if (act1) alpha[c1] = dot1;
    }
  }
  if (lanczos) {
    const float b0 = act0 ? beta[c0] : 0.f, b1 = act1 ? beta[c1] : 0.f;
    const float* p0 = Xp + (size_t)c0 * ldp;
    const float* p1 = Xp + (size_t)c1 * ldp;
    for (int a = threadIdx.x; a < N; a += blockDim.x) {
      const float2 yv = sbuf32[a];
      if (act0) y0[a] = yv.x - dot0 * x0[a] - b0 * p0[a];
      if (act1) y1[a] = yv.y - dot1 * x1[a] - b1 * p1[a];
    }
  }
}

__global__ void tables32_kernel(int N, int ntw, const double* __restrict__ kin, const double* __restrict__ V,
                                const double2* __restrict__ tw, float* __restrict__ kin32, float* __restrict__ V32,
                                float2* __restrict__ tw32) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    kin32[a] = (float)kin[a];
    V32[a] = (float)V[a];
    if (a < ntw) tw32[a] = make_float2((float)tw[a].x, (float)tw[a].y);
  }
}

}  // namespace

// FP32 tables (kinetic symbol, V_eff, twiddles) in the workspace; rebuilt with the orbitals.
acp_status tables32(acp_ctx* ctx, const float** kin32, const float** V32, const float2** tw32) {
  float* buf = nullptr;
  const int N = ctx->N;
  ACP_TRY(ws(ctx, "tables32", (size_t)4 * N, &buf));
  if (ctx->tables32_stale) {
    ::acp::note_launch(ctx);
    const int ntw = (ctx->dim == 2) ? ctx->nx + ctx->ny : N;  // 2D: x twiddles, then y twiddles
    tables32_kernel<<<(N + 255) / 256, 256, 0, ctx->stream>>>(N, ntw, ctx->d_kin, ctx->d_V, ctx->d_tw, buf, buf + N,
                                                             reinterpret_cast<float2*>(buf + 2 * N));
    ACP_LAUNCH(ctx);
    // raised once per device to the opt-in maximum, never lowered (the limit is shared by all
    // contexts; occupancy follows the size of each launch)
    std::lock_guard<std::mutex> lock(device_mutex());
    static int configured_device = -1;
    if (configured_device != ctx->device) {
      ACP_TRY(raise_smem_limit(ctx, reinterpret_cast<const void*>(spectral32_kernel<false>)));
      ACP_TRY(raise_smem_limit(ctx, reinterpret_cast<const void*>(spectral32_kernel<true>)));
      configured_device = ctx->device;
    }
    ctx->tables32_stale = false;
  }
  *kin32 = buf;
  *V32 = buf + N;
  *tw32 = reinterpret_cast<const float2*>(buf + 2 * N);
  return ACP_OK;
}

acp_status spectral32_apply(acp_ctx* ctx, const float* X, int ldx, int ncol, const float* shift_d, float* Y, int ldy,
                            float* alpha_d, const int* active_d, const float* Xprev, int ldp, const float* beta_d,
                            const int* kdev, long long kstride) {
  if (ncol <= 0) return ACP_OK;
  const float *kin = nullptr, *V = nullptr;
  const float2* tw = nullptr;
  ACP_TRY(tables32(ctx, &kin, &V, &tw));
  if (ctx->dim == 2)
    return spectral2d_apply_f32(ctx, X, ldx, ncol, kin, V, shift_d, Y, ldy, alpha_d, active_d, Xprev, ldp, beta_d, tw,
                                tw + ctx->nx, kdev, kstride);
  PlanArgF pa{};
  pa.n = ctx->plan.n;
  pa.nst = ctx->plan.nst;
  for (int i = 0; i < pa.nst; ++i) pa.rad[i] = ctx->plan.rad[i];
  const int blocks = (ncol + 1) / 2;
  ::acp::note_launch(ctx);
  cudaEvent_t ev0 = prof_begin(ctx);
  auto kernel = ctx->plan.wide ? spectral32_kernel<true> : spectral32_kernel<false>;
  kernel<<<blocks, ctx->plan.threads, ctx->N * sizeof(float2), ctx->stream>>>(
      X, ldx, ncol, pa, tw, kin, V, shift_d, Y, ldy, alpha_d, active_d, Xprev, ldp, beta_d, kdev, kstride);
  ACP_LAUNCH(ctx);
  const double lg = std::log2((double)ctx->N);
  const double flops = 2.0 * 5.0 * ctx->N * lg * blocks + 6.0 * (double)ctx->N * ncol;
  const double bytes = 4.0 * ctx->N * ncol * (Xprev ? 3.0 : 2.0);
  prof_end(ctx, "spectral32", ev0, flops, bytes);
  return ACP_OK;
}

}  // namespace acp
