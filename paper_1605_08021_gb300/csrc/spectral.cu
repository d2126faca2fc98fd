// Spectral operators on the periodic grid: the kinetic part of H (Eq. Hamil), the Yukawa
// convolution K and its inverse (Eq. yukawa, v_hxc = K), and the perturbation potentials
// g_I = dV_I/dR_I, B = K^{-1} G, d2V_I (Eq. pseudocharge, Sec. 2.2, Sec. 3.2).
//
// Each CTA owns whole grid functions: two real columns are packed as one complex signal
// z = x0 + i x1, transformed by a mixed-radix (4, 2, 3, 5) Stockham FFT that lives entirely in
// shared memory, multiplied by a real even symbol (which keeps the two halves separate), and
// transformed back.  Because the CTA holds complete columns it can also finish reductions over
// the grid (e.g. the Lanczos coefficient v . Hv) without atomics.
#include "internal.cuh"

namespace acp {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// i * s * a
__device__ __forceinline__ double2 cimul(double2 a, double s) { return make_double2(-a.y * s, a.x * s); }

// DFT of length R with kernel exp(dir * 2 pi i r m / R), dir = -1 forward, +1 inverse.
template <int R>
__device__ __forceinline__ void dft(double2 (&a)[R], double dir);

template <>
__device__ __forceinline__ void dft<2>(double2 (&a)[2], double) {
  double2 t = a[0];
  a[0] = cadd(t, a[1]);
  a[1] = csub(t, a[1]);
}

template <>
__device__ __forceinline__ void dft<4>(double2 (&a)[4], double dir) {
  double2 s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
  double2 s13 = cadd(a[1], a[3]), d13 = cimul(csub(a[1], a[3]), dir);
  a[0] = cadd(s02, s13);
  a[2] = csub(s02, s13);
  a[1] = cadd(d02, d13);
  a[3] = csub(d02, d13);
}

template <>
__device__ __forceinline__ void dft<3>(double2 (&a)[3], double dir) {
  const double c = -0.5, s = 0.86602540378443864676;  // cos(2 pi/3), sin(2 pi/3)
  double2 t1 = cadd(a[1], a[2]), t2 = cimul(csub(a[1], a[2]), dir * s);
  double2 m = cadd(a[0], cscale(t1, c));
  a[0] = cadd(a[0], t1);
  a[1] = cadd(m, t2);
  a[2] = csub(m, t2);
}

template <>
__device__ __forceinline__ void dft<5>(double2 (&a)[5], double dir) {
  const double c1 = 0.30901699437494742410, s1 = 0.95105651629515357212;   // 2 pi / 5
  const double c2 = -0.80901699437494742410, s2 = 0.58778525229247312917;  // 4 pi / 5
  double2 t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
  double2 d1 = csub(a[1], a[4]), d2 = csub(a[2], a[3]);
  double2 m1 = cadd(a[0], cadd(cscale(t1, c1), cscale(t2, c2)));
  double2 m2 = cadd(a[0], cadd(cscale(t1, c2), cscale(t2, c1)));
  double2 e1 = cimul(cadd(cscale(d1, s1), cscale(d2, s2)), dir);
  double2 e2 = cimul(csub(cscale(d1, s2), cscale(d2, s1)), dir);
  a[0] = cadd(a[0], cadd(t1, t2));
  a[1] = cadd(m1, e1);
  a[4] = csub(m1, e1);
  a[2] = cadd(m2, e2);
  a[3] = csub(m2, e2);
}

// Butterflies per thread and stage, by radix; the plan sizes the CTA so that these suffice.
// Every grid up to 4096 points fits CTAs of at most 512 threads; the wide form (CTAs of up to
// 1024 threads, five radix-2 butterflies per thread) covers every 2^a 3^b 5^c grid up to 10240
// points.  The FP32 kernels use the same counts (one plan serves both).
template <int R, bool Wide> struct MaxB;
template <bool W> struct MaxB<2, W> { static constexpr int v = W ? 5 : 4; };
template <bool W> struct MaxB<3, W> { static constexpr int v = 4; };
template <bool W> struct MaxB<4, W> { static constexpr int v = 3; };
template <bool W> struct MaxB<5, W> { static constexpr int v = 2; };

// One in-place Stockham stage: all inputs of the thread are loaded to registers before the CTA
// barrier, outputs are stored after it.  tw[m] = exp(-2 pi i m / N).
template <int R, bool Wide>
__device__ __noinline__ void fft_stage(double2* s, int N, int Ns, const double2* __restrict__ tw, double dir) {
  constexpr int B = MaxB<R, Wide>::v;
  const int nb = N / R;
  const int stride = N / (Ns * R);
  double2 a[B][R];
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
        double2 w = __ldg(&tw[r * k * stride]);
        if (dir > 0) w.y = -w.y;
        a[b][r] = cmul(a[b][r], w);
      }
      dft<R>(a[b], dir);
      const int base = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) s[base + r * Ns] = a[b][r];
    }
  }
  __syncthreads();
}

constexpr int kMaxThreads = 512;
constexpr int kMaxThreadsWide = 1024;

struct PlanArg {
  int n, nst;
  int rad[24];
};

// Unnormalised DFT of the N values in shared memory: sum_a s[a] exp(dir 2 pi i a n / N).
template <bool Wide>
__device__ void fft(double2* s, const PlanArg& p, const double2* __restrict__ tw, double dir) {
  int Ns = 1;
  for (int st = 0; st < p.nst; ++st) {
    const int R = p.rad[st];
    switch (R) {
      case 4: fft_stage<4, Wide>(s, p.n, Ns, tw, dir); break;
      case 2: fft_stage<2, Wide>(s, p.n, Ns, tw, dir); break;
      case 3: fft_stage<3, Wide>(s, p.n, Ns, tw, dir); break;
      default: fft_stage<5, Wide>(s, p.n, Ns, tw, dir); break;
    }
    Ns *= R;
  }
}

PlanArg plan_arg(const FftPlan& p) {
  PlanArg a{};
  a.n = p.n;
  a.nst = p.nst;
  for (int i = 0; i < p.nst; ++i) a.rad[i] = p.rad[i];
  return a;
}

template <bool Wide>
__global__ void __launch_bounds__(Wide ? kMaxThreadsWide : kMaxThreads) spectral_kernel(const double* __restrict__ X, int ldx, int ncol, PlanArg plan,
                                const double2* __restrict__ tw, const double* __restrict__ mult,
                                const double* __restrict__ V, const double* __restrict__ shift,
                                double* __restrict__ Y, int ldy, double* __restrict__ alpha,
                                const int* __restrict__ active, const double* __restrict__ Xp,
                                const double* __restrict__ beta) {
  extern __shared__ double2 sbuf[];
  __shared__ double red[32];
  const int c0 = 2 * blockIdx.x, c1 = c0 + 1;
  const bool act0 = (active == nullptr) || active[c0] != 0;
  const bool act1 = (c1 < ncol) && ((active == nullptr) || active[c1] != 0);
  if (!act0 && !act1) return;  // uniform over the CTA
  const int N = plan.n;
  const double* x0 = X + (size_t)c0 * ldx;
  const double* x1 = X + (size_t)c1 * ldx;
  for (int a = threadIdx.x; a < N; a += blockDim.x)
    sbuf[a] = make_double2(act0 ? x0[a] : 0.0, act1 ? x1[a] : 0.0);
  __syncthreads();
  fft<Wide>(sbuf, plan, tw, -1.0);
  for (int a = threadIdx.x; a < N; a += blockDim.x) sbuf[a] = cscale(sbuf[a], __ldg(&mult[a]));
  __syncthreads();
  fft<Wide>(sbuf, plan, tw, 1.0);
  const double invN = 1.0 / N;
  const double sh0 = (shift && act0) ? shift[c0] : 0.0;
  const double sh1 = (shift && act1) ? shift[c1] : 0.0;
  double dot0 = 0.0, dot1 = 0.0;
  double* y0 = Y + (size_t)c0 * ldy;
  double* y1 = Y + (size_t)c1 * ldy;
  const bool lanczos = (Xp != nullptr);
  for (int a = threadIdx.x; a < N; a += blockDim.x) {
    const double2 z = sbuf[a];
    const double v = V ? __ldg(&V[a]) : 0.0;
    const double xa0 = act0 ? x0[a] : 0.0, xa1 = act1 ? x1[a] : 0.0;
    const double ya0 = z.x * invN + (v - sh0) * xa0;
    const double ya1 = z.y * invN + (v - sh1) * xa1;
    dot0 += xa0 * ya0;
    dot1 += xa1 * ya1;
    if (lanczos) {
      sbuf[a] = make_double2(ya0, ya1);
    } else {
      if (act0) y0[a] = ya0;
      if (act1) y1[a] = ya1;
    }
  }
  if (alpha || lanczos) {
    dot0 = block_sum(dot0, red);
    dot1 = block_sum(dot1, red);
    if (alpha && threadIdx.x == 0) {
      if (act0) alpha[c0] = dot0;
      if (act1) alpha[c1] = dot1;
    }
  }
  if (lanczos) {
    // Lanczos three-term recurrence: P = (H - s) v - alpha v - beta v_prev
    const double b0 = act0 ? beta[c0] : 0.0, b1 = act1 ? beta[c1] : 0.0;
    const double* p0 = Xp + (size_t)c0 * ldx;
    const double* p1 = Xp + (size_t)c1 * ldx;
    for (int a = threadIdx.x; a < N; a += blockDim.x) {
      const double2 yv = sbuf[a];
      if (act0) y0[a] = yv.x - dot0 * x0[a] - b0 * p0[a];
      if (act1) y1[a] = yv.y - dot1 * x1[a] - b1 * p1[a];
    }
  }
}

// Fourier coefficient of the pseudocharge of atom I at signed wavenumber index n:
// -Z exp(-sigma^2 k^2 / 2) exp(-i k R), k = 2 pi n / L.
__device__ __forceinline__ double2 pseudo_coeff(int n, double L, double Z, double sig, double R) {
  const double k = 2.0 * M_PI * n / L;
  const double amp = -Z * exp(-0.5 * sig * sig * k * k);
  double t = fmod((double)n * (R / L), 1.0);  // phase -2 pi n R / L reduced to one turn
  double sn, cs;
  sincospi(-2.0 * t, &sn, &cs);
  return make_double2(amp * cs, amp * sn);
}

// One CTA per atom: G[:, I] + i B[:, I] from one inverse transform, D2[:, I] from a second.
template <bool Wide>
__global__ void __launch_bounds__(Wide ? kMaxThreadsWide : kMaxThreads) perturbation_kernel(PlanArg plan, const double2* __restrict__ tw, double L, double kappa,
                                    double scale, const double* __restrict__ R, const double* __restrict__ Z,
                                    const double* __restrict__ sig, double* G, double* B, double* D2) {
  extern __shared__ double2 sbuf[];
  const int I = blockIdx.x;
  const int N = plan.n;
  const double RI = R[I], ZI = Z[I], sI = sig[I];
  const double invL = 1.0 / L;
  if (G || B) {
    for (int a = threadIdx.x; a < N; a += blockDim.x) {
      const int n = (a < (N + 1) / 2) ? a : a - N;
      const double k = 2.0 * M_PI * n / L;
      const double kodd = (2 * a == N) ? 0.0 : k;  // Nyquist term of odd symbols dropped
      const double khat = 4.0 * M_PI * scale / (k * k + kappa * kappa);
      const double2 c = pseudo_coeff(n, L, ZI, sI, RI);
      // b^ = -i k c ; g^ = Khat b^ ; pack z^ = g^ + i b^
      const double2 bh = make_double2(kodd * c.y, -kodd * c.x);
      const double2 gh = cscale(bh, khat);
      sbuf[a] = make_double2(gh.x - bh.y, gh.y + bh.x);
    }
    __syncthreads();
    fft<Wide>(sbuf, plan, tw, 1.0);
    for (int a = threadIdx.x; a < N; a += blockDim.x) {
      if (G) G[(size_t)I * N + a] = sbuf[a].x * invL;
      if (B) B[(size_t)I * N + a] = sbuf[a].y * invL;
    }
    __syncthreads();
  }
  if (D2) {
    for (int a = threadIdx.x; a < N; a += blockDim.x) {
      const int n = (a < (N + 1) / 2) ? a : a - N;
      const double k = 2.0 * M_PI * n / L;
      const double khat = 4.0 * M_PI * scale / (k * k + kappa * kappa);
      sbuf[a] = cscale(pseudo_coeff(n, L, ZI, sI, RI), -k * k * khat);
    }
    __syncthreads();
    fft<Wide>(sbuf, plan, tw, 1.0);
    for (int a = threadIdx.x; a < N; a += blockDim.x) D2[(size_t)I * N + a] = sbuf[a].x * invL;
  }
}

}  // namespace

// The dynamic shared-memory limit is a property of the kernel, shared by every context in the
// process: it is raised once to the device's opt-in maximum (a context with a smaller grid must
// not lower it under another context's feet); occupancy follows the size of each launch.
acp_status spectral_configure(acp_ctx* ctx) {
  std::lock_guard<std::mutex> lock(device_mutex());
  static int configured_device = -1;
  if (configured_device == ctx->device) return ACP_OK;
  ACP_TRY(raise_smem_limit(ctx, reinterpret_cast<const void*>(spectral_kernel<false>)));
  ACP_TRY(raise_smem_limit(ctx, reinterpret_cast<const void*>(spectral_kernel<true>)));
  ACP_TRY(raise_smem_limit(ctx, reinterpret_cast<const void*>(perturbation_kernel<false>)));
  ACP_TRY(raise_smem_limit(ctx, reinterpret_cast<const void*>(perturbation_kernel<true>)));
  configured_device = ctx->device;
  return ACP_OK;
}

// Dynamic shared-memory limit of `func` = the device's opt-in maximum minus its static shared memory.
acp_status raise_smem_limit(acp_ctx* ctx, const void* func) {
  int optin = 0;
  ACP_CUDA(ctx, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
  cudaFuncAttributes fa{};
  ACP_CUDA(ctx, cudaFuncGetAttributes(&fa, func));
  ACP_CUDA(ctx, cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
  return ACP_OK;
}

bool make_fft_plan(int n, FftPlan* plan) {
  if (n < 8 || n > kMaxFftN) return false;
  FftPlan p{};
  p.n = n;
  int m = n;
  auto push = [&](int r) { p.rad[p.nst++] = r; m /= r; };
  while (m % 4 == 0) push(4);
  while (m % 2 == 0) push(2);
  while (m % 3 == 0) push(3);
  while (m % 5 == 0) push(5);
  if (m != 1 || p.nst > 24) return false;
  // the smallest CTA (a multiple of 32 threads, at least 64) in which every stage's butterflies
  // fit the per-thread counts MaxB of the narrow form, else of the wide form
  for (int wide = 0; wide < 2; ++wide) {
    int t = 64;
    for (int s = 0; s < p.nst; ++s) {
      const int r = p.rad[s];
      const int mb = (r == 2) ? (wide ? MaxB<2, true>::v : MaxB<2, false>::v) : (r == 3) ? MaxB<3, false>::v
                     : (r == 4) ? MaxB<4, false>::v : MaxB<5, false>::v;
      const int need = (n / r + mb - 1) / mb;
      if (need > t) t = need;
    }
    t = (t + 31) / 32 * 32;
    if (t <= (wide ? kMaxThreadsWide : kMaxThreads)) {
      p.threads = t;
      p.wide = wide != 0;
      *plan = p;
      return true;
    }
  }
  return false;
}

acp_status spectral_apply(acp_ctx* ctx, const double* X, int ldx, int ncol, SpectralMult mult, bool with_v,
                          const double* shift_d, double* Y, int ldy, double* alpha_d, const int* active_d,
                          const double* Xprev, const double* beta_d) {
  if (ncol <= 0) return ACP_OK;
  const double* m = (mult == MULT_KINETIC) ? ctx->d_kin : (mult == MULT_KHAT) ? ctx->d_khat : ctx->d_khat_inv;
  if (ctx->dim == 2)
    return spectral2d_apply_f64(ctx, X, ldx, ncol, m, with_v ? ctx->d_V : nullptr, shift_d, Y, ldy, alpha_d, active_d,
                                Xprev, ldx, beta_d);
  const int blocks = (ncol + 1) / 2;
  ::acp::note_launch(ctx);
  cudaEvent_t ev0 = prof_begin(ctx);
  auto kernel = ctx->plan.wide ? spectral_kernel<true> : spectral_kernel<false>;
  kernel<<<blocks, ctx->plan.threads, ctx->N * sizeof(double2), ctx->stream>>>(
      X, ldx, ncol, plan_arg(ctx->plan), ctx->d_tw, m, with_v ? ctx->d_V : nullptr, shift_d, Y, ldy, alpha_d,
      active_d, Xprev, beta_d);
  ACP_LAUNCH(ctx);
  {
    // algorithmic work of the launch (all columns counted, active or not): two complex FFTs of
    // length N per column pair, and the column reads/writes of the operator
    const double lg = std::log2((double)ctx->N);
    const double flops = 2.0 * 5.0 * ctx->N * lg * blocks + 4.0 * (double)ctx->N * ncol;
    const double bytes = 8.0 * ctx->N * ncol * (Xprev ? 3.0 : 2.0);
    prof_end(ctx, "spectral", ev0, flops, bytes);
  }
  return ACP_OK;
}

acp_status perturbations_1d(acp_ctx* ctx, int n_atoms, const double* R_d, const double* Z_d, const double* sig_d,
                            double* G, double* B, double* D2) {
  if (n_atoms <= 0) return ACP_OK;
  ::acp::note_launch(ctx);
  auto kernel = ctx->plan.wide ? perturbation_kernel<true> : perturbation_kernel<false>;
  kernel<<<n_atoms, ctx->plan.threads, ctx->N * sizeof(double2), ctx->stream>>>(
      plan_arg(ctx->plan), ctx->d_tw, ctx->L, ctx->kappa, ctx->scale, R_d, Z_d, sig_d, G, B, D2);
  ACP_LAUNCH(ctx);
  return ACP_OK;
}

}  // namespace acp
