// Batched MINRES (Paige-Saunders) for the projected Sternheimer equations
// Q(H - s)Q x = Q b (Sec. 2.2 below Eq. Sternheimer; Alg. 1 and Eq. eqncompressU).
//
// One Lanczos step of every active right-hand side per iteration:
//   1. spectral kernel (one CTA owns whole columns): alpha = v . (H - s) v and
//      P = (H - s) v - alpha v - beta v_prev
//   2. projector GEMMs: P = Q P.  Projecting after the three-term recurrence matters: rounding
//      leaves tiny occupied (null-space) components in every Lanczos vector, and the recurrence
//      multiplies them by the Lanczos polynomials at 0, outside the spectrum [gap, E_max], which
//      grow geometrically; hundreds of iterations would otherwise make them O(1).
//   3. update kernel (one CTA per column): beta' = ||P||, Givens QR of the growing tridiagonal
//      matrix, direction vectors and iterate, v <- P / beta'.
// The multi-shift variant runs one Lanczos process per right-hand side for the unshifted
// operator QHQ and carries one Givens recurrence and one iterate per shift: the Krylov spaces of
// Q(H - s)Q for all shifts coincide (shift invariance), so the N_c Chebyshev shifts of
// Eq. eqncompressU share every H and Q application.
#include "internal.cuh"

namespace acp {

namespace {

constexpr int kThreads = 256;

// ---- single-shift batched MINRES ------------------------------------------------------------
struct MinresState {
  double *V, *Vp, *P, *W1, *W2;  // N x ncol
  double *alpha, *beta, *beta1, *cs, *sn, *dbar, *epsln, *phibar;
  int *active, *iters;
};

__global__ void __launch_bounds__(kThreads) minres_init_kernel(int N, const double* __restrict__ Bm, MinresState s,
                                                               double* __restrict__ X, int* nan_flag) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  const double* b = Bm + (size_t)j * N;
  double acc = 0.0;
  for (int a = threadIdx.x; a < N; a += blockDim.x) acc += b[a] * b[a];
  const double nrm = sqrt(block_sum(acc, red));
  const bool ok = isfinite(nrm);
  const double inv = (nrm > 0.0 && ok) ? 1.0 / nrm : 0.0;
  const size_t off = (size_t)j * N;
  for (int a = threadIdx.x; a < N; a += blockDim.x) {
    s.V[off + a] = b[a] * inv;
    s.Vp[off + a] = 0.0;
    s.W1[off + a] = 0.0;
    s.W2[off + a] = 0.0;
    X[off + a] = 0.0;
  }
  if (threadIdx.x == 0) {
    s.beta1[j] = ok ? nrm : 0.0;
    s.beta[j] = 0.0;
    s.cs[j] = -1.0;
    s.sn[j] = 0.0;
    s.dbar[j] = 0.0;
    s.epsln[j] = 0.0;
    s.phibar[j] = ok ? nrm : 0.0;
    s.iters[j] = 0;
    s.active[j] = (nrm > 0.0 && ok) ? 1 : 0;
    if (!ok) atomicExch(nan_flag, 1);
  }
}

__global__ void __launch_bounds__(kThreads) minres_step_kernel(int N, MinresState s, double* __restrict__ X,
                                                               double tol, int maxit, int* nan_flag) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  if (!s.active[j]) return;
  const size_t off = (size_t)j * N;
  const double a = s.alpha[j];
  const double* P = s.P + off;  // Q[(H - s) v - alpha v - beta v_prev], already projected
  double acc = 0.0;
  for (int r = threadIdx.x; r < N; r += blockDim.x) acc += P[r] * P[r];
  const double bn = sqrt(block_sum(acc, red));
  const double oldeps = s.epsln[j], c = s.cs[j], sg = s.sn[j], db = s.dbar[j], pb = s.phibar[j];
  const double delta = c * db + sg * a;
  const double gbar = sg * db - c * a;
  const double gamma = fmax(hypot(gbar, bn), 1e-300);
  const double cn = gbar / gamma, sn_ = bn / gamma;
  const double phi = cn * pb, pbn = sn_ * pb;
  const double ig = 1.0 / gamma, ib = (bn > 0.0) ? 1.0 / bn : 0.0;
  double* W1 = s.W1 + off;
  double* W2 = s.W2 + off;
  double* Vw = s.V + off;
  double* Vpw = s.Vp + off;
  double* x = X + off;
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    const double v = Vw[r];
    const double w1 = W1[r];
    const double w = (v - oldeps * W2[r] - delta * w1) * ig;
    W2[r] = w1;
    W1[r] = w;
    x[r] += phi * w;
    Vpw[r] = v;
    Vw[r] = P[r] * ib;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s.epsln[j] = sg * bn;
    s.dbar[j] = -c * bn;
    s.cs[j] = cn;
    s.sn[j] = sn_;
    s.phibar[j] = pbn;
    s.beta[j] = bn;
    const int it = s.iters[j] + 1;
    s.iters[j] = it;
    const bool bad = !isfinite(bn) || !isfinite(pbn);
    if (bad) atomicExch(nan_flag, 1);
    if (bad || fabs(pbn) <= tol * s.beta1[j] || bn == 0.0 || it >= maxit) s.active[j] = 0;
  }
}

__global__ void count_active_kernel(const int* __restrict__ active, int n, int* out) {
  int c = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) c += active[i] != 0;
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void minres_report_kernel(int n, const int* __restrict__ iters, const double* __restrict__ phibar,
                                     const double* __restrict__ beta1, double tol, unsigned long long* steps,
                                     int* max_it, unsigned long long* conv, double* max_res) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    atomicAdd(steps, (unsigned long long)iters[i]);
    atomicMax(max_it, iters[i]);
    const double r = (beta1[i] > 0.0) ? fabs(phibar[i]) / beta1[i] : 0.0;
    if (r <= tol) atomicAdd(conv, 1ull);
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(max_res), (unsigned long long)__double_as_longlong(r));
  }
}

__global__ void ms_report_kernel(int nmu, int nc, const int* __restrict__ iters, const double* __restrict__ phibar,
                                 const double* __restrict__ beta1, double tol, unsigned long long* steps, int* max_it,
                                 unsigned long long* conv, double* max_res) {
  const size_t nq = (size_t)nmu * nc;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nq; i += (size_t)gridDim.x * blockDim.x) {
    const int mu = (int)(i / nc), c = (int)(i % nc);
    if (c == 0) {
      atomicAdd(steps, (unsigned long long)iters[mu]);
      atomicMax(max_it, iters[mu]);
    }
    const double r = (beta1[mu] > 0.0) ? fabs(phibar[i]) / beta1[mu] : 0.0;
    if (r <= tol) atomicAdd(conv, 1ull);
    atomicMax(reinterpret_cast<unsigned long long*>(max_res), (unsigned long long)__double_as_longlong(r));
  }
}

// ---- multi-shift MINRES ------------------------------------------------------------------------
constexpr int kMaxShifts = 64;

struct MsState {
  double *V, *Vp, *P;                 // N x nmu
  double *W1, *W2;                    // N x (nc nmu), column mu + c nmu
  double *alpha, *beta, *beta1;       // nmu
  double *cs, *sn, *dbar, *epsln, *phibar;  // nc x nmu (index c + nc mu)
  int *act_c;                         // nc x nmu
  int *active, *iters;                // nmu
  const double* nodes;                // nc
};

__global__ void __launch_bounds__(kThreads) ms_init_kernel(int N, int nmu, int nc, const double* __restrict__ Bm,
                                                           MsState s, double* __restrict__ X, int* nan_flag) {
  __shared__ double red[32];
  const int mu = blockIdx.x;
  const double* b = Bm + (size_t)mu * N;
  double acc = 0.0;
  for (int a = threadIdx.x; a < N; a += blockDim.x) acc += b[a] * b[a];
  const double nrm = sqrt(block_sum(acc, red));
  const bool ok = isfinite(nrm) && nrm > 0.0;
  const double inv = ok ? 1.0 / nrm : 0.0;
  const size_t off = (size_t)mu * N;
  for (int a = threadIdx.x; a < N; a += blockDim.x) {
    s.V[off + a] = b[a] * inv;
    s.Vp[off + a] = 0.0;
  }
  for (int c = 0; c < nc; ++c) {
    const size_t o = ((size_t)mu + (size_t)c * nmu) * N;
    for (int a = threadIdx.x; a < N; a += blockDim.x) {
      s.W1[o + a] = 0.0;
      s.W2[o + a] = 0.0;
      X[o + a] = 0.0;
    }
  }
  if (threadIdx.x < nc) {
    const int q = threadIdx.x + nc * mu;
    s.cs[q] = -1.0;
    s.sn[q] = 0.0;
    s.dbar[q] = 0.0;
    s.epsln[q] = 0.0;
    s.phibar[q] = ok ? nrm : 0.0;
    s.act_c[q] = ok ? 1 : 0;
  }
  if (threadIdx.x == 0) {
    s.beta1[mu] = ok ? nrm : 0.0;
    s.beta[mu] = 0.0;
    s.iters[mu] = 0;
    s.active[mu] = ok ? 1 : 0;
    if (!isfinite(nrm)) atomicExch(nan_flag, 1);
  }
}

__global__ void __launch_bounds__(kThreads) ms_step_kernel(int N, int nmu, int nc, MsState s, double* __restrict__ X,
                                                           double tol, int maxit, int* nan_flag) {
  __shared__ double red[32];
  __shared__ double c_oldeps[kMaxShifts], c_delta[kMaxShifts], c_ig[kMaxShifts], c_phi[kMaxShifts];
  __shared__ int c_upd[kMaxShifts];
  __shared__ int any_active;
  const int mu = blockIdx.x;
  if (!s.active[mu]) return;
  const size_t off = (size_t)mu * N;
  const double a = s.alpha[mu];
  const double* P = s.P + off;  // Q[H v - alpha v - beta v_prev], already projected
  double* V = s.V + off;
  double* Vp = s.Vp + off;
  double acc = 0.0;
  for (int r = threadIdx.x; r < N; r += blockDim.x) acc += P[r] * P[r];
  const double bn = sqrt(block_sum(acc, red));
  if (threadIdx.x == 0) any_active = 0;
  __syncthreads();
  if (threadIdx.x < nc) {
    const int c = threadIdx.x;
    const int q = c + nc * mu;
    const int upd = s.act_c[q];
    c_upd[c] = upd;
    if (upd) {
      const double ac = a - s.nodes[c];  // Lanczos coefficient of the shifted operator
      const double cs = s.cs[q], sg = s.sn[q], db = s.dbar[q], pb = s.phibar[q];
      const double delta = cs * db + sg * ac;
      const double gbar = sg * db - cs * ac;
      const double gamma = fmax(hypot(gbar, bn), 1e-300);
      const double cn = gbar / gamma, sn_ = bn / gamma;
      c_oldeps[c] = s.epsln[q];
      c_delta[c] = delta;
      c_ig[c] = 1.0 / gamma;
      c_phi[c] = cn * pb;
      const double pbn = sn_ * pb;
      s.epsln[q] = sg * bn;
      s.dbar[q] = -cs * bn;
      s.cs[q] = cn;
      s.sn[q] = sn_;
      s.phibar[q] = pbn;
      const bool bad = !isfinite(pbn);
      if (bad) atomicExch(nan_flag, 1);
      const bool done = bad || fabs(pbn) <= tol * s.beta1[mu] || bn == 0.0 || s.iters[mu] + 1 >= maxit;
      if (done) s.act_c[q] = 0;
      else atomicOr(&any_active, 1);
    }
  }
  __syncthreads();
  const double ib = (bn > 0.0) ? 1.0 / bn : 0.0;
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    const double v = V[r];
    for (int c = 0; c < nc; ++c) {
      if (!c_upd[c]) continue;
      const size_t o = ((size_t)mu + (size_t)c * nmu) * N + r;
      const double w1 = s.W1[o];
      const double w = (v - c_oldeps[c] * s.W2[o] - c_delta[c] * w1) * c_ig[c];
      s.W2[o] = w1;
      s.W1[o] = w;
      X[o] += c_phi[c] * w;
    }
    Vp[r] = v;
    V[r] = P[r] * ib;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s.beta[mu] = bn;
    s.iters[mu] += 1;
    if (!isfinite(bn)) atomicExch(nan_flag, 1);
    if (!any_active || !isfinite(bn)) s.active[mu] = 0;
  }
}

// ---- multi-shift MINRES with a stored Lanczos basis -----------------------------------------
// Instead of carrying w_{k-1}, w_{k-2} and x for every shift (6 vector passes per shift and
// step), the normalised Lanczos vectors v_1..v_k of each mu are kept, together with the per-step
// coefficients of every shift's Givens factorisation R (diagonal gamma_j, first superdiagonal
// delta_{j+1}, second eps_{j+2}) and phi_j.  MINRES's iterate is x_c = V R_c^{-1} phi_c, so at the
// end y_c = R_c^{-1} phi_c is a banded back substitution and X_mu = V_mu Y_mu one small GEMM.
struct MsBasis {
  double* Vb;        // slot s of mu at Vb + mu * slot_ld + s * N; slot 0 = v_0 = 0
  size_t slot_ld;    // (kmax + 2) * N
  double* P;         // N x nmu, the unnormalised next Lanczos vector
  double *alpha, *beta, *beta1;             // nmu
  double *cs, *sn, *dbar, *epsln, *phibar;  // nc x nmu (c + nc mu)
  double* coef;      // (gamma, delta, eps, phi) of step j: coef[(((size_t)mu * nc + c) * kmax + j) * 4 + q]
  double* Y;         // y_{c, j}: Y[((size_t)mu * nc + c) * kmax + j]
  int *active, *iters;
  const double* nodes;
  int kmax;
};

__global__ void __launch_bounds__(kThreads) msb_init_kernel(int N, int nmu, int nc, const double* __restrict__ Bm,
                                                            MsBasis s, int* nan_flag) {
  __shared__ double red[32];
  const int mu = blockIdx.x;
  const double* b = Bm + (size_t)mu * N;
  double acc = 0.0;
  for (int a = threadIdx.x; a < N; a += blockDim.x) acc += b[a] * b[a];
  const double nrm = sqrt(block_sum(acc, red));
  const bool ok = isfinite(nrm) && nrm > 0.0;
  const double inv = ok ? 1.0 / nrm : 0.0;
  double* v0 = s.Vb + (size_t)mu * s.slot_ld;
  for (int a = threadIdx.x; a < N; a += blockDim.x) {
    v0[a] = 0.0;
    v0[N + a] = b[a] * inv;
  }
  if (threadIdx.x < nc) {
    const int q = threadIdx.x + nc * mu;
    s.cs[q] = -1.0;
    s.sn[q] = 0.0;
    s.dbar[q] = 0.0;
    s.epsln[q] = 0.0;
    s.phibar[q] = ok ? nrm : 0.0;
  }
  if (threadIdx.x == 0) {
    s.beta1[mu] = ok ? nrm : 0.0;
    s.beta[mu] = 0.0;
    s.iters[mu] = 0;
    s.active[mu] = ok ? 1 : 0;
    if (!isfinite(nrm)) atomicExch(nan_flag, 1);
  }
}

// Step k (1-based): P = Q[H v_k - alpha v_k - beta_k v_{k-1}] is given; store v_{k+1} = P/||P|| in
// slot k+1 and advance every shift's Givens factorisation.
__global__ void __launch_bounds__(kThreads) msb_step_kernel(int N, int nmu, int nc, int k, MsBasis s, double tol,
                                                            int* nan_flag) {
  __shared__ double red[32];
  __shared__ int any_active;
  const int mu = blockIdx.x;
  if (!s.active[mu]) return;
  const double* P = s.P + (size_t)mu * N;
  double acc = 0.0;
  for (int r = threadIdx.x; r < N; r += blockDim.x) acc += P[r] * P[r];
  const double bn = sqrt(block_sum(acc, red));
  const double ib = (bn > 0.0) ? 1.0 / bn : 0.0;
  double* vn = s.Vb + (size_t)mu * s.slot_ld + (size_t)(k + 1) * N;
  for (int r = threadIdx.x; r < N; r += blockDim.x) vn[r] = P[r] * ib;
  if (threadIdx.x == 0) any_active = 0;
  __syncthreads();
  const double a = s.alpha[mu];
  if (threadIdx.x < nc) {
    const int c = threadIdx.x;
    const int q = c + nc * mu;
    const double ac = a - s.nodes[c];
    const double cs = s.cs[q], sg = s.sn[q], db = s.dbar[q], pb = s.phibar[q], oldeps = s.epsln[q];
    const double delta = cs * db + sg * ac;
    const double gbar = sg * db - cs * ac;
    const double gamma = fmax(hypot(gbar, bn), 1e-300);
    const double cn = gbar / gamma, sn_ = bn / gamma;
    const double phi = cn * pb, pbn = sn_ * pb;
    double* cf = s.coef + (((size_t)mu * nc + c) * s.kmax + (k - 1)) * 4;
    cf[0] = gamma;
    cf[1] = delta;
    cf[2] = oldeps;
    cf[3] = phi;
    s.epsln[q] = sg * bn;
    s.dbar[q] = -cs * bn;
    s.cs[q] = cn;
    s.sn[q] = sn_;
    s.phibar[q] = pbn;
    if (!isfinite(pbn)) atomicExch(nan_flag, 1);
    if (isfinite(pbn) && !(fabs(pbn) <= tol * s.beta1[mu])) atomicOr(&any_active, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s.beta[mu] = bn;
    const int it = s.iters[mu] + 1;
    s.iters[mu] = it;
    if (!isfinite(bn)) atomicExch(nan_flag, 1);
    if (!any_active || !isfinite(bn) || bn == 0.0 || it >= s.kmax) s.active[mu] = 0;
  }
}

// y_c = R_c^{-1} phi_c, one thread per (mu, c): y_j = (phi_j - delta_{j+1} y_{j+1} - eps_{j+2} y_{j+2}) / gamma_j
__global__ void msb_backsub_kernel(int nmu, int nc, MsBasis s) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)nmu * nc) return;
  const int mu = (int)(t / nc);
  const int kk = s.iters[mu];
  const double* cf = s.coef + t * s.kmax * 4;
  double* y = s.Y + t * s.kmax;
  double y1 = 0.0, y2 = 0.0;  // y_{j+1}, y_{j+2}
  for (int j = kk - 1; j >= 0; --j) {
    const double d1 = (j + 1 < kk) ? cf[(j + 1) * 4 + 1] : 0.0;
    const double e2 = (j + 2 < kk) ? cf[(j + 2) * 4 + 2] : 0.0;
    const double yj = (cf[j * 4 + 3] - d1 * y1 - e2 * y2) / cf[j * 4 + 0];
    y[j] = yj;
    y2 = y1;
    y1 = yj;
  }
}

// X[:, mu + c nmu] = sum_j v_{j+1} y_{c, j}: grid (row tiles, mu); 16 shifts per pass.
__global__ void __launch_bounds__(256) msb_assemble_kernel(int N, int nmu, int nc, MsBasis s, double* __restrict__ X) {
  __shared__ double ys[64][16];
  const int mu = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int kk = s.iters[mu];
  const double* V = s.Vb + (size_t)mu * s.slot_ld + N;  // v_1 in slot 1
  for (int c0 = 0; c0 < nc; c0 += 16) {
    const int cw = (nc - c0 < 16) ? nc - c0 : 16;
    double acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = 0.0;
    for (int j0 = 0; j0 < kk; j0 += 64) {
      const int jw = (kk - j0 < 64) ? kk - j0 : 64;
      __syncthreads();
      for (int e = threadIdx.x; e < 64 * 16; e += blockDim.x) {
        const int j = e / 16, c = e % 16;
        ys[j][c] = (j < jw && c < cw) ? s.Y[((size_t)mu * nc + c0 + c) * s.kmax + j0 + j] : 0.0;
      }
      __syncthreads();
      if (r < N) {
        for (int j = 0; j < jw; ++j) {
          const double v = V[(size_t)(j0 + j) * N + r];
#pragma unroll
          for (int c = 0; c < 16; ++c) acc[c] = fma(v, ys[j][c], acc[c]);
        }
      }
    }
    if (r < N) {
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < cw) X[((size_t)mu + (size_t)(c0 + c) * nmu) * N + r] = acc[c];
    }
  }
}

acp_status count_active(acp_ctx* ctx, const int* active, int n, int* out_h) {
  int* cnt = ctx->d_flag + 4;
  ACP_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(int), ctx->stream));
  int blocks = (n + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  ::acp::note_launch(ctx);
  count_active_kernel<<<blocks, 256, 0, ctx->stream>>>(active, n, cnt);
  ACP_LAUNCH(ctx);
  ACP_CUDA(ctx, cudaMemcpyAsync(out_h, cnt, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ACP_OK;
}

acp_status check_nan(acp_ctx* ctx) {
  int h = 0;
  ACP_CUDA(ctx, cudaMemcpyAsync(&h, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (h) return set_error(ctx, ACP_E_NUMERIC, "NaN or Inf met in a Sternheimer solve");
  return ACP_OK;
}

struct Report {
  unsigned long long steps, conv;
  int max_it;
  int pad;
  double max_res;
};

acp_status collect_report(acp_ctx* ctx, int n, const int* iters, const double* phibar, const double* beta1,
                          double tol, SolveReport* rep, long long pairs_per_entry) {
  Report* d = nullptr;
  ACP_TRY(ws(ctx, "minres_report", 1, &d));
  ACP_CUDA(ctx, cudaMemsetAsync(d, 0, sizeof(Report), ctx->stream));
  int blocks = (n + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  ::acp::note_launch(ctx);
  minres_report_kernel<<<blocks, 256, 0, ctx->stream>>>(n, iters, phibar, beta1, tol, &d->steps, &d->max_it, &d->conv,
                                                        &d->max_res);
  ACP_LAUNCH(ctx);
  Report h{};
  ACP_CUDA(ctx, cudaMemcpyAsync(&h, d, sizeof(Report), cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  rep->steps += (long long)h.steps * pairs_per_entry;
  rep->converged += (long long)h.conv;
  if (h.max_it > rep->max_iters) rep->max_iters = h.max_it;
  if (h.max_res > rep->max_rel_res) rep->max_rel_res = h.max_res;
  if ((long long)h.conv < (long long)n) rep->all_converged = false;
  return ACP_OK;
}

}  // namespace

// Projection period of the Lanczos vectors.  Rounding puts occupied components into each new
// vector; the shifts of Alg. 1 (eps_i) and of Eq. eqncompressU (Chebyshev nodes) lie inside the
// occupied band, where H - s has eigenvalues eps_j - s close to zero (the orbitals of distant,
// nearly isolated atoms are almost degenerate).  Left in the Lanczos basis for a few steps, those
// components make MINRES resolve the near-zero eigenvalues and its residual stalls (on the
// 128-atom chain at 1e-8 with a period of 15, while projecting every step converges in ~220
// steps).  The automatic period is therefore 1; a caller may ask for a longer one.
int projection_period(const acp_ctx* ctx) {
  if (ctx->opt.project_every > 0) return ctx->opt.project_every;
  return 1;
}

acp_status minres_batched(acp_ctx* ctx, const double* B, int ncol, const double* shift_d, double* X,
                          SolveReport* rep, double t0_ms) {
  if (ncol <= 0) return ACP_OK;
  if (ctx->opt.precision == ACP_PREC_MIXED) return minres_batched_mixed(ctx, B, ncol, shift_d, X, rep, t0_ms);
  return minres_batched_fp64(ctx, B, ncol, shift_d, X, ctx->opt.stern_tol, rep, t0_ms);
}

acp_status minres_batched_fp64(acp_ctx* ctx, const double* B, int ncol, const double* shift_d, double* X,
                               double tol, SolveReport* rep, double t0_ms) {
  if (ncol <= 0) return ACP_OK;
  const int N = ctx->N;
  const size_t nv = (size_t)N * ncol;
  MinresState s{};
  double* vec = nullptr;
  double* sc = nullptr;
  int* iv = nullptr;
  ACP_TRY(ws(ctx, "minres_vec", 5 * nv, &vec));
  ACP_TRY(ws(ctx, "minres_sc", 8 * (size_t)ncol, &sc));
  ACP_TRY(ws(ctx, "minres_iv", 2 * (size_t)ncol, &iv));
  s.V = vec; s.Vp = vec + nv; s.P = vec + 2 * nv; s.W1 = vec + 3 * nv; s.W2 = vec + 4 * nv;
  s.alpha = sc; s.beta = sc + ncol; s.beta1 = sc + 2 * ncol; s.cs = sc + 3 * ncol; s.sn = sc + 4 * ncol;
  s.dbar = sc + 5 * ncol; s.epsln = sc + 6 * ncol; s.phibar = sc + 7 * ncol;
  s.active = iv; s.iters = iv + ncol;
  ACP_CUDA(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
  ::acp::note_launch(ctx);
  minres_init_kernel<<<ncol, kThreads, 0, ctx->stream>>>(N, B, s, X, ctx->d_flag);
  ACP_LAUNCH(ctx);
  const int maxit = ctx->opt.stern_maxit;
  const int period = projection_period(ctx);
  for (int it = 0; it < maxit; ++it) {
    ACP_TRY(spectral_apply(ctx, s.V, N, ncol, MULT_KINETIC, true, shift_d, s.P, N, s.alpha, s.active, s.Vp, s.beta));
    if (it % period == period - 1 || it < 2) ACP_TRY(project(ctx, s.P, N, ncol, s.P, N));
    ::acp::note_launch(ctx);
    minres_step_kernel<<<ncol, kThreads, 0, ctx->stream>>>(N, s, X, tol, maxit, ctx->d_flag);
    ACP_LAUNCH(ctx);
    if ((it & 15) == 15 || it == maxit - 1) {
      int n_act = 0;
      ACP_TRY(count_active(ctx, s.active, ncol, &n_act));
      if (n_act == 0) break;
      if (deadline_passed(ctx, t0_ms)) return set_error(ctx, ACP_E_TIMEOUT, "deadline passed in MINRES");
    }
  }
  ACP_TRY(check_nan(ctx));
  ACP_TRY(collect_report(ctx, ncol, s.iters, s.phibar, s.beta1, tol, rep, 1));
  return ACP_OK;
}

static acp_status minres_multishift_vectors(acp_ctx* ctx, const double* B, int nmu, const double* nodes_d, int nc,
                                            double* X, SolveReport* rep, double t0_ms) {
  if (nmu <= 0) return ACP_OK;
  if (nc < 1 || nc > kMaxShifts) return set_error(ctx, ACP_E_ARG, "number of shifts %d outside [1, %d]", nc, kMaxShifts);
  const int N = ctx->N;
  const size_t nv = (size_t)N * nmu;
  MsState s{};
  double* vec = nullptr;
  double* sc = nullptr;
  int* iv = nullptr;
  ACP_TRY(ws(ctx, "ms_vec", (3 + 2 * (size_t)nc) * nv, &vec));
  ACP_TRY(ws(ctx, "ms_sc", (3 + 5 * (size_t)nc) * nmu, &sc));
  ACP_TRY(ws(ctx, "ms_iv", (2 + (size_t)nc) * nmu, &iv));
  s.V = vec; s.Vp = vec + nv; s.P = vec + 2 * nv; s.W1 = vec + 3 * nv; s.W2 = vec + (3 + nc) * nv;
  s.alpha = sc; s.beta = sc + nmu; s.beta1 = sc + 2 * nmu;
  double* q = sc + 3 * nmu;
  const size_t nq = (size_t)nc * nmu;
  s.cs = q; s.sn = q + nq; s.dbar = q + 2 * nq; s.epsln = q + 3 * nq; s.phibar = q + 4 * nq;
  s.active = iv; s.iters = iv + nmu; s.act_c = iv + 2 * nmu;
  s.nodes = nodes_d;
  ACP_CUDA(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
  ::acp::note_launch(ctx);
  ms_init_kernel<<<nmu, kThreads, 0, ctx->stream>>>(N, nmu, nc, B, s, X, ctx->d_flag);
  ACP_LAUNCH(ctx);
  const double tol = ctx->opt.stern_tol;
  const int maxit = ctx->opt.stern_maxit;
  const int period = projection_period(ctx);
  for (int it = 0; it < maxit; ++it) {
    ACP_TRY(spectral_apply(ctx, s.V, N, nmu, MULT_KINETIC, true, nullptr, s.P, N, s.alpha, s.active, s.Vp, s.beta));
    if (it % period == period - 1 || it < 2) ACP_TRY(project(ctx, s.P, N, nmu, s.P, N));
    ::acp::note_launch(ctx);
    ms_step_kernel<<<nmu, kThreads, 0, ctx->stream>>>(N, nmu, nc, s, X, tol, maxit, ctx->d_flag);
    ACP_LAUNCH(ctx);
    if ((it & 15) == 15 || it == maxit - 1) {
      int n_act = 0;
      ACP_TRY(count_active(ctx, s.active, nmu, &n_act));
      if (n_act == 0) break;
      if (deadline_passed(ctx, t0_ms)) return set_error(ctx, ACP_E_TIMEOUT, "deadline passed in MINRES");
    }
  }
  ACP_TRY(check_nan(ctx));
  // per (shift, mu) residual estimates; iteration counts are per mu (shared Lanczos process)
  Report* d = nullptr;
  ACP_TRY(ws(ctx, "minres_report", 1, &d));
  ACP_CUDA(ctx, cudaMemsetAsync(d, 0, sizeof(Report), ctx->stream));
  int blocks = (int)((nq + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  ::acp::note_launch(ctx);
  ms_report_kernel<<<blocks, 256, 0, ctx->stream>>>(nmu, nc, s.iters, s.phibar, s.beta1, tol, &d->steps, &d->max_it,
                                                    &d->conv, &d->max_res);
  ACP_LAUNCH(ctx);
  Report h{};
  ACP_CUDA(ctx, cudaMemcpyAsync(&h, d, sizeof(Report), cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  rep->steps += (long long)h.steps;
  rep->converged += (long long)h.conv;
  if (h.max_it > rep->max_iters) rep->max_iters = h.max_it;
  if (h.max_res > rep->max_rel_res) rep->max_rel_res = h.max_res;
  if ((long long)h.conv < (long long)nq) rep->all_converged = false;
  return ACP_OK;
}


static acp_status ms_report(acp_ctx* ctx, int nmu, int nc, const int* iters, const double* phibar, const double* beta1,
                            double tol, SolveReport* rep) {
  const size_t nq = (size_t)nc * nmu;
  Report* d = nullptr;
  ACP_TRY(ws(ctx, "minres_report", 1, &d));
  ACP_CUDA(ctx, cudaMemsetAsync(d, 0, sizeof(Report), ctx->stream));
  int blocks = (int)((nq + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  ::acp::note_launch(ctx);
  ms_report_kernel<<<blocks, 256, 0, ctx->stream>>>(nmu, nc, iters, phibar, beta1, tol, &d->steps, &d->max_it,
                                                    &d->conv, &d->max_res);
  ACP_LAUNCH(ctx);
  Report h{};
  ACP_CUDA(ctx, cudaMemcpyAsync(&h, d, sizeof(Report), cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  rep->steps += (long long)h.steps;
  rep->converged += (long long)h.conv;
  if (h.max_it > rep->max_iters) rep->max_iters = h.max_it;
  if (h.max_res > rep->max_rel_res) rep->max_rel_res = h.max_res;
  if ((long long)h.conv < (long long)nq) rep->all_converged = false;
  return ACP_OK;
}

static acp_status minres_multishift_basis(acp_ctx* ctx, const double* B, int nmu, const double* nodes_d, int nc,
                                          double* X, int kmax, SolveReport* rep, double t0_ms) {
  const int N = ctx->N;
  MsBasis s{};
  s.kmax = kmax;
  s.slot_ld = (size_t)(kmax + 2) * N;
  double *vb = nullptr, *sc = nullptr, *cf = nullptr, *yb = nullptr, *pb = nullptr;
  int* iv = nullptr;
  const size_t nq = (size_t)nc * nmu;
  ACP_TRY(ws(ctx, "msb_basis", s.slot_ld * nmu, &vb));
  ACP_TRY(ws(ctx, "msb_p", (size_t)N * nmu, &pb));
  ACP_TRY(ws(ctx, "msb_sc", 3 * (size_t)nmu + 5 * nq, &sc));
  ACP_TRY(ws(ctx, "msb_coef", 4 * nq * kmax, &cf));
  ACP_TRY(ws(ctx, "msb_y", nq * kmax, &yb));
  ACP_TRY(ws(ctx, "msb_iv", 2 * (size_t)nmu, &iv));
  s.Vb = vb; s.P = pb; s.coef = cf; s.Y = yb;
  s.alpha = sc; s.beta = sc + nmu; s.beta1 = sc + 2 * nmu;
  double* q = sc + 3 * nmu;
  s.cs = q; s.sn = q + nq; s.dbar = q + 2 * nq; s.epsln = q + 3 * nq; s.phibar = q + 4 * nq;
  s.active = iv; s.iters = iv + nmu;
  s.nodes = nodes_d;
  ACP_CUDA(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
  ::acp::note_launch(ctx);
  msb_init_kernel<<<nmu, kThreads, 0, ctx->stream>>>(N, nmu, nc, B, s, ctx->d_flag);
  ACP_LAUNCH(ctx);
  const double tol = ctx->opt.stern_tol;
  const int period = projection_period(ctx);
  int k = 1;
  for (; k <= kmax; ++k) {
    const double* vk = s.Vb + (size_t)k * N;
    const double* vkm = s.Vb + (size_t)(k - 1) * N;
    ACP_TRY(spectral_apply(ctx, vk, (int)s.slot_ld, nmu, MULT_KINETIC, true, nullptr, s.P, N, s.alpha, s.active, vkm,
                           s.beta));
    if ((k - 1) % period == period - 1 || k <= 2) ACP_TRY(project(ctx, s.P, N, nmu, s.P, N));
    ::acp::note_launch(ctx);
    msb_step_kernel<<<nmu, kThreads, 0, ctx->stream>>>(N, nmu, nc, k, s, tol, ctx->d_flag);
    ACP_LAUNCH(ctx);
    if ((k & 15) == 0 || k == kmax) {
      int n_act = 0;
      ACP_TRY(count_active(ctx, s.active, nmu, &n_act));
      if (n_act == 0) break;
      if (deadline_passed(ctx, t0_ms)) return set_error(ctx, ACP_E_TIMEOUT, "deadline passed in MINRES");
    }
  }
  ACP_TRY(check_nan(ctx));
  ::acp::note_launch(ctx);
  msb_backsub_kernel<<<(int)((nq + 127) / 128), 128, 0, ctx->stream>>>(nmu, nc, s);
  ACP_LAUNCH(ctx);
  ::acp::note_launch(ctx);
  msb_assemble_kernel<<<dim3((N + 255) / 256, nmu), 256, 0, ctx->stream>>>(N, nmu, nc, s, X);
  ACP_LAUNCH(ctx);
  return ms_report(ctx, nmu, nc, s.iters, s.phibar, s.beta1, tol, rep);
}

acp_status minres_multishift(acp_ctx* ctx, const double* B, int nmu, const double* nodes_d, int nc, double* X,
                             SolveReport* rep, double t0_ms) {
  if (nmu <= 0) return ACP_OK;
  if (nc < 1 || nc > kMaxShifts) return set_error(ctx, ACP_E_ARG, "number of shifts %d outside [1, %d]", nc, kMaxShifts);
  if (ctx->opt.precision == ACP_PREC_MIXED) return minres_multishift_mixed(ctx, B, nmu, nodes_d, nc, X, rep, t0_ms);
  if (ctx->opt.ms_variant != 2) {
    // stored-basis variant: up to 512 Lanczos steps, within min(32 GB, half the free memory)
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    auto it = ctx->ws.bufs.find("msb_basis");  // memory this buffer already holds counts as available
    if (it != ctx->ws.bufs.end()) free_b += it->second.second;
    size_t budget = free_b / 2;
    if (budget > (size_t(32) << 30)) budget = size_t(32) << 30;
    const size_t per_slot = (size_t)ctx->N * nmu * sizeof(double) + (size_t)nc * nmu * 5 * sizeof(double);
    const size_t fit = per_slot ? budget / per_slot : 0;
    int kmax = ctx->opt.stern_maxit;
    if (kmax > 512) kmax = 512;
    if ((size_t)kmax + 2 > fit) kmax = (int)fit - 2;
    // the basis must hold a whole solve: with fewer than 384 slots (large grids with many
    // points) the per-shift-vector variant is used instead
    if (kmax >= 384 || ctx->opt.ms_variant == 1)
      return minres_multishift_basis(ctx, B, nmu, nodes_d, nc, X, kmax < 1 ? 1 : kmax, rep, t0_ms);
  }
  return minres_multishift_vectors(ctx, B, nmu, nodes_d, nc, X, rep, t0_ms);
}

}  // namespace acp
