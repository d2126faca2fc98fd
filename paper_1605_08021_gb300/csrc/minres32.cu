// Mixed-precision Sternheimer solves: FP32 MINRES with the tensor-core (3xTF32) projector,
// recovered to the FP64 tolerance by iterative refinement.
//
//   refine:   X (FP64) starts from 0 or from a given iterate; each round forms the FP64 residual
//             R = B - (H - s) X with the FP64 spectral operator (X stays in the unoccupied space,
//             where Q(H - s)Q = H - s), scales it to unit norm, projects it in FP32 and solves
//             Q(H - s)Q D = R / |R| by FP32 MINRES to a relative 1e-6; X += |R| D in FP64.
//             Converged columns are masked out of the later rounds.
//   multi-shift (Eq. eqncompressU): the first pass runs one FP32 Lanczos process per selected
//             point for all N_c Chebyshev shifts (stored FP32 basis, per-shift Givens recurrences
//             in FP64); the refinement rounds then correct every (shift, point) pair on its own,
//             because the residuals of different shifts no longer share a Krylov space.
//
// FP32 blocks use the leading dimension ctx->ld32 (N rounded up to 32; the padding is zero).
#include "internal.cuh"

#include <vector>

namespace acp {

int projection_period(const acp_ctx* ctx);

namespace {

constexpr int kThreads = 256;
constexpr double kInnerTol = 1e-6;   // relative residual of every FP32 inner solve
constexpr int kMaxRounds = 8;        // refinement rounds

__device__ __forceinline__ float block_sum32(float v, float* red) {
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

int grid_for(size_t total) {
  size_t b = (total + 255) / 256;
  if (b > 65535) b = 65535;
  return b < 1 ? 1 : (int)b;
}

// ---- FP32 single-shift batched MINRES -----------------------------------------------------
// Solve state of the n columns being iterated (compact index j); the caller's blocks (right-hand
// sides R, corrections D, iteration counts) keep their own column order, map[j] being column j's
// index there.  When most columns have converged the state is gathered into a smaller set.
struct M32 {
  float *V, *Vp, *P, *W1, *W2;         // ld x n
  float *alpha, *beta;                 // n (Lanczos coefficients, read by the spectral kernel)
  double *beta1, *cs, *sn, *dbar, *epsln, *phibar;
  double* tolc;                        // n: relative tolerance of each column
  float* shift;                        // n
  int *active, *iters;                 // n
  int* map;                            // n: column in the caller's blocks
  int* iters_out;                      // iteration count by the caller's column
  int ld;
};

// Column j starts from R[:, map[j]] / ||R[:, map[j]]|| with D[:, map[j]] = 0; its shift and
// tolerance are copied from the caller's per-column arrays.
__global__ void __launch_bounds__(kThreads) m32_init_kernel(int N, const float* __restrict__ R, M32 s,
                                                           float* __restrict__ D, const float* __restrict__ shift_full,
                                                           const double* __restrict__ tol_full, double tol) {
  __shared__ float red[32];
  const int j = blockIdx.x;
  const int col = s.map[j];
  const size_t off = (size_t)j * s.ld, offc = (size_t)col * s.ld;
  float acc = 0.f;
  for (int a = threadIdx.x; a < N; a += blockDim.x) acc = fmaf(R[offc + a], R[offc + a], acc);
  const float nrm = sqrtf(block_sum32(acc, red));
  const bool ok = isfinite(nrm) && nrm > 0.f;
  const float inv = ok ? 1.f / nrm : 0.f;
  for (int a = threadIdx.x; a < N; a += blockDim.x) {
    s.V[off + a] = R[offc + a] * inv;
    s.Vp[off + a] = 0.f;
    s.W1[off + a] = 0.f;
    s.W2[off + a] = 0.f;
    D[offc + a] = 0.f;
  }
  if (threadIdx.x == 0) {
    s.beta1[j] = ok ? nrm : 0.0;
    s.beta[j] = 0.f;
    s.cs[j] = -1.0;
    s.sn[j] = 0.0;
    s.dbar[j] = 0.0;
    s.epsln[j] = 0.0;
    s.phibar[j] = ok ? nrm : 0.0;
    s.iters[j] = 0;
    s.active[j] = ok ? 1 : 0;
    s.shift[j] = shift_full[col];
    s.tolc[j] = tol_full ? tol_full[col] : tol;
    s.iters_out[col] = 0;
  }
}

__global__ void __launch_bounds__(kThreads) m32_step_kernel(int N, M32 s, float* __restrict__ D, int maxit) {
  __shared__ float red[32];
  __shared__ float coef[4];
  const int j = blockIdx.x;
  if (!s.active[j]) return;
  const size_t off = (size_t)j * s.ld;
  const float* P = s.P + off;
  float acc = 0.f;
  for (int r = threadIdx.x; r < N; r += blockDim.x) acc = fmaf(P[r], P[r], acc);
  const float bnf = sqrtf(block_sum32(acc, red));
  if (threadIdx.x == 0) {
    const double bn = bnf, a = s.alpha[j];
    const double oldeps = s.epsln[j], c = s.cs[j], sg = s.sn[j], db = s.dbar[j], pb = s.phibar[j];
    const double delta = c * db + sg * a;
    const double gbar = sg * db - c * a;
    const double gamma = fmax(hypot(gbar, bn), 1e-300);
    const double cn = gbar / gamma, sn_ = bn / gamma;
    const double phi = cn * pb, pbn = sn_ * pb;
    coef[0] = (float)oldeps;
    coef[1] = (float)delta;
    coef[2] = (float)(1.0 / gamma);
    coef[3] = (float)phi;
    s.epsln[j] = sg * bn;
    s.dbar[j] = -c * bn;
    s.cs[j] = cn;
    s.sn[j] = sn_;
    s.phibar[j] = pbn;
    s.beta[j] = bnf;
    const int it = s.iters[j] + 1;
    s.iters[j] = it;
    s.iters_out[s.map[j]] = it;
    const bool bad = !isfinite(bn) || !isfinite(pbn);
    if (bad || fabs(pbn) <= s.tolc[j] * s.beta1[j] || bn == 0.0 || it >= maxit) s.active[j] = 0;
  }
  __syncthreads();
  const float oe = coef[0], de = coef[1], ig = coef[2], ph = coef[3];
  const float ib = (bnf > 0.f) ? 1.f / bnf : 0.f;
  float* W1 = s.W1 + off;
  float* W2 = s.W2 + off;
  float* V = s.V + off;
  float* Vp = s.Vp + off;
  float* d = D + (size_t)s.map[j] * s.ld;
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    const float v = V[r];
    const float w1 = W1[r];
    const float w = (v - oe * W2[r] - de * w1) * ig;
    W2[r] = w1;
    W1[r] = w;
    d[r] = fmaf(ph, w, d[r]);
    Vp[r] = v;
    V[r] = P[r] * ib;
  }
}

// Compaction: column k of the new state is column idx[k] of the old one (vectors V, Vp, W1, W2 of
// N rows; grid (row tiles, n)); the new columns are all active.
__global__ void m32_gather_vectors_kernel(int N, int n, const int* __restrict__ idx, M32 o, M32 t) {
  const int k = blockIdx.y;
  const size_t src = (size_t)idx[k] * o.ld, dst = (size_t)k * t.ld;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < N; a += gridDim.x * blockDim.x) {
    t.V[dst + a] = o.V[src + a];
    t.Vp[dst + a] = o.Vp[src + a];
    t.W1[dst + a] = o.W1[src + a];
    t.W2[dst + a] = o.W2[src + a];
  }
}

__global__ void m32_gather_scalars_kernel(int n, const int* __restrict__ idx, M32 o, M32 t) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int q = idx[k];
    t.alpha[k] = o.alpha[q];
    t.beta[k] = o.beta[q];
    t.beta1[k] = o.beta1[q];
    t.cs[k] = o.cs[q];
    t.sn[k] = o.sn[q];
    t.dbar[k] = o.dbar[q];
    t.epsln[k] = o.epsln[q];
    t.phibar[k] = o.phibar[q];
    t.tolc[k] = o.tolc[q];
    t.shift[k] = o.shift[q];
    t.iters[k] = o.iters[q];
    t.map[k] = o.map[q];
    t.active[k] = 1;
  }
}

__global__ void iota32_kernel(int* p, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

__global__ void count_active32(const int* __restrict__ active, int n, int* out) {
  int c = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) c += active[i] != 0;
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void sum_iters_kernel(const int* __restrict__ iters, int n, unsigned long long* steps, int* max_it) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    atomicAdd(steps, (unsigned long long)iters[i]);
    atomicMax(max_it, iters[i]);
  }
}

// ---- refinement kernels (FP64 <-> FP32) ---------------------------------------------------------
// Per column: rn = ||R_j|| (FP64); R32_j = R_j / rn in FP32 (zero for a zero column); scale_j = rn.
__global__ void __launch_bounds__(kThreads) scale_to_f32_kernel(int N, int ld32, const double* __restrict__ R,
                                                                float* __restrict__ R32, double* __restrict__ scale,
                                                                int* nan_flag) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  const double* r = R + (size_t)j * N;
  double acc = 0.0;
  for (int a = threadIdx.x; a < N; a += blockDim.x) acc += r[a] * r[a];
  const double rn = sqrt(block_sum(acc, red));
  const bool go = isfinite(rn) && rn > 0.0;
  const double inv = go ? 1.0 / rn : 0.0;
  float* o = R32 + (size_t)j * ld32;
  for (int a = threadIdx.x; a < N; a += blockDim.x) o[a] = (float)(r[a] * inv);
  if (threadIdx.x == 0) {
    scale[j] = go ? rn : 0.0;
    if (!isfinite(rn)) atomicExch(nan_flag, 1);
  }
}

// After the FP32 projection of R32: the projected residual norm is ||R32_j|| * scale_j, relative
// rel_j = that / ||B_j||.  The FP64 residual B - (H - s)X cannot be evaluated more accurately than
// the rounding of its own evaluation: the FFT of the kinetic term errs by ~log2(N) u ||x|| times the
// largest multiplier (the standard forward-error bound of the radix FFT), so
//   floor_j = (log2 N + 4) u (||H||_bound + |s_j|) ||X_j|| / ||B_j||,  u = 2^-53,
// with ||H||_bound = max k^2/2 + max |V| (hbound).  Column j is converged when rel_j <= max(tol,
// floor_j): masked, and its R32 zeroed.  From the third round on, a column whose round gained less
// than 10x has met the attainable accuracy of its FP32 inner solves (shifts close to an eigenvalue
// make Q(H - s)Q ill conditioned, and FP32 Lanczos then stalls at its own floor): it leaves the FP32
// rounds and is finished by FP64 MINRES (polish_fp64 below).
// The inner solve of column j only has to reduce its residual by the factor tol / rel_j that is
// still missing (with a margin of 4, never below the FP32 floor kInnerTol, never above 1e-2).
__global__ void __launch_bounds__(kThreads) refine_check_kernel(int N, int ld32, float* __restrict__ R32,
                                                                const double* __restrict__ X,
                                                                const double* __restrict__ shift,
                                                                const double* __restrict__ hbound, double log_fac,
                                                                const double* __restrict__ scale,
                                                                const double* __restrict__ bnorm, double tol,
                                                                double* __restrict__ rel, double* __restrict__ prev,
                                                                double* __restrict__ floor_out, int round,
                                                                int* __restrict__ act,
                                                                double* __restrict__ tol_in, double floor_tol) {
  __shared__ float red[32];
  __shared__ double red64[32];
  const int j = blockIdx.x;
  float* o = R32 + (size_t)j * ld32;
  const double* x = X + (size_t)j * N;
  float acc = 0.f;
  double xacc = 0.0;
  for (int a = threadIdx.x; a < N; a += blockDim.x) {
    acc = fmaf(o[a], o[a], acc);
    xacc += x[a] * x[a];
  }
  const double pn = sqrt((double)block_sum32(acc, red));
  const double xn = sqrt(block_sum(xacc, red64));
  const double bn = bnorm[j];
  const double rl = (bn > 0.0) ? pn * scale[j] / bn : 0.0;
  const double fl = (bn > 0.0) ? log_fac * 0x1p-53 * (hbound[0] + fabs(shift[j])) * xn / bn : 0.0;
  const double lim = fmax(tol, fl);
  const bool stalled = round > 1 && rl > 0.1 * prev[j];
  const bool go = rl > lim && !stalled;
  if (!go)
    for (int a = threadIdx.x; a < N; a += blockDim.x) o[a] = 0.f;
  if (threadIdx.x == 0) {
    rel[j] = rl;
    prev[j] = rl;
    floor_out[j] = fl;
    act[j] = go ? 1 : 0;
    const double want = (rl > 0.0) ? 0.25 * lim / rl : 1e-2;
    tol_in[j] = fmin(1e-2, fmax(floor_tol, want));
  }
}

// hbound[0] = max_a kin[a] + max_a |V[a]|: a bound of ||H||_2 (H = T + V, T diagonal in Fourier
// space with entries kin >= 0, V diagonal in real space); one CTA.
__global__ void __launch_bounds__(kThreads) hbound_kernel(int N, const double* __restrict__ kin,
                                                          const double* __restrict__ V, double* __restrict__ hbound) {
  __shared__ double rk[kThreads], rv[kThreads];
  double mk = 0.0, mv = 0.0;
  for (int a = threadIdx.x; a < N; a += blockDim.x) {
    mk = fmax(mk, kin[a]);
    mv = fmax(mv, fabs(V[a]));
  }
  rk[threadIdx.x] = mk;
  rv[threadIdx.x] = mv;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      rk[threadIdx.x] = fmax(rk[threadIdx.x], rk[threadIdx.x + o]);
      rv[threadIdx.x] = fmax(rv[threadIdx.x], rv[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) hbound[0] = rk[0] + rv[0];
}

// X_j += scale_j * D32_j for the active columns
__global__ void refine_update_kernel(int N, int ncol, int ld32, const float* __restrict__ D32,
                                     const double* __restrict__ scale, const int* __restrict__ act,
                                     double* __restrict__ X) {
  const size_t total = (size_t)N * ncol;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % N), j = (int)(e / N);
    if (act[j]) X[e] += scale[j] * (double)D32[(size_t)j * ld32 + a];
  }
}

// R_j = B_j - Y_j for the active columns
__global__ void residual_kernel(int N, int ncol, const double* __restrict__ B, const double* __restrict__ Y,
                                const int* __restrict__ act, double* __restrict__ R) {
  const size_t total = (size_t)N * ncol;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / N);
    if (act[j]) R[e] = B[e] - Y[e];
  }
}

__global__ void col_norms64(int N, int ncol, const double* __restrict__ X, double* __restrict__ out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= ncol) return;
  const double* x = X + (size_t)warp * N;
  double s = 0.0;
  for (int r = lane; r < N; r += 32) s += x[r] * x[r];
  s = warp_sum(s);
  if (lane == 0) out[warp] = sqrt(s);
}

__global__ void to_float_kernel(size_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] = (float)x[e];
}

// dst[:, k] = src[:, idx[k]] (N x n from N-row columns); shifts likewise when sh_src is given.
__global__ void gather_cols_kernel(int N, int n, const int* __restrict__ idx, const double* __restrict__ src,
                                   double* __restrict__ dst, const double* __restrict__ sh_src,
                                   double* __restrict__ sh_dst) {
  const size_t total = (size_t)N * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % N), k = (int)(e / N);
    dst[e] = src[(size_t)idx[k] * N + a];
    if (sh_src && a == 0) sh_dst[k] = sh_src[idx[k]];
  }
}

// dst[:, idx[k]] += src[:, k]
__global__ void scatter_add_cols_kernel(int N, int n, const int* __restrict__ idx, const double* __restrict__ src,
                                        double* __restrict__ dst) {
  const size_t total = (size_t)N * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % N), k = (int)(e / N);
    dst[(size_t)idx[k] * N + a] += src[e];
  }
}

// act[j] = 1 for the listed columns, 0 for the others
__global__ void mark_cols_kernel(int ncol, int n, const int* __restrict__ idx, int* __restrict__ act) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ncol; j += gridDim.x * blockDim.x) act[j] = 0;
}
__global__ void mark_cols2_kernel(int n, const int* __restrict__ idx, int* __restrict__ act) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) act[idx[k]] = 1;
}

// rel[idx[k]] = ||R_k|| / ||B_idx[k]|| for the N x n block R (FP64, already projected); one warp a column
__global__ void polish_rel_kernel(int N, int n, const int* __restrict__ idx, const double* __restrict__ R,
                                  const double* __restrict__ bnorm, double* __restrict__ rel) {
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (k >= n) return;
  const double* r = R + (size_t)k * N;
  double acc = 0.0;
  for (int a = lane; a < N; a += 32) acc += r[a] * r[a];
  acc = warp_sum(acc);
  if (lane == 0) {
    const double bn = bnorm[idx[k]];
    rel[idx[k]] = (bn > 0.0) ? sqrt(acc) / bn : 0.0;
  }
}

__global__ void refine_report_kernel(int n, const double* __restrict__ rel, const double* __restrict__ bnorm,
                                     const double* __restrict__ floor_in, double tol, unsigned long long* conv,
                                     double* max_res) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double r = (bnorm[i] > 0.0) ? rel[i] : 0.0;
    if (r <= fmax(tol, floor_in[i])) atomicAdd(conv, 1ull);
    atomicMax(reinterpret_cast<unsigned long long*>(max_res), (unsigned long long)__double_as_longlong(r));
  }
}

// ---- FP32 multi-shift MINRES with a stored basis --------------------------------------------
struct MsB32 {
  float* Vb;          // slot s of mu at Vb + mu * slot_ld + s * ld; slot 0 = 0
  size_t slot_ld;
  int ld;
  float* P;           // ld x nmu
  float *alpha, *beta;                       // nmu
  double* beta1;                             // nmu
  double *cs, *sn, *dbar, *epsln, *phibar;   // nc x nmu (c + nc mu)
  double* coef;       // (gamma, delta, eps, phi) per (mu, c, step)
  float* Y;           // y per (mu, c, step)
  int *active, *iters;
  const double* nodes;
  int kmax;
};

__global__ void __launch_bounds__(kThreads) msb32_init_kernel(int N, int nc, const float* __restrict__ Bm, MsB32 s) {
  __shared__ float red[32];
  const int mu = blockIdx.x;
  const float* b = Bm + (size_t)mu * s.ld;
  float acc = 0.f;
  for (int a = threadIdx.x; a < N; a += blockDim.x) acc = fmaf(b[a], b[a], acc);
  const float nrm = sqrtf(block_sum32(acc, red));
  const bool ok = isfinite(nrm) && nrm > 0.f;
  const float inv = ok ? 1.f / nrm : 0.f;
  float* v0 = s.Vb + (size_t)mu * s.slot_ld;
  for (int a = threadIdx.x; a < s.ld; a += blockDim.x) {
    v0[a] = 0.f;
    v0[s.ld + a] = (a < N) ? b[a] * inv : 0.f;
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
    s.beta[mu] = 0.f;
    s.iters[mu] = 0;
    s.active[mu] = ok ? 1 : 0;
  }
}

__global__ void __launch_bounds__(kThreads) msb32_step_kernel(int N, int nc, const int* __restrict__ kdev, MsB32 s,
                                                              double tol) {
  __shared__ float red[32];
  __shared__ int any_active;
  const int k = *kdev;  // step index from device memory, so that captured steps can be replayed
  const int mu = blockIdx.x;
  if (!s.active[mu]) return;
  const float* P = s.P + (size_t)mu * s.ld;
  float acc = 0.f;
  for (int r = threadIdx.x; r < N; r += blockDim.x) acc = fmaf(P[r], P[r], acc);
  const float bnf = sqrtf(block_sum32(acc, red));
  const float ib = (bnf > 0.f) ? 1.f / bnf : 0.f;
  float* vn = s.Vb + (size_t)mu * s.slot_ld + (size_t)(k + 1) * s.ld;
  for (int r = threadIdx.x; r < N; r += blockDim.x) vn[r] = P[r] * ib;
  if (threadIdx.x == 0) any_active = 0;
  __syncthreads();
  const double bn = bnf, a = s.alpha[mu];
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
    if (isfinite(pbn) && !(fabs(pbn) <= tol * s.beta1[mu])) atomicOr(&any_active, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s.beta[mu] = bnf;
    const int it = s.iters[mu] + 1;
    s.iters[mu] = it;
    if (!any_active || !isfinite(bn) || bn == 0.0 || it >= s.kmax) s.active[mu] = 0;
  }
}

__global__ void advance_k_kernel(int* kdev) { *kdev += 1; }

__global__ void msb32_backsub_kernel(int nmu, int nc, MsB32 s) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)nmu * nc) return;
  const int mu = (int)(t / nc);
  const int kk = s.iters[mu];
  const double* cf = s.coef + t * s.kmax * 4;
  float* y = s.Y + t * s.kmax;
  double y1 = 0.0, y2 = 0.0;
  for (int j = kk - 1; j >= 0; --j) {
    const double d1 = (j + 1 < kk) ? cf[(j + 1) * 4 + 1] : 0.0;
    const double e2 = (j + 2 < kk) ? cf[(j + 2) * 4 + 2] : 0.0;
    const double yj = (cf[j * 4 + 3] - d1 * y1 - e2 * y2) / cf[j * 4 + 0];
    y[j] = (float)yj;
    y2 = y1;
    y1 = yj;
  }
}

// X (FP64, N x nc nmu, column mu + c nmu) = scale_mu * sum_j v_{j+1} y_{c, j}
__global__ void __launch_bounds__(256) msb32_assemble_kernel(int N, int nmu, int nc, MsB32 s,
                                                             const double* __restrict__ scale,
                                                             double* __restrict__ X) {
  __shared__ float ys[64][16];
  const int mu = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int kk = s.iters[mu];
  const float* V = s.Vb + (size_t)mu * s.slot_ld + s.ld;
  const double sc = scale[mu];
  for (int c0 = 0; c0 < nc; c0 += 16) {
    const int cw = (nc - c0 < 16) ? nc - c0 : 16;
    float acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = 0.f;
    for (int j0 = 0; j0 < kk; j0 += 64) {
      const int jw = (kk - j0 < 64) ? kk - j0 : 64;
      __syncthreads();
      for (int e = threadIdx.x; e < 64 * 16; e += blockDim.x) {
        const int j = e / 16, c = e % 16;
        ys[j][c] = (j < jw && c < cw) ? s.Y[((size_t)mu * nc + c0 + c) * s.kmax + j0 + j] : 0.f;
      }
      __syncthreads();
      if (r < N) {
        for (int j = 0; j < jw; ++j) {
          const float v = V[(size_t)(j0 + j) * s.ld + r];
#pragma unroll
          for (int c = 0; c < 16; ++c) acc[c] = fmaf(v, ys[j][c], acc[c]);
        }
      }
    }
    if (r < N) {
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < cw) X[((size_t)mu + (size_t)(c0 + c) * nmu) * N + r] = sc * (double)acc[c];
    }
  }
}

// B_rep[:, mu + c nmu] = B[:, mu]; shifts[mu + c nmu] = nodes[c]
__global__ void replicate_kernel(int N, int nmu, int nc, const double* __restrict__ B, const double* __restrict__ nodes,
                                 double* __restrict__ Brep, double* __restrict__ shifts) {
  const size_t total = (size_t)N * nmu * nc;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % N);
    const size_t col = e / N;
    const int mu = (int)(col % nmu), c = (int)(col / nmu);
    Brep[e] = B[(size_t)mu * N + a];
    if (a == 0) shifts[col] = nodes[c];
  }
}

// Number of active columns; also fails fast when a tensor-core pipeline wait ran out (status word
// d_flag[8]), so that a broken pipeline cannot keep a long solve going.
acp_status count32(acp_ctx* ctx, const int* active, int n, int* out_h) {
  int* cnt = ctx->d_flag + 12;
  ACP_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(int), ctx->stream));
  int blocks = (n + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  ::acp::note_launch(ctx);
  count_active32<<<blocks, 256, 0, ctx->stream>>>(active, n, cnt);
  ACP_LAUNCH(ctx);
  int h[5] = {0, 0, 0, 0, 0};
  ACP_CUDA(ctx, cudaMemcpyAsync(h, ctx->d_flag + 8, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (h[0]) return tc_check(ctx);
  *out_h = h[4];
  return ACP_OK;
}

struct IterSum {
  unsigned long long steps;
  int max_it;
  int pad;
};

acp_status sum_iters(acp_ctx* ctx, const int* iters, int n, long long* steps, long long* max_it) {
  IterSum* d = nullptr;
  ACP_TRY(ws(ctx, "m32_itsum", 1, &d));
  ACP_CUDA(ctx, cudaMemsetAsync(d, 0, sizeof(IterSum), ctx->stream));
  int blocks = (n + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  ::acp::note_launch(ctx);
  sum_iters_kernel<<<blocks, 256, 0, ctx->stream>>>(iters, n, &d->steps, &d->max_it);
  ACP_LAUNCH(ctx);
  IterSum h{};
  ACP_CUDA(ctx, cudaMemcpyAsync(&h, d, sizeof(IterSum), cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *steps += (long long)h.steps;
  if (h.max_it > *max_it) *max_it = h.max_it;
  return ACP_OK;
}

// ---- CUDA-graph replay of the Lanczos loops ------------------------------------------------------
constexpr int kChunk = 16;  // steps between convergence checks

struct ChunkGraph {
  cudaGraphExec_t exec = nullptr;
  long long nodes = 0;
  bool warm = false;  // a chunk has run eagerly with the current buffers and column count
  ~ChunkGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

// Runs n Lanczos steps starting at step it0.  With `graphs`, a full chunk is captured once into a
// CUDA graph (the step functions launch the same kernels with the same arguments in every chunk:
// step indices live in device memory) and replayed for every later chunk; the first chunk, and the
// first after the buffers or the column count change, run eagerly, so that one-time work (tile
// autotuning, workspace growth) happens outside capture.
template <class Step>
acp_status run_chunk(acp_ctx* ctx, ChunkGraph& g, bool graphs, int it0, int n, Step step) {
  if (!graphs || n != kChunk || it0 == 0 || !g.warm) {
    for (int i = 0; i < n; ++i) ACP_TRY(step(it0 + i));
    g.warm = true;
    return ACP_OK;
  }
  if (!g.exec) {
    std::lock_guard<std::mutex> lock(device_mutex());
    const bool prof_on = ctx->prof.on;
    ctx->prof.on = false;
    const long long l0 = ctx->prof.launches;
    ACP_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    acp_status st = ACP_OK;
    for (int i = 0; i < n && st == ACP_OK; ++i) st = step(it0 + i);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    ctx->prof.on = prof_on;
    g.nodes = ctx->prof.launches - l0;
    ctx->prof.launches = l0;
    if (st != ACP_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return st != ACP_OK ? st : set_error(ctx, ACP_E_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
    }
    const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      g.exec = nullptr;
      return set_error(ctx, ACP_E_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
    }
  }
  ACP_CUDA(ctx, cudaGraphLaunch(g.exec, ctx->stream));
  ctx->prof.launches += g.nodes;
  return ACP_OK;
}

// FP32 inner solve of Q(H - s_j)Q D_j = R32_j (R32 projected, unit or zero columns).
// FP32 MINRES on the columns cols[0..n) of the caller's blocks (all ncol columns when cols is
// null): Q(H - shift32[c])Q D[:, c] = R32[:, c] to the relative tolerance tolc[c] (or tol).  Every
// chunk of steps, when fewer than 60% of the iterated columns are still active, the state of the
// active ones is gathered into a second buffer set, so that the spectral, projector and step
// kernels of the later steps only touch columns that still iterate.
acp_status minres32(acp_ctx* ctx, const float* R32, int ncol, const int* cols, int n, const float* shift32, float* D32,
                    double tol, const double* tolc, long long* steps, long long* max_it, double t0_ms) {
  const int N = ctx->N, ld = ctx->ld32;
  if (n <= 0) return ACP_OK;
  M32 st[2];
  for (int b = 0; b < 2; ++b) {
    const size_t nv = (size_t)ld * n;
    float* vec = nullptr;
    float* fsc = nullptr;
    double* dsc = nullptr;
    int* iv = nullptr;
    const char* names[2][4] = {{"m32_vec", "m32_fsc", "m32_dsc", "m32_iv"}, {"m32_vec2", "m32_fsc2", "m32_dsc2", "m32_iv2"}};
    // the second set is only touched once the first compaction shrinks the problem
    const size_t nvb = (b == 0) ? nv : (size_t)ld * ((n * 3 + 4) / 5);
    const size_t nb = (b == 0) ? (size_t)n : (size_t)((n * 3 + 4) / 5);
    ACP_TRY(ws(ctx, names[b][0], 5 * nvb, &vec));
    ACP_TRY(ws(ctx, names[b][1], 3 * nb, &fsc));
    ACP_TRY(ws(ctx, names[b][2], 7 * nb, &dsc));
    ACP_TRY(ws(ctx, names[b][3], 3 * nb, &iv));
    M32& s = st[b];
    s.ld = ld;
    s.V = vec; s.Vp = vec + nvb; s.P = vec + 2 * nvb; s.W1 = vec + 3 * nvb; s.W2 = vec + 4 * nvb;
    s.alpha = fsc; s.beta = fsc + nb; s.shift = fsc + 2 * nb;
    s.beta1 = dsc; s.cs = dsc + nb; s.sn = dsc + 2 * nb; s.dbar = dsc + 3 * nb; s.epsln = dsc + 4 * nb;
    s.phibar = dsc + 5 * nb; s.tolc = dsc + 6 * nb;
    s.active = iv; s.iters = iv + nb; s.map = iv + 2 * nb;
  }
  int* iters_out = nullptr;
  ACP_TRY(ws(ctx, "m32_itout", (size_t)ncol, &iters_out));
  ACP_CUDA(ctx, cudaMemsetAsync(iters_out, 0, sizeof(int) * ncol, ctx->stream));
  st[0].iters_out = st[1].iters_out = iters_out;
  if (cols) {
    ACP_CUDA(ctx, cudaMemcpyAsync(st[0].map, cols, sizeof(int) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  } else {
    ::acp::note_launch(ctx);
    iota32_kernel<<<grid_for(n), 256, 0, ctx->stream>>>(st[0].map, n);
    ACP_LAUNCH(ctx);
  }
  ::acp::note_launch(ctx);
  m32_init_kernel<<<n, kThreads, 0, ctx->stream>>>(N, R32, st[0], D32, shift32, tolc, tol);
  ACP_LAUNCH(ctx);
  const int maxit = ctx->opt.stern_maxit;
  const int period = projection_period(ctx);
  int cur = 0, ncur = n;
  auto step = [&](int it) -> acp_status {
    M32& s = st[cur];
    ACP_TRY(spectral32_apply(ctx, s.V, ld, ncur, s.shift, s.P, ld, s.alpha, s.active, s.Vp, ld, s.beta));
    if (it % period == period - 1 || it < 2) ACP_TRY(project32(ctx, s.P, ld, ncur, s.P, ld));
    ::acp::note_launch(ctx);
    cudaEvent_t ev0 = prof_begin(ctx);
    m32_step_kernel<<<ncur, kThreads, 0, ctx->stream>>>(N, s, D32, maxit);
    ACP_LAUNCH(ctx);
    // per iterated column: P read, V, W1, W2, D read and V, Vp, W1, W2, D written (FP32); columns
    // that converged inside the chunk return early, so this counts at most the bytes moved
    prof_end(ctx, "m32_step", ev0, 0.0, 40.0 * N * (double)ncur);
    return ACP_OK;
  };
  ChunkGraph graph;
  const bool graphs = ctx->opt.use_graphs && period == 1 && ctx->stream != nullptr;
  std::vector<int> hact;
  for (int it = 0; it < maxit;) {
    const int nstep = (maxit - it < kChunk) ? maxit - it : kChunk;
    ACP_TRY(run_chunk(ctx, graph, graphs, it, nstep, step));
    it += nstep;
    int n_act = 0;
    ACP_TRY(count32(ctx, st[cur].active, ncur, &n_act));
    if (n_act == 0) break;
    if (deadline_passed(ctx, t0_ms)) return set_error(ctx, ACP_E_TIMEOUT, "deadline passed in FP32 MINRES");
    if (n_act * 5 < ncur * 3 && it < maxit) {
      // gather the active columns into the other buffer set (sized 60% of n, enough for them)
      hact.resize(ncur);
      ACP_CUDA(ctx, cudaMemcpyAsync(hact.data(), st[cur].active, sizeof(int) * ncur, cudaMemcpyDeviceToHost,
                                    ctx->stream));
      ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      std::vector<int> idx;
      idx.reserve(n_act);
      for (int j = 0; j < ncur; ++j)
        if (hact[j]) idx.push_back(j);
      const int nn = (int)idx.size();
      int* d_idx = nullptr;
      ACP_TRY(ws(ctx, "m32_cidx", (size_t)(nn > 0 ? nn : 1), &d_idx));
      ACP_CUDA(ctx, cudaMemcpyAsync(d_idx, idx.data(), sizeof(int) * nn, cudaMemcpyHostToDevice, ctx->stream));
      const int nxt = 1 - cur;
      ::acp::note_launch(ctx);
      m32_gather_vectors_kernel<<<dim3((N + 255) / 256, nn), 256, 0, ctx->stream>>>(N, nn, d_idx, st[cur], st[nxt]);
      ACP_LAUNCH(ctx);
      ::acp::note_launch(ctx);
      m32_gather_scalars_kernel<<<grid_for(nn), 256, 0, ctx->stream>>>(nn, d_idx, st[cur], st[nxt]);
      ACP_LAUNCH(ctx);
      cur = nxt;
      ncur = nn;
      if (graph.exec) {  // the captured steps name the old buffers and column count
        cudaGraphExecDestroy(graph.exec);
        graph.exec = nullptr;
      }
      graph.warm = false;  // one eager chunk first: tile autotuning at the new column count
    }
  }
  ACP_TRY(tc_check(ctx));
  return sum_iters(ctx, iters_out, ncol, steps, max_it);
}

// FP64 finish of the columns the FP32 rounds left above their tolerance (stalled, or at the round
// cap): gather their FP64 residuals R (current for X), project them in FP64, solve
// Q(H - s)Q D = Q R by FP64 MINRES to the largest reduction any of them still needs, X += D, and
// re-evaluate the true FP64 residuals; at most three passes.  rel is updated for those columns.
acp_status polish_fp64(acp_ctx* ctx, const double* B, int ncol, const double* shift_d, double* X, double* R,
                       double* Y, int* act, const double* bnorm, double* rel, const double* floor_j,
                       SolveReport* rep, double t0_ms) {
  const int N = ctx->N;
  const double tol = ctx->opt.stern_tol;
  std::vector<double> hr(ncol), hf(ncol);
  ACP_CUDA(ctx, cudaMemcpyAsync(hf.data(), floor_j, sizeof(double) * ncol, cudaMemcpyDeviceToHost, ctx->stream));
  for (int pass = 0; pass < 3; ++pass) {
    ACP_CUDA(ctx, cudaMemcpyAsync(hr.data(), rel, sizeof(double) * ncol, cudaMemcpyDeviceToHost, ctx->stream));
    ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<int> idx;
    double need = 1.0;
    for (int j = 0; j < ncol; ++j) {
      const double lim = fmax(tol, hf[j]);
      if (hr[j] > lim) {
        idx.push_back(j);
        need = fmin(need, lim / hr[j]);
      }
    }
    if (idx.empty()) return ACP_OK;
    if (deadline_passed(ctx, t0_ms)) return set_error(ctx, ACP_E_TIMEOUT, "deadline passed in refinement");
    const int n = (int)idx.size();
    const size_t nv = (size_t)N * n;
    int* d_idx = nullptr;
    double *Rp = nullptr, *Dp = nullptr, *sp = nullptr;
    ACP_TRY(ws(ctx, "pl_idx", (size_t)n, &d_idx));
    ACP_TRY(ws(ctx, "pl_r", nv, &Rp));
    ACP_TRY(ws(ctx, "pl_d", nv, &Dp));
    ACP_TRY(ws(ctx, "pl_sh", (size_t)n, &sp));
    ACP_CUDA(ctx, cudaMemcpyAsync(d_idx, idx.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream));
    ::acp::note_launch(ctx);
    gather_cols_kernel<<<grid_for(nv), 256, 0, ctx->stream>>>(N, n, d_idx, R, Rp, shift_d, sp);
    ACP_LAUNCH(ctx);
    ACP_TRY(project(ctx, Rp, N, n, Rp, N));
    SolveReport sub{};
    ACP_TRY(minres_batched_fp64(ctx, Rp, n, sp, Dp, 0.5 * need, &sub, t0_ms));
    rep->steps += sub.steps;
    if (sub.max_iters > rep->max_iters) rep->max_iters = sub.max_iters;
    ::acp::note_launch(ctx);
    scatter_add_cols_kernel<<<grid_for(nv), 256, 0, ctx->stream>>>(N, n, d_idx, Dp, X);
    ACP_LAUNCH(ctx);
    ::acp::note_launch(ctx);
    mark_cols_kernel<<<grid_for(ncol), 256, 0, ctx->stream>>>(ncol, n, d_idx, act);
    ACP_LAUNCH(ctx);
    ::acp::note_launch(ctx);
    mark_cols2_kernel<<<grid_for(n), 256, 0, ctx->stream>>>(n, d_idx, act);
    ACP_LAUNCH(ctx);
    ACP_TRY(spectral_apply(ctx, X, N, ncol, MULT_KINETIC, true, shift_d, Y, N, nullptr, act));
    ::acp::note_launch(ctx);
    residual_kernel<<<grid_for((size_t)N * ncol), 256, 0, ctx->stream>>>(N, ncol, B, Y, act, R);
    ACP_LAUNCH(ctx);
    ::acp::note_launch(ctx);
    gather_cols_kernel<<<grid_for(nv), 256, 0, ctx->stream>>>(N, n, d_idx, R, Rp, nullptr, nullptr);
    ACP_LAUNCH(ctx);
    ACP_TRY(project(ctx, Rp, N, n, Rp, N));
    ::acp::note_launch(ctx);
    polish_rel_kernel<<<(n * 32 + 255) / 256, 256, 0, ctx->stream>>>(N, n, d_idx, Rp, bnorm, rel);
    ACP_LAUNCH(ctx);
  }
  return ACP_OK;
}

// Refinement rounds over ncol columns: B (FP64, projected), shift_d (FP64), X in/out.
acp_status refine(acp_ctx* ctx, const double* B, int ncol, const double* shift_d, double* X, bool x_zero,
                  SolveReport* rep, double t0_ms) {
  ACP_TRY(mixed_prepare(ctx));
  const int N = ctx->N, ld = ctx->ld32;
  const size_t nv = (size_t)N * ncol;
  double *R = nullptr, *Y = nullptr, *dsc = nullptr;
  float *R32 = nullptr, *D32 = nullptr, *sh32 = nullptr;
  int* act = nullptr;
  ACP_TRY(ws(ctx, "rf_r", nv, &R));
  ACP_TRY(ws(ctx, "rf_y", nv, &Y));
  ACP_TRY(ws(ctx, "rf_dsc", 6 * (size_t)ncol + 1, &dsc));
  ACP_TRY(ws(ctx, "rf_r32", (size_t)ld * ncol, &R32));
  ACP_TRY(ws(ctx, "rf_d32", (size_t)ld * ncol, &D32));
  ACP_TRY(ws(ctx, "rf_sh32", (size_t)ncol, &sh32));
  ACP_TRY(ws(ctx, "rf_act", (size_t)ncol, &act));
  double* bnorm = dsc;
  double* scale = dsc + ncol;
  double* rel = dsc + 2 * ncol;
  double* tol_in = dsc + 3 * ncol;
  double* prev = dsc + 4 * ncol;
  double* floor_j = dsc + 5 * ncol;
  double* hbound = dsc + 6 * ncol;
  int lg = 0;
  while ((1 << lg) < N) ++lg;
  const double log_fac = lg + 4.0;
  ::acp::note_launch(ctx);
  hbound_kernel<<<1, kThreads, 0, ctx->stream>>>(N, ctx->d_kin, ctx->d_V, hbound);
  ACP_LAUNCH(ctx);
  ACP_CUDA(ctx, cudaMemsetAsync(R32, 0, sizeof(float) * ld * ncol, ctx->stream));
  ::acp::note_launch(ctx);
  col_norms64<<<(ncol * 32 + 255) / 256, 256, 0, ctx->stream>>>(N, ncol, B, bnorm);
  ACP_LAUNCH(ctx);
  ::acp::note_launch(ctx);
  to_float_kernel<<<grid_for(ncol), 256, 0, ctx->stream>>>((size_t)ncol, shift_d, sh32);
  ACP_LAUNCH(ctx);
  if (x_zero) {
    ACP_CUDA(ctx, cudaMemsetAsync(X, 0, sizeof(double) * nv, ctx->stream));
    ACP_CUDA(ctx, cudaMemcpyAsync(R, B, sizeof(double) * nv, cudaMemcpyDeviceToDevice, ctx->stream));
  } else {
    ACP_TRY(spectral_apply(ctx, X, N, ncol, MULT_KINETIC, true, shift_d, Y, N, nullptr, nullptr));
    ACP_CUDA(ctx, cudaMemsetAsync(act, 0xff, sizeof(int) * ncol, ctx->stream));  // all columns
    ::acp::note_launch(ctx);
    residual_kernel<<<grid_for(nv), 256, 0, ctx->stream>>>(N, ncol, B, Y, act, R);
    ACP_LAUNCH(ctx);
  }
  ACP_CUDA(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
  const double tol = ctx->opt.stern_tol;
  for (int round = 0;; ++round) {
    ::acp::note_launch(ctx);
    scale_to_f32_kernel<<<ncol, kThreads, 0, ctx->stream>>>(N, ld, R, R32, scale, ctx->d_flag);
    ACP_LAUNCH(ctx);
    ACP_TRY(project32(ctx, R32, ld, ncol, R32, ld));
    ::acp::note_launch(ctx);
    refine_check_kernel<<<ncol, kThreads, 0, ctx->stream>>>(N, ld, R32, X, shift_d, hbound, log_fac, scale, bnorm,
                                                            tol, rel, prev, floor_j, round, act, tol_in, kInnerTol);
    ACP_LAUNCH(ctx);
    int n_act = 0;
    ACP_TRY(count32(ctx, act, ncol, &n_act));
    if (n_act == 0 || round == kMaxRounds) break;
    if (deadline_passed(ctx, t0_ms)) return set_error(ctx, ACP_E_TIMEOUT, "deadline passed in refinement");
    // the inner solve iterates only the columns still refining
    {
      std::vector<int> hact(ncol), cols;
      ACP_CUDA(ctx, cudaMemcpyAsync(hact.data(), act, sizeof(int) * ncol, cudaMemcpyDeviceToHost, ctx->stream));
      ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      cols.reserve(n_act);
      for (int j = 0; j < ncol; ++j)
        if (hact[j]) cols.push_back(j);
      int* d_cols = nullptr;
      ACP_TRY(ws(ctx, "rf_cols", (size_t)ncol, &d_cols));
      ACP_CUDA(ctx, cudaMemcpyAsync(d_cols, cols.data(), sizeof(int) * cols.size(), cudaMemcpyHostToDevice,
                                    ctx->stream));
      ACP_TRY(minres32(ctx, R32, ncol, d_cols, (int)cols.size(), sh32, D32, kInnerTol, tol_in, &rep->steps,
                       &rep->max_iters, t0_ms));
    }
    ::acp::note_launch(ctx);
    refine_update_kernel<<<grid_for(nv), 256, 0, ctx->stream>>>(N, ncol, ld, D32, scale, act, X);
    ACP_LAUNCH(ctx);
    ACP_TRY(spectral_apply(ctx, X, N, ncol, MULT_KINETIC, true, shift_d, Y, N, nullptr, act));
    ::acp::note_launch(ctx);
    residual_kernel<<<grid_for(nv), 256, 0, ctx->stream>>>(N, ncol, B, Y, act, R);
    ACP_LAUNCH(ctx);
  }
  ACP_TRY(polish_fp64(ctx, B, ncol, shift_d, X, R, Y, act, bnorm, rel, floor_j, rep, t0_ms));
  int h_nan = 0;
  ACP_CUDA(ctx, cudaMemcpyAsync(&h_nan, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (h_nan) return set_error(ctx, ACP_E_NUMERIC, "NaN or Inf met in a mixed-precision Sternheimer solve");
  struct Rep {
    unsigned long long conv;
    double max_res;
  };
  Rep* d = nullptr;
  ACP_TRY(ws(ctx, "rf_rep", 1, &d));
  ACP_CUDA(ctx, cudaMemsetAsync(d, 0, sizeof(Rep), ctx->stream));
  ::acp::note_launch(ctx);
  refine_report_kernel<<<grid_for(ncol), 256, 0, ctx->stream>>>(ncol, rel, bnorm, floor_j, tol, &d->conv,
                                                                 &d->max_res);
  ACP_LAUNCH(ctx);
  Rep h{};
  ACP_CUDA(ctx, cudaMemcpyAsync(&h, d, sizeof(Rep), cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  rep->converged += (long long)h.conv;
  if (h.max_res > rep->max_rel_res) rep->max_rel_res = h.max_res;
  if ((long long)h.conv < (long long)ncol) rep->all_converged = false;
  return ACP_OK;
}

}  // namespace

acp_status minres_batched_mixed(acp_ctx* ctx, const double* B, int ncol, const double* shift_d, double* X,
                                SolveReport* rep, double t0_ms) {
  if (ncol <= 0) return ACP_OK;
  if (ctx->opt.learned && ctx->dim == 2) {
    // start from the learned guess, projected onto range(Q) where the solution lies
    ACP_TRY(cnn_initial_guess(ctx, B, ctx->N, ncol, shift_d, X, ctx->N));
    ACP_TRY(project(ctx, X, ctx->N, ncol, X, ctx->N));
    return refine(ctx, B, ncol, shift_d, X, false, rep, t0_ms);
  }
  return refine(ctx, B, ncol, shift_d, X, true, rep, t0_ms);
}

acp_status minres_multishift_mixed(acp_ctx* ctx, const double* B, int nmu, const double* nodes_d, int nc, double* X,
                                   SolveReport* rep, double t0_ms) {
  if (nmu <= 0) return ACP_OK;
  ACP_TRY(mixed_prepare(ctx));
  const int N = ctx->N, ld = ctx->ld32;
  // ---- first pass: FP32 multi-shift on B / ||B|| --------------------------------------------
  double* bsc = nullptr;
  float* B32 = nullptr;
  ACP_TRY(ws(ctx, "ms32_bsc", (size_t)nmu, &bsc));
  ACP_TRY(ws(ctx, "ms32_b", (size_t)ld * nmu, &B32));
  ACP_CUDA(ctx, cudaMemsetAsync(B32, 0, sizeof(float) * ld * nmu, ctx->stream));
  ACP_CUDA(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
  ::acp::note_launch(ctx);
  scale_to_f32_kernel<<<nmu, kThreads, 0, ctx->stream>>>(N, ld, B, B32, bsc, ctx->d_flag);
  ACP_LAUNCH(ctx);
  ACP_TRY(project32(ctx, B32, ld, nmu, B32, ld));
  // stored basis within min(16 GB, half the free memory), at most 512 steps (a larger basis
  // lengthens the FP32 pass without shortening the refinement much: measured on the 2D lattice)
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  auto itb = ctx->ws.bufs.find("ms32_basis");
  if (itb != ctx->ws.bufs.end()) free_b += itb->second.second;
  size_t budget = free_b / 2;
  if (budget > (size_t(16) << 30)) budget = size_t(16) << 30;
  const size_t per_slot = (size_t)ld * nmu * sizeof(float) + (size_t)nc * nmu * 5 * sizeof(double);
  int kmax = ctx->opt.stern_maxit < 512 ? ctx->opt.stern_maxit : 512;
  if ((size_t)kmax + 2 > budget / per_slot) kmax = (int)(budget / per_slot) - 2;
  if (kmax < 8) return set_error(ctx, ACP_E_OOM, "no room for the FP32 Lanczos basis");
  MsB32 s{};
  s.kmax = kmax;
  s.ld = ld;
  s.slot_ld = (size_t)(kmax + 2) * ld;
  const size_t nq = (size_t)nc * nmu;
  float *vb = nullptr, *pb = nullptr, *fsc = nullptr, *yb = nullptr;
  double *dsc = nullptr, *cf = nullptr;
  int* iv = nullptr;
  ACP_TRY(ws(ctx, "ms32_basis", s.slot_ld * nmu, &vb));
  ACP_TRY(ws(ctx, "ms32_p", (size_t)ld * nmu, &pb));
  ACP_TRY(ws(ctx, "ms32_fsc", 2 * (size_t)nmu, &fsc));
  ACP_TRY(ws(ctx, "ms32_dsc", (size_t)nmu + 5 * nq, &dsc));
  ACP_TRY(ws(ctx, "ms32_coef", 4 * nq * kmax, &cf));
  ACP_TRY(ws(ctx, "ms32_y", nq * kmax, &yb));
  ACP_TRY(ws(ctx, "ms32_iv", 2 * (size_t)nmu, &iv));
  ACP_CUDA(ctx, cudaMemsetAsync(pb, 0, sizeof(float) * ld * nmu, ctx->stream));
  s.Vb = vb; s.P = pb; s.coef = cf; s.Y = yb;
  s.alpha = fsc; s.beta = fsc + nmu;
  s.beta1 = dsc;
  double* q = dsc + nmu;
  s.cs = q; s.sn = q + nq; s.dbar = q + 2 * nq; s.epsln = q + 3 * nq; s.phibar = q + 4 * nq;
  s.active = iv; s.iters = iv + nmu;
  s.nodes = nodes_d;
  ::acp::note_launch(ctx);
  msb32_init_kernel<<<nmu, kThreads, 0, ctx->stream>>>(N, nc, B32, s);
  ACP_LAUNCH(ctx);
  const int period = projection_period(ctx);
  int* kdev = nullptr;
  ACP_TRY(ws(ctx, "ms32_k", 1, &kdev));
  {
    const int one = 1;
    ACP_CUDA(ctx, cudaMemcpyAsync(kdev, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  }
  auto step = [&](int k0) -> acp_status {  // k0: 0-based step; the basis slot k = k0 + 1 is on the device
    ACP_TRY(spectral32_apply(ctx, s.Vb, (int)s.slot_ld, nmu, nullptr, s.P, ld, s.alpha, s.active, s.Vb,
                             (int)s.slot_ld, s.beta, kdev, ld));
    if (k0 % period == period - 1 || k0 < 2) ACP_TRY(project32(ctx, s.P, ld, nmu, s.P, ld));
    ::acp::note_launch(ctx);
    cudaEvent_t ev0 = prof_begin(ctx);
    msb32_step_kernel<<<nmu, kThreads, 0, ctx->stream>>>(N, nc, kdev, s, kInnerTol);
    ACP_LAUNCH(ctx);
    // per selected point: P read and the next basis vector written (FP32)
    prof_end(ctx, "msb32_step", ev0, 0.0, 8.0 * N * (double)nmu);
    ::acp::note_launch(ctx);
    advance_k_kernel<<<1, 1, 0, ctx->stream>>>(kdev);
    ACP_LAUNCH(ctx);
    return ACP_OK;
  };
  ChunkGraph graph;
  const bool graphs = ctx->opt.use_graphs && period == 1 && ctx->stream != nullptr;
  for (int k0 = 0; k0 < kmax;) {
    const int n = (kmax - k0 < kChunk) ? kmax - k0 : kChunk;
    ACP_TRY(run_chunk(ctx, graph, graphs, k0, n, step));
    k0 += n;
    int n_act = 0;
    ACP_TRY(count32(ctx, s.active, nmu, &n_act));
    if (n_act == 0) break;
    if (deadline_passed(ctx, t0_ms)) return set_error(ctx, ACP_E_TIMEOUT, "deadline passed in FP32 MINRES");
  }
  ACP_TRY(tc_check(ctx));
  ::acp::note_launch(ctx);
  msb32_backsub_kernel<<<(int)((nq + 127) / 128), 128, 0, ctx->stream>>>(nmu, nc, s);
  ACP_LAUNCH(ctx);
  ::acp::note_launch(ctx);
  msb32_assemble_kernel<<<dim3((N + 255) / 256, nmu), 256, 0, ctx->stream>>>(N, nmu, nc, s, bsc, X);
  ACP_LAUNCH(ctx);
  ACP_TRY(sum_iters(ctx, s.iters, nmu, &rep->steps, &rep->max_iters));
  if (!ctx->mixed_refine) return ACP_OK;  // inexact outer iteration: the FP32 pass is the answer
  // ---- refinement of every (shift, point) pair ----------------------------------------------
  double *Brep = nullptr, *shifts = nullptr;
  const size_t ncol = nq;
  ACP_TRY(ws(ctx, "ms32_brep", (size_t)N * ncol, &Brep));
  ACP_TRY(ws(ctx, "ms32_shifts", ncol, &shifts));
  ::acp::note_launch(ctx);
  replicate_kernel<<<grid_for((size_t)N * ncol), 256, 0, ctx->stream>>>(N, nmu, nc, B, nodes_d, Brep, shifts);
  ACP_LAUNCH(ctx);
  return refine(ctx, Brep, (int)ncol, shifts, X, false, rep, t0_ms);
}

}  // namespace acp
