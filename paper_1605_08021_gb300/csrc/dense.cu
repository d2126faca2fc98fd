// Small dense FP64 kernels: the N_mu x N_mu solve of the Sherman-Morrison-Woodbury update
// (Eq. dyson4), the eigendecomposition of the dynamical matrix (Sec. 2.2, D u = omega^2 u),
// and helpers (row gathers, Frobenius norms).
#include "internal.cuh"

namespace acp {

namespace {

// Step k of LU with partial pivoting (single CTA): choose the pivot row, swap rows of A and B.
__global__ void lu_pivot_kernel(double* A, int n, int k, double* B, int nrhs, int* singular) {
  __shared__ double sv[32];
  __shared__ int si[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double best = -1.0;
  int bi = n;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    const double v = fabs(A[i + (size_t)k * n]);
    if (v > best || (v == best && i < bi)) { best = v; bi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if (lane == 0) { sv[wid] = best; si[wid] = bi; }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    best = (lane < nw) ? sv[lane] : -1.0;
    bi = (lane < nw) ? si[lane] : n;
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { si[0] = bi; sv[0] = best; }
  }
  __syncthreads();
  const int p = si[0];
  if (threadIdx.x == 0 && !(sv[0] > 0.0)) atomicExch(singular, 1);
  if (p == k || p >= n) return;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double t = A[k + (size_t)j * n];
    A[k + (size_t)j * n] = A[p + (size_t)j * n];
    A[p + (size_t)j * n] = t;
  }
  for (int j = threadIdx.x; j < nrhs; j += blockDim.x) {
    const double t = B[k + (size_t)j * n];
    B[k + (size_t)j * n] = B[p + (size_t)j * n];
    B[p + (size_t)j * n] = t;
  }
}

// Eliminate below the pivot: rows i > k of A (columns > k) and of B.
__global__ void lu_update_kernel(double* A, int n, int k, double* B, int nrhs) {
  const int i = k + 1 + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double piv = A[k + (size_t)k * n];
  const double l = (piv != 0.0) ? A[i + (size_t)k * n] / piv : 0.0;
  const int j0 = blockIdx.y;
  for (int j = k + 1 + j0; j < n; j += gridDim.y) A[i + (size_t)j * n] -= l * A[k + (size_t)j * n];
  for (int j = j0; j < nrhs; j += gridDim.y) B[i + (size_t)j * n] -= l * B[k + (size_t)j * n];
}

// Back substitution U x = b, one CTA per right-hand side.
__global__ void back_subst_kernel(const double* __restrict__ A, int n, double* B) {
  __shared__ double xk;
  double* b = B + (size_t)blockIdx.x * n;
  for (int k = n - 1; k >= 0; --k) {
    if (threadIdx.x == 0) {
      const double u = A[k + (size_t)k * n];
      xk = (u != 0.0) ? b[k] / u : 0.0;
      b[k] = xk;
    }
    __syncthreads();
    const double x = xk;
    for (int i = threadIdx.x; i < k; i += blockDim.x) b[i] -= A[i + (size_t)k * n] * x;
    __syncthreads();
  }
}

// Parallel cyclic Jacobi (round-robin pairing) on one CTA; A (n x n, column-major) is
// diagonalised in place, V accumulates the rotations.
__global__ void jacobi_kernel(double* A, int n, double* V, double* w, int max_sweeps, double tol) {
  __shared__ double rc[512], rs[512];
  __shared__ int rp[512], rq[512];
  __shared__ double red[32];
  const int ne = n + (n & 1);
  const int half = ne / 2;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) V[e] = ((e % n) == (e / n)) ? 1.0 : 0.0;
  __syncthreads();
  double fro = 0.0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) fro += A[e] * A[e];
  fro = sqrt(block_sum(fro, red));
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x)
      if ((e % n) != (e / n)) off += A[e] * A[e];
    off = sqrt(block_sum(off, red));
    if (off <= tol * fro || fro == 0.0) break;
    for (int r = 0; r < ne - 1; ++r) {
      for (int q = threadIdx.x; q < half; q += blockDim.x) {
        int a, b;
        if (q == 0) { a = r; b = ne - 1; }
        else { a = (r + q) % (ne - 1); b = (r - q + ne - 1) % (ne - 1); }
        const int p = a < b ? a : b, qq = a < b ? b : a;
        double c = 1.0, s = 0.0;
        if (qq < n) {
          const double apq = A[p + (size_t)qq * n];
          if (apq != 0.0) {
            const double app = A[p + (size_t)p * n], aqq = A[qq + (size_t)qq * n];
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        rc[q] = c; rs[q] = s; rp[q] = p; rq[q] = qq;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = threadIdx.x; e < half * n; e += blockDim.x) {
        const int q = e / n, j = e % n;
        const int p = rp[q], qq = rq[q];
        if (qq >= n || rs[q] == 0.0) continue;
        const double c = rc[q], s = rs[q];
        const double ap = A[p + (size_t)j * n], aq = A[qq + (size_t)j * n];
        A[p + (size_t)j * n] = c * ap - s * aq;
        A[qq + (size_t)j * n] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = threadIdx.x; e < half * n; e += blockDim.x) {
        const int q = e / n, i = e % n;
        const int p = rp[q], qq = rq[q];
        if (qq >= n || rs[q] == 0.0) continue;
        const double c = rc[q], s = rs[q];
        const double ap = A[i + (size_t)p * n], aq = A[i + (size_t)qq * n];
        A[i + (size_t)p * n] = c * ap - s * aq;
        A[i + (size_t)qq * n] = s * ap + c * aq;
        const double vp = V[i + (size_t)p * n], vq = V[i + (size_t)qq * n];
        V[i + (size_t)p * n] = c * vp - s * vq;
        V[i + (size_t)qq * n] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = A[i + (size_t)i * n];
  __syncthreads();
  // odd-even transposition sort of (w, V columns), ascending
  for (int pass = 0; pass < n; ++pass) {
    for (int i = 2 * threadIdx.x + (pass & 1); i + 1 < n; i += 2 * blockDim.x) {
      if (w[i] > w[i + 1]) {
        const double t = w[i]; w[i] = w[i + 1]; w[i + 1] = t;
        for (int r = 0; r < n; ++r) {
          const double u = V[r + (size_t)i * n];
          V[r + (size_t)i * n] = V[r + (size_t)(i + 1) * n];
          V[r + (size_t)(i + 1) * n] = u;
        }
      }
    }
    __syncthreads();
  }
}

__global__ void diff_norms_kernel(const double* __restrict__ A, const double* __restrict__ B, size_t count,
                                  double* out) {
  double d = 0.0, a = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const double x = A[e], y = B ? B[e] : 0.0;
    d += (x - y) * (x - y);
    a += x * x;
  }
  d = warp_sum(d);
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], d);
    atomicAdd(&out[1], a);
  }
}

__global__ void gather_rows_kernel(const double* __restrict__ X, int ldx, int ncol, const int* __restrict__ rows,
                                   int nrows, double* __restrict__ Y, int ldy) {
  const size_t total = (size_t)nrows * ncol;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % nrows), c = (int)(e / nrows);
    Y[r + (size_t)c * ldy] = X[rows[r] + (size_t)c * ldx];
  }
}

int grid_for(size_t total) {
  size_t b = (total + 255) / 256;
  if (b > 65535) b = 65535;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

acp_status lu_solve(acp_ctx* ctx, double* A, int n, double* B, int nrhs) {
  int* sing = ctx->d_flag + 8;
  ACP_CUDA(ctx, cudaMemsetAsync(sing, 0, sizeof(int), ctx->stream));
  for (int k = 0; k < n; ++k) {
    ::acp::note_launch(ctx);
    lu_pivot_kernel<<<1, 1024, 0, ctx->stream>>>(A, n, k, B, nrhs, sing);
    const int rows = n - k - 1;
    if (rows > 0) {
      dim3 g((rows + 127) / 128, 32);
      ::acp::note_launch(ctx);
      lu_update_kernel<<<g, 128, 0, ctx->stream>>>(A, n, k, B, nrhs);
    }
  }
  ACP_LAUNCH(ctx);
  ::acp::note_launch(ctx);
  back_subst_kernel<<<nrhs, 256, 0, ctx->stream>>>(A, n, B);
  ACP_LAUNCH(ctx);
  int h = 0;
  ACP_CUDA(ctx, cudaMemcpyAsync(&h, sing, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (h) return set_error(ctx, ACP_E_NUMERIC, "singular matrix in the Sherman-Morrison-Woodbury solve");
  return ACP_OK;
}

acp_status jacobi_eig(acp_ctx* ctx, double* A, int n, double* w_d, double* V_d) {
  if (n < 1 || n > 1024) return set_error(ctx, ACP_E_ARG, "eigensolver size %d outside [1, 1024]", n);
  ::acp::note_launch(ctx);
  jacobi_kernel<<<1, 1024, 0, ctx->stream>>>(A, n, V_d, w_d, 60, 1e-15);
  ACP_LAUNCH(ctx);
  return ACP_OK;
}

acp_status diff_norms(acp_ctx* ctx, const double* A, const double* B, size_t count, double* out_h) {
  double* d = ctx->d_flag ? reinterpret_cast<double*>(ctx->d_flag + 10) : nullptr;
  ACP_CUDA(ctx, cudaMemsetAsync(d, 0, 2 * sizeof(double), ctx->stream));
  ::acp::note_launch(ctx);
  diff_norms_kernel<<<grid_for(count) > 2048 ? 2048 : grid_for(count), 256, 0, ctx->stream>>>(A, B, count, d);
  ACP_LAUNCH(ctx);
  ACP_CUDA(ctx, cudaMemcpyAsync(out_h, d, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ACP_OK;
}

acp_status gather_rows(acp_ctx* ctx, const double* X, int ldx, int ncol, const int* rows_d, int nrows, double* Y,
                       int ldy) {
  if (nrows <= 0 || ncol <= 0) return ACP_OK;
  ::acp::note_launch(ctx);
  gather_rows_kernel<<<grid_for((size_t)nrows * ncol), 256, 0, ctx->stream>>>(X, ldx, ncol, rows_d, nrows, Y, ldy);
  ACP_LAUNCH(ctx);
  return ACP_OK;
}

}  // namespace acp
