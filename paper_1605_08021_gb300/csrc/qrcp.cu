// Interpolative decomposition of M_ij = psi_i * g_j (Eq. MID) by Alg. 2 in the form of its
// Remark: the SRFT acts on G only (G_tilde = G Omega), row alpha of M_tilde is the Kronecker
// product psi(r_alpha, :) (x) G_tilde(r_alpha, :), a column-pivoted Householder QR of
// M_tilde^T (m = n_orb * sketch_cols rows, N columns) selects the points r_mu, and
// Xi^T = R_11^{-1} R_{1:N_mu, :} Pi^{-1} gives the interpolation vectors (Alg. 2 steps 2-4).
//
// The QR runs right-looking: per step one single-CTA kernel chooses the pivot (largest
// downdated column norm, lowest index on ties), swaps it in and forms the Householder vector;
// a second kernel applies the reflector to all trailing columns (one warp per column) and
// downdates their norms with the usual cancellation safeguard (recompute when the downdated
// norm has lost about half its digits).  The loop stops at the first |R_jj| < id_tol |R_11|.
#include "internal.cuh"

namespace acp {

namespace {

// A (m x N, ld m): A[t * no + i + alpha * m] = psiT[i + alpha * no] * Gt[alpha + t * N]
__global__ void build_sketch_rows(int N, int no, int sc, const double* __restrict__ psiT,
                                  const double* __restrict__ Gt, double* __restrict__ A) {
  const int alpha = blockIdx.x;
  const int m = no * sc;
  double* col = A + (size_t)alpha * m;
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    const int i = r % no, t = r / no;
    col[r] = psiT[i + (size_t)alpha * no] * Gt[alpha + (size_t)t * N];
  }
}

// column norms: vn1 = vn2 = ||A[:, c]||
__global__ void column_norms(int m, int n, const double* __restrict__ A, double* vn1, double* vn2) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* col = A + (size_t)warp * m;
  double s = 0.0;
  for (int r = lane; r < m; r += 32) s += col[r] * col[r];
  s = warp_sum(s);
  if (lane == 0) {
    vn1[warp] = sqrt(s);
    vn2[warp] = sqrt(s);
  }
}

struct QrState {
  double* A;      // m x n
  double* vn1;    // n
  double* vn2;    // n
  int* perm;      // n
  double* v;      // m: Householder vector of the current step (entries j..m-1)
  double* tau;    // [0]: 2 / (v^T v); [1]: R_11 magnitude
  double* rdiag;  // kmax
  int* stop;      // [0]: 1 once the threshold stopped the loop; [1]: N_mu
};

// Single CTA: pivot choice, column swap, Householder vector for step j.
__global__ void qr_pivot_kernel(int m, int n, int j, double id_tol, QrState s) {
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ double red[32];
  if (s.stop[0]) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // argmax of vn1 over [j, n), lowest index on ties
  double best = -1.0;
  int bi = n;
  for (int c = j + threadIdx.x; c < n; c += blockDim.x) {
    const double v = s.vn1[c];
    if (v > best || (v == best && c < bi)) { best = v; bi = c; }
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
    if (lane == 0) si[0] = bi;
  }
  __syncthreads();
  const int p = si[0];
  __syncthreads();
  double* cj = s.A + (size_t)j * m;
  if (p != j) {
    double* cp = s.A + (size_t)p * m;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
      const double t = cj[r];
      cj[r] = cp[r];
      cp[r] = t;
    }
    if (threadIdx.x == 0) {
      double t = s.vn1[j]; s.vn1[j] = s.vn1[p]; s.vn1[p] = t;
      t = s.vn2[j]; s.vn2[j] = s.vn2[p]; s.vn2[p] = t;
      const int q = s.perm[j]; s.perm[j] = s.perm[p]; s.perm[p] = q;
    }
  }
  __syncthreads();
  // Householder: x = A[j:m, j], alpha = -sign(x0) ||x||, v = x - alpha e1
  double acc = 0.0;
  for (int r = j + threadIdx.x; r < m; r += blockDim.x) acc += cj[r] * cj[r];
  const double nrm = sqrt(block_sum(acc, red));
  const double x0 = cj[j];
  const double alpha = (x0 >= 0.0) ? -nrm : nrm;
  const double r11 = (j == 0) ? fabs(alpha) : s.tau[1];
  const bool below = !(fabs(alpha) >= id_tol * r11) || nrm == 0.0;
  if (below) {
    if (threadIdx.x == 0) {
      s.stop[0] = 1;
      s.stop[1] = j;
    }
    return;
  }
  const double v0 = x0 - alpha;
  const double vtv = nrm * nrm - x0 * x0 + v0 * v0;
  for (int r = j + threadIdx.x; r < m; r += blockDim.x) s.v[r] = (r == j) ? v0 : cj[r];
  __syncthreads();
  for (int r = j + threadIdx.x; r < m; r += blockDim.x) cj[r] = (r == j) ? alpha : 0.0;
  if (threadIdx.x == 0) {
    s.tau[0] = (vtv > 0.0) ? 2.0 / vtv : 0.0;
    if (j == 0) s.tau[1] = fabs(alpha);
    s.rdiag[j] = fabs(alpha);
    s.stop[1] = j + 1;
  }
}

// Apply H = I - tau v v^T to the trailing columns c > j (one warp per column) and downdate
// their norms.
__global__ void qr_update_kernel(int m, int n, int j, QrState s) {
  if (s.stop[0]) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int c = j + 1 + warp;
  if (c >= n) return;
  const double tau = s.tau[0];
  double* col = s.A + (size_t)c * m;
  const double* v = s.v;
  double d = 0.0;
  for (int r = j + lane; r < m; r += 32) d += v[r] * col[r];
  d = warp_sum(d) * tau;
  double tail = 0.0;
  for (int r = j + lane; r < m; r += 32) {
    const double a = col[r] - d * v[r];
    col[r] = a;
    if (r > j) tail += a * a;
  }
  const double arj = col[j];  // written by lane (j % 32) above
  __syncwarp();
  const double vn1 = s.vn1[c];
  if (vn1 != 0.0) {
    double temp = fabs(col[j]) / vn1;
    temp = fmax(0.0, (1.0 + temp) * (1.0 - temp));
    const double r = vn1 / s.vn2[c];
    const double temp2 = temp * r * r;
    const double tol3z = 1.4901161193847656e-08;  // sqrt(2^-52)
    if (temp2 <= tol3z) {
      tail = warp_sum(tail);
      if (lane == 0) {
        s.vn1[c] = sqrt(tail);
        s.vn2[c] = sqrt(tail);
      }
    } else if (lane == 0) {
      s.vn1[c] = vn1 * sqrt(temp);
    }
  }
  (void)arj;
}

// Back substitution of a diagonal block: X[r0:r1, c] = R[r0:r1, r0:r1]^{-1} X[r0:r1, c].
__global__ void trsm_diag_kernel(int nb, const double* __restrict__ R, int ldr, double* X, int ldx, int ncol) {
  extern __shared__ double tri[];  // nb x nb, column-major
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int r = e % nb, c = e / nb;
    tri[e] = (r <= c) ? R[r + (size_t)c * ldr] : 0.0;
  }
  __syncthreads();
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncol) return;
  double* x = X + (size_t)col * ldx;
  for (int i = nb - 1; i >= 0; --i) {
    double v = x[i];
    for (int k = i + 1; k < nb; ++k) v -= tri[i + k * nb] * x[k];
    x[i] = v / tri[i + i * nb];
  }
}

// Xi (N x k): Xi[perm[mu], mu] = 1; Xi[perm[k + c], mu] = X[mu + c * k].
__global__ void assemble_xi(int N, int k, const int* __restrict__ perm, const double* __restrict__ X,
                            double* __restrict__ Xi) {
  const size_t total = (size_t)N * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int mu = (int)(e % k);
    const int q = (int)(e / k);  // position in the pivot order
    const int row = perm[q];
    const double v = (q < k) ? (q == mu ? 1.0 : 0.0) : X[mu + (size_t)(q - k) * k];
    Xi[row + (size_t)mu * N] = v;
  }
}

__global__ void iota_kernel(int* p, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

__global__ void transpose_kernel(int rows, int cols, const double* __restrict__ A, double* __restrict__ At) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int r = bx + threadIdx.x, c = by + y;
    if (r < rows && c < cols) tile[y][threadIdx.x] = A[r + (size_t)c * rows];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = by + threadIdx.x, r = bx + y;
    if (r < rows && c < cols) At[c + (size_t)r * cols] = tile[threadIdx.x][y];
  }
}

}  // namespace

acp_status transpose(acp_ctx* ctx, int rows, int cols, const double* A, double* At) {
  dim3 g((rows + 31) / 32, (cols + 31) / 32), b(32, 8);
  ::acp::note_launch(ctx);
  transpose_kernel<<<g, b, 0, ctx->stream>>>(rows, cols, A, At);
  ACP_LAUNCH(ctx);
  return ACP_OK;
}

acp_status compress(acp_ctx* ctx, const double* G, int ncol, const double* sketch_h, int sketch_cols, double id_tol,
                    int max_rank, Compression* out) {
  const int N = ctx->N, no = ctx->n_orb, sc = sketch_cols;
  if (sc <= 0 || !sketch_h) return set_error(ctx, ACP_E_ARG, "ACP compression needs a sketch (sketch_cols > 0)");
  const int m = no * sc;
  int kmax = (m < N) ? m : N;
  if (max_rank > 0 && max_rank < kmax) kmax = max_rank;
  double *om = nullptr, *Gt = nullptr, *A = nullptr, *psiT = nullptr;
  ACP_TRY(ws(ctx, "id_omega", (size_t)ncol * sc, &om));
  ACP_TRY(ws(ctx, "id_gt", (size_t)N * sc, &Gt));
  ACP_TRY(ws(ctx, "id_a", (size_t)m * N, &A));
  ACP_TRY(ws(ctx, "id_psit", (size_t)no * N, &psiT));
  ACP_CUDA(ctx, cudaMemcpyAsync(om, sketch_h, sizeof(double) * ncol * sc, cudaMemcpyHostToDevice, ctx->stream));
  // G_tilde = G Omega (Alg. 2 step 1, Remark)
  ACP_TRY(dgemm(ctx, false, false, N, sc, ncol, 1.0, G, N, om, ncol, 0.0, Gt, N));
  ACP_TRY(transpose(ctx, N, no, ctx->d_psi, psiT));
  ::acp::note_launch(ctx);
  build_sketch_rows<<<N, 256, 0, ctx->stream>>>(N, no, sc, psiT, Gt, A);
  ACP_LAUNCH(ctx);

  QrState s{};
  s.A = A;
  double* dv = nullptr;
  ACP_TRY(ws(ctx, "qr_dv", 2 * (size_t)N + m + 2 + kmax, &dv));
  s.vn1 = dv; s.vn2 = dv + N; s.v = dv + 2 * N; s.tau = dv + 2 * N + m; s.rdiag = s.tau + 2;
  int* iv = nullptr;
  ACP_TRY(ws(ctx, "qr_iv", (size_t)N + 2, &iv));
  s.perm = iv; s.stop = iv + N;
  ACP_CUDA(ctx, cudaMemsetAsync(s.stop, 0, 2 * sizeof(int), ctx->stream));
  ::acp::note_launch(ctx);
  iota_kernel<<<(N + 255) / 256, 256, 0, ctx->stream>>>(s.perm, N);
  ACP_LAUNCH(ctx);
  ::acp::note_launch(ctx);
  column_norms<<<(N * 32 + 255) / 256, 256, 0, ctx->stream>>>(m, N, A, s.vn1, s.vn2);
  ACP_LAUNCH(ctx);
  int host_stop[2] = {0, 0};
  for (int j = 0; j < kmax; ++j) {
    ::acp::note_launch(ctx);
    qr_pivot_kernel<<<1, 1024, 0, ctx->stream>>>(m, N, j, id_tol, s);
    const int rest = N - j - 1;
    if (rest > 0) {
      ::acp::note_launch(ctx);
      qr_update_kernel<<<(rest * 32 + 255) / 256, 256, 0, ctx->stream>>>(m, N, j, s);
    }
    ACP_LAUNCH(ctx);
    if ((j & 63) == 63) {
      ACP_CUDA(ctx, cudaMemcpyAsync(host_stop, s.stop, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      if (host_stop[0]) break;
    }
  }
  ACP_CUDA(ctx, cudaMemcpyAsync(host_stop, s.stop, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int k = host_stop[1];
  if (k <= 0) return set_error(ctx, ACP_E_RANK, "pivoted QR found rank 0 (is G zero?)");
  out->n_mu = k;
  out->piv.resize(N);
  out->rdiag.resize(k);
  ACP_CUDA(ctx, cudaMemcpyAsync(out->piv.data(), s.perm, sizeof(int) * N, cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaMemcpyAsync(out->rdiag.data(), s.rdiag, sizeof(double) * k, cudaMemcpyDeviceToHost, ctx->stream));

  // X = R11^{-1} R12 by blocked back substitution (diagonal blocks in shared memory, GEMM updates)
  const int nr = N - k;
  double* X = nullptr;
  ACP_TRY(ws(ctx, "id_x", (size_t)k * (nr > 0 ? nr : 1), &X));
  if (nr > 0) {
    ACP_CUDA(ctx, cudaMemcpy2DAsync(X, sizeof(double) * k, A + (size_t)k * m, sizeof(double) * m, sizeof(double) * k,
                                    nr, cudaMemcpyDeviceToDevice, ctx->stream));
    const int nb = 64;
    const int nblk = (k + nb - 1) / nb;
    for (int b = nblk - 1; b >= 0; --b) {
      const int r0 = b * nb, r1 = (r0 + nb < k) ? r0 + nb : k, w = r1 - r0;
      ::acp::note_launch(ctx);
      trsm_diag_kernel<<<(nr + 127) / 128, 128, w * w * sizeof(double), ctx->stream>>>(
          w, A + r0 + (size_t)r0 * m, m, X + r0, k, nr);
      ACP_LAUNCH(ctx);
      if (r0 > 0)
        ACP_TRY(dgemm(ctx, false, false, r0, nr, w, -1.0, A + (size_t)r0 * m, m, X + r0, k, 1.0, X, k));
    }
  }
  double* Xi = nullptr;
  int* dpiv = nullptr;
  ACP_TRY(ws(ctx, "xi", (size_t)N * k, &Xi));
  ACP_TRY(ws(ctx, "xi_piv", (size_t)N, &dpiv));
  ACP_CUDA(ctx, cudaMemcpyAsync(dpiv, s.perm, sizeof(int) * N, cudaMemcpyDeviceToDevice, ctx->stream));
  {
    const size_t total = (size_t)N * k;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 65535) blocks = 65535;
    ::acp::note_launch(ctx);
    assemble_xi<<<blocks, 256, 0, ctx->stream>>>(N, k, dpiv, X, Xi);
    ACP_LAUNCH(ctx);
  }
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  out->piv.resize(k);
  out->d_piv = dpiv;
  out->d_xi = Xi;
  return ACP_OK;
}

}  // namespace acp
