// FP64 GEMM for the projector Q = I - Psi Psi^T h (Sec. 2.2), the W construction of Eq. eqnW,
// the products W G(r_mu, :) (Eq. chi0gcompress2) and W X (Eq. dyson4), and the dynamical matrix
// term G^T U (Eq. SecDeriv).  tcgen05 has no FP64 kind, so this path is a register-blocked DFMA
// kernel: 64 x 64 output tiles, 16-deep shared-memory k-slices, 4 x 4 outputs per thread.
#include <mutex>

#include "internal.cuh"

namespace acp {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

// Split over K (gridDim.z > 1): slice z takes k in [z kchunk, (z+1) kchunk) and writes its own
// C block at C + z cz (the partial sums are added up by slice_sum_kernel).
template <bool TA, bool TB, bool HAD>
__global__ void __launch_bounds__(256) dgemm_kernel(int M, int N, int K, double alpha, const double* __restrict__ A,
                                                    int lda, const double* __restrict__ B, int ldb, double beta,
                                                    double* __restrict__ C, int ldc, const double* __restrict__ Hz,
                                                    int ldh, int kchunk, size_t cz) {
  if (gridDim.z > 1) {
    const int kz0 = blockIdx.z * kchunk;
    K = min(K - kz0, kchunk);
    A += TA ? (size_t)kz0 : (size_t)kz0 * lda;
    B += TB ? (size_t)kz0 * ldb : (size_t)kz0;
    C += blockIdx.z * cz;
  }
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int e0 = 0; e0 < BM * BK; e0 += 256) {
      const int e = e0 + tid;
      int mm, kk;
      if (!TA) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      const int gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < K) v = TA ? A[gk + (size_t)gm * lda] : A[gm + (size_t)gk * lda];
      As[kk][mm] = v;
    }
#pragma unroll
    for (int e0 = 0; e0 < BN * BK; e0 += 256) {
      const int e = e0 + tid;
      int nn, kk;
      if (!TB) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
      const int gn = n0 + nn, gk = k0 + kk;
      double v = 0.0;
      if (gn < N && gk < K) v = TB ? B[gn + (size_t)gk * ldb] : B[gk + (size_t)gn * ldb];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int gn = n0 + ty + 16 * j;
    if (gn >= N) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gm = m0 + tx + 16 * i;
      if (gm >= M) continue;
      double* c = &C[gm + (size_t)gn * ldc];
      if (HAD) {
        *c += alpha * Hz[gm + (size_t)gn * ldh] * acc[i][j];
      } else {
        *c = alpha * acc[i][j] + (beta == 0.0 ? 0.0 : beta * *c);
      }
    }
  }
}

template <bool TA, bool TB>
void launch(dim3 g, cudaStream_t s, int m, int n, int k, double alpha, const double* A, int lda, const double* B,
            int ldb, double beta, double* C, int ldc, const double* hz, int ldh, int kchunk = 0, size_t cz = 0) {
  if (hz)
    dgemm_kernel<TA, TB, true><<<g, 256, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, hz, ldh, kchunk, cz);
  else
    dgemm_kernel<TA, TB, false><<<g, 256, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, hz, ldh, kchunk, cz);
}

// C = alpha * sum_z P[z] (+ beta C), column-major m x n with leading dimension ldc; P slices m x n.
__global__ void slice_sum_kernel(int m, int n, int slices, const double* __restrict__ P, double alpha, double beta,
                                 double* __restrict__ C, int ldc) {
  const size_t total = (size_t)m * n, mn = (size_t)m * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int z = 0; z < slices; ++z) acc += P[z * mn + e];
    double* c = &C[(e % m) + (e / m) * (size_t)ldc];
    *c = alpha * acc + (beta == 0.0 ? 0.0 : beta * *c);
  }
}

}  // namespace

acp_status dgemm(acp_ctx* ctx, bool ta, bool tb, int m, int n, int k, double alpha, const double* A, int lda,
                 const double* B, int ldb, double beta, double* C, int ldc, const double* hz, int ldhz) {
  if (m <= 0 || n <= 0) return ACP_OK;
  const unsigned gy = (unsigned)((n + BN - 1) / BN);
  if (gy > 65535u) {
    // split very wide products into column slabs (grid.y limit)
    const int slab = 65535 * BN;
    for (int c0 = 0; c0 < n; c0 += slab) {
      const int nc = (n - c0 < slab) ? n - c0 : slab;
      const double* Bp = tb ? B + c0 : B + (size_t)c0 * ldb;
      ACP_TRY(dgemm(ctx, ta, tb, m, nc, k, alpha, A, lda, Bp, ldb, beta, C + (size_t)c0 * ldc, ldc,
                    hz ? hz + (size_t)c0 * ldhz : nullptr, ldhz));
    }
    return ACP_OK;
  }
  dim3 g((m + BM - 1) / BM, gy);
  if (k <= 0) {
    // C = beta C (or unchanged for the Hadamard epilogue)
    if (hz) return ACP_OK;
    ::acp::note_launch(ctx);
    launch<false, false>(g, ctx->stream, m, n, 0, alpha, A, lda, B, ldb, beta, C, ldc, nullptr, 0);
    ACP_LAUNCH(ctx);
    return ACP_OK;
  }
  // Few output tiles and a long K (the projector's h Psi^T X): split K over gridDim.z so that
  // the launch fills the GPU, then add the slices up.
  const long long tiles = (long long)g.x * g.y;
  if (!hz && tiles < 152 && k >= 1024) {
    int slices = (int)((304 + tiles - 1) / tiles);
    if (slices > k / 256) slices = k / 256;
    if (slices > 64) slices = 64;
    if (slices >= 2) {
      const int kchunk = ((k + slices - 1) / slices + BK - 1) / BK * BK;
      slices = (k + kchunk - 1) / kchunk;
      double* part = nullptr;
      const size_t mn = (size_t)m * n;
      ACP_TRY(ws(ctx, "dgemm_slices", mn * slices, &part));
      ::acp::note_launch(ctx);
      cudaEvent_t ev0 = prof_begin(ctx);
      const dim3 gz(g.x, g.y, slices);
      if (ta && !tb) launch<true, false>(gz, ctx->stream, m, n, k, 1.0, A, lda, B, ldb, 0.0, part, m, nullptr, 0, kchunk, mn);
      else if (!ta && !tb) launch<false, false>(gz, ctx->stream, m, n, k, 1.0, A, lda, B, ldb, 0.0, part, m, nullptr, 0, kchunk, mn);
      else if (!ta && tb) launch<false, true>(gz, ctx->stream, m, n, k, 1.0, A, lda, B, ldb, 0.0, part, m, nullptr, 0, kchunk, mn);
      else launch<true, true>(gz, ctx->stream, m, n, k, 1.0, A, lda, B, ldb, 0.0, part, m, nullptr, 0, kchunk, mn);
      ACP_LAUNCH(ctx);
      size_t blocks = (mn + 255) / 256;
      if (blocks > 4096) blocks = 4096;
      ::acp::note_launch(ctx);
      slice_sum_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(m, n, slices, part, alpha, beta, C, ldc);
      ACP_LAUNCH(ctx);
      prof_end(ctx, "dgemm", ev0, 2.0 * m * n * k,
               8.0 * ((double)m * k + (double)k * n + (double)m * n * (beta != 0.0 ? 2 : 1)));
      return ACP_OK;
    }
  }
  ::acp::note_launch(ctx);
  const double e_flops = 2.0 * m * n * k;
  const double e_bytes = 8.0 * ((double)m * k + (double)k * n + (double)m * n * ((beta != 0.0 || hz) ? 2 : 1) +
                                (hz ? (double)m * n : 0.0));
  cudaEvent_t ev0 = prof_begin(ctx);
  if (!ta && !tb) launch<false, false>(g, ctx->stream, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, hz, ldhz);
  else if (ta && !tb) launch<true, false>(g, ctx->stream, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, hz, ldhz);
  else if (!ta && tb) launch<false, true>(g, ctx->stream, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, hz, ldhz);
  else launch<true, true>(g, ctx->stream, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, hz, ldhz);
  ACP_LAUNCH(ctx);
  prof_end(ctx, "dgemm", ev0, e_flops, e_bytes);
  return ACP_OK;
}

acp_status project(acp_ctx* ctx, const double* X, int ldx, int ncol, double* Y, int ldy) {
  if (ncol <= 0) return ACP_OK;
  const int N = ctx->N, no = ctx->n_orb;
  double* C = nullptr;
  ACP_TRY(ws(ctx, "proj_c", (size_t)no * ncol, &C));
  // C = h Psi^T X
  ACP_TRY(dgemm(ctx, true, false, no, ncol, N, ctx->h, ctx->d_psi, N, X, ldx, 0.0, C, no));
  if (Y != X)
    ACP_CUDA(ctx, cudaMemcpy2DAsync(Y, (size_t)ldy * sizeof(double), X, (size_t)ldx * sizeof(double),
                                    (size_t)N * sizeof(double), ncol, cudaMemcpyDeviceToDevice, ctx->stream));
  // Y -= Psi C
  ACP_TRY(dgemm(ctx, false, false, N, ncol, no, -1.0, ctx->d_psi, N, C, no, 1.0, Y, ldy));
  return ACP_OK;
}

}  // namespace acp

// ---- projector for callers that cannot allocate device memory ----------------------------------
// The intermediate C = h Psi^T X lives in a fixed array of device memory that the library owns
// for the lifetime of the process (on every GPU that loads it), so this entry point needs no
// context and no cudaMalloc.  Host code may not use the array's name as a device address: the
// address is looked up once per device with cudaGetSymbolAddress.
namespace acp {
namespace {

constexpr size_t kNoAllocElems = size_t(1) << 20;  // 8 MiB of FP64: n_orb * ncol <= 1,048,576
__device__ __align__(256) double g_noalloc_c[kNoAllocElems];

std::mutex g_noalloc_mu;
double* g_noalloc_addr[64] = {};  // per device ordinal, filled on the first call on that device

}  // namespace

}  // namespace acp

extern "C" acp_status acp_project_noalloc(const double* psi_d, int n_grid, int n_orb, double h, const double* X_d,
                                          int ncol, double* Y_d, void* stream) {
  using namespace acp;
  if (!psi_d || !X_d || !Y_d || n_grid < 1 || n_orb < 1 || ncol < 0 || !(h > 0.0)) return ACP_E_ARG;
  if (ncol == 0) return ACP_OK;
  if ((size_t)n_orb * (size_t)ncol > kNoAllocElems) return ACP_E_ARG;
  // an error left by earlier, unrelated work would otherwise be read (and cleared) by the launch
  // checks below and reported as this call's; refuse to enqueue onto a context in that state
  if (cudaPeekAtLastError() != cudaSuccess) return ACP_E_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return ACP_E_CUDA;
  }
  if (dev < 0 || dev >= 64) return ACP_E_ARG;
  double* C = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_c);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return ACP_E_CUDA;
      }
      g_noalloc_addr[dev] = static_cast<double*>(p);
    }
    C = g_noalloc_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // C = h Psi^T X: beta = 0, so every entry is written and nothing needs clearing beforehand
  launch<true, false>(dim3((n_orb + BM - 1) / BM, (ncol + BN - 1) / BN), s, n_orb, ncol, n_grid, h, psi_d, n_grid,
                      X_d, n_grid, 0.0, C, n_orb, nullptr, 0);
  if (cudaGetLastError() != cudaSuccess) return ACP_E_CUDA;  // the first GEMM did not launch
  if (Y_d != X_d) {
    if (cudaMemcpyAsync(Y_d, X_d, sizeof(double) * (size_t)n_grid * ncol, cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess) {
      cudaGetLastError();
      return ACP_E_CUDA;
    }
  }
  // Y -= Psi C
  launch<false, false>(dim3((n_grid + BM - 1) / BM, (ncol + BN - 1) / BN), s, n_grid, ncol, n_orb, -1.0, psi_d,
                       n_grid, C, n_orb, 1.0, Y_d, n_grid, nullptr, 0);
  if (cudaGetLastError() != cudaSuccess) return ACP_E_CUDA;  // the second GEMM did not launch
  return ACP_OK;
}
