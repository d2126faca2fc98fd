// Projector Q = I - Psi Psi^T h (Sec. 2.2) on FP32 blocks of grid functions, as two tcgen05
// tensor-core GEMMs with FP32 accuracy (3xTF32: every operand is split as hi + lo with hi
// representable in TF32, and A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi, accumulated in FP32 in TMEM):
//
//   GEMM 1 (split over K = grid):  C^T = X^T Psi      (ncol x n_orb), partial sums per K slice
//   reduce:                        C^T = h sum_slices, split into hi / lo
//   GEMM 2 (K = n_orb):            Y^T = X^T - C^T Psi^T   (fused subtract epilogue)
//
// Both GEMMs see K-major operands only: an FP32 block X (ncol grid functions of leading dimension
// ld, a multiple of 32) is K-major for GEMM 1 as it stands; Psi is kept as hi / lo FP32 copies in
// both orientations (orbital rows for GEMM 1, grid rows for GEMM 2), zero padded.
//
// One CTA computes one 128 x BN output tile with warp-specialised roles: warp 0 issues the TMA
// loads (128-byte swizzled boxes of 32 FP32 along K), warp 1 owns the TMEM accumulator and issues
// tcgen05.mma, warps 4-7 split the FP32 A tile into hi / lo in shared memory (GEMM 1) and run the
// epilogue (tcgen05.ld of their 32 TMEM lanes).  Two pipeline stages; every wait is bounded.
#include "internal.cuh"
#include "tc.cuh"

#include <cudaTypedefs.h>

#include <atomic>

namespace acp {

namespace {

constexpr int kBM = 128;      // rows of the output tile (TMEM lanes)
constexpr int kBK = 32;       // FP32 elements along K per stage: one 128-byte swizzle row
constexpr int kStages = 2;
constexpr int kThreads = 256;
constexpr uint64_t kWaitNs = 200000000ull;  // 0.2 s: far beyond any legitimate wait

struct TcArgs {
  int M;             // rows of A = output rows
  int Nd;            // valid output columns (rows of B)
  int BN;            // output tile width (multiple of 16, <= 256)
  int kb_per;        // k-blocks of 32 per CTA (split over blockIdx.y)
  int kb_total;      // k-blocks in total
  uint32_t tmem_cols;
  int split_a;       // 1: A is loaded once in FP32 and split into hi / lo in shared memory
  int mode;          // 0: store D (partials, slice blockIdx.y); 1: Y = X - D
  float* out;
  int ldo;
  long long slice_stride;
  const float* X;
  int ldx;
  float* Y;
  int ldy;
  int* status;
  uint64_t wait_ns;  // bound of every barrier wait (kWaitNs; shorter in the failure self-test)
  int withhold;      // failure self-test: the producer issues no TMA load, so no barrier completes
};

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__global__ void __launch_bounds__(kThreads, 1)
    tc3_gemm_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mAlo,
                    const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo, TcArgs p) {
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t conv_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  extern __shared__ uint8_t dyn_smem[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~uintptr_t(1023));
  const uint32_t a_bytes = kBM * kBK * 4;
  const uint32_t b_bytes = (uint32_t)p.BN * kBK * 4;
  const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM;
  const int n0 = blockIdx.z * p.BN;
  const int kb0 = blockIdx.y * p.kb_per;
  const int nkb = min(p.kb_per, p.kb_total - kb0);
  const uint64_t deadline = tc::globaltimer_ns() + p.wait_ns;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&conv_bar[s], 128);
      tc::mbar_init(&empty_bar[s], 1);
    }
    tc::mbar_init(&done_bar, 1);
    abort_sh = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(&tmem_base_sh, p.tmem_cols);
    tc::tmem_relinquish();
  }
  if (warp == 0 && lane == 0) {
    tc::tma_prefetch(&mA);
    tc::tma_prefetch(&mBhi);
    tc::tma_prefetch(&mBlo);
    if (!p.split_a) tc::tma_prefetch(&mAlo);
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0) {
    if (lane == 0) {
      bool ok = true;
      int issued = 0;
      for (int i = 0; i < (p.withhold ? 0 : nkb); ++i) {
        const int s = i % kStages, u = i / kStages;
        if (u > 0 && !tc::mbar_wait(&empty_bar[s], (u - 1) & 1, deadline)) {
          ok = false;
          break;
        }
        ++issued;
        uint8_t* st = base + s * stage_bytes;
        tc::mbar_arrive_expect_tx(&full_bar[s], (p.split_a ? a_bytes : 2 * a_bytes) + 2 * b_bytes);
        const int kx = (kb0 + i) * kBK;
        tc::tma_load_2d(st, &mA, &full_bar[s], kx, m0);
        if (!p.split_a) tc::tma_load_2d(st + a_bytes, &mAlo, &full_bar[s], kx, m0);
        tc::tma_load_2d(st + 2 * a_bytes, &mBhi, &full_bar[s], kx, n0);
        tc::tma_load_2d(st + 2 * a_bytes + b_bytes, &mBlo, &full_bar[s], kx, n0);
      }
      // no copy may still be landing in shared memory when the CTA exits: wait (bounded) for the
      // last load of every stage; each load completes its stage's full barrier once, so the
      // phase of load i is i / kStages (already complete on the normal path)
      const uint64_t drain = tc::globaltimer_ns() + p.wait_ns;
      for (int i = issued > kStages ? issued - kStages : 0; i < issued; ++i)
        if (!tc::mbar_wait(&full_bar[i % kStages], (uint32_t)(i / kStages) & 1u, drain)) ok = false;
      if (!ok) atomicExch(&abort_sh, 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      const uint32_t idesc = tc::idesc_tf32(kBM, p.BN);
      for (int i = 0; i < nkb; ++i) {
        const int s = i % kStages, u = i / kStages;
        if (!tc::mbar_wait(p.split_a ? &conv_bar[s] : &full_bar[s], u & 1, deadline)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        uint8_t* st = base + s * stage_bytes;
        const uint64_t ah = tc::desc_k_sw128(st), al = tc::desc_k_sw128(st + a_bytes);
        const uint64_t bh = tc::desc_k_sw128(st + 2 * a_bytes), bl = tc::desc_k_sw128(st + 2 * a_bytes + b_bytes);
#pragma unroll
        for (int kk = 0; kk < kBK / 8; ++kk) {
          const uint64_t off = (uint64_t)((kk * 8 * 4) >> 4);  // 8 TF32 = 32 bytes per MMA k-step
          tc::mma_tf32(tmem, al + off, bh + off, idesc, (i > 0 || kk > 0) ? 1u : 0u);
          tc::mma_tf32(tmem, ah + off, bl + off, idesc, 1u);
          tc::mma_tf32(tmem, ah + off, bh + off, idesc, 1u);
        }
        tc::mma_commit(&empty_bar[s]);
      }
      tc::mma_commit(&done_bar);
      if (!ok) atomicExch(&abort_sh, 1);
    }
  } else if (warp >= 4) {
    const int q = warp - 4;
    bool ok = true;
    if (p.split_a) {
      for (int i = 0; i < nkb; ++i) {
        const int s = i % kStages, u = i / kStages;
        if (!tc::mbar_wait(&full_bar[s], u & 1, deadline)) {
          ok = false;
          break;
        }
        float4* hi = reinterpret_cast<float4*>(base + s * stage_bytes);
        float4* lo = reinterpret_cast<float4*>(base + s * stage_bytes + a_bytes);
        for (int e = threadIdx.x - 128; e < (int)(a_bytes / 16); e += 128) {
          const float4 v = hi[e];
          const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
          hi[e] = h;
          lo[e] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
        }
        tc::fence_proxy_async_smem();
        tc::mbar_arrive(&conv_bar[s]);
      }
    }
    if (ok) ok = tc::mbar_wait(&done_bar, 0, deadline);
    ok = __all_sync(0xffffffffu, ok);
    tc::tc_fence_after();
    if (ok) {
      const int row = m0 + q * 32 + lane;
      const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
      for (int c0 = 0; c0 < p.BN; c0 += 32) {
        const int col0 = n0 + c0;
        const int nvalid = (row < p.M) ? min(min(32, p.BN - c0), p.Nd - col0) : 0;
        float4 xv[8];
        if (p.mode == 1 && nvalid == 32) {
          // issue the loads of X before waiting on the accumulator
          const float4* x4 = reinterpret_cast<const float4*>(p.X + (size_t)row * p.ldx + col0);
#pragma unroll
          for (int j = 0; j < 8; ++j) xv[j] = __ldg(x4 + j);
        }
        float v[32];
        tc::tmem_ld_32x32(trow + (uint32_t)c0, v);
        if (nvalid <= 0) continue;
        if (p.mode == 0) {
          float* o = p.out + (size_t)blockIdx.y * p.slice_stride + (size_t)row * p.ldo + col0;
          if (nvalid == 32) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) *reinterpret_cast<float4*>(o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
          } else {
            for (int j = 0; j < nvalid; ++j) o[j] = v[j];
          }
        } else {
          float* y = p.Y + (size_t)row * p.ldy + col0;
          if (nvalid == 32) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
              *reinterpret_cast<float4*>(y + 4 * j) =
                  make_float4(xv[j].x - v[4 * j], xv[j].y - v[4 * j + 1], xv[j].z - v[4 * j + 2], xv[j].w - v[4 * j + 3]);
          } else {
            const float* x = p.X + (size_t)row * p.ldx + col0;
            for (int j = 0; j < nvalid; ++j) y[j] = x[j] - v[j];
          }
        }
      }
    } else if (lane == 0) {
      atomicExch(&abort_sh, 1);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    // the MMAs must be done with the accumulator before it is freed (complete on the normal
    // path, where the epilogue has waited for the same phase)
    if (!tc::mbar_wait(&done_bar, 0, tc::globaltimer_ns() + p.wait_ns) && lane == 0) atomicExch(p.status, 1);
    __syncwarp();  // the dealloc is warp-collective (.sync.aligned): reconverge after the wait
    tc::tmem_dealloc(tmem, p.tmem_cols);
  }
  if (threadIdx.x == 0 && abort_sh) atomicExch(p.status, 1);
}

// C^T (ncol x no_pad) = h * sum of the K-slice partials, split into TF32 hi and FP32 lo parts.
__global__ void slice_reduce_kernel(int ncol, int no, int no_pad, int slices, long long stride,
                                    const float* __restrict__ part, double h, float* __restrict__ ct_hi,
                                    float* __restrict__ ct_lo) {
  const size_t total = (size_t)ncol * no_pad;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % no_pad);
    double s = 0.0;
    if (i < no)
      for (int sl = 0; sl < slices; ++sl) s += (double)part[(size_t)sl * stride + e];
    const float v = (float)(s * h);
    const float hi = tf32_hi(v);
    ct_hi[e] = hi;
    ct_lo[e] = v - hi;
  }
}

// FP64 orbitals -> hi / lo FP32 copies in both orientations (zero padding is set beforehand).
__global__ void psi_split_kernel(int N, int no, int ld32, int no_pad, const double* __restrict__ psi,
                                 float* __restrict__ psi_hi, float* __restrict__ psi_lo, float* __restrict__ psit_hi,
                                 float* __restrict__ psit_lo) {
  const size_t total = (size_t)N * no;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % N), i = (int)(e / N);
    const double v = psi[e];
    const float hi = tf32_hi((float)v);
    const float lo = (float)(v - (double)hi);
    psi_hi[(size_t)i * ld32 + a] = hi;
    psi_lo[(size_t)i * ld32 + a] = lo;
    psit_hi[(size_t)a * no_pad + i] = hi;
    psit_lo[(size_t)a * no_pad + i] = lo;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
    return nullptr;
  }();
  return fn;
}

// 2D FP32 tensor map: `rows` rows of `inner` elements, row stride `ld` elements, box 32 x box_rows,
// 128-byte swizzle, out-of-range elements read as zero.
acp_status make_map(acp_ctx* ctx, CUtensorMap* m, const float* ptr, int inner, int rows, int ld, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return set_error(ctx, ACP_E_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) || (ld % 4))
    return set_error(ctx, ACP_E_ARG, "TMA operand must be 16-byte aligned with a row stride multiple of 4 floats");
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(ctx, ACP_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return ACP_OK;
}

uint32_t tmem_cols_for(int bn) {
  uint32_t c = 32;
  while ((int)c < bn) c <<= 1;
  return c;
}

size_t smem_for(int bn) { return (size_t)kStages * (2 * kBM * kBK * 4 + 2 * (size_t)bn * kBK * 4) + 1024; }

acp_status launch_tc3(acp_ctx* ctx, dim3 grid, const CUtensorMap& a, const CUtensorMap& alo, const CUtensorMap& bhi,
                      const CUtensorMap& blo, const TcArgs& p) {
  static std::atomic<bool> configured{false};
  if (!configured.load()) {
    std::lock_guard<std::mutex> lock(device_mutex());
    ACP_CUDA(ctx, cudaFuncSetAttribute(tc3_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_for(256)));
    configured.store(true);
  }
  ::acp::note_launch(ctx);
  tc3_gemm_kernel<<<grid, kThreads, smem_for(p.BN), ctx->stream>>>(a, alo, bhi, blo, p);
  ACP_LAUNCH(ctx);
  return ACP_OK;
}

}  // namespace

acp_status mixed_prepare(acp_ctx* ctx) {
  if (!ctx->psi32_stale) return ACP_OK;
  const int N = ctx->N, no = ctx->n_orb;
  ctx->ld32 = (N + 31) / 32 * 32;
  ctx->no_pad = (no + 31) / 32 * 32;
  float* buf = nullptr;
  const size_t a = (size_t)no * ctx->ld32, b = (size_t)N * ctx->no_pad;
  ACP_TRY(ws(ctx, "psi32", 2 * a + 2 * b, &buf));
  ACP_CUDA(ctx, cudaMemsetAsync(buf, 0, (2 * a + 2 * b) * sizeof(float), ctx->stream));
  ctx->d_psi_hi = buf;
  ctx->d_psi_lo = buf + a;
  ctx->d_psiT_hi = buf + 2 * a;
  ctx->d_psiT_lo = buf + 2 * a + b;
  size_t blocks = ((size_t)N * no + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  ::acp::note_launch(ctx);
  psi_split_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(N, no, ctx->ld32, ctx->no_pad, ctx->d_psi, ctx->d_psi_hi,
                                                              ctx->d_psi_lo, ctx->d_psiT_hi, ctx->d_psiT_lo);
  ACP_LAUNCH(ctx);
  ctx->psi32_stale = false;
  return ACP_OK;
}

namespace {

// One projector application with a given tile configuration: GEMM 1 over `slices` K-slices
// (0: automatic, about one CTA per SM), GEMM 2 with output tiles 128 x bn2.
acp_status project32_cfg(acp_ctx* ctx, const float* X, int ldx, int ncol, float* Y, int ldy, int bn2,
                         int slice_mul) {
  const int N = ctx->N, no = ctx->n_orb, no_pad = ctx->no_pad;
  int* status = ctx->d_flag + 8;
  const int m_tiles = (ncol + kBM - 1) / kBM;

  // GEMM 1: C^T = X^T Psi, split over the grid
  const int n_tiles1 = (no + 255) / 256;
  int bn1 = (no + n_tiles1 - 1) / n_tiles1;
  bn1 = (bn1 + 15) / 16 * 16;
  const int kb_total1 = (N + kBK - 1) / kBK;
  int slices = 148 * slice_mul / (m_tiles * n_tiles1);
  if (slices < 1) slices = 1;
  if (slices > kb_total1) slices = kb_total1;
  const int kb_per1 = (kb_total1 + slices - 1) / slices;
  slices = (kb_total1 + kb_per1 - 1) / kb_per1;
  float *part = nullptr, *ct = nullptr;
  const long long slice_stride = (long long)ncol * no_pad;
  ACP_TRY(ws(ctx, "p32_part", (size_t)slices * slice_stride, &part));
  ACP_TRY(ws(ctx, "p32_ct", 2 * (size_t)slice_stride, &ct));
  float* ct_hi = ct;
  float* ct_lo = ct + slice_stride;

  CUtensorMap mX, mPh, mPl, mCh, mCl, mTh, mTl;
  ACP_TRY(make_map(ctx, &mX, X, N, ncol, ldx, kBM));
  ACP_TRY(make_map(ctx, &mPh, ctx->d_psi_hi, N, no, ctx->ld32, bn1));
  ACP_TRY(make_map(ctx, &mPl, ctx->d_psi_lo, N, no, ctx->ld32, bn1));
  TcArgs a1{};
  a1.M = ncol;
  a1.Nd = no;
  a1.BN = bn1;
  a1.kb_per = kb_per1;
  a1.kb_total = kb_total1;
  a1.tmem_cols = tmem_cols_for(bn1);
  a1.split_a = 1;
  a1.mode = 0;
  a1.out = part;
  a1.ldo = no_pad;
  a1.slice_stride = slice_stride;
  a1.status = status;
  a1.wait_ns = kWaitNs;
  const double fl = 2.0 * (double)ncol * no * N;  // algorithmic (the tensor pipe runs 3 passes)
  cudaEvent_t ev = prof_begin(ctx);
  ACP_TRY(launch_tc3(ctx, dim3(m_tiles, slices, n_tiles1), mX, mX, mPh, mPl, a1));
  prof_end(ctx, "tc_gemm", ev, fl, 4.0 * ((double)ncol * N + 2.0 * no * N + (double)slices * ncol * no));

  {
    size_t blocks = ((size_t)slice_stride + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    ::acp::note_launch(ctx);
    slice_reduce_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(ncol, no, no_pad, slices, slice_stride, part,
                                                                   ctx->h, ct_hi, ct_lo);
    ACP_LAUNCH(ctx);
  }

  // GEMM 2: Y^T = X^T - C^T Psi^T
  if (N < bn2) bn2 = (N + 15) / 16 * 16;
  ACP_TRY(make_map(ctx, &mCh, ct_hi, no_pad, ncol, no_pad, kBM));
  ACP_TRY(make_map(ctx, &mCl, ct_lo, no_pad, ncol, no_pad, kBM));
  ACP_TRY(make_map(ctx, &mTh, ctx->d_psiT_hi, no_pad, N, no_pad, bn2));
  ACP_TRY(make_map(ctx, &mTl, ctx->d_psiT_lo, no_pad, N, no_pad, bn2));
  TcArgs a2{};
  a2.M = ncol;
  a2.Nd = N;
  a2.BN = bn2;
  a2.kb_total = no_pad / kBK;
  a2.kb_per = a2.kb_total;
  a2.tmem_cols = tmem_cols_for(bn2);
  a2.split_a = 0;
  a2.mode = 1;
  a2.X = X;
  a2.ldx = ldx;
  a2.Y = Y;
  a2.ldy = ldy;
  a2.status = status;
  a2.wait_ns = kWaitNs;
  ev = prof_begin(ctx);
  ACP_TRY(launch_tc3(ctx, dim3(m_tiles, 1, (N + bn2 - 1) / bn2), mCh, mCl, mTh, mTl, a2));
  prof_end(ctx, "tc_gemm", ev, fl, 4.0 * (2.0 * ncol * N + 2.0 * no * N + 2.0 * (double)ncol * no_pad));
  return ACP_OK;
}

constexpr int kTileCandidates[][2] = {{256, 1}, {128, 1}, {64, 1}, {256, 2}, {128, 2}};

}  // namespace

// Y = Q X.  The tile configuration (GEMM 2 tile width, GEMM 1 K-slices) is chosen per problem
// shape by timing every candidate once on the caller's data (Q is idempotent, so the extra
// applications leave Y = Q X unchanged up to rounding) and kept in the context.
acp_status project32(acp_ctx* ctx, const float* X, int ldx, int ncol, float* Y, int ldy) {
  if (ncol <= 0) return ACP_OK;
  ACP_TRY(mixed_prepare(ctx));
  const int N = ctx->N;
  if ((ldx % 4) || (ldy % 4) || ldx < N || ldy < N)
    return set_error(ctx, ACP_E_ARG, "FP32 blocks need a leading dimension >= N and a multiple of 4");
  int lg = 0;
  while ((1 << (lg + 1)) <= ncol) ++lg;
  const long long key = ((long long)lg << 48) ^ ((long long)N << 20) ^ (long long)ctx->n_orb;
  auto it = ctx->tc_tune.find(key);
  if (it == ctx->tc_tune.end()) {
    // first application at this shape: Y = Q X once, then time each candidate on Y in place
    ACP_TRY(project32_cfg(ctx, X, ldx, ncol, Y, ldy, 256, 1));
    const bool prof_on = ctx->prof.on;
    ctx->prof.on = false;
    cudaEvent_t e0, e1;
    ACP_CUDA(ctx, cudaEventCreate(&e0));
    ACP_CUDA(ctx, cudaEventCreate(&e1));
    float best = 1e30f;
    int best_i = 0;
    const int ncand = (int)(sizeof(kTileCandidates) / sizeof(kTileCandidates[0]));
    for (int c = 0; c < ncand; ++c) {
      ACP_TRY(project32_cfg(ctx, Y, ldy, ncol, Y, ldy, kTileCandidates[c][0], kTileCandidates[c][1]));  // warm
      ACP_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
      ACP_TRY(project32_cfg(ctx, Y, ldy, ncol, Y, ldy, kTileCandidates[c][0], kTileCandidates[c][1]));
      ACP_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
      ACP_CUDA(ctx, cudaEventSynchronize(e1));
      float ms = 0.f;
      ACP_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        best_i = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->prof.on = prof_on;
    ctx->tc_tune[key] = {kTileCandidates[best_i][0], kTileCandidates[best_i][1]};
    return ACP_OK;
  }
  return project32_cfg(ctx, X, ldx, ncol, Y, ldy, it->second.first, it->second.second);
}

namespace {
__global__ void narrow_kernel(int N, int ncol, int ld32, const double* __restrict__ X, float* __restrict__ Y) {
  const size_t total = (size_t)N * ncol;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    Y[(e / N) * ld32 + e % N] = (float)X[e];
}
__global__ void widen_kernel(int N, int ncol, int ld32, const float* __restrict__ X, double* __restrict__ Y) {
  const size_t total = (size_t)N * ncol;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    Y[e] = (double)X[(e / N) * ld32 + e % N];
}
}  // namespace

// Y = Q X through the FP32 tensor-core projector (FP64 in and out; stage check of project32).
acp_status project_mixed64(acp_ctx* ctx, const double* X, int ncol, double* Y) {
  if (ncol <= 0) return ACP_OK;
  ACP_TRY(mixed_prepare(ctx));
  const int N = ctx->N, ld = ctx->ld32;
  float* x32 = nullptr;
  ACP_TRY(ws(ctx, "pm_x32", (size_t)ld * ncol, &x32));
  ACP_CUDA(ctx, cudaMemsetAsync(x32, 0, sizeof(float) * ld * ncol, ctx->stream));
  size_t blocks = ((size_t)N * ncol + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  ::acp::note_launch(ctx);
  narrow_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(N, ncol, ld, X, x32);
  ACP_LAUNCH(ctx);
  ACP_TRY(project32(ctx, x32, ld, ncol, x32, ld));
  ::acp::note_launch(ctx);
  widen_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(N, ncol, ld, x32, Y);
  ACP_LAUNCH(ctx);
  return tc_check(ctx);
}

// Failure self-test of the bounded waits: GEMM 1 of the projector on a zero block of 128 columns
// with its TMA loads withheld, so the split warps' and the MMA warp's barrier waits run out after
// wait_ns; the kernel then skips its MMAs and epilogue, waits (bounded) for the empty commit,
// frees its TMEM, sets the status word and returns.  Returns what tc_check reports
// (ACP_E_TIMEOUT when the abort path ran).
acp_status tc_selftest_timeout(acp_ctx* ctx, uint64_t wait_ns) {
  ACP_TRY(mixed_prepare(ctx));
  const int N = ctx->N, no = ctx->n_orb, no_pad = ctx->no_pad, ld = ctx->ld32;
  const int ncol = kBM;
  float *x = nullptr, *part = nullptr;
  ACP_TRY(ws(ctx, "st_x", (size_t)ld * ncol, &x));
  ACP_TRY(ws(ctx, "st_part", (size_t)ncol * no_pad, &part));
  ACP_CUDA(ctx, cudaMemsetAsync(x, 0, sizeof(float) * ld * ncol, ctx->stream));
  const int n_tiles1 = (no + 255) / 256;
  int bn1 = (no + n_tiles1 - 1) / n_tiles1;
  bn1 = (bn1 + 15) / 16 * 16;
  CUtensorMap mX, mPh, mPl;
  ACP_TRY(make_map(ctx, &mX, x, N, ncol, ld, kBM));
  ACP_TRY(make_map(ctx, &mPh, ctx->d_psi_hi, N, no, ld, bn1));
  ACP_TRY(make_map(ctx, &mPl, ctx->d_psi_lo, N, no, ld, bn1));
  TcArgs a{};
  a.M = ncol;
  a.Nd = no;
  a.BN = bn1;
  a.kb_total = (N + kBK - 1) / kBK;
  a.kb_per = a.kb_total;
  a.tmem_cols = tmem_cols_for(bn1);
  a.split_a = 1;
  a.mode = 0;
  a.out = part;
  a.ldo = no_pad;
  a.slice_stride = (long long)ncol * no_pad;
  a.status = ctx->d_flag + 8;
  a.wait_ns = wait_ns;
  a.withhold = 1;
  ACP_TRY(launch_tc3(ctx, dim3(1, 1, n_tiles1), mX, mX, mPh, mPl, a));
  return tc_check(ctx);
}

// Device status word of the tensor-core kernels: nonzero after a bounded wait ran out.
acp_status tc_check(acp_ctx* ctx) {
  int h = 0;
  ACP_CUDA(ctx, cudaMemcpyAsync(&h, ctx->d_flag + 8, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (h) {
    ACP_CUDA(ctx, cudaMemsetAsync(ctx->d_flag + 8, 0, sizeof(int), ctx->stream));
    return set_error(ctx, ACP_E_TIMEOUT, "a tensor-core GEMM pipeline wait timed out");
  }
  return ACP_OK;
}

}  // namespace acp
