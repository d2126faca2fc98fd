// Internal declarations of the ACP library: context, workspace, error plumbing, device helpers.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/acp.h"

namespace acp {

// ---- FFT plan: N = prod rad[s], radices in {2, 3, 4, 5}; threads per transform --------------
// Largest 1D grid: one FP64 column pair (16 bytes a point) stays within a CTA's shared memory.
constexpr int kMaxFftN = 10240;

struct FftPlan {
  int n = 0;
  int nst = 0;
  int rad[24];
  int threads = 0;     // CTA size of the spectral kernels
  bool wide = false;   // CTAs of up to 1024 threads (grids the 512-thread form does not cover)
};

bool make_fft_plan(int n, FftPlan* plan);

// ---- instrumentation: per-kernel device time from CUDA events on the context's stream --------
struct Profiler {
  bool on = false;
  long long launches = 0;  // every kernel launch of the library, counted whether on or not
  std::vector<cudaEvent_t> pool;
  size_t next = 0;
  struct Pending {
    const char* name;
    cudaEvent_t a, b;
    double flops, bytes;
  };
  std::vector<Pending> pending;
  struct Acc {
    double ms = 0, flops = 0, bytes = 0;
    long long n = 0;
  };
  std::map<std::string, Acc> acc;
  ~Profiler();
};

// ---- workspace: named device buffers that grow on demand ------------------------------------
struct Workspace {
  std::map<std::string, std::pair<void*, size_t>> bufs;
  ~Workspace();
};

}  // namespace acp

struct acp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int N = 0;
  double L = 0, h = 0;            // h: quadrature weight of a grid point (hx in 1D, hx hy in 2D)
  int dim = 1;                    // 2D: N = nx ny, x fastest
  int nx = 0, ny = 0;
  double Lx = 0, Ly = 0;
  acp::FftPlan plan_x, plan_y;    // 2D: per-axis plans of the multi-pass transforms
  double2* d_twx = nullptr;       // 2D: exp(-2 pi i m / nx), then exp(-2 pi i m / ny) (d_twy)
  double2* d_twy = nullptr;
  size_t smem_optin = 0;          // dynamic shared memory a CTA may use on this device
  double kappa = 0, scale = 0;
  int n_orb = 0;
  acp_options opt{};
  std::vector<double> eps;        // host copy, ascending
  double* d_V = nullptr;          // N
  double* d_psi = nullptr;        // N x n_orb
  double* d_eps = nullptr;        // n_orb
  double* d_kin = nullptr;        // N: k^2/2
  double* d_khat = nullptr;       // N: Khat(k)
  double* d_khat_inv = nullptr;   // N: 1/Khat(k)
  double* d_kvec = nullptr;       // N: k with the Nyquist entry zeroed (odd multipliers)
  double2* d_tw = nullptr;        // N: exp(-2 pi i m / N)
  int* d_flag = nullptr;          // device status word / counters (16 ints)
  // mixed precision: FP32 blocks use leading dimension ld32 (N rounded up to 32); the orbitals
  // are kept as TF32 hi + FP32 lo parts in both orientations for the tensor-core projector.
  int ld32 = 0, no_pad = 0;
  float* d_psi_hi = nullptr;   // n_orb x ld32 (orbital rows)
  float* d_psi_lo = nullptr;
  float* d_psiT_hi = nullptr;  // N x no_pad (grid rows, orbitals contiguous)
  float* d_psiT_lo = nullptr;
  bool psi32_stale = true;
  bool tables32_stale = true;     // FP32 copies of the kinetic symbol, V_eff and twiddles
  std::map<long long, std::pair<int, int>> tc_tune;  // projector tile choice per shape
  bool mixed_refine = true;       // mixed precision: refine the multi-shift solves to stern_tol
  long long graph_launch_nodes = 0;  // kernels replayed through CUDA graphs (launch counter)
  bool cnn_ready = false;         // weights of the learned initial guess are set (2D)
  long long cnn_steps = 0;        // Adam steps taken since the weights were set
  acp::FftPlan plan;
  acp::Workspace ws;
  acp::Profiler prof;
  std::string err;
};

namespace acp {

// ---- errors ---------------------------------------------------------------------------------
acp_status set_error(acp_ctx* ctx, acp_status st, const char* fmt, ...);

#define ACP_CUDA(ctx, call)                                                                    \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return ::acp::set_error((ctx), ACP_E_CUDA, "%s failed: %s (%s:%d)", #call,               \
                              cudaGetErrorString(e_), __FILE__, __LINE__);                     \
  } while (0)

#define ACP_LAUNCH(ctx)                                                                        \
  do {                                                                                         \
    cudaError_t e_ = cudaGetLastError();                                                       \
    if (e_ != cudaSuccess)                                                                     \
      return ::acp::set_error((ctx), ACP_E_CUDA, "kernel launch failed: %s (%s:%d)",           \
                              cudaGetErrorString(e_), __FILE__, __LINE__);                     \
  } while (0)

#define ACP_TRY(x)                                                                             \
  do {                                                                                         \
    acp_status s_ = (x);                                                                       \
    if (s_ != ACP_OK) return s_;                                                               \
  } while (0)

// Serialises the calls that may synchronise the device (workspace cudaMalloc / cudaFree, function
// attributes) with CUDA-graph captures, when several host threads drive contexts at once.
std::mutex& device_mutex();

// Device buffer from the context's workspace, grown (never shrunk) to hold `bytes`.
acp_status ws_get(acp_ctx* ctx, const char* name, size_t bytes, void** out);
template <class T>
inline acp_status ws(acp_ctx* ctx, const char* name, size_t count, T** out) {
  return ws_get(ctx, name, count * sizeof(T), reinterpret_cast<void**>(out));
}

double now_ms();
bool deadline_passed(const acp_ctx* ctx, double t0_ms);

inline void note_launch(acp_ctx* ctx) { ++ctx->prof.launches; }
// Event recorded on the context's stream before a timed launch (nullptr when profiling is off).
cudaEvent_t prof_begin(acp_ctx* ctx);
// Records the end event of a timed launch with its algorithmic flops and bytes.
void prof_end(acp_ctx* ctx, const char* name, cudaEvent_t begin, double flops, double bytes);
// Accumulates the elapsed times of completed launches (the stream must be synchronised).
void prof_flush(acp_ctx* ctx);
// Sets the work of the last recorded launch of `name` (known only after the launch completes).
void prof_amend_last(acp_ctx* ctx, const char* name, double flops, double bytes);

// ---- host wrappers of the kernels (one translation unit each) -------------------------------
// spectral.cu
enum SpectralMult { MULT_KINETIC = 0, MULT_KHAT = 1, MULT_KHAT_INV = 2 };
// Y[:, j] = IFFT(mult * FFT(X[:, j])) + (with_v ? V .* X[:, j] : 0) - shift_d[j] X[:, j]
// alpha_d (nullable): alpha_d[j] = X[:, j] . Y[:, j] (no weight).  Columns with active_d[j] == 0
// are skipped when active_d is not null.  Lanczos form (Xprev != nullptr): the output is
// Y - alpha_j X_j - beta_d[j] Xprev_j, the unprojected next Lanczos vector.
acp_status spectral_apply(acp_ctx* ctx, const double* X, int ldx, int ncol, SpectralMult mult, bool with_v,
                          const double* shift_d, double* Y, int ldy, double* alpha_d, const int* active_d,
                          const double* Xprev = nullptr, const double* beta_d = nullptr);
// Raise the dynamic shared-memory limit of the spectral kernels (once per device, never lowered).
acp_status spectral_configure(acp_ctx* ctx);
// Set the dynamic shared-memory limit of a kernel to the opt-in maximum minus its static usage.
acp_status raise_smem_limit(acp_ctx* ctx, const void* func);
// 2D (spectral2d.cu): per-axis FFT plans, the multi-pass spectral operator in FP64 or FP32 (same
// semantics as spectral_apply / spectral32_apply), perturbation potentials (G, B: N x 2 nA,
// column 2I + a; D2: N x 3 nA, columns 3I + {xx, xy, yy}), the ion-ion Hessian blocks and the
// assembly of D.
bool make_axis_plan(int n, FftPlan* plan);
acp_status spectral2d_apply_f64(acp_ctx* ctx, const double* X, int ldx, int ncol, const double* mult, const double* V,
                                const double* shift_d, double* Y, int ldy, double* alpha_d, const int* active_d,
                                const double* Xp, int ldp, const double* beta_d);
acp_status spectral2d_apply_f32(acp_ctx* ctx, const float* X, int ldx, int ncol, const float* mult, const float* V,
                                const float* shift_d, float* Y, int ldy, float* alpha_d, const int* active_d,
                                const float* Xp, int ldp, const float* beta_d, const float2* twx, const float2* twy,
                                const int* kdev, long long kstride);
acp_status perturbations_2d(acp_ctx* ctx, int nA, const double* R_d, const double* Z_d, const double* sig_d,
                            double* G, double* B, double* D2);
acp_status ion_hessian_2d(acp_ctx* ctx, int nA, const double* R_h, const double* R_d, double* Hp);
acp_status assemble_2d(acp_ctx* ctx, int nA, const double* Hm, const double* dv, const double* Hp, const double* Z_d,
                       const double* M_d, double* D);
// Perturbation potentials of n_atoms atoms (1D): G, B, d2V (each nullable, N x n_atoms).
acp_status perturbations_1d(acp_ctx* ctx, int n_atoms, const double* R_d, const double* Z_d, const double* sig_d,
                            double* G, double* B, double* D2);

// dgemm.cu: C = alpha op(A) op(B) + beta C (column-major).  If hz != nullptr the epilogue is
// C += alpha * hz .* (op(A) op(B)) (Hadamard accumulate; ldhz = leading dimension).
acp_status dgemm(acp_ctx* ctx, bool ta, bool tb, int m, int n, int k, double alpha, const double* A, int lda,
                 const double* B, int ldb, double beta, double* C, int ldc, const double* hz = nullptr,
                 int ldhz = 0);

// projector: Y = Q X (Y may alias X).  Columns processed in chunks through workspace "proj".
acp_status project(acp_ctx* ctx, const double* X, int ldx, int ncol, double* Y, int ldy);

// minres.cu
struct SolveReport {
  long long converged = 0;
  long long steps = 0;
  long long max_iters = 0;
  double max_rel_res = 0;
  bool all_converged = true;
};
// Solve Q(H - shift_d[j])Q X_j = B_j (B must already be projected) for ncol columns.
acp_status minres_batched(acp_ctx* ctx, const double* B, int ncol, const double* shift_d, double* X,
                          SolveReport* rep, double t0_ms);
// The FP64 batched solve whatever opt.precision says, to relative residual tol (X starts at 0).
acp_status minres_batched_fp64(acp_ctx* ctx, const double* B, int ncol, const double* shift_d, double* X,
                               double tol, SolveReport* rep, double t0_ms);
// Multi-shift: for each column mu of B solve Q(H - nodes[c])Q X_{c,mu} = B_mu for all c.
// X layout: column mu + c * ncol of an N x (nc * ncol) block.
acp_status minres_multishift(acp_ctx* ctx, const double* B, int ncol, const double* nodes_d, int nc, double* X,
                             SolveReport* rep, double t0_ms);

// qrcp.cu: Alg. 2 (Remark form) on G (N x ncol).  Writes n_mu, pivots (device, int), Xi (N x n_mu,
// workspace "xi"), and |R_mm| on the host.
struct Compression {
  int n_mu = 0;
  int* d_piv = nullptr;   // workspace-owned
  double* d_xi = nullptr; // workspace-owned, N x n_mu
  std::vector<int> piv;
  std::vector<double> rdiag;
};
acp_status compress(acp_ctx* ctx, const double* G, int ncol, const double* sketch_h, int sketch_cols,
                    double id_tol, int max_rank, Compression* out);

// minres32.cu: the same solves with FP32 MINRES (tensor-core projector) and FP64 iterative
// refinement; used when opt.precision == ACP_PREC_MIXED.
acp_status minres_batched_mixed(acp_ctx* ctx, const double* B, int ncol, const double* shift_d, double* X,
                                SolveReport* rep, double t0_ms);
acp_status minres_multishift_mixed(acp_ctx* ctx, const double* B, int nmu, const double* nodes_d, int nc, double* X,
                                   SolveReport* rep, double t0_ms);
// spectral32.cu: FP32 (H - s) X, or the Lanczos form when Xprev is given (see spectral_apply).
// With kdev (stored basis), X and Xprev are slot 0 of the basis and the kernel uses slots k and
// k - 1, k = *kdev, slot stride kstride elements.
acp_status spectral32_apply(acp_ctx* ctx, const float* X, int ldx, int ncol, const float* shift_d, float* Y, int ldy,
                            float* alpha_d, const int* active_d, const float* Xprev, int ldp, const float* beta_d,
                            const int* kdev = nullptr, long long kstride = 0);

// tc_gemm.cu: FP32 projector Y = Q X on the tensor cores (3xTF32 tcgen05 GEMMs); X, Y FP32 blocks
// with leading dimensions that are multiples of 4 (Y may alias X).  mixed_prepare builds the FP32
// orbital copies when the orbitals changed; tc_check reads the tensor-core status word.
acp_status mixed_prepare(acp_ctx* ctx);
acp_status project32(acp_ctx* ctx, const float* X, int ldx, int ncol, float* Y, int ldy);
acp_status tc_check(acp_ctx* ctx);
acp_status tc_selftest_timeout(acp_ctx* ctx, uint64_t wait_ns);
acp_status project_mixed64(acp_ctx* ctx, const double* X, int ncol, double* Y);

// cnn.cu: the learned initial guess of the 2D Sternheimer solves.  cnn_set_weights copies the
// packed FP32 weights (host) and builds the bfloat16 copies; cnn_initial_guess writes
// X0 = rms(R_j) net(R_j / rms(R_j), V_eff - shift_j) per column (not projected).
acp_status cnn_set_weights(acp_ctx* ctx, const float* w_h);
acp_status cnn_initial_guess(acp_ctx* ctx, const double* R, int ldr, int ncol, const double* shift_d, double* X0,
                             int ldx);
// cnn_train.cu: one Adam step on nsamp solved samples (R, V - s, X*) on an nx x ny grid, FP32
// master weights; loss before the step to *loss_h; the gradient to grad_h if not null (host,
// ACP_CNN_WEIGHTS values).
acp_status cnn_train_step(acp_ctx* ctx, int nx, int ny, const double* R, const double* VS, const double* Xs,
                          int nsamp, float lr, double* loss_h, float* grad_h);

// dense.cu: LU solve of an n x n system with nrhs right-hand sides (A, B overwritten; X in B).
acp_status lu_solve(acp_ctx* ctx, double* A, int n, double* B, int nrhs);
// Jacobi eigensolver of a symmetric n x n device matrix; eigenvalues (ascending) and vectors.
acp_status jacobi_eig(acp_ctx* ctx, double* A, int n, double* w_d, double* V_d);
// Frobenius norms: out_h[0] = ||A - B||_F^2, out_h[1] = ||A||_F^2 (N x ncol blocks)
acp_status diff_norms(acp_ctx* ctx, const double* A, const double* B, size_t count, double* out_h);
// small helpers
acp_status gather_rows(acp_ctx* ctx, const double* X, int ldx, int ncol, const int* rows_d, int nrows, double* Y,
                       int ldy);

}  // namespace acp

// ---- device helpers ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA; every thread gets the result.  red must hold 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (wid == 0) {
    t = warp_sum(t);
    if (lane == 0) red[0] = t;
  }
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}
