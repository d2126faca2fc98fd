// C ABI entry points (include/acp.h): context life cycle, workspace, options and dispatch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <thread>

#include "internal.cuh"

namespace acp {

acp_status chi0_plain(acp_ctx* ctx, const double* G, int ncol, double* out, SolveReport* rep, double t0);
acp_status chi0_acp(acp_ctx* ctx, const double* G, int ncol, double* out, acp_stats* st, SolveReport* rep, double t0);
acp_status dyson(acp_ctx* ctx, const double* G, int ncol, double* U, acp_stats* st, SolveReport* rep, double t0);
acp_status dynamical(acp_ctx* ctx, const acp_atoms* at, const double* rho, double* D_h, double* U_user,
                     acp_stats* st, SolveReport* rep, double t0);

Workspace::~Workspace() {
  for (auto& kv : bufs)
    if (kv.second.first) cudaFree(kv.second.first);
}

acp_status set_error(acp_ctx* ctx, acp_status st, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

std::mutex& device_mutex() {
  static std::mutex mu;
  return mu;
}

acp_status ws_get(acp_ctx* ctx, const char* name, size_t bytes, void** out) {
  if (bytes == 0) bytes = 8;
  auto it = ctx->ws.bufs.find(name);
  if (it != ctx->ws.bufs.end() && it->second.second >= bytes) {
    *out = it->second.first;
    return ACP_OK;
  }
  // cudaFree synchronises the device, which must not overlap another thread's stream capture
  std::lock_guard<std::mutex> lock(device_mutex());
  if (it != ctx->ws.bufs.end()) {
    cudaFree(it->second.first);  // synchronises the device before the memory is reused
    ctx->ws.bufs.erase(it);
  }
  void* p = nullptr;
  const size_t cap = bytes + bytes / 8;  // headroom against small regrowths
  cudaError_t e = cudaMalloc(&p, cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(ctx, ACP_E_OOM, "cudaMalloc of %zu bytes for workspace '%s' failed: %s", cap, name,
                     cudaGetErrorString(e));
  }
  ctx->ws.bufs[name] = {p, cap};
  *out = p;
  return ACP_OK;
}

Profiler::~Profiler() {
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

cudaEvent_t prof_begin(acp_ctx* ctx) {
  Profiler& p = ctx->prof;
  if (!p.on) return nullptr;
  if (p.next + 2 > p.pool.size()) {
    if (p.pool.size() >= 200000) return nullptr;  // bounded; the remaining launches go untimed
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      p.pool.push_back(e);
    }
  }
  cudaEvent_t e = p.pool[p.next++];
  cudaEventRecord(e, ctx->stream);
  return e;
}

void prof_end(acp_ctx* ctx, const char* name, cudaEvent_t begin, double flops, double bytes) {
  Profiler& p = ctx->prof;
  if (!p.on || !begin || p.next >= p.pool.size()) return;
  cudaEvent_t e = p.pool[p.next++];
  cudaEventRecord(e, ctx->stream);
  p.pending.push_back({name, begin, e, flops, bytes});
}

void prof_amend_last(acp_ctx* ctx, const char* name, double flops, double bytes) {
  Profiler& p = ctx->prof;
  if (!p.on || p.pending.empty() || std::strcmp(p.pending.back().name, name) != 0) return;
  p.pending.back().flops = flops;
  p.pending.back().bytes = bytes;
}

void prof_flush(acp_ctx* ctx) {
  Profiler& p = ctx->prof;
  if (p.pending.empty()) {
    p.next = 0;
    return;
  }
  cudaStreamSynchronize(ctx->stream);
  for (const auto& q : p.pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, q.a, q.b) != cudaSuccess) continue;
    auto& a = p.acc[q.name];
    a.ms += ms;
    a.flops += q.flops;
    a.bytes += q.bytes;
    a.n += 1;
  }
  cudaGetLastError();
  p.pending.clear();
  p.next = 0;
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

bool deadline_passed(const acp_ctx* ctx, double t0_ms) {
  return ctx->opt.deadline_s > 0 && (now_ms() - t0_ms) > ctx->opt.deadline_s * 1e3;
}

namespace {

acp_status validate_options(acp_ctx* ctx, const acp_options* o) {
  if (o->method != ACP_METHOD_PLAIN && o->method != ACP_METHOD_ACP)
    return set_error(ctx, ACP_E_ARG, "unknown method %d", o->method);
  if (!(o->occ > 0)) return set_error(ctx, ACP_E_ARG, "occupation must be positive");
  if (o->n_cheb < 1 || o->n_cheb > 64) return set_error(ctx, ACP_E_ARG, "n_cheb %d outside [1, 64]", o->n_cheb);
  if (!(o->stern_tol > 0) || o->stern_maxit < 1) return set_error(ctx, ACP_E_ARG, "bad Sternheimer tolerance/maxit");
  if (!(o->dyson_tol > 0)) return set_error(ctx, ACP_E_ARG, "bad Dyson tolerance");
  if (o->sketch_cols < 0) return set_error(ctx, ACP_E_ARG, "negative sketch_cols");
  if (o->project_every < 0) return set_error(ctx, ACP_E_ARG, "negative project_every");
  if (o->ms_variant < 0 || o->ms_variant > 2) return set_error(ctx, ACP_E_ARG, "ms_variant must be 0, 1 or 2");
  if (o->precision != ACP_PREC_FP64 && o->precision != ACP_PREC_MIXED)
    return set_error(ctx, ACP_E_ARG, "unknown precision %d", o->precision);
  if (o->learned != 0 && o->learned != 1) return set_error(ctx, ACP_E_ARG, "learned must be 0 or 1");
  return ACP_OK;
}

void fill_stats(acp_stats* st, const SolveReport& rep, double t0) {
  if (!st) return;
  st->ms_total = 0;
  st->rhs_solved += rep.converged;
  st->lanczos_steps += rep.steps;
  if (rep.max_iters > st->max_iters) st->max_iters = rep.max_iters;
  if (rep.max_rel_res > st->max_rel_res) st->max_rel_res = rep.max_rel_res;
  st->ms_total = now_ms() - t0;
}

acp_status check_ctx(acp_ctx* ctx) {
  if (!ctx) return ACP_E_ARG;
  ctx->err.clear();
  prof_flush(ctx);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return set_error(ctx, ACP_E_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  return ACP_OK;
}

}  // namespace
}  // namespace acp

using namespace acp;

extern "C" {

void acp_options_default(acp_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->method = ACP_METHOD_ACP;
  o->occ = 1.0;
  o->n_cheb = 16;
  o->id_tol = 1e-5;
  o->sketch_cols = 0;
  o->sketch = nullptr;
  o->max_rank = 0;
  o->stern_tol = 1e-11;
  o->stern_maxit = 5000;
  o->dyson_tol = 1e-10;
  o->dyson_maxit = 30;
  o->rhs_batch = 0;
  o->deadline_s = 0;
}

const char* acp_status_string(acp_status s) {
  switch (s) {
    case ACP_OK: return "ok";
    case ACP_E_ARG: return "invalid argument";
    case ACP_E_CUDA: return "CUDA error";
    case ACP_E_OOM: return "out of device memory";
    case ACP_E_NOCONV: return "iteration did not converge";
    case ACP_E_TIMEOUT: return "deadline exceeded";
    case ACP_E_GAP: return "eigenvalues not ascending / no gap";
    case ACP_E_RANK: return "pivoted QR rank is zero";
    case ACP_E_NUMERIC: return "NaN or Inf";
  }
  return "unknown status";
}

const char* acp_last_error(const acp_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

acp_status acp_grid_supported(const acp_grid* g) {
  if (!g) return ACP_E_ARG;
  acp::FftPlan p;
  if (g->dim == 1) return acp::make_fft_plan(g->n[0], &p) ? ACP_OK : ACP_E_ARG;
  if (g->dim == 2) return (acp::make_axis_plan(g->n[0], &p) && acp::make_axis_plan(g->n[1], &p)) ? ACP_OK : ACP_E_ARG;
  return ACP_E_ARG;
}

acp_status acp_phonon_dos(const double* omega_h, int n, const double* w_h, int n_w, double sigma, double* rho_h) {
  if (!omega_h || n < 1 || n_w < 0 || !(sigma > 0.0) || !std::isfinite(sigma)) return ACP_E_ARG;
  if (n_w == 0) return ACP_OK;
  if (!w_h || !rho_h) return ACP_E_ARG;
  for (int k = 0; k < n; ++k)
    if (!std::isfinite(omega_h[k])) return ACP_E_ARG;
  for (int j = 0; j < n_w; ++j)
    if (!std::isfinite(w_h[j])) return ACP_E_ARG;
  // delta_sigma(x) = exp(-x^2 / (2 sigma^2)) / sqrt(2 pi sigma^2); the 1 / n of the spectrum is
  // folded into the prefactor
  const double inv2s2 = 0.5 / (sigma * sigma);
  const double pref = 1.0 / (std::sqrt(2.0 * M_PI * sigma * sigma) * n);
  for (int j = 0; j < n_w; ++j) {
    double acc = 0.0;
    for (int k = 0; k < n; ++k) {
      const double x = w_h[j] - omega_h[k];
      acc += std::exp(-x * x * inv2s2);
    }
    rho_h[j] = pref * acc;
  }
  return ACP_OK;
}

acp_status acp_init(acp_ctx** out, const acp_grid* g, const acp_kernel* k, const double* v_eff_d,
                    const double* psi_d, const double* eps_h, int n_orb, const acp_options* opt, void* stream) {
  if (!out || !g || !k || !v_eff_d || !psi_d || !eps_h || !opt) return ACP_E_ARG;
  *out = nullptr;
  acp_ctx* ctx = new acp_ctx();
  auto fail = [&](acp_status st) {
    // keep the context so the caller can read the message, then destroy
    *out = ctx;
    return st;
  };
  if (g->dim != 1 && g->dim != 2) return fail(set_error(ctx, ACP_E_ARG, "only dim = 1 or 2 grids are supported"));
  ctx->dim = g->dim;
  int N = g->n[0];
  if (g->dim == 1) {
    if (!make_fft_plan(N, &ctx->plan))
      return fail(set_error(ctx, ACP_E_ARG,
                            "grid size %d is not supported: it must be 2^a 3^b 5^c in [8, %d]", N, kMaxFftN));
  } else {
    if (!make_axis_plan(g->n[0], &ctx->plan_x) || !make_axis_plan(g->n[1], &ctx->plan_y))
      return fail(set_error(ctx, ACP_E_ARG, "2D grid sizes %d x %d must be 2^a 3^b 5^c in [8, 4096]", g->n[0],
                            g->n[1]));
    if (!(g->L[1] > 0)) return fail(set_error(ctx, ACP_E_ARG, "bad box length"));
    ctx->nx = g->n[0];
    ctx->ny = g->n[1];
    ctx->Lx = g->L[0];
    ctx->Ly = g->L[1];
    N = ctx->nx * ctx->ny;
    ctx->plan = ctx->plan_x;
  }
  if (!(g->L[0] > 0) || !(k->kappa > 0) || n_orb < 1 || n_orb >= N)
    return fail(set_error(ctx, ACP_E_ARG, "bad box length, kappa or n_orb"));
  for (int i = 0; i < n_orb; ++i) {
    if (!std::isfinite(eps_h[i])) return fail(set_error(ctx, ACP_E_NUMERIC, "eigenvalue %d is not finite", i));
    if (i && eps_h[i] < eps_h[i - 1]) return fail(set_error(ctx, ACP_E_GAP, "eigenvalues must be ascending"));
  }
  acp_status st = validate_options(ctx, opt);
  if (st != ACP_OK) return fail(st);
  cudaGetDevice(&ctx->device);
  ctx->stream = static_cast<cudaStream_t>(stream);
  ctx->N = N;
  ctx->L = g->L[0];
  ctx->h = (g->dim == 1) ? ctx->L / N : (g->L[0] / g->n[0]) * (g->L[1] / g->n[1]);
  ctx->kappa = k->kappa;
  ctx->scale = k->scale;
  ctx->n_orb = n_orb;
  ctx->opt = *opt;
  ctx->eps.assign(eps_h, eps_h + n_orb);
  // grid tables on the host (FP64, host libm), copied once
  std::vector<double> kin(N), khat(N), kinv(N), kodd(N, 0.0);
  std::vector<double2> tw(N);
  if (g->dim == 1) {
    for (int a = 0; a < N; ++a) {
      const int n = (a < (N + 1) / 2) ? a : a - N;
      const double kk = 2.0 * M_PI * n / ctx->L;
      kin[a] = 0.5 * kk * kk;
      khat[a] = 4.0 * M_PI * ctx->scale / (kk * kk + ctx->kappa * ctx->kappa);
      kinv[a] = 1.0 / khat[a];
      kodd[a] = (2 * a == N) ? 0.0 : kk;
      const double ang = 2.0 * M_PI * (double)a / N;
      tw[a] = make_double2(std::cos(ang), -std::sin(ang));
    }
  } else {
    // symbols on the (ky, kx) grid, kx fastest; twiddles of the x axis then of the y axis
    const int nx = ctx->nx, ny = ctx->ny;
    for (int iy = 0; iy < ny; ++iy) {
      const int my = (iy < (ny + 1) / 2) ? iy : iy - ny;
      const double ky = 2.0 * M_PI * my / ctx->Ly;
      for (int ix = 0; ix < nx; ++ix) {
        const int mx = (ix < (nx + 1) / 2) ? ix : ix - nx;
        const double kx = 2.0 * M_PI * mx / ctx->Lx;
        const double k2 = kx * kx + ky * ky;
        const int a = ix + nx * iy;
        kin[a] = 0.5 * k2;
        khat[a] = 4.0 * M_PI * ctx->scale / (k2 + ctx->kappa * ctx->kappa);
        kinv[a] = 1.0 / khat[a];
      }
    }
    for (int m = 0; m < nx; ++m) {
      const double ang = 2.0 * M_PI * (double)m / nx;
      tw[m] = make_double2(std::cos(ang), -std::sin(ang));
    }
    for (int m = 0; m < ny; ++m) {
      const double ang = 2.0 * M_PI * (double)m / ny;
      tw[nx + m] = make_double2(std::cos(ang), -std::sin(ang));
    }
  }
  auto alloc = [&](void** p, size_t bytes) -> acp_status {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return set_error(ctx, ACP_E_OOM, "cudaMalloc: %s", cudaGetErrorString(e));
    return ACP_OK;
  };
  if ((st = alloc((void**)&ctx->d_V, N * sizeof(double))) != ACP_OK) return fail(st);
  if ((st = alloc((void**)&ctx->d_psi, (size_t)N * n_orb * sizeof(double))) != ACP_OK) return fail(st);
  if ((st = alloc((void**)&ctx->d_eps, n_orb * sizeof(double))) != ACP_OK) return fail(st);
  if ((st = alloc((void**)&ctx->d_kin, 4 * N * sizeof(double))) != ACP_OK) return fail(st);
  if ((st = alloc((void**)&ctx->d_tw, N * sizeof(double2))) != ACP_OK) return fail(st);
  if ((st = alloc((void**)&ctx->d_flag, 64 * sizeof(int))) != ACP_OK) return fail(st);
  ctx->d_khat = ctx->d_kin + N;
  ctx->d_khat_inv = ctx->d_kin + 2 * N;
  ctx->d_kvec = ctx->d_kin + 3 * N;
  ctx->d_twx = ctx->d_tw;
  ctx->d_twy = ctx->d_tw + ctx->nx;
  cudaStream_t s = ctx->stream;
#define INIT_CUDA(call)                                                                                   \
  do {                                                                                                    \
    cudaError_t e_ = (call);                                                                              \
    if (e_ != cudaSuccess) return fail(set_error(ctx, ACP_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_))); \
  } while (0)
  INIT_CUDA(cudaMemcpyAsync(ctx->d_V, v_eff_d, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  INIT_CUDA(cudaMemcpyAsync(ctx->d_psi, psi_d, (size_t)N * n_orb * sizeof(double), cudaMemcpyDeviceToDevice, s));
  INIT_CUDA(cudaMemcpyAsync(ctx->d_eps, eps_h, n_orb * sizeof(double), cudaMemcpyHostToDevice, s));
  INIT_CUDA(cudaMemcpyAsync(ctx->d_kin, kin.data(), N * sizeof(double), cudaMemcpyHostToDevice, s));
  INIT_CUDA(cudaMemcpyAsync(ctx->d_khat, khat.data(), N * sizeof(double), cudaMemcpyHostToDevice, s));
  INIT_CUDA(cudaMemcpyAsync(ctx->d_khat_inv, kinv.data(), N * sizeof(double), cudaMemcpyHostToDevice, s));
  INIT_CUDA(cudaMemcpyAsync(ctx->d_kvec, kodd.data(), N * sizeof(double), cudaMemcpyHostToDevice, s));
  INIT_CUDA(cudaMemcpyAsync(ctx->d_tw, tw.data(), N * sizeof(double2), cudaMemcpyHostToDevice, s));
  INIT_CUDA(cudaMemsetAsync(ctx->d_flag, 0, 64 * sizeof(int), s));
  INIT_CUDA(cudaStreamSynchronize(s));
#undef INIT_CUDA
  st = spectral_configure(ctx);
  if (st != ACP_OK) return fail(st);
  {
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device) == cudaSuccess)
      ctx->smem_optin = (size_t)optin;
    cudaGetLastError();
  }
  *out = ctx;
  return ACP_OK;
}

acp_status acp_set_options(acp_ctx* ctx, const acp_options* opt) {
  ACP_TRY(check_ctx(ctx));
  if (!opt) return set_error(ctx, ACP_E_ARG, "null options");
  ACP_TRY(validate_options(ctx, opt));
  ctx->opt = *opt;
  return ACP_OK;
}

void acp_destroy(acp_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  cudaFree(ctx->d_V);
  cudaFree(ctx->d_psi);
  cudaFree(ctx->d_eps);
  cudaFree(ctx->d_kin);
  cudaFree(ctx->d_tw);
  cudaFree(ctx->d_flag);
  delete ctx;
}

acp_status acp_apply_chi0(acp_ctx* ctx, const double* G_d, int ncol, double* out_d, acp_stats* stats) {
  ACP_TRY(check_ctx(ctx));
  if (ncol == 0) return ACP_OK;
  if (!G_d || !out_d || ncol < 0) return set_error(ctx, ACP_E_ARG, "null pointer or negative ncol");
  const double t0 = now_ms();
  SolveReport rep;
  acp_status st;
  if (ctx->opt.method == ACP_METHOD_ACP) st = chi0_acp(ctx, G_d, ncol, out_d, stats, &rep, t0);
  else st = chi0_plain(ctx, G_d, ncol, out_d, &rep, t0);
  if (st == ACP_OK) ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  fill_stats(stats, rep, t0);
  if (st == ACP_OK && !rep.all_converged)
    return set_error(ctx, ACP_E_NOCONV, "some Sternheimer solves hit the iteration cap (max rel. res %.3e)",
                     rep.max_rel_res);
  return st;
}

acp_status acp_dyson_solve(acp_ctx* ctx, const double* G_d, int ncol, double* U_d, acp_stats* stats) {
  ACP_TRY(check_ctx(ctx));
  if (ncol == 0) return ACP_OK;
  if (!G_d || !U_d || ncol < 0) return set_error(ctx, ACP_E_ARG, "null pointer or negative ncol");
  const double t0 = now_ms();
  SolveReport rep;
  acp_status st = dyson(ctx, G_d, ncol, U_d, stats, &rep, t0);
  if (st == ACP_OK) ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  fill_stats(stats, rep, t0);
  if (st == ACP_OK && !rep.all_converged)
    return set_error(ctx, ACP_E_NOCONV, "some Sternheimer solves hit the iteration cap (max rel. res %.3e)",
                     rep.max_rel_res);
  return st;
}

acp_status acp_perturbations(acp_ctx* ctx, const acp_atoms* atoms, double* G_d, double* B_d, double* d2V_d) {
  ACP_TRY(check_ctx(ctx));
  if (!atoms || atoms->n_atoms < 0 || (atoms->n_atoms > 0 && (!atoms->R || !atoms->Z || !atoms->sigma)))
    return set_error(ctx, ACP_E_ARG, "bad atoms");
  const int nA = atoms->n_atoms;
  if (nA == 0) return ACP_OK;
  const int d = ctx->dim;
  double* hv = nullptr;
  ACP_TRY(ws(ctx, "pt_atoms", (size_t)(d + 2) * nA, &hv));
  std::vector<double> host((size_t)(d + 2) * nA);
  for (int I = 0; I < nA; ++I) {
    for (int a = 0; a < d; ++a) host[(size_t)d * I + a] = atoms->R[(size_t)d * I + a];
    host[(size_t)d * nA + I] = atoms->Z[I];
    host[(size_t)(d + 1) * nA + I] = atoms->sigma[I];
  }
  ACP_CUDA(ctx, cudaMemcpyAsync(hv, host.data(), sizeof(double) * (d + 2) * nA, cudaMemcpyHostToDevice, ctx->stream));
  if (d == 2) ACP_TRY(perturbations_2d(ctx, nA, hv, hv + 2 * nA, hv + 3 * nA, G_d, B_d, d2V_d));
  else ACP_TRY(perturbations_1d(ctx, nA, hv, hv + nA, hv + 2 * nA, G_d, B_d, d2V_d));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ACP_OK;
}

acp_status acp_dynamical_matrix(acp_ctx* ctx, const acp_atoms* atoms, const double* rho_d, double* D_h,
                                double* U_d, acp_stats* stats) {
  ACP_TRY(check_ctx(ctx));
  if (!atoms || atoms->n_atoms < 1 || !atoms->R || !atoms->Z || !atoms->sigma || !rho_d || !D_h)
    return set_error(ctx, ACP_E_ARG, "bad atoms, density or output");
  const double t0 = now_ms();
  SolveReport rep;
  acp_status st = dynamical(ctx, atoms, rho_d, D_h, U_d, stats, &rep, t0);
  fill_stats(stats, rep, t0);
  if (st == ACP_OK && !rep.all_converged)
    return set_error(ctx, ACP_E_NOCONV, "some Sternheimer solves hit the iteration cap (max rel. res %.3e)",
                     rep.max_rel_res);
  return st;
}

acp_status acp_batch_dynamical_matrix(acp_ctx* const* ctxs, int n_sys, const acp_atoms* atoms,
                                      const double* const* rho_d, double* const* D_h, acp_stats* stats,
                                      acp_status* status_out, int n_workers) {
  if (!ctxs || n_sys < 0 || !atoms || !rho_d || !D_h) return ACP_E_ARG;
  for (int i = 0; i < n_sys; ++i)
    if (!ctxs[i]) return ACP_E_ARG;
  if (n_sys == 0) return ACP_OK;
  int workers = n_workers > 0 ? n_workers : (int)std::thread::hardware_concurrency();
  if (workers < 1) workers = 1;
  if (workers > n_sys) workers = n_sys;
  if (workers > 64) workers = 64;
  std::vector<acp_status> st(n_sys, ACP_OK);
  std::atomic<int> next{0};
  // work queue over systems, largest first (the callers' order is kept in the outputs)
  std::vector<int> order(n_sys);
  for (int i = 0; i < n_sys; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ctxs[a]->N > ctxs[b]->N; });
  // Each worker carries one set of workspace buffers from system to system (moved into the
  // context before its run and back out after), so the batch holds memory for the systems in
  // flight only and allocates (cudaMalloc / cudaFree synchronise the device) only when a larger
  // system needs more; what the workers hold at the end is freed.
  std::vector<std::map<std::string, std::pair<void*, size_t>>> held(workers);
  // Each worker runs its systems on a stream of its own.  The callers' streams may coincide (a
  // pool of library streams can hand the same one to several contexts), and a worker that captures
  // its Lanczos steps as a CUDA graph must not see another worker's launches on the same stream.
  std::vector<cudaStream_t> wstream(workers, nullptr);
  for (int w = 0; w < workers; ++w)
    if (cudaStreamCreateWithFlags(&wstream[w], cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      for (int v = 0; v < w; ++v) cudaStreamDestroy(wstream[v]);
      return ACP_E_CUDA;
    }
  // Admission by device memory: a system enters only while the workspace estimates of the systems
  // in flight fit in 85% of the memory free at the start (one system always runs).  Estimate, per
  // grid point and (shift, point) pair of the N_c x N_mu Sternheimer equations (N_mu ~ 7 n_orb):
  // four FP64 blocks (solutions, replicated right-hand sides, residuals, operator products) and ten
  // FP32 ones (refinement residual and correction, the MINRES vectors and their compacted copy),
  // 72 bytes with 1/8 allocation headroom, plus the stored FP32 Lanczos basis (512 steps, at most
  // 16 GB).  A system that still runs out of memory is run again alone after the others.
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const double budget = 0.85 * (double)free_b;
  std::vector<double> need(n_sys);
  for (int i = 0; i < n_sys; ++i) {
    const acp_ctx* c = ctxs[i];
    const double nmu = 7.0 * c->n_orb, nc = c->opt.n_cheb > 0 ? c->opt.n_cheb : 16;
    need[i] = 81.0 * c->N * nc * nmu + std::min(16.0e9, 512.0 * 4.0 * c->N * nmu);
  }
  std::mutex adm_mu;
  std::condition_variable adm_cv;
  double in_flight = 0.0;
  int running = 0;
  auto release_held = [&](int w) {
    std::lock_guard<std::mutex> lock(device_mutex());
    for (auto& kv : held[w])
      if (kv.second.first) cudaFree(kv.second.first);
    held[w].clear();
  };
  auto worker = [&](int w) {
    for (;;) {
      const int q = next.fetch_add(1);
      if (q >= n_sys) return;
      const int i = order[q];
      acp_ctx* c = ctxs[i];
      {
        // buffers kept from a larger system would exceed this system's estimate: give them back
        double held_b = 0.0;
        for (const auto& kv : held[w]) held_b += (double)kv.second.second;
        if (held_b > 1.25 * need[i]) release_held(w);
        std::unique_lock<std::mutex> lk(adm_mu);
        if (!(running == 0 || in_flight + need[i] <= budget)) {
          lk.unlock();
          release_held(w);  // waiting: give the memory back to the systems in flight
          lk.lock();
          adm_cv.wait(lk, [&] { return running == 0 || in_flight + need[i] <= budget; });
        }
        in_flight += need[i];
        ++running;
      }
      cudaSetDevice(c->device);
      cudaStreamSynchronize(c->stream);  // the caller's inputs are ready
      cudaStream_t caller_stream = c->stream;
      c->stream = wstream[w];
      for (auto& kv : c->ws.bufs) {  // the context's own buffers join the worker's set
        auto it = held[w].find(kv.first);
        if (it == held[w].end() || it->second.second < kv.second.second) {
          if (it != held[w].end()) {
            std::lock_guard<std::mutex> lock(device_mutex());
            cudaFree(it->second.first);
          }
          held[w][kv.first] = kv.second;
        } else {
          std::lock_guard<std::mutex> lock(device_mutex());
          cudaFree(kv.second.first);
        }
      }
      c->ws.bufs = std::move(held[w]);
      held[w].clear();
      c->psi32_stale = true;  // the buffers hold another system's data
      c->tables32_stale = true;
      st[i] = acp_dynamical_matrix(c, &atoms[i], rho_d[i], D_h[i], nullptr, stats ? &stats[i] : nullptr);
      cudaStreamSynchronize(c->stream);
      c->stream = caller_stream;
      held[w] = std::move(c->ws.bufs);
      c->ws.bufs.clear();
      c->psi32_stale = true;
      c->tables32_stale = true;
      {
        std::lock_guard<std::mutex> lk(adm_mu);
        in_flight -= need[i];
        --running;
      }
      adm_cv.notify_all();
    }
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < workers; ++w) pool.emplace_back(worker, w);
  worker(0);
  for (auto& t : pool) t.join();
  for (int w = 0; w < workers; ++w) release_held(w);
  auto destroy_streams = [&]() {
    for (cudaStream_t x : wstream)
      if (x) cudaStreamDestroy(x);
  };
  // systems that ran out of memory beside others run again, one at a time, largest first
  {
    std::vector<int> retry;
    for (int q = 0; q < n_sys; ++q)
      if (st[order[q]] == ACP_E_OOM) retry.push_back(order[q]);
    if (!retry.empty()) {
      next.store(0);
      std::vector<int> saved = order;
      order = retry;
      const int saved_n = n_sys;
      n_sys = (int)retry.size();
      worker(0);
      release_held(0);
      order = saved;
      n_sys = saved_n;
    }
  }
  destroy_streams();
  acp_status worst = ACP_OK;
  for (int i = 0; i < n_sys; ++i) {
    if (status_out) status_out[i] = st[i];
    if (worst == ACP_OK && st[i] != ACP_OK) worst = st[i];
  }
  return worst;
}

acp_status acp_phonons(acp_ctx* ctx, const double* D_h, int n, double* omega_h, double* modes_h) {
  ACP_TRY(check_ctx(ctx));
  if (!D_h || !omega_h || n < 1 || n > 1024) return set_error(ctx, ACP_E_ARG, "bad matrix or size");
  double* buf = nullptr;
  ACP_TRY(ws(ctx, "ph_buf", 2 * (size_t)n * n + n, &buf));
  double* A = buf;
  double* V = buf + (size_t)n * n;
  double* w = V + (size_t)n * n;
  // the row-major symmetric input is its own column-major transpose
  ACP_CUDA(ctx, cudaMemcpyAsync(A, D_h, sizeof(double) * n * n, cudaMemcpyHostToDevice, ctx->stream));
  ACP_TRY(jacobi_eig(ctx, A, n, w, V));
  std::vector<double> lam(n);
  ACP_CUDA(ctx, cudaMemcpyAsync(lam.data(), w, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
  if (modes_h)
    ACP_CUDA(ctx, cudaMemcpyAsync(modes_h, V, sizeof(double) * n * n, cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < n; ++i) omega_h[i] = (lam[i] < 0 ? -1.0 : 1.0) * std::sqrt(std::fabs(lam[i]));
  return ACP_OK;
}

acp_status acp_hamiltonian_apply(acp_ctx* ctx, const double* X_d, int ncol, const double* shift_h, double* Y_d) {
  ACP_TRY(check_ctx(ctx));
  if (ncol == 0) return ACP_OK;
  if (!X_d || !Y_d || ncol < 0) return set_error(ctx, ACP_E_ARG, "bad arguments");
  double* sh = nullptr;
  if (shift_h) {
    ACP_TRY(ws(ctx, "ha_shift", ncol, &sh));
    ACP_CUDA(ctx, cudaMemcpyAsync(sh, shift_h, sizeof(double) * ncol, cudaMemcpyHostToDevice, ctx->stream));
  }
  ACP_TRY(spectral_apply(ctx, X_d, ctx->N, ncol, MULT_KINETIC, true, sh, Y_d, ctx->N, nullptr, nullptr));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ACP_OK;
}

acp_status acp_project(acp_ctx* ctx, const double* X_d, int ncol, double* Y_d) {
  ACP_TRY(check_ctx(ctx));
  if (!X_d || !Y_d || ncol < 0) return set_error(ctx, ACP_E_ARG, "bad arguments");
  ACP_TRY(project(ctx, X_d, ctx->N, ncol, Y_d, ctx->N));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ACP_OK;
}

acp_status acp_project_mixed(acp_ctx* ctx, const double* X_d, int ncol, double* Y_d) {
  ACP_TRY(check_ctx(ctx));
  if (!X_d || !Y_d || ncol < 0) return set_error(ctx, ACP_E_ARG, "bad arguments");
  ACP_TRY(project_mixed64(ctx, X_d, ncol, Y_d));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ACP_OK;
}

acp_status acp_selftest_wait_timeout(acp_ctx* ctx, double wait_s) {
  ACP_TRY(check_ctx(ctx));
  if (!(wait_s > 0.0) || wait_s > 1.0) return set_error(ctx, ACP_E_ARG, "wait_s must lie in (0, 1]");
  return tc_selftest_timeout(ctx, (uint64_t)(wait_s * 1e9));
}

acp_status acp_kernel_apply(acp_ctx* ctx, const double* X_d, int ncol, int kernel_op, double* Y_d) {
  ACP_TRY(check_ctx(ctx));
  if (!X_d || !Y_d || ncol < 0 || (kernel_op != 1 && kernel_op != -1))
    return set_error(ctx, ACP_E_ARG, "bad arguments");
  ACP_TRY(spectral_apply(ctx, X_d, ctx->N, ncol, kernel_op == 1 ? MULT_KHAT : MULT_KHAT_INV, false, nullptr, Y_d,
                         ctx->N, nullptr, nullptr));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ACP_OK;
}

acp_status acp_sternheimer_solve(acp_ctx* ctx, const double* B_d, int ncol, const double* shift_h, double* X_d,
                                 acp_stats* stats) {
  ACP_TRY(check_ctx(ctx));
  if (ncol == 0) return ACP_OK;
  if (!B_d || !X_d || !shift_h || ncol < 0) return set_error(ctx, ACP_E_ARG, "bad arguments");
  const double t0 = now_ms();
  double *R = nullptr, *sh = nullptr;
  ACP_TRY(ws(ctx, "ss_rhs", (size_t)ctx->N * ncol, &R));
  ACP_TRY(ws(ctx, "ss_shift", ncol, &sh));
  ACP_CUDA(ctx, cudaMemcpyAsync(sh, shift_h, sizeof(double) * ncol, cudaMemcpyHostToDevice, ctx->stream));
  ACP_TRY(project(ctx, B_d, ctx->N, ncol, R, ctx->N));
  SolveReport rep;
  ACP_TRY(minres_batched(ctx, R, ncol, sh, X_d, &rep, t0));
  ACP_TRY(project(ctx, X_d, ctx->N, ncol, X_d, ctx->N));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  fill_stats(stats, rep, t0);
  if (!rep.all_converged) return set_error(ctx, ACP_E_NOCONV, "MINRES hit the iteration cap");
  return ACP_OK;
}

acp_status acp_cnn_set_weights(acp_ctx* ctx, const float* w_h, long long n) {
  ACP_TRY(check_ctx(ctx));
  if (!w_h || n != ACP_CNN_WEIGHTS)
    return set_error(ctx, ACP_E_ARG, "expected %d weights, got %lld", (int)ACP_CNN_WEIGHTS, n);
  if (ctx->dim != 2) return set_error(ctx, ACP_E_ARG, "the learned initial guess is defined on 2D grids");
  return cnn_set_weights(ctx, w_h);
}

acp_status acp_cnn_apply(acp_ctx* ctx, const double* R_d, int ncol, const double* shift_h, double* X0_d) {
  ACP_TRY(check_ctx(ctx));
  if (ncol == 0) return ACP_OK;
  if (!R_d || !X0_d || !shift_h || ncol < 0) return set_error(ctx, ACP_E_ARG, "bad arguments");
  double* sh = nullptr;
  ACP_TRY(ws(ctx, "cnn_shift", ncol, &sh));
  ACP_CUDA(ctx, cudaMemcpyAsync(sh, shift_h, sizeof(double) * ncol, cudaMemcpyHostToDevice, ctx->stream));
  ACP_TRY(cnn_initial_guess(ctx, R_d, ctx->N, ncol, sh, X0_d, ctx->N));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // shift_h may go away
  return ACP_OK;
}

acp_status acp_cnn_train_step(acp_ctx* ctx, int nx, int ny, const double* R_d, const double* VS_d,
                              const double* Xstar_d, int nsamp, float lr, double* loss_h, float* grad_h) {
  ACP_TRY(check_ctx(ctx));
  if (!R_d || !VS_d || !Xstar_d || nsamp < 1 || !(lr >= 0.f)) return set_error(ctx, ACP_E_ARG, "bad arguments");
  return cnn_train_step(ctx, nx, ny, R_d, VS_d, Xstar_d, nsamp, lr, loss_h, grad_h);
}

acp_status acp_cnn_get_weights(acp_ctx* ctx, float* w_h) {
  ACP_TRY(check_ctx(ctx));
  if (!w_h) return set_error(ctx, ACP_E_ARG, "null pointer");
  if (!ctx->cnn_ready) return set_error(ctx, ACP_E_ARG, "no network weights (acp_cnn_set_weights)");
  float* w = nullptr;
  ACP_TRY(ws(ctx, "cnn_w32", (size_t)ACP_CNN_WEIGHTS, &w));
  ACP_CUDA(ctx, cudaMemcpyAsync(w_h, w, sizeof(float) * ACP_CNN_WEIGHTS, cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ACP_OK;
}

acp_status acp_compress(acp_ctx* ctx, const double* G_d, int ncol, int cap, int* n_mu, int* pivots_h, double* Xi_d,
                        double* Rdiag_h) {
  ACP_TRY(check_ctx(ctx));
  if (!G_d || ncol < 1 || !n_mu || !pivots_h || cap < 1) return set_error(ctx, ACP_E_ARG, "bad arguments");
  Compression comp;
  ACP_TRY(compress(ctx, G_d, ncol, ctx->opt.sketch, ctx->opt.sketch_cols, ctx->opt.id_tol, ctx->opt.max_rank, &comp));
  *n_mu = comp.n_mu;
  const int k = comp.n_mu < cap ? comp.n_mu : cap;
  for (int i = 0; i < k; ++i) pivots_h[i] = comp.piv[i];
  if (Rdiag_h)
    for (int i = 0; i < k; ++i) Rdiag_h[i] = comp.rdiag[i];
  if (Xi_d)
    ACP_CUDA(ctx, cudaMemcpyAsync(Xi_d, comp.d_xi, sizeof(double) * ctx->N * k, cudaMemcpyDeviceToDevice, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (comp.n_mu > cap) return set_error(ctx, ACP_E_ARG, "N_mu = %d exceeds the capacity %d", comp.n_mu, cap);
  return ACP_OK;
}

acp_status acp_update(acp_ctx* ctx, const double* v_eff_d, const double* psi_d, const double* eps_h, int n_orb) {
  ACP_TRY(check_ctx(ctx));
  if (!v_eff_d || !psi_d || !eps_h || n_orb != ctx->n_orb)
    return set_error(ctx, ACP_E_ARG, "acp_update needs V, Psi and %d eigenvalues", ctx->n_orb);
  for (int i = 0; i < n_orb; ++i) {
    if (!std::isfinite(eps_h[i])) return set_error(ctx, ACP_E_NUMERIC, "eigenvalue %d is not finite", i);
    if (i && eps_h[i] < eps_h[i - 1]) return set_error(ctx, ACP_E_GAP, "eigenvalues must be ascending");
  }
  ctx->eps.assign(eps_h, eps_h + n_orb);
  const int N = ctx->N;
  ACP_CUDA(ctx, cudaMemcpyAsync(ctx->d_V, v_eff_d, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  ACP_CUDA(ctx, cudaMemcpyAsync(ctx->d_psi, psi_d, (size_t)N * n_orb * sizeof(double), cudaMemcpyDeviceToDevice,
                                ctx->stream));
  ACP_CUDA(ctx, cudaMemcpyAsync(ctx->d_eps, eps_h, n_orb * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->psi32_stale = true;
  ctx->tables32_stale = true;
  return ACP_OK;
}

acp_status acp_profile_enable(acp_ctx* ctx, int enable) {
  ACP_TRY(check_ctx(ctx));
  ctx->prof.acc.clear();
  ctx->prof.on = enable != 0;
  return ACP_OK;
}

acp_status acp_profile_get(acp_ctx* ctx, const char* kernel, double* total_ms, long long* launches, double* flops,
                           double* bytes) {
  ACP_TRY(check_ctx(ctx));
  if (!kernel) return set_error(ctx, ACP_E_ARG, "null kernel name");
  auto it = ctx->prof.acc.find(kernel);
  const Profiler::Acc a = (it == ctx->prof.acc.end()) ? Profiler::Acc{} : it->second;
  if (total_ms) *total_ms = a.ms;
  if (launches) *launches = a.n;
  if (flops) *flops = a.flops;
  if (bytes) *bytes = a.bytes;
  return ACP_OK;
}

long long acp_launch_count(const acp_ctx* ctx) { return ctx ? ctx->prof.launches : -1; }

}  // extern "C"
