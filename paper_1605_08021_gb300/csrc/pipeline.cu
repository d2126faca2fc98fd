// The polarizability pipelines:
//   chi0_plain  Alg. 1: one projected Sternheimer solve per (occupied orbital, column) pair,
//               u_j = 2f sum_i psi_i * zeta_ij with Q(eps_i - H)Q zeta_ij = Q(psi_i * g_j).
//   acp_build   Alg. 3: compression of psi_i * g_j (Alg. 2, Remark form), the compressed
//               equations Q(eps_c - H)Q zeta_{c mu} = Q xi_mu at the Chebyshev nodes
//               (Eq. eqncompressU), and W_mu = 2f sum_i psi_i (sum_c zeta_{c mu} L_c(eps_i)) psi_i(r_mu)
//               (Eq. eqnW), so that chi0~ = W Pi^T (Eq. chi0gcompress2).
//   dyson_acp   Alg. 4 with the Sherman-Morrison-Woodbury update of Eq. dyson4.
//   dyson_gmres the exact Dyson equation (I - chi0 K) U = chi0 G by GMRES (Eq. dyson).
//   dynamical   Eq. SecDeriv with U = chi G.
#include "internal.cuh"

namespace acp {

acp_status transpose(acp_ctx* ctx, int rows, int cols, const double* A, double* At);

namespace {

int grid_for(size_t total, int cap = 65535) {
  size_t b = (total + 255) / 256;
  if (b > (size_t)cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// RHS[:, i + jl*no] = psi_i .* G[:, c0 + jl]; shift[p] = eps_i; ref[p] = ||psi_i .* g_j||
__global__ void build_pair_rhs(int N, int no, int ncols, const double* __restrict__ psi, const double* __restrict__ G,
                               const double* __restrict__ eps, double* __restrict__ R, double* __restrict__ shift) {
  const size_t total = (size_t)N * no * ncols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % N);
    const size_t p = e / N;
    const int i = (int)(p % no), jl = (int)(p / no);
    R[e] = psi[a + (size_t)i * N] * G[a + (size_t)jl * N];
    if (a == 0) shift[p] = eps[i];
  }
}

__global__ void col_norms_kernel(int N, int ncol, const double* __restrict__ X, double* __restrict__ out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= ncol) return;
  const double* x = X + (size_t)warp * N;
  double s = 0.0;
  for (int r = lane; r < N; r += 32) s += x[r] * x[r];
  s = warp_sum(s);
  if (lane == 0) out[warp] = sqrt(s);
}

// Zero the columns that Q annihilated (their norm fell below 1e-13 of the unprojected norm):
// they lie in the occupied space and their rounding residue must not be solved for.
__global__ void zero_annihilated(int N, int ncol, double* __restrict__ X, const double* __restrict__ before,
                                 const double* __restrict__ after) {
  const int c = blockIdx.x;
  if (c >= ncol || !(after[c] <= 1e-13 * before[c])) return;
  for (int a = threadIdx.x; a < N; a += blockDim.x) X[a + (size_t)c * N] = 0.0;
}

// out[:, jl] = -2f sum_i psi_i .* X[:, i + jl*no]   (zeta = -x)
__global__ void accumulate_pairs(int N, int no, int ncols, double f2, const double* __restrict__ psi,
                                 const double* __restrict__ X, double* __restrict__ out) {
  const size_t total = (size_t)N * ncols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % N), jl = (int)(e / N);
    double s = 0.0;
    for (int i = 0; i < no; ++i) s += psi[a + (size_t)i * N] * X[a + ((size_t)i + (size_t)jl * no) * N];
    out[a + (size_t)jl * N] = -f2 * s;
  }
}

// Chebyshev nodes on [eps_1, eps_Ne] (Sec. 3.1) and Lagrange weights L_c(eps_i) (Eq. LagPoly).
__global__ void cheb_lagrange_kernel(int nc, int no, const double* __restrict__ eps, double* __restrict__ nodes,
                                     double* __restrict__ Lw) {
  __shared__ double x[64];
  const double e1 = eps[0], eN = eps[no - 1];
  if (threadIdx.x < nc) {
    x[threadIdx.x] = (nc == 1) ? 0.5 * (e1 + eN)
                               : 0.5 * (e1 + eN) + 0.5 * (e1 - eN) * cospi((threadIdx.x + 0.5) / nc);
    nodes[threadIdx.x] = x[threadIdx.x];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nc * no; e += blockDim.x) {
    const int c = e % nc, i = e / nc;
    double l = 1.0;
    for (int cp = 0; cp < nc; ++cp)
      if (cp != c) l *= (eps[i] - x[cp]) / (x[c] - x[cp]);
    Lw[c + (size_t)nc * i] = l;
  }
}

// Bc[i, mu] = L_c(eps_i) psi_i(r_mu)
__global__ void build_bc(int no, int k, int nc, int c, const double* __restrict__ Lw, const double* __restrict__ psiT,
                         const int* __restrict__ piv, double* __restrict__ Bc) {
  const size_t total = (size_t)no * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % no), mu = (int)(e / no);
    Bc[e] = Lw[c + (size_t)nc * i] * psiT[i + (size_t)piv[mu] * no];
  }
}

__global__ void identity_minus(int n, double* S) {
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % n), c = (int)(e / n);
    S[e] = (r == c ? 1.0 : 0.0) - S[e];
  }
}

__global__ void axpby_kernel(size_t n, double a, const double* __restrict__ X, double b, const double* __restrict__ Y,
                             double* __restrict__ Z) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    Z[e] = a * X[e] + b * Y[e];
}

// ---- GMRES (modified Gram-Schmidt Arnoldi, Givens least squares), one CTA per column ---------
struct GmresState {
  double* Vb;     // (m+1) blocks of N x ncol
  double* H;      // ncol x (m+1) x m, column-major per column
  double* cs;     // ncol x m
  double* sn;
  double* g;      // ncol x (m+1)
  double* beta0;  // ncol
  int m;
};

__global__ void gmres_start(int N, int ncol, const double* __restrict__ Bm, GmresState s) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  const double* b = Bm + (size_t)j * N;
  double acc = 0.0;
  for (int a = threadIdx.x; a < N; a += blockDim.x) acc += b[a] * b[a];
  const double nrm = sqrt(block_sum(acc, red));
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  double* v = s.Vb + (size_t)j * N;
  for (int a = threadIdx.x; a < N; a += blockDim.x) v[a] = b[a] * inv;
  if (threadIdx.x == 0) {
    s.beta0[j] = nrm;
    s.g[(size_t)j * (s.m + 1)] = nrm;
  }
}

// w (block k+1 of Vb, holds A v_k on entry) is orthogonalised against v_0..v_k, normalised,
// and the new Hessenberg column is reduced by the Givens rotations.  res[j] = |g_{k+1}| / beta0.
__global__ void gmres_arnoldi(int N, int ncol, int k, GmresState s, double* res) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  const size_t blk = (size_t)N * ncol;
  double* w = s.Vb + (size_t)(k + 1) * blk + (size_t)j * N;
  double* Hc = s.H + (size_t)j * (s.m + 1) * s.m + (size_t)k * (s.m + 1);
  for (int pass = 0; pass < 2; ++pass) {  // MGS with one re-orthogonalisation pass
    for (int i = 0; i <= k; ++i) {
      const double* v = s.Vb + (size_t)i * blk + (size_t)j * N;
      double acc = 0.0;
      for (int a = threadIdx.x; a < N; a += blockDim.x) acc += v[a] * w[a];
      const double hij = block_sum(acc, red);
      for (int a = threadIdx.x; a < N; a += blockDim.x) w[a] -= hij * v[a];
      if (threadIdx.x == 0) Hc[i] = (pass == 0 ? hij : Hc[i] + hij);
      __syncthreads();
    }
  }
  double acc = 0.0;
  for (int a = threadIdx.x; a < N; a += blockDim.x) acc += w[a] * w[a];
  const double hn = sqrt(block_sum(acc, red));
  const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
  for (int a = threadIdx.x; a < N; a += blockDim.x) w[a] *= inv;
  if (threadIdx.x == 0) {
    Hc[k + 1] = hn;
    double* cs = s.cs + (size_t)j * s.m;
    double* sn = s.sn + (size_t)j * s.m;
    double* g = s.g + (size_t)j * (s.m + 1);
    for (int i = 0; i < k; ++i) {
      const double t = cs[i] * Hc[i] + sn[i] * Hc[i + 1];
      Hc[i + 1] = -sn[i] * Hc[i] + cs[i] * Hc[i + 1];
      Hc[i] = t;
    }
    double r = hypot(Hc[k], Hc[k + 1]);
    if (r == 0.0) r = 1.0;
    cs[k] = Hc[k] / r;
    sn[k] = Hc[k + 1] / r;
    Hc[k] = r;
    Hc[k + 1] = 0.0;
    g[k + 1] = -sn[k] * g[k];
    g[k] = cs[k] * g[k];
    res[j] = s.beta0[j] > 0.0 ? fabs(g[k + 1]) / s.beta0[j] : 0.0;
  }
}

// y = H^{-1} g (k x k upper triangular, per column), then U[:, j] = sum_i y_i v_i.
__global__ void gmres_finish(int N, int ncol, int k, GmresState s, double* __restrict__ U) {
  __shared__ double y[128];
  const int j = blockIdx.x;
  if (threadIdx.x == 0) {
    const double* Hj = s.H + (size_t)j * (s.m + 1) * s.m;
    const double* g = s.g + (size_t)j * (s.m + 1);
    for (int i = k - 1; i >= 0; --i) {
      double v = g[i];
      for (int c = i + 1; c < k; ++c) v -= Hj[i + (size_t)c * (s.m + 1)] * y[c];
      const double d = Hj[i + (size_t)i * (s.m + 1)];
      y[i] = (d != 0.0 && s.beta0[j] > 0.0) ? v / d : 0.0;
    }
  }
  __syncthreads();
  const size_t blk = (size_t)N * ncol;
  for (int a = threadIdx.x; a < N; a += blockDim.x) {
    double u = 0.0;
    for (int i = 0; i < k; ++i) u += y[i] * s.Vb[(size_t)i * blk + (size_t)j * N + a];
    U[(size_t)j * N + a] = u;
  }
}

__global__ void max_kernel(const double* __restrict__ x, int n, double* out) {
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, x[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, sm[w]);
    *out = r;
  }
}

// ---- dynamical matrix ------------------------------------------------------------------------
// D[I, J] (row-major out) = (Hm[I, J] + delta_IJ dv[I] + Eii[I, J]) / sqrt(M_I M_J), where
// Eii is the Hessian of E_II = 1/2 sum_{I != J} Z_I Z_J K(R_I - R_J) over periodic images:
// sum_n exp(-kappa |x + nL|) = cosh(kappa (x - L/2)) / sinh(kappa L / 2), K'' = kappa^2 K.
__global__ void assemble_dmat(int nA, const double* __restrict__ Hm, const double* __restrict__ dv,
                              const double* __restrict__ R, const double* __restrict__ Z,
                              const double* __restrict__ M, double L, double kappa, double scale,
                              double* __restrict__ D) {
  const double pref = 2.0 * M_PI * scale / kappa / sinh(0.5 * kappa * L) * kappa * kappa;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nA * nA; e += gridDim.x * blockDim.x) {
    const int I = e / nA, J = e % nA;
    double eii = 0.0;
    if (I != J) {
      double x = fmod(R[I] - R[J], L);
      if (x < 0) x += L;
      eii = -Z[I] * Z[J] * pref * cosh(kappa * (x - 0.5 * L));
    } else {
      for (int K = 0; K < nA; ++K) {
        if (K == I) continue;
        double x = fmod(R[I] - R[K], L);
        if (x < 0) x += L;
        eii += Z[I] * Z[K] * pref * cosh(kappa * (x - 0.5 * L));
      }
    }
    const double h = Hm[I + (size_t)J * nA] + (I == J ? dv[I] : 0.0) + eii;
    D[(size_t)I * nA + J] = h / sqrt(M[I] * M[J]);
  }
}

__global__ void symmetrize_kernel(int n, const double* __restrict__ D, double* __restrict__ Ds, double* out) {
  double d = 0.0, a = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int r = e / n, c = e % n;
    const double x = D[(size_t)r * n + c], y = D[(size_t)c * n + r];
    Ds[(size_t)r * n + c] = 0.5 * (x + y);
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

}  // namespace

// ---- Alg. 1 ---------------------------------------------------------------------------------
acp_status chi0_plain(acp_ctx* ctx, const double* G, int ncol, double* out, SolveReport* rep, double t0) {
  const int N = ctx->N, no = ctx->n_orb;
  int batch = ctx->opt.rhs_batch > 0 ? ctx->opt.rhs_batch : 16384;
  int cols_per = batch / no;
  if (cols_per < 1) cols_per = 1;
  if (cols_per > ncol) cols_per = ncol;
  const size_t maxr = (size_t)cols_per * no;
  double *R = nullptr, *X = nullptr, *sh = nullptr, *nb = nullptr;
  ACP_TRY(ws(ctx, "p_rhs", (size_t)N * maxr, &R));
  ACP_TRY(ws(ctx, "p_x", (size_t)N * maxr, &X));
  ACP_TRY(ws(ctx, "p_shift", maxr, &sh));
  ACP_TRY(ws(ctx, "p_norms", 2 * maxr, &nb));
  for (int c0 = 0; c0 < ncol; c0 += cols_per) {
    const int nc = (ncol - c0 < cols_per) ? ncol - c0 : cols_per;
    const int nr = nc * no;
    ::acp::note_launch(ctx);
    build_pair_rhs<<<grid_for((size_t)N * nr), 256, 0, ctx->stream>>>(N, no, nc, ctx->d_psi, G + (size_t)c0 * N,
                                                                         ctx->d_eps, R, sh);
    ACP_LAUNCH(ctx);
    ::acp::note_launch(ctx);
    col_norms_kernel<<<(nr * 32 + 255) / 256, 256, 0, ctx->stream>>>(N, nr, R, nb);
    ACP_LAUNCH(ctx);
    ACP_TRY(project(ctx, R, N, nr, R, N));
    ::acp::note_launch(ctx);
    col_norms_kernel<<<(nr * 32 + 255) / 256, 256, 0, ctx->stream>>>(N, nr, R, nb + maxr);
    ::acp::note_launch(ctx);
    zero_annihilated<<<nr, 256, 0, ctx->stream>>>(N, nr, R, nb, nb + maxr);
    ACP_LAUNCH(ctx);
    ACP_TRY(minres_batched(ctx, R, nr, sh, X, rep, t0));
    ACP_TRY(project(ctx, X, N, nr, X, N));  // outer Q of Eq. Sternheimer
    ::acp::note_launch(ctx);
    accumulate_pairs<<<grid_for((size_t)N * nc), 256, 0, ctx->stream>>>(N, no, nc, 2.0 * ctx->opt.occ, ctx->d_psi,
                                                                         X, out + (size_t)c0 * N);
    ACP_LAUNCH(ctx);
  }
  return ACP_OK;
}

// ---- Alg. 3: W (N x k, workspace "acp_w") and the compression of Gk -------------------------
acp_status acp_build(acp_ctx* ctx, const double* Gk, int ncol, Compression* comp, double** W_out, SolveReport* rep,
                     double t0, double* ms_compress, double* ms_solve) {
  const int N = ctx->N, no = ctx->n_orb;
  const double tc = now_ms();
  ACP_TRY(compress(ctx, Gk, ncol, ctx->opt.sketch, ctx->opt.sketch_cols, ctx->opt.id_tol, ctx->opt.max_rank, comp));
  if (ms_compress) *ms_compress += now_ms() - tc;
  const int k = comp->n_mu;
  // Chebyshev nodes (a degenerate occupied band collapses to a single node)
  int nc = ctx->opt.n_cheb;
  const double e1 = ctx->eps.front(), eN = ctx->eps.back();
  if (eN - e1 < 1e-10 * fmax(1.0, fabs(e1))) nc = 1;
  double *nodes = nullptr, *Lw = nullptr, *rhs = nullptr, *X = nullptr, *W = nullptr, *Bc = nullptr, *psiT = nullptr;
  ACP_TRY(ws(ctx, "acp_nodes", 64, &nodes));
  ACP_TRY(ws(ctx, "acp_lw", (size_t)64 * no, &Lw));
  ::acp::note_launch(ctx);
  cheb_lagrange_kernel<<<1, 256, 0, ctx->stream>>>(nc, no, ctx->d_eps, nodes, Lw);
  ACP_LAUNCH(ctx);
  // right-hand sides Q xi_mu (Eq. eqncompressU)
  ACP_TRY(ws(ctx, "acp_rhs", (size_t)N * k, &rhs));
  ACP_TRY(project(ctx, comp->d_xi, N, k, rhs, N));
  ACP_TRY(ws(ctx, "acp_x", (size_t)N * k * nc, &X));
  const double ts = now_ms();
  ACP_TRY(minres_multishift(ctx, rhs, k, nodes, nc, X, rep, t0));
  // zeta lies in the unoccupied space: the outer Q of Eq. eqncompressU.  An inexact Alg. 4
  // iteration of the mixed form (FP32 solves only, relative error ~1e-6) takes Q through the
  // tensor-core projector, accurate to FP32 like the solves; solutions refined to stern_tol take
  // the FP64 one.
  if (ctx->opt.precision == ACP_PREC_MIXED && !ctx->mixed_refine)
    ACP_TRY(project_mixed64(ctx, X, k * nc, X));
  else
    ACP_TRY(project(ctx, X, N, k * nc, X, N));
  if (ms_solve) *ms_solve += now_ms() - ts;
  // W = sum_c (-2f) X_c .* (Psi diag(L_c) Psi(r_mu, :)^T)   (Eq. eqnW, zeta = -x)
  ACP_TRY(ws(ctx, "acp_w", (size_t)N * k, &W));
  ACP_TRY(ws(ctx, "acp_bc", (size_t)no * k, &Bc));
  ACP_TRY(ws(ctx, "id_psit", (size_t)no * N, &psiT));
  ACP_TRY(transpose(ctx, N, no, ctx->d_psi, psiT));
  ACP_CUDA(ctx, cudaMemsetAsync(W, 0, sizeof(double) * N * k, ctx->stream));
  for (int c = 0; c < nc; ++c) {
    ::acp::note_launch(ctx);
    build_bc<<<grid_for((size_t)no * k), 256, 0, ctx->stream>>>(no, k, nc, c, Lw, psiT, comp->d_piv, Bc);
    ACP_LAUNCH(ctx);
    ACP_TRY(dgemm(ctx, false, false, N, k, no, -2.0 * ctx->opt.occ, ctx->d_psi, N, Bc, no, 1.0, W, N,
                  X + (size_t)c * k * N, N));
  }
  *W_out = W;
  return ACP_OK;
}

acp_status chi0_acp(acp_ctx* ctx, const double* G, int ncol, double* out, acp_stats* st, SolveReport* rep, double t0) {
  Compression comp;
  double* W = nullptr;
  double msc = 0, mss = 0;
  ACP_TRY(acp_build(ctx, G, ncol, &comp, &W, rep, t0, &msc, &mss));
  const int k = comp.n_mu;
  double* Gp = nullptr;
  ACP_TRY(ws(ctx, "acp_gpiv", (size_t)k * ncol, &Gp));
  ACP_TRY(gather_rows(ctx, G, ctx->N, ncol, comp.d_piv, k, Gp, k));
  ACP_TRY(dgemm(ctx, false, false, ctx->N, ncol, k, 1.0, W, ctx->N, Gp, k, 0.0, out, ctx->N));
  if (st) {
    st->n_mu = k;
    st->ms_compress += msc;
    st->ms_solve += mss;
  }
  return ACP_OK;
}

// ---- Alg. 4 -----------------------------------------------------------------------------------
acp_status dyson_acp(acp_ctx* ctx, const double* G, int ncol, double* U, acp_stats* st, SolveReport* rep, double t0) {
  const int N = ctx->N;
  const size_t nv = (size_t)N * ncol;
  double *B = nullptr, *Ut = nullptr, *Un = nullptr, *Gk = nullptr;
  ACP_TRY(ws(ctx, "d_b", nv, &B));
  ACP_TRY(ws(ctx, "d_ut", nv, &Ut));
  ACP_TRY(ws(ctx, "d_un", nv, &Un));
  ACP_TRY(ws(ctx, "d_gk", nv, &Gk));
  // U~^0 = B = K^{-1} G
  ACP_TRY(spectral_apply(ctx, G, N, ncol, MULT_KHAT_INV, false, nullptr, B, N, nullptr, nullptr));
  ACP_CUDA(ctx, cudaMemcpyAsync(Ut, B, nv * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  double msc = 0, mss = 0;
  int it = 0;
  double change = 1e300;
  const int maxit = ctx->opt.dyson_maxit > 0 ? ctx->opt.dyson_maxit : 8;
  // Mixed precision: while the iterates still change by more than kRefineSwitch, the compressed
  // equations are solved by the FP32 pass alone (an inexact outer iteration, whose error ~1e-6
  // is below the change); from then on every solve is refined to stern_tol, and Alg. 4 may only
  // stop after a refined iteration.  An FP32-only iteration that shrinks the change by less than
  // 2x has met the noise floor of its solves (above kRefineSwitch when Alg. 4 amplifies them):
  // refinement then starts at once.
  constexpr double kRefineSwitch = 1e-4;
  bool refining = false;
  double prev_change = 1e300;
  const bool mixed = ctx->opt.precision == ACP_PREC_MIXED;
  struct RefineReset {
    acp_ctx* c;
    ~RefineReset() { c->mixed_refine = true; }
  } reset{ctx};
  for (it = 0; it < maxit; ++it) {
    refining = refining || change <= kRefineSwitch || (it >= 2 && change > 0.5 * prev_change) || it == maxit - 1;
    ctx->mixed_refine = !mixed || refining;
    ACP_TRY(spectral_apply(ctx, Ut, N, ncol, MULT_KHAT, false, nullptr, Gk, N, nullptr, nullptr));
    Compression comp;
    double* W = nullptr;
    ACP_TRY(acp_build(ctx, Gk, ncol, &comp, &W, rep, t0, &msc, &mss));
    const int k = comp.n_mu;
    double *KW = nullptr, *S = nullptr, *Y = nullptr;
    ACP_TRY(ws(ctx, "d_kw", (size_t)N * k, &KW));
    ACP_TRY(ws(ctx, "d_s", (size_t)k * k, &S));
    ACP_TRY(ws(ctx, "d_y", (size_t)k * ncol, &Y));
    // S = Pi^T K W, X = (I - S)^{-1} Pi^T G  (Pi^T K B = Pi^T G)
    ACP_TRY(spectral_apply(ctx, W, N, k, MULT_KHAT, false, nullptr, KW, N, nullptr, nullptr));
    ACP_TRY(gather_rows(ctx, KW, N, k, comp.d_piv, k, S, k));
    ::acp::note_launch(ctx);
    identity_minus<<<grid_for((size_t)k * k), 256, 0, ctx->stream>>>(k, S);
    ACP_LAUNCH(ctx);
    ACP_TRY(gather_rows(ctx, G, N, ncol, comp.d_piv, k, Y, k));
    ACP_TRY(lu_solve(ctx, S, k, Y, ncol));
    // U~^{k+1} = B + W X
    ACP_CUDA(ctx, cudaMemcpyAsync(Un, B, nv * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    ACP_TRY(dgemm(ctx, false, false, N, ncol, k, 1.0, W, N, Y, k, 1.0, Un, N));
    double nrm[2];
    ACP_TRY(diff_norms(ctx, Un, Ut, nv, nrm));
    prev_change = change;
    change = nrm[1] > 0 ? sqrt(nrm[0] / nrm[1]) : 0.0;
    double* t = Ut; Ut = Un; Un = t;
    if (st) st->n_mu = k;
    if (!std::isfinite(change)) return set_error(ctx, ACP_E_NUMERIC, "NaN in the adaptive Dyson iteration");
    if (change < ctx->opt.dyson_tol && ctx->mixed_refine) { ++it; break; }
    if (deadline_passed(ctx, t0)) return set_error(ctx, ACP_E_TIMEOUT, "deadline passed in Alg. 4");
  }
  // U = U~ - B
  ::acp::note_launch(ctx);
  axpby_kernel<<<grid_for(nv), 256, 0, ctx->stream>>>(nv, 1.0, Ut, -1.0, B, U);
  ACP_LAUNCH(ctx);
  if (st) {
    st->outer_iters = it > maxit ? maxit : it;
    st->ms_compress += msc;
    st->ms_solve += mss;
  }
  if (change >= ctx->opt.dyson_tol)
    return set_error(ctx, ACP_E_NOCONV, "Alg. 4 stopped after %d iterations at relative change %.3e", maxit, change);
  return ACP_OK;
}

// ---- GMRES on (I - chi0 K) U = chi0 G ---------------------------------------------------------
acp_status dyson_gmres(acp_ctx* ctx, const double* G, int ncol, double* U, acp_stats* st, SolveReport* rep, double t0) {
  const int N = ctx->N;
  const size_t nv = (size_t)N * ncol;
  int m = ctx->opt.dyson_maxit > 0 ? ctx->opt.dyson_maxit : 60;
  if (m > 120) m = 120;
  GmresState s{};
  s.m = m;
  double *rhs = nullptr, *tmp = nullptr, *tmp2 = nullptr, *res = nullptr, *mx = nullptr;
  ACP_TRY(ws(ctx, "g_vb", nv * (m + 1), &s.Vb));
  ACP_TRY(ws(ctx, "g_h", (size_t)ncol * (m + 1) * m, &s.H));
  ACP_TRY(ws(ctx, "g_cs", (size_t)ncol * m, &s.cs));
  ACP_TRY(ws(ctx, "g_sn", (size_t)ncol * m, &s.sn));
  ACP_TRY(ws(ctx, "g_g", (size_t)ncol * (m + 1), &s.g));
  ACP_TRY(ws(ctx, "g_b0", ncol, &s.beta0));
  ACP_TRY(ws(ctx, "g_res", ncol + 1, &res));
  mx = res + ncol;
  ACP_TRY(ws(ctx, "g_rhs", nv, &rhs));
  ACP_TRY(ws(ctx, "g_tmp", nv, &tmp));
  ACP_TRY(ws(ctx, "g_tmp2", nv, &tmp2));
  ACP_CUDA(ctx, cudaMemsetAsync(s.g, 0, sizeof(double) * ncol * (m + 1), ctx->stream));
  ACP_TRY(chi0_plain(ctx, G, ncol, rhs, rep, t0));
  ::acp::note_launch(ctx);
  gmres_start<<<ncol, 256, 0, ctx->stream>>>(N, ncol, rhs, s);
  ACP_LAUNCH(ctx);
  int k = 0;
  double r = 1.0;
  for (k = 0; k < m; ++k) {
    const double* vk = s.Vb + (size_t)k * nv;
    double* w = s.Vb + (size_t)(k + 1) * nv;
    ACP_TRY(spectral_apply(ctx, vk, N, ncol, MULT_KHAT, false, nullptr, tmp, N, nullptr, nullptr));
    ACP_TRY(chi0_plain(ctx, tmp, ncol, tmp2, rep, t0));
    ::acp::note_launch(ctx);
    axpby_kernel<<<grid_for(nv), 256, 0, ctx->stream>>>(nv, 1.0, vk, -1.0, tmp2, w);
    ACP_LAUNCH(ctx);
    ::acp::note_launch(ctx);
    gmres_arnoldi<<<ncol, 256, 0, ctx->stream>>>(N, ncol, k, s, res);
    ::acp::note_launch(ctx);
    max_kernel<<<1, 1024, 0, ctx->stream>>>(res, ncol, mx);
    ACP_LAUNCH(ctx);
    ACP_CUDA(ctx, cudaMemcpyAsync(&r, mx, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (!std::isfinite(r)) return set_error(ctx, ACP_E_NUMERIC, "NaN in GMRES");
    if (r <= ctx->opt.dyson_tol) { ++k; break; }
    if (deadline_passed(ctx, t0)) return set_error(ctx, ACP_E_TIMEOUT, "deadline passed in GMRES");
  }
  if (k > m) k = m;
  ::acp::note_launch(ctx);
  gmres_finish<<<ncol, 256, 0, ctx->stream>>>(N, ncol, k, s, U);
  ACP_LAUNCH(ctx);
  if (st) st->outer_iters = k;
  if (r > ctx->opt.dyson_tol)
    return set_error(ctx, ACP_E_NOCONV, "GMRES stopped after %d iterations at relative residual %.3e", k, r);
  return ACP_OK;
}

acp_status dyson(acp_ctx* ctx, const double* G, int ncol, double* U, acp_stats* st, SolveReport* rep, double t0) {
  if (ctx->opt.method == ACP_METHOD_ACP) return dyson_acp(ctx, G, ncol, U, st, rep, t0);
  return dyson_gmres(ctx, G, ncol, U, st, rep, t0);
}

// ---- Eq. SecDeriv ------------------------------------------------------------------------------
// 2D: perturbation columns 2I + a; D is (2 nA) x (2 nA) with a 2 x 2 local block per atom and the
// ion-ion Hessian blocks of spectral2d.cu.
acp_status dynamical_2d(acp_ctx* ctx, const acp_atoms* at, const double* rho, double* D_h, double* U_user,
                        acp_stats* st, SolveReport* rep, double t0) {
  const int N = ctx->N, nA = at->n_atoms, nP = 2 * nA;
  double *hv = nullptr, *G = nullptr, *D2 = nullptr, *U = nullptr, *Hm = nullptr, *nrm = nullptr;
  ACP_TRY(ws(ctx, "dm_atoms", 5 * (size_t)nA, &hv));  // R (2 per atom), Z, sigma, mass
  std::vector<double> host(5 * (size_t)nA);
  for (int I = 0; I < nA; ++I) {
    host[2 * I] = at->R[2 * I];
    host[2 * I + 1] = at->R[2 * I + 1];
    host[2 * nA + I] = at->Z[I];
    host[3 * nA + I] = at->sigma[I];
    host[4 * nA + I] = at->mass ? at->mass[I] : 1.0;
  }
  ACP_CUDA(ctx, cudaMemcpyAsync(hv, host.data(), sizeof(double) * 5 * nA, cudaMemcpyHostToDevice, ctx->stream));
  ACP_TRY(ws(ctx, "dm_g", (size_t)N * nP, &G));
  ACP_TRY(ws(ctx, "dm_d2", (size_t)N * 3 * nA, &D2));
  if (U_user) U = U_user;
  else ACP_TRY(ws(ctx, "dm_u", (size_t)N * nP, &U));
  ACP_TRY(ws(ctx, "dm_h", (size_t)nP * nP * 3 + 3 * (size_t)nA + 4 * (size_t)nA * nA + 2, &Hm));
  double* D = Hm + (size_t)nP * nP;
  double* Ds = D + (size_t)nP * nP;
  double* dv = Ds + (size_t)nP * nP;
  double* Hp = dv + 3 * (size_t)nA;
  nrm = Hp + 4 * (size_t)nA * nA;
  ACP_TRY(perturbations_2d(ctx, nA, hv, hv + 2 * nA, hv + 3 * nA, G, nullptr, D2));
  acp_status sd = dyson(ctx, G, nP, U, st, rep, t0);
  if (sd != ACP_OK && sd != ACP_E_NOCONV) return sd;
  ACP_TRY(dgemm(ctx, true, false, nP, nP, N, ctx->h, G, N, U, N, 0.0, Hm, nP));
  ACP_TRY(dgemm(ctx, true, false, 3 * nA, 1, N, ctx->h, D2, N, rho, N, 0.0, dv, 3 * nA));
  ACP_TRY(ion_hessian_2d(ctx, nA, at->R, hv, Hp));
  ACP_TRY(assemble_2d(ctx, nA, Hm, dv, Hp, hv + 2 * nA, hv + 4 * nA, D));
  ACP_CUDA(ctx, cudaMemsetAsync(nrm, 0, 2 * sizeof(double), ctx->stream));
  ::acp::note_launch(ctx);
  symmetrize_kernel<<<grid_for((size_t)nP * nP, 1024), 256, 0, ctx->stream>>>(nP, D, Ds, nrm);
  ACP_LAUNCH(ctx);
  double hn[2];
  ACP_CUDA(ctx, cudaMemcpyAsync(D_h, Ds, sizeof(double) * nP * nP, cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaMemcpyAsync(hn, nrm, sizeof(double) * 2, cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (st) st->asymmetry = hn[1] > 0 ? sqrt(hn[0] / hn[1]) : 0.0;
  return sd;
}

acp_status dynamical(acp_ctx* ctx, const acp_atoms* at, const double* rho, double* D_h, double* U_user,
                     acp_stats* st, SolveReport* rep, double t0) {
  if (ctx->dim == 2) return dynamical_2d(ctx, at, rho, D_h, U_user, st, rep, t0);
  const int N = ctx->N, nA = at->n_atoms;
  double *hv = nullptr, *G = nullptr, *D2 = nullptr, *U = nullptr, *Hm = nullptr, *dv = nullptr, *D = nullptr,
         *Ds = nullptr, *nrm = nullptr;
  ACP_TRY(ws(ctx, "dm_atoms", 4 * (size_t)nA, &hv));
  std::vector<double> host(4 * (size_t)nA);
  for (int I = 0; I < nA; ++I) {
    host[I] = at->R[I];
    host[nA + I] = at->Z[I];
    host[2 * nA + I] = at->sigma[I];
    host[3 * nA + I] = at->mass ? at->mass[I] : 1.0;
  }
  ACP_CUDA(ctx, cudaMemcpyAsync(hv, host.data(), sizeof(double) * 4 * nA, cudaMemcpyHostToDevice, ctx->stream));
  ACP_TRY(ws(ctx, "dm_g", (size_t)N * nA, &G));
  ACP_TRY(ws(ctx, "dm_d2", (size_t)N * nA, &D2));
  if (U_user) U = U_user;
  else ACP_TRY(ws(ctx, "dm_u", (size_t)N * nA, &U));
  ACP_TRY(ws(ctx, "dm_h", (size_t)nA * nA * 3 + nA + 2, &Hm));
  D = Hm + (size_t)nA * nA;
  Ds = D + (size_t)nA * nA;
  dv = Ds + (size_t)nA * nA;
  nrm = dv + nA;
  ACP_TRY(perturbations_1d(ctx, nA, hv, hv + nA, hv + 2 * nA, G, nullptr, D2));
  acp_status sd = dyson(ctx, G, nA, U, st, rep, t0);
  if (sd != ACP_OK && sd != ACP_E_NOCONV) return sd;
  // first term h G^T U, second term h d2V^T rho (Eq. SecDeriv)
  ACP_TRY(dgemm(ctx, true, false, nA, nA, N, ctx->h, G, N, U, N, 0.0, Hm, nA));
  ACP_TRY(dgemm(ctx, true, false, nA, 1, N, ctx->h, D2, N, rho, N, 0.0, dv, nA));
  ::acp::note_launch(ctx);
  assemble_dmat<<<grid_for((size_t)nA * nA), 256, 0, ctx->stream>>>(nA, Hm, dv, hv, hv + nA, hv + 3 * nA, ctx->L,
                                                                     ctx->kappa, ctx->scale, D);
  ACP_LAUNCH(ctx);
  ACP_CUDA(ctx, cudaMemsetAsync(nrm, 0, 2 * sizeof(double), ctx->stream));
  ::acp::note_launch(ctx);
  symmetrize_kernel<<<grid_for((size_t)nA * nA, 1024), 256, 0, ctx->stream>>>(nA, D, Ds, nrm);
  ACP_LAUNCH(ctx);
  double hn[2];
  ACP_CUDA(ctx, cudaMemcpyAsync(D_h, Ds, sizeof(double) * nA * nA, cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaMemcpyAsync(hn, nrm, sizeof(double) * 2, cudaMemcpyDeviceToHost, ctx->stream));
  ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (st) st->asymmetry = hn[1] > 0 ? sqrt(hn[0] / hn[1]) : 0.0;
  return sd;
}

}  // namespace acp
