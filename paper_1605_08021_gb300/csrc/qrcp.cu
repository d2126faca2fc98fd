// Interpolative decomposition of M_ij = psi_i * g_j (Eq. MID) by Alg. 2 in the form of its
// Remark: the SRFT acts on G only (G_tilde = G Omega), row alpha of M_tilde is the Kronecker
// product psi(r_alpha, :) (x) G_tilde(r_alpha, :), a column-pivoted Householder QR of
// M_tilde^T (m = n_orb * sketch_cols rows, N columns) selects the points r_mu, and
// Xi^T = R_11^{-1} R_{1:N_mu, :} Pi^{-1} gives the interpolation vectors (Alg. 2 steps 2-4).
//
// The QR runs right-looking with the pivot rule of LAPACK's geqp3: at step j the pivot is the
// trailing column of largest downdated norm (lowest position in the swapped column order on
// ties); its Householder reflector is applied to every trailing column and their norms are
// downdated with the usual cancellation safeguard (recompute when the downdated norm has lost
// about half its digits).  The loop stops at the first |R_jj| < id_tol |R_11|.
//
// Persistent form (qr_persistent_kernel): one cooperative launch with one CTA per SM.  Columns
// are dealt round-robin to the CTAs, which keep their norms and positions in shared memory and
// never move columns (the swapped order is tracked as positions).  Per step: every CTA reduces
// the per-CTA pivot candidates, reads the pivot column and forms the same Householder vector
// (identical arithmetic in every CTA), updates its own trailing columns (one warp per column),
// downdates their norms and publishes its next candidate; one grid barrier (bounded wait) ends
// the step.  The pivot column is only read during its own step, so no CTA writes what another
// reads.  R_jj and the pivot order are recorded per step; a gather builds R in pivot order.
// Fallback (per-step kernels qr_pivot_kernel + qr_update_kernel, physical swaps) when the
// cooperative launch or its shared memory is not available.
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

// ---- persistent pivoted QR ----------------------------------------------------------------------
struct PqrArgs {
  double* A;        // m x N (ld m), updated in place; columns never move
  int m, N, kmax;
  double id_tol;
  double* rdiag;    // |R_jj|, kmax
  double* alpha;    // R_jj (signed), kmax
  int* perm;        // perm[q] = column at position q of the final swapped order (N)
  double* cand_v;   // per CTA and step parity: candidate norm (-1: none), 2 x gridDim
  int* cand_pos;    // its position
  int* cand_col;    // its column
  unsigned* bar;    // [0] arrivals, [1] generation (zeroed before the launch)
  int* status;      // [0] N_mu; [1] 1 if a grid barrier ran out of time
};

constexpr unsigned long long kBarrierNs = 500000000ull;  // 0.5 s per grid barrier

__device__ __forceinline__ unsigned long long qr_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier over the co-resident CTAs of a cooperative launch; the wait is bounded (a CTA that
// gives up sets status[1] and returns false).  Makes the CTA's global writes visible to all CTAs.
__device__ bool qr_grid_barrier(unsigned* bar, int* status, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long deadline = qr_globaltimer() + kBarrierNs;
      unsigned spins = 0;
      while (*gen == g) {
        __nanosleep(64);
        if ((++spins & 255u) == 0 && (qr_globaltimer() > deadline || spins > (1u << 30))) {
          ok = 0;
          atomicExch(status + 1, 1);
          break;
        }
      }
    }
    __threadfence();
    *s_ok = ok && (*((volatile int*)(status + 1)) == 0);
  }
  __syncthreads();
  return *s_ok != 0;
}

// A column group of W warps shares one trailing column per pass, each thread holding R of its rows
// in registers: one read and one write per element, R loads in flight, and two FP64 FMAs per
// element (the dot product and the update; GB300's FP64 rate bounds this kernel).  The tail norm
// of the column is formed from the registers only when the norm downdate needs a recomputation.
constexpr int kQrThreads = 512;

__device__ __forceinline__ void group_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int R, int W>
__global__ void __launch_bounds__(kQrThreads, 1) qr_persistent_kernel(PqrArgs a) {
  constexpr int THREADS = kQrThreads;
  constexpr int G = 32 * W;
  extern __shared__ double qsm[];
  const int m = a.m, N = a.N, nb = gridDim.x, b = blockIdx.x;
  const int ncl = (N + nb - 1) / nb;     // columns of this CTA: c = b + t nb
  double* v = qsm;                       // m: Householder vector of the step
  double* vn1 = v + m;                   // ncl (negative: chosen)
  double* vn2 = vn1 + ncl;               // ncl
  int* cpos = reinterpret_cast<int*>(vn2 + ncl);  // ncl: position in the swapped order
  __shared__ double red[32];
  __shared__ double part_d[THREADS / G][G / 32], part_t[THREADS / G][G / 32];
  __shared__ int flag_s[THREADS / G];
  __shared__ double wv[32];
  __shared__ int wp[32], wc[32];
  __shared__ int s_ok, s_p, s_pp;
  __shared__ double s_best;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;

  // initial norms
  for (int t = wid; t < ncl; t += nw) {
    const int c = b + t * nb;
    double sacc = 0.0;
    if (c < N) {
      const double* col = a.A + (size_t)c * m;
      for (int r = lane; r < m; r += 32) sacc += col[r] * col[r];
      sacc = warp_sum(sacc);
    }
    if (lane == 0) {
      vn1[t] = (c < N) ? sqrt(sacc) : -1.0;
      vn2[t] = vn1[t];
      cpos[t] = c;
    }
  }
  __syncthreads();
  // local candidate: largest vn1, lowest position on ties
  // candidates of step j live in buffer j & 1: a CTA that has finished step j writes buffer
  // (j + 1) & 1 while slower CTAs may still read buffer j & 1 (the barrier keeps them one step apart)
  auto publish = [&](int buf) {
    double best = -1.0;
    int bp = 0x7fffffff, bc = -1;
    for (int t = threadIdx.x; t < ncl; t += blockDim.x) {
      const double x = vn1[t];
      if (x > best || (x == best && x >= 0.0 && cpos[t] < bp)) { best = x; bp = cpos[t]; bc = b + t * nb; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int op = __shfl_xor_sync(0xffffffffu, bp, o), oc = __shfl_xor_sync(0xffffffffu, bc, o);
      if (ob > best || (ob == best && op < bp)) { best = ob; bp = op; bc = oc; }
    }
    if (lane == 0) { wv[wid] = best; wp[wid] = bp; wc[wid] = bc; }
    __syncthreads();
    if (wid == 0) {
      best = (lane < nw) ? wv[lane] : -1.0;
      bp = (lane < nw) ? wp[lane] : 0x7fffffff;
      bc = (lane < nw) ? wc[lane] : -1;
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o), oc = __shfl_xor_sync(0xffffffffu, bc, o);
        if (ob > best || (ob == best && op < bp)) { best = ob; bp = op; bc = oc; }
      }
      if (lane == 0) {
        a.cand_v[buf * nb + b] = best;
        a.cand_pos[buf * nb + b] = bp;
        a.cand_col[buf * nb + b] = bc;
      }
    }
  };
  publish(0);
  if (!qr_grid_barrier(a.bar, a.status, &s_ok)) return;

  double r11 = 0.0;
  int k = a.kmax;
  for (int j = 0; j < a.kmax; ++j) {
    // global pivot from the CTA candidates (L2 reads: they change every step)
    if (wid == 0) {
      double best = -1.0;
      int bp = 0x7fffffff, bc = -1;
      const int off = (j & 1) * nb;
      for (int q = lane; q < nb; q += 32) {
        const double x = __ldcg(a.cand_v + off + q);
        const int qp = __ldcg(a.cand_pos + off + q);
        if (x > best || (x == best && qp < bp)) { best = x; bp = qp; bc = __ldcg(a.cand_col + off + q); }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o), oc = __shfl_xor_sync(0xffffffffu, bc, o);
        if (ob > best || (ob == best && op < bp)) { best = ob; bp = op; bc = oc; }
      }
      if (lane == 0) { s_best = best; s_p = bc; s_pp = bp; }
    }
    __syncthreads();
    const int p = s_p, pos_p = s_pp;
    if (p < 0 || s_best < 0.0) { k = j; break; }
    // Householder vector of column p, rows j..m-1 (same arithmetic in every CTA)
    const double* cp = a.A + (size_t)p * m;
    double acc = 0.0;
    for (int r = j + threadIdx.x; r < m; r += blockDim.x) {
      const double x = __ldcg(cp + r);
      v[r] = x;
      acc += x * x;
    }
    const double nrm = sqrt(block_sum(acc, red));
    const double x0 = v[j];
    const double alpha = (x0 >= 0.0) ? -nrm : nrm;
    if (j == 0) r11 = fabs(alpha);
    if (!(fabs(alpha) >= a.id_tol * r11) || nrm == 0.0) { k = j; break; }
    const double v0 = x0 - alpha;
    const double vtv = nrm * nrm - x0 * x0 + v0 * v0;
    const double tau = (vtv > 0.0) ? 2.0 / vtv : 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
      v[j] = v0;
      if (b == 0) { a.rdiag[j] = fabs(alpha); a.alpha[j] = alpha; }
    }
    // positions: p moves to j, the column at position j moves to p's old position
    for (int t = threadIdx.x; t < ncl; t += blockDim.x) {
      const int c = b + t * nb;
      if (c == p) { vn1[t] = -1.0; cpos[t] = j; }
      else if (vn1[t] >= 0.0 && cpos[t] == j) cpos[t] = pos_p;
    }
    __syncthreads();
    // reflector on this CTA's trailing columns (one column per group pass), norm downdate
    const int rem = m - j;  // chunk i (rows j + i G ...) is live while i G < rem: a uniform branch
    {
      const int ngr = THREADS / G, g = threadIdx.x / G, gt = threadIdx.x % G;
      const int wig = gt >> 5;  // warp in group
      for (int t = g; t < ncl; t += ngr) {
        const double vn1t = vn1[t];
        if (vn1t < 0.0) continue;  // uniform in the group
        double* col = a.A + (size_t)(b + t * nb) * m;
        double x[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
          if (i * G < rem) {
            const int r = j + gt + i * G;
            x[i] = (r < m) ? col[r] : 0.0;
          }
        }
        double pd0 = 0.0, pd1 = 0.0;
#pragma unroll
        for (int i = 0; i < R; i += 2) {
          if (i * G < rem) {
            const int r = j + gt + i * G;
            if (r < m) pd0 = fma(v[r], x[i], pd0);
          }
          if (i + 1 < R && (i + 1) * G < rem) {
            const int r = j + gt + (i + 1) * G;
            if (r < m) pd1 = fma(v[r], x[i + 1], pd1);
          }
        }
        const double pd = warp_sum(pd0 + pd1);
        if (lane == 0) part_d[g][wig] = pd;
        group_sync(1 + g, G);
        double d = 0.0;
#pragma unroll
        for (int w = 0; w < W; ++w) d += part_d[g][w];
        d *= tau;
#pragma unroll
        for (int i = 0; i < R; ++i) {
          if (i * G < rem) {
            const int r = j + gt + i * G;
            if (r < m) {
              x[i] = fma(-d, v[r], x[i]);
              col[r] = x[i];
            }
          }
        }
        // norm downdate, decided by the group's thread 0 (it holds row j: i = 0); flag_s[g] = 1 asks
        // the group for the tail norm
        if (gt == 0) {
          int rec = 0;
          if (vn1t != 0.0) {
            double temp = fabs(x[0]) / vn1t;
            temp = fmax(0.0, (1.0 + temp) * (1.0 - temp));
            const double rr = vn1t / vn2[t];
            if (temp * rr * rr <= 1.4901161193847656e-08) rec = 1;  // sqrt(2^-52)
            else vn1[t] = vn1t * sqrt(temp);
          }
          flag_s[g] = rec;
        }
        group_sync(1 + g, G);
        if (flag_s[g]) {
          double tail = 0.0;
#pragma unroll
          for (int i = 0; i < R; ++i) {
            if (i * G < rem) {
              const int r = j + gt + i * G;
              if (r > j && r < m) tail = fma(x[i], x[i], tail);
            }
          }
          tail = warp_sum(tail);
          if (lane == 0) part_t[g][wig] = tail;
          group_sync(1 + g, G);
          if (gt == 0) {
            double tl = 0.0;
#pragma unroll
            for (int w = 0; w < W; ++w) tl += part_t[g][w];
            vn1[t] = sqrt(tl);
            vn2[t] = sqrt(tl);
          }
        }
      }
    }
    __syncthreads();
    publish((j + 1) & 1);
    if (!qr_grid_barrier(a.bar, a.status, &s_ok)) return;
  }
  // final positions (chosen columns: their step; the others: their swapped slot)
  for (int t = threadIdx.x; t < ncl; t += blockDim.x) {
    const int c = b + t * nb;
    if (c < N) a.perm[cpos[t]] = c;
  }
  if (b == 0 && threadIdx.x == 0) a.status[0] = k;
}

// Rs (k x N, ld k) in pivot order: column q = A[0:k, perm[q]] above the diagonal (and every row
// for q >= k), alpha on it, zero below.
__global__ void gather_r_kernel(int m, int N, int k, const double* __restrict__ A, const int* __restrict__ perm,
                                const double* __restrict__ alpha, double* __restrict__ Rs) {
  const size_t total = (size_t)k * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % k), q = (int)(e / k);
    double x;
    if (q >= k || r < q) x = A[r + (size_t)perm[q] * m];
    else x = (r == q) ? alpha[q] : 0.0;
    Rs[e] = x;
  }
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

  // persistent form when one CTA per SM can hold the step's shared memory and launch cooperatively;
  // rows per thread R covers m rows with a group of 256 threads (R <= 12 at 1024 threads, up to 48
  // at 256 threads, within the register budget of one CTA per SM)
  int coop = 0, n_sm = 0;
  ACP_CUDA(ctx, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device));
  ACP_CUDA(ctx, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, ctx->device));
  const int ncl = (N + n_sm - 1) / (n_sm > 0 ? n_sm : 1);
  const size_t pq_smem = sizeof(double) * ((size_t)m + 2 * (size_t)ncl) + sizeof(int) * (size_t)ncl;
  const void* pq_fn = nullptr;
  const int pq_threads = kQrThreads;
  {
    // groups of 2 warps while 48 rows a thread hold a column (registers of 512 threads at one CTA per
    // SM), wider groups beyond; fewer rows a thread for short columns
    struct Inst { int rows; const void* fn; };
    const Inst inst[] = {{64 * 16, reinterpret_cast<const void*>(qr_persistent_kernel<16, 2>)},
                         {64 * 32, reinterpret_cast<const void*>(qr_persistent_kernel<32, 2>)},
                         {64 * 48, reinterpret_cast<const void*>(qr_persistent_kernel<48, 2>)},
                         {128 * 48, reinterpret_cast<const void*>(qr_persistent_kernel<48, 4>)},
                         {256 * 48, reinterpret_cast<const void*>(qr_persistent_kernel<48, 8>)}};
    for (const Inst& in : inst)
      if (m <= in.rows) { pq_fn = in.fn; break; }
  }
  bool persistent = pq_fn && coop && n_sm > 0 && pq_smem + 4096 <= ctx->smem_optin;
  if (persistent) {
    ACP_TRY(raise_smem_limit(ctx, pq_fn));
    int per_sm = 0;
    ACP_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pq_fn, pq_threads, pq_smem));
    persistent = per_sm >= 1;
  }
  const double* Rb = A;  // R in pivot order: the swapped A (ld m) or the gathered Rs (ld k)
  int ldr = m;
  int* perm_d = nullptr;
  int k = 0;
  if (persistent) {
    double* dv = nullptr;
    ACP_TRY(ws(ctx, "pq_dv", 2 * (size_t)kmax + 2 * (size_t)n_sm, &dv));
    int* iv = nullptr;
    ACP_TRY(ws(ctx, "pq_iv", (size_t)N + 4 * (size_t)n_sm + 4, &iv));
    PqrArgs pa{};
    pa.A = A; pa.m = m; pa.N = N; pa.kmax = kmax; pa.id_tol = id_tol;
    pa.rdiag = dv; pa.alpha = dv + kmax; pa.cand_v = dv + 2 * kmax;
    pa.perm = iv; pa.cand_pos = iv + N; pa.cand_col = iv + N + 2 * n_sm;
    pa.status = iv + N + 4 * n_sm;
    pa.bar = reinterpret_cast<unsigned*>(iv + N + 4 * n_sm + 2);
    ACP_CUDA(ctx, cudaMemsetAsync(pa.status, 0, 4 * sizeof(int), ctx->stream));
    void* kargs[] = {&pa};
    ::acp::note_launch(ctx);
    cudaEvent_t ev0 = prof_begin(ctx);
    ACP_CUDA(ctx, cudaLaunchCooperativeKernel(pq_fn, dim3(n_sm), dim3(pq_threads), kargs, pq_smem, ctx->stream));
    prof_end(ctx, "qrcp", ev0, 0.0, 0.0);
    int hs[2] = {0, 0};
    ACP_CUDA(ctx, cudaMemcpyAsync(hs, pa.status, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    ACP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (hs[1]) return set_error(ctx, ACP_E_TIMEOUT, "pivoted QR: a grid barrier of the persistent kernel timed out");
    k = hs[0];
    {
      // algorithmic work of the k steps: the reflector's dot product and update on the trailing
      // (m - j) x (N - j - 1) block, 2 FMAs and one read and one write of each FP64 element
      double el = 0.0;
      for (int j = 0; j < k; ++j) el += (double)(m - j) * (double)(N - j - 1);
      prof_amend_last(ctx, "qrcp", 4.0 * el, 16.0 * el);
    }
    if (k <= 0) return set_error(ctx, ACP_E_RANK, "pivoted QR found rank 0 (is G zero?)");
    out->n_mu = k;
    out->piv.resize(N);
    out->rdiag.resize(k);
    ACP_CUDA(ctx, cudaMemcpyAsync(out->piv.data(), pa.perm, sizeof(int) * N, cudaMemcpyDeviceToHost, ctx->stream));
    ACP_CUDA(ctx, cudaMemcpyAsync(out->rdiag.data(), pa.rdiag, sizeof(double) * k, cudaMemcpyDeviceToHost,
                                  ctx->stream));
    double* Rs = nullptr;
    ACP_TRY(ws(ctx, "pq_rs", (size_t)k * N, &Rs));
    {
      const size_t total = (size_t)k * N;
      int blocks = (int)((total + 255) / 256);
      if (blocks > 65535) blocks = 65535;
      ::acp::note_launch(ctx);
      gather_r_kernel<<<blocks, 256, 0, ctx->stream>>>(m, N, k, A, pa.perm, pa.alpha, Rs);
      ACP_LAUNCH(ctx);
    }
    Rb = Rs;
    ldr = k;
    perm_d = pa.perm;
  } else {
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
    k = host_stop[1];
    if (k <= 0) return set_error(ctx, ACP_E_RANK, "pivoted QR found rank 0 (is G zero?)");
    out->n_mu = k;
    out->piv.resize(N);
    out->rdiag.resize(k);
    ACP_CUDA(ctx, cudaMemcpyAsync(out->piv.data(), s.perm, sizeof(int) * N, cudaMemcpyDeviceToHost, ctx->stream));
    ACP_CUDA(ctx, cudaMemcpyAsync(out->rdiag.data(), s.rdiag, sizeof(double) * k, cudaMemcpyDeviceToHost,
                                  ctx->stream));
    perm_d = s.perm;
  }

  // X = R11^{-1} R12 by blocked back substitution (diagonal blocks in shared memory, GEMM updates)
  const int nr = N - k;
  double* X = nullptr;
  ACP_TRY(ws(ctx, "id_x", (size_t)k * (nr > 0 ? nr : 1), &X));
  if (nr > 0) {
    ACP_CUDA(ctx, cudaMemcpy2DAsync(X, sizeof(double) * k, Rb + (size_t)k * ldr, sizeof(double) * ldr,
                                    sizeof(double) * k, nr, cudaMemcpyDeviceToDevice, ctx->stream));
    const int nb = 64;
    const int nblk = (k + nb - 1) / nb;
    for (int bb = nblk - 1; bb >= 0; --bb) {
      const int r0 = bb * nb, r1 = (r0 + nb < k) ? r0 + nb : k, w = r1 - r0;
      ::acp::note_launch(ctx);
      trsm_diag_kernel<<<(nr + 127) / 128, 128, w * w * sizeof(double), ctx->stream>>>(
          w, Rb + r0 + (size_t)r0 * ldr, ldr, X + r0, k, nr);
      ACP_LAUNCH(ctx);
      if (r0 > 0)
        ACP_TRY(dgemm(ctx, false, false, r0, nr, w, -1.0, Rb + (size_t)r0 * ldr, ldr, X + r0, k, 1.0, X, k));
    }
  }
  double* Xi = nullptr;
  int* dpiv = nullptr;
  ACP_TRY(ws(ctx, "xi", (size_t)N * k, &Xi));
  ACP_TRY(ws(ctx, "xi_piv", (size_t)N, &dpiv));
  ACP_CUDA(ctx, cudaMemcpyAsync(dpiv, perm_d, sizeof(int) * N, cudaMemcpyDeviceToDevice, ctx->stream));
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
