// Spectral operators on the periodic 2D grid (the 2D model of Sec. 4; Eq. Hamil, Eq. yukawa,
// Eq. pseudocharge in two dimensions), in FP64 and FP32.
//
// A 2D grid function has N = nx * ny values, x fastest.  Two real columns are packed as one
// complex signal z = x0 + i x1 (the symbols of H, K and K^-1 are real and even, so the halves
// stay apart) and transformed in three passes through a complex scratch block Z:
//   rows  forward FFT along x of every row            (CTA: a group of threads per row, several rows)
//   cols  forward FFT along y, symbol, inverse FFT    (CTA: a group per column, several columns)
//   rows  inverse FFT along x + the local potential, the shift and the Lanczos coefficient
// Each FFT runs in shared memory (mixed-radix Stockham, radices 4, 2, 3, 5).  The Lanczos form adds
// alpha_j = x_j . (H - s_j) x_j across the CTAs of a column (atomics) and a fourth, elementwise pass
// P = (H - s)x - alpha x - beta x_prev.
//
// The ion-ion Hessian of E_II (point charges, periodic Yukawa kernel) is evaluated spectrally:
// for two charges smeared into Gaussians of width sg, the kernel becomes
// exp(sg^2 kappa^2) [K(d) - S(d)] with S(d) ~ exp(-d^2 / 4 sg^2) (heat-kernel identity), so
// K(d) = exp(-sg^2 kappa^2) (1/A) sum_k Khat(k) exp(-sg^2 |k|^2) exp(i k.d) up to S; sg is chosen
// as a twelfth of the smallest pair distance (S/K < 1e-15) and the k-sum is cut where
// exp(-sg^2 |k|^2) < 1e-18.
#include "internal.cuh"

namespace acp {

namespace {

template <class T> struct Cx;
template <> struct Cx<double> { using t = double2; };
template <> struct Cx<float> { using t = float2; };

template <class T2, class T>
__device__ __forceinline__ T2 mk(T a, T b) {
  T2 r;
  r.x = a;
  r.y = b;
  return r;
}
template <class T2> __device__ __forceinline__ T2 cmul2(T2 a, T2 b) {
  return mk<T2>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class T2> __device__ __forceinline__ T2 cadd2(T2 a, T2 b) { return mk<T2>(a.x + b.x, a.y + b.y); }
template <class T2> __device__ __forceinline__ T2 csub2(T2 a, T2 b) { return mk<T2>(a.x - b.x, a.y - b.y); }
template <class T2, class T> __device__ __forceinline__ T2 cscale2(T2 a, T s) { return mk<T2>(a.x * s, a.y * s); }
template <class T2, class T> __device__ __forceinline__ T2 cimul2(T2 a, T s) { return mk<T2>(-a.y * s, a.x * s); }

template <int R, class T2, class T> struct Dft;
template <class T2, class T> struct Dft<2, T2, T> {
  static __device__ __forceinline__ void run(T2 (&a)[2], T) {
    const T2 t = a[0];
    a[0] = cadd2(t, a[1]);
    a[1] = csub2(t, a[1]);
  }
};
template <class T2, class T> struct Dft<4, T2, T> {
  static __device__ __forceinline__ void run(T2 (&a)[4], T dir) {
    const T2 s02 = cadd2(a[0], a[2]), d02 = csub2(a[0], a[2]);
    const T2 s13 = cadd2(a[1], a[3]), d13 = cimul2<T2, T>(csub2(a[1], a[3]), dir);
    a[0] = cadd2(s02, s13);
    a[2] = csub2(s02, s13);
    a[1] = cadd2(d02, d13);
    a[3] = csub2(d02, d13);
  }
};
template <class T2, class T> struct Dft<3, T2, T> {
  static __device__ __forceinline__ void run(T2 (&a)[3], T dir) {
    const T c = T(-0.5), s = T(0.86602540378443864676);
    const T2 t1 = cadd2(a[1], a[2]), t2 = cimul2<T2, T>(csub2(a[1], a[2]), dir * s);
    const T2 m = cadd2(a[0], cscale2<T2, T>(t1, c));
    a[0] = cadd2(a[0], t1);
    a[1] = cadd2(m, t2);
    a[2] = csub2(m, t2);
  }
};
template <class T2, class T> struct Dft<5, T2, T> {
  static __device__ __forceinline__ void run(T2 (&a)[5], T dir) {
    const T c1 = T(0.30901699437494742410), s1 = T(0.95105651629515357212);
    const T c2 = T(-0.80901699437494742410), s2 = T(0.58778525229247312917);
    const T2 t1 = cadd2(a[1], a[4]), t2 = cadd2(a[2], a[3]);
    const T2 d1 = csub2(a[1], a[4]), d2 = csub2(a[2], a[3]);
    const T2 m1 = cadd2(a[0], cadd2(cscale2<T2, T>(t1, c1), cscale2<T2, T>(t2, c2)));
    const T2 m2 = cadd2(a[0], cadd2(cscale2<T2, T>(t1, c2), cscale2<T2, T>(t2, c1)));
    const T2 e1 = cimul2<T2, T>(cadd2(cscale2<T2, T>(d1, s1), cscale2<T2, T>(d2, s2)), dir);
    const T2 e2 = cimul2<T2, T>(csub2(cscale2<T2, T>(d1, s2), cscale2<T2, T>(d2, s1)), dir);
    a[0] = cadd2(a[0], cadd2(t1, t2));
    a[1] = cadd2(m1, e1);
    a[4] = csub2(m1, e1);
    a[2] = cadd2(m2, e2);
    a[3] = csub2(m2, e2);
  }
};

template <int R> struct Mb;
template <> struct Mb<2> { static constexpr int v = 4; };
template <> struct Mb<3> { static constexpr int v = 4; };
template <> struct Mb<4> { static constexpr int v = 3; };
template <> struct Mb<5> { static constexpr int v = 2; };

struct AxisPlan {
  int n, nst, nt;  // length, stages, threads per transform
  int rad[16];
};

// One in-place Stockham stage of every transform of the CTA: thread `tid` of a group of `nt`
// threads works on the length-n signal at s.  All groups call it together (CTA barriers);
// groups without a signal pass valid = false.
// wsync: the group is one whole warp working on its own signal, so the stage synchronises the warp
// only (no CTA barrier; warps then run their transforms independently).
template <int R, class T2, class T>
__device__ __noinline__ void stage2(T2* s, int n, int Ns, const T2* __restrict__ tw, T dir, int tid, int nt,
                                    bool valid, int es, bool wsync) {
  constexpr int B = Mb<R>::v;
  const int nb = n / R;
  const int stride = n / (Ns * R);
  T2 a[B][R];
  if (valid) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = tid + b * nt;
      if (j < nb) {
#pragma unroll
        for (int r = 0; r < R; ++r) a[b][r] = s[(j + r * nb) * es];
      }
    }
  }
  if (wsync) __syncwarp();
  else __syncthreads();
  if (valid) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = tid + b * nt;
      if (j < nb) {
        const int k = j % Ns;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          T2 w = tw[r * k * stride];
          if (dir > 0) w.y = -w.y;
          a[b][r] = cmul2(a[b][r], w);
        }
        Dft<R, T2, T>::run(a[b], dir);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) s[(base + r * Ns) * es] = a[b][r];
      }
    }
  }
  if (wsync) __syncwarp();
  else __syncthreads();
}

// Transform of a length-n signal whose element i sits at s[i * es] (es = 1: contiguous).
template <class T2, class T>
__device__ void fft_grp(T2* s, const AxisPlan& p, const T2* __restrict__ tw, T dir, int tid, bool valid, int es = 1,
                        bool wsync = false) {
  int Ns = 1;
  for (int st = 0; st < p.nst; ++st) {
    switch (p.rad[st]) {
      case 4: stage2<4, T2, T>(s, p.n, Ns, tw, dir, tid, p.nt, valid, es, wsync); break;
      case 2: stage2<2, T2, T>(s, p.n, Ns, tw, dir, tid, p.nt, valid, es, wsync); break;
      case 3: stage2<3, T2, T>(s, p.n, Ns, tw, dir, tid, p.nt, valid, es, wsync); break;
      default: stage2<5, T2, T>(s, p.n, Ns, tw, dir, tid, p.nt, valid, es, wsync); break;
    }
    Ns *= p.rad[st];
  }
}

// Block reduction of a value of type T; every thread gets the sum.
template <class T>
__device__ T block_sum_t(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = (threadIdx.x < nw) ? red[threadIdx.x] : T(0);
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[0] = t;
  }
  __syncthreads();
  const T r = red[0];
  __syncthreads();
  return r;
}

// Column pointers of a pair, with the stored-basis slot offset when kdev is given.
template <class T>
__device__ __forceinline__ const T* colptr(const T* X, int ldx, int c, const int* kdev, long long kstride, int koff) {
  const T* base = X;
  if (kdev) base += ((long long)(*kdev) + koff) * kstride;
  return base + (size_t)c * ldx;
}

struct PassArgs {
  int nx, ny, ncol;
  AxisPlan px, py;
  const int* active;
  const int* kdev;
  long long kstride;
};

// rows, forward: Z[p] = FFT_x(x_{2p} + i x_{2p+1}) row by row.
template <class T>
__global__ void __launch_bounds__(512) rows_fwd_kernel(PassArgs a, const T* __restrict__ X, int ldx,
                                                       const typename Cx<T>::t* __restrict__ twx,
                                                       typename Cx<T>::t* __restrict__ Z) {
  using T2 = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char smem2d[];
  T2* s = reinterpret_cast<T2*>(smem2d);
  const int p = blockIdx.y, c0 = 2 * p, c1 = c0 + 1;
  const bool act0 = !a.active || a.active[c0];
  const bool act1 = c1 < a.ncol && (!a.active || a.active[c1]);
  if (!act0 && !act1) return;
  const int rpc = blockDim.x / a.px.nt;
  const int g = threadIdx.x / a.px.nt, tid = threadIdx.x % a.px.nt;
  const int iy = blockIdx.x * rpc + g;
  const bool valid = g < rpc && iy < a.ny;
  const T* x0 = colptr(X, ldx, c0, a.kdev, a.kstride, 0);
  const T* x1 = colptr(X, ldx, c1, a.kdev, a.kstride, 0);
  T2* row = s + (size_t)g * a.nx;
  if (valid)
    for (int ix = tid; ix < a.nx; ix += a.px.nt) {
      const size_t e = (size_t)iy * a.nx + ix;
      row[ix] = mk<T2>(act0 ? x0[e] : T(0), act1 ? x1[e] : T(0));
    }
  __syncthreads();
  fft_grp<T2, T>(row, a.px, twx, T(-1), tid, valid);
  if (valid) {
    T2* z = Z + (size_t)p * a.nx * a.ny + (size_t)iy * a.nx;
    for (int ix = tid; ix < a.nx; ix += a.px.nt) z[ix] = row[ix];
  }
}

// cols: along y, forward FFT (flag 1), multiply by mult (flag 2), inverse FFT (flag 4).
template <class T>
__global__ void __launch_bounds__(512) cols_kernel(PassArgs a, int flags, const T* __restrict__ mult,
                                                   const typename Cx<T>::t* __restrict__ twy,
                                                   typename Cx<T>::t* __restrict__ Z, int nsig) {
  using T2 = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char smem2d[];
  T2* s = reinterpret_cast<T2*>(smem2d);
  const int p = blockIdx.y;
  if (a.active) {
    const int c0 = 2 * p, c1 = c0 + 1;
    if (!a.active[c0] && !(c1 < a.ncol && a.active[c1])) return;
  }
  if (p >= nsig) return;
  const int cpc = blockDim.x / a.py.nt;
  const int kx0 = blockIdx.x * cpc;
  T2* zp = Z + (size_t)p * a.nx * a.ny;
  for (int e = threadIdx.x; e < cpc * a.ny; e += blockDim.x) {
    const int iy = e / cpc, c = e % cpc;
    if (kx0 + c < a.nx) s[(size_t)c * a.ny + iy] = zp[(size_t)iy * a.nx + kx0 + c];
  }
  __syncthreads();
  const int g = threadIdx.x / a.py.nt, tid = threadIdx.x % a.py.nt;
  const int kx = kx0 + g;
  const bool valid = g < cpc && kx < a.nx;
  T2* col = s + (size_t)g * a.ny;
  if (flags & 1) fft_grp<T2, T>(col, a.py, twy, T(-1), tid, valid);
  if (flags & 2) {
    if (valid)
      for (int iy = tid; iy < a.ny; iy += a.py.nt) col[iy] = cscale2<T2, T>(col[iy], mult[(size_t)iy * a.nx + kx]);
    __syncthreads();
  }
  if (flags & 4) fft_grp<T2, T>(col, a.py, twy, T(1), tid, valid);
  for (int e = threadIdx.x; e < cpc * a.ny; e += blockDim.x) {
    const int iy = e / cpc, c = e % cpc;
    if (kx0 + c < a.nx) zp[(size_t)iy * a.nx + kx0 + c] = s[(size_t)c * a.ny + iy];
  }
}

// rows, inverse: z = IFFT_x(Z[p]) / N.  mode 0: Y_j = Re/Im z + (V - s_j) x_j (V, shift nullable)
// and alpha_j += x_j . Y_j when alpha is given; mode 1: outA[:, p] = scale Re z, outB[:, p] =
// scale Im z (signals that are not column pairs: perturbation potentials).
template <class T>
__global__ void __launch_bounds__(512) rows_inv_kernel(PassArgs a, int mode, const typename Cx<T>::t* __restrict__ twx,
                                                       const typename Cx<T>::t* __restrict__ Z, const T* __restrict__ X,
                                                       int ldx, const T* __restrict__ V, const T* __restrict__ shift,
                                                       T* __restrict__ Y, int ldy, T* __restrict__ alpha, T scale,
                                                       T* __restrict__ outA, T* __restrict__ outB, int nsig) {
  using T2 = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char smem2d[];
  __shared__ T red[32];
  T2* s = reinterpret_cast<T2*>(smem2d);
  const int p = blockIdx.y, c0 = 2 * p, c1 = c0 + 1;
  bool act0 = true, act1 = true;
  if (mode == 0) {
    act0 = !a.active || a.active[c0];
    act1 = c1 < a.ncol && (!a.active || a.active[c1]);
    if (!act0 && !act1) return;
  } else if (p >= nsig) {
    return;
  }
  const int rpc = blockDim.x / a.px.nt;
  const int g = threadIdx.x / a.px.nt, tid = threadIdx.x % a.px.nt;
  const int iy = blockIdx.x * rpc + g;
  const bool valid = g < rpc && iy < a.ny;
  T2* row = s + (size_t)g * a.nx;
  const T2* zr = Z + (size_t)p * a.nx * a.ny + (size_t)iy * a.nx;
  if (valid)
    for (int ix = tid; ix < a.nx; ix += a.px.nt) row[ix] = zr[ix];
  __syncthreads();
  fft_grp<T2, T>(row, a.px, twx, T(1), tid, valid);
  const size_t N = (size_t)a.nx * a.ny;
  if (mode == 1) {
    if (valid)
      for (int ix = tid; ix < a.nx; ix += a.px.nt) {
        const size_t e = (size_t)iy * a.nx + ix;
        if (outA) outA[(size_t)p * N + e] = row[ix].x * scale;
        if (outB) outB[(size_t)p * N + e] = row[ix].y * scale;
      }
    return;
  }
  const T invN = T(1) / T(N);
  const T* x0 = colptr(X, ldx, c0, a.kdev, a.kstride, 0);
  const T* x1 = colptr(X, ldx, c1, a.kdev, a.kstride, 0);
  const T sh0 = (shift && act0) ? shift[c0] : T(0);
  const T sh1 = (shift && act1) ? shift[c1] : T(0);
  T dot0 = 0, dot1 = 0;
  if (valid)
    for (int ix = tid; ix < a.nx; ix += a.px.nt) {
      const size_t e = (size_t)iy * a.nx + ix;
      const T v = V ? V[e] : T(0);
      const T xa0 = act0 ? x0[e] : T(0), xa1 = act1 ? x1[e] : T(0);
      const T y0 = row[ix].x * invN + (v - sh0) * xa0;
      const T y1 = row[ix].y * invN + (v - sh1) * xa1;
      dot0 += xa0 * y0;
      dot1 += xa1 * y1;
      if (act0) Y[(size_t)c0 * ldy + e] = y0;
      if (act1) Y[(size_t)c1 * ldy + e] = y1;
    }
  if (alpha) {
    dot0 = block_sum_t(dot0, red);
    dot1 = block_sum_t(dot1, red);
    if (threadIdx.x == 0) {
      if (act0) atomicAdd(&alpha[c0], dot0);
      if (act1) atomicAdd(&alpha[c1], dot1);
    }
  }
}

// Whole 2D transform of one column pair in shared memory (one CTA per pair; the ny x nx signal is
// stored with a row stride of nx + 1 to spread column accesses over the banks): row FFTs, column
// FFTs, symbol, inverse column and row FFTs, then y = z / N + (V - s) x, alpha = x . y within the
// CTA, and in the Lanczos form P = y - alpha x - beta x_prev -- the 1D kernel's structure, for
// grids whose signal fits in shared memory.
template <class T>
__global__ void __launch_bounds__(512) fused2d_kernel(PassArgs a, const T* __restrict__ X, int ldx,
                                                      const typename Cx<T>::t* __restrict__ twx,
                                                      const typename Cx<T>::t* __restrict__ twy,
                                                      const T* __restrict__ mult, const T* __restrict__ V,
                                                      const T* __restrict__ shift, T* __restrict__ Y, int ldy,
                                                      T* __restrict__ alpha, const T* __restrict__ Xp, int ldp,
                                                      const T* __restrict__ beta) {
  using T2 = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char smem2d[];
  __shared__ T red[32];
  T2* s = reinterpret_cast<T2*>(smem2d);
  const int p = blockIdx.x, c0 = 2 * p, c1 = c0 + 1;
  const bool act0 = !a.active || a.active[c0];
  const bool act1 = c1 < a.ncol && (!a.active || a.active[c1]);
  if (!act0 && !act1) return;
  const int nx = a.nx, ny = a.ny, ld = nx + 1;
  const int N = nx * ny;
  const T* x0 = colptr(X, ldx, c0, a.kdev, a.kstride, 0);
  const T* x1 = colptr(X, ldx, c1, a.kdev, a.kstride, 0);
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    const int ix = e % nx, iy = e / nx;
    s[iy * ld + ix] = mk<T2>(act0 ? x0[e] : T(0), act1 ? x1[e] : T(0));
  }
  __syncthreads();
  if (a.px.nt == 32 && a.py.nt == 32) {
    // one warp per row / column, each warp through its own signals without CTA barriers
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int iy = warp; iy < ny; iy += nw) fft_grp<T2, T>(s + (size_t)iy * ld, a.px, twx, T(-1), lane, true, 1, true);
    __syncthreads();
    for (int kx = warp; kx < nx; kx += nw) {
      T2* col = s + kx;
      fft_grp<T2, T>(col, a.py, twy, T(-1), lane, true, ld, true);
      for (int iy = lane; iy < ny; iy += 32) col[iy * ld] = cscale2<T2, T>(col[iy * ld], mult[iy * nx + kx]);
      __syncwarp();
      fft_grp<T2, T>(col, a.py, twy, T(1), lane, true, ld, true);
    }
    __syncthreads();
    for (int iy = warp; iy < ny; iy += nw) fft_grp<T2, T>(s + (size_t)iy * ld, a.px, twx, T(1), lane, true, 1, true);
    __syncthreads();
  } else {
    const int gx = blockDim.x / a.px.nt, gy = blockDim.x / a.py.nt;
    const int rx = threadIdx.x / a.px.nt, tx = threadIdx.x % a.px.nt;
    const int ry = threadIdx.x / a.py.nt, ty = threadIdx.x % a.py.nt;
    for (int r0 = 0; r0 < ny; r0 += gx) {
      const int iy = r0 + rx;
      fft_grp<T2, T>(s + (size_t)(iy < ny ? iy : 0) * ld, a.px, twx, T(-1), tx, rx < gx && iy < ny);
    }
    for (int q0 = 0; q0 < nx; q0 += gy) {
      const int kx = q0 + ry;
      const bool valid = ry < gy && kx < nx;
      T2* col = s + (valid ? kx : 0);
      fft_grp<T2, T>(col, a.py, twy, T(-1), ty, valid, ld);
      if (valid)
        for (int iy = ty; iy < ny; iy += a.py.nt) col[iy * ld] = cscale2<T2, T>(col[iy * ld], mult[iy * nx + kx]);
      __syncthreads();
      fft_grp<T2, T>(col, a.py, twy, T(1), ty, valid, ld);
    }
    for (int r0 = 0; r0 < ny; r0 += gx) {
      const int iy = r0 + rx;
      fft_grp<T2, T>(s + (size_t)(iy < ny ? iy : 0) * ld, a.px, twx, T(1), tx, rx < gx && iy < ny);
    }
  }
  const T invN = T(1) / T(N);
  const T sh0 = (shift && act0) ? shift[c0] : T(0);
  const T sh1 = (shift && act1) ? shift[c1] : T(0);
  T dot0 = 0, dot1 = 0;
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    const int ix = e % nx, iy = e / nx;
    const T v = V ? V[e] : T(0);
    const T xa0 = act0 ? x0[e] : T(0), xa1 = act1 ? x1[e] : T(0);
    const T2 z = s[iy * ld + ix];
    const T y0 = z.x * invN + (v - sh0) * xa0;
    const T y1 = z.y * invN + (v - sh1) * xa1;
    dot0 += xa0 * y0;
    dot1 += xa1 * y1;
    s[iy * ld + ix] = mk<T2>(y0, y1);
  }
  const bool lanczos = Xp != nullptr;
  if (alpha || lanczos) {
    dot0 = block_sum_t(dot0, red);
    dot1 = block_sum_t(dot1, red);
    if (alpha && threadIdx.x == 0) {
      if (act0) alpha[c0] = dot0;
      if (act1) alpha[c1] = dot1;
    }
  }
  __syncthreads();
  const T b0 = (lanczos && act0) ? beta[c0] : T(0), b1 = (lanczos && act1) ? beta[c1] : T(0);
  const T* p0 = lanczos ? colptr(Xp, ldp, c0, a.kdev, a.kstride, -1) : nullptr;
  const T* p1 = lanczos ? colptr(Xp, ldp, c1, a.kdev, a.kstride, -1) : nullptr;
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    const int ix = e % nx, iy = e / nx;
    const T2 yv = s[iy * ld + ix];
    if (lanczos) {
      if (act0) Y[(size_t)c0 * ldy + e] = yv.x - dot0 * x0[e] - b0 * p0[e];
      if (act1) Y[(size_t)c1 * ldy + e] = yv.y - dot1 * x1[e] - b1 * p1[e];
    } else {
      if (act0) Y[(size_t)c0 * ldy + e] = yv.x;
      if (act1) Y[(size_t)c1 * ldy + e] = yv.y;
    }
  }
}

// P = Y - alpha x - beta x_prev for the active columns (Lanczos three-term recurrence)
template <class T>
__global__ void lanczos2d_kernel(int N, int ncol, const int* __restrict__ active, const T* __restrict__ X, int ldx,
                                 const T* __restrict__ Xp, int ldp, const int* __restrict__ kdev, long long kstride,
                                 const T* __restrict__ alpha, const T* __restrict__ beta, T* __restrict__ Y,
                                 int ldy) {
  const int c = blockIdx.y;
  if (c >= ncol || (active && !active[c])) return;
  const T* x = colptr(X, ldx, c, kdev, kstride, 0);
  const T* xp = colptr(Xp, ldp, c, kdev, kstride, -1);
  const T al = alpha[c], be = beta[c];
  T* y = Y + (size_t)c * ldy;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x)
    y[e] = y[e] - al * x[e] - be * xp[e];
}

__global__ void zero_kernel_d(int n, double* p) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0.0;
}
__global__ void zero_kernel_f(int n, float* p) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0.f;
}

// ---- perturbation potentials (2D) -----------------------------------------------------------
// One complex spectrum per output column; the column is the real part of its inverse transform.
// (Packing two outputs into one complex signal, as the 1D kernel does, would mix them here: on a
// grid with an even number of points the Nyquist row or column of the other axis breaks the
// Hermitian symmetry of the pseudocharge coefficients, so each inverse transform has a small
// imaginary part, which the real part discards.)
// kind 0: g_{I,a} = Khat (-i k_a) m^ (signal 2I + a); kind 1: b_{I,a} = (-i k_a) m^;
// kind 2: d2V_I, signal 3I + c, c = 0: -k_x^2 Khat m^, 1: -k_x k_y Khat m^ (odd factors), 2: -k_y^2 Khat m^.
struct Atoms2D {
  const double* R;  // 2 per atom (x, y)
  const double* Z;
  const double* sig;
  int nA;
};

__global__ void pert_spectra_2d(int nx, int ny, double Lx, double Ly, double kappa, double scale, Atoms2D at,
                                int kind, double2* __restrict__ Z) {
  const size_t N = (size_t)nx * ny;
  const int per = (kind == 2) ? 3 : 2;
  const int nsig = per * at.nA;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N * nsig; e += (size_t)gridDim.x * blockDim.x) {
    const int sidx = (int)(e / N);
    const size_t q = e % N;
    const int ix = (int)(q % nx), iy = (int)(q / nx);
    const int I = sidx / per, comp = sidx % per;
    const int mx = (ix < (nx + 1) / 2) ? ix : ix - nx;
    const int my = (iy < (ny + 1) / 2) ? iy : iy - ny;
    const double kx = 2.0 * M_PI * mx / Lx, ky = 2.0 * M_PI * my / Ly;
    const double kxo = (2 * ix == nx) ? 0.0 : kx, kyo = (2 * iy == ny) ? 0.0 : ky;
    const double k2 = kx * kx + ky * ky;
    const double khat = 4.0 * M_PI * scale / (k2 + kappa * kappa);
    const double Rx = at.R[2 * I], Ry = at.R[2 * I + 1], sg = at.sig[I];
    const double amp = -at.Z[I] * exp(-0.5 * sg * sg * k2);
    double t = fmod((double)mx * (Rx / Lx) + (double)my * (Ry / Ly), 1.0);  // phase -2 pi t
    double sn, cs;
    sincospi(-2.0 * t, &sn, &cs);
    const double2 m = make_double2(amp * cs, amp * sn);  // pseudocharge coefficient
    double2 z;
    if (kind < 2) {
      const double ka = comp == 0 ? kxo : kyo;
      const double f = (kind == 0) ? khat * ka : ka;
      z = make_double2(f * m.y, -f * m.x);  // -i f m^
    } else {
      const double f = (comp == 0) ? -kx * kx * khat : (comp == 1) ? -kxo * kyo * khat : -ky * ky * khat;
      z = make_double2(f * m.x, f * m.y);
    }
    Z[e] = z;
  }
}

// Hessian blocks of the periodic point-charge Yukawa energy for every ordered pair I != J:
// H[(I nA + J) * 4 + 2a + b] = d^2 K_per(d) / dd_a dd_b at d = R_I - R_J (see the file header).
__global__ void ion_pair_hessian_2d(int nA, const double* __restrict__ R, double Lx, double Ly, double kappa,
                                    double scale, double sg, int Mx, int My, double* __restrict__ H) {
  __shared__ double red[32];
  const int pair = blockIdx.x;
  const int I = pair / nA, J = pair % nA;
  if (I == J) {
    if (threadIdx.x < 4) H[(size_t)pair * 4 + threadIdx.x] = 0.0;
    return;
  }
  const double dx = R[2 * I] - R[2 * J], dy = R[2 * I + 1] - R[2 * J + 1];
  double hxx = 0, hxy = 0, hyy = 0;
  const int nkx = 2 * Mx + 1, nky = 2 * My + 1;
  for (int e = threadIdx.x; e < nkx * nky; e += blockDim.x) {
    const int mx = e % nkx - Mx, my = e / nkx - My;
    const double kx = 2.0 * M_PI * mx / Lx, ky = 2.0 * M_PI * my / Ly;
    const double k2 = kx * kx + ky * ky;
    const double w = 4.0 * M_PI * scale / (k2 + kappa * kappa) * exp(-sg * sg * k2);
    double t = fmod((double)mx * (dx / Lx) + (double)my * (dy / Ly), 1.0);
    const double c = cospi(2.0 * t) * w;
    hxx -= kx * kx * c;
    hxy -= kx * ky * c;
    hyy -= ky * ky * c;
  }
  const double f = exp(-sg * sg * kappa * kappa) / (Lx * Ly);
  hxx = block_sum_t(hxx, red) * f;
  hxy = block_sum_t(hxy, red) * f;
  hyy = block_sum_t(hyy, red) * f;
  if (threadIdx.x == 0) {
    double* o = H + (size_t)pair * 4;
    o[0] = hxx;
    o[1] = hxy;
    o[2] = hxy;
    o[3] = hyy;
  }
}

// D (row-major, n = 2 nA) = (Hm + local blocks + ion Hessian) / sqrt(M_I M_J)
__global__ void assemble_dmat_2d(int nA, const double* __restrict__ Hm, const double* __restrict__ dv,
                                 const double* __restrict__ Hp, const double* __restrict__ Z,
                                 const double* __restrict__ M, double* __restrict__ D) {
  const int n = 2 * nA;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int p = e / n, q = e % n;
    const int I = p / 2, a = p % 2, J = q / 2, b = q % 2;
    double v = Hm[p + (size_t)q * n];
    if (I == J) {
      // local term: dv[3I + {0: xx, 1: xy, 2: yy}]
      v += dv[3 * I + a + b];
      for (int K = 0; K < nA; ++K)
        if (K != I) v += Z[I] * Z[K] * Hp[((size_t)I * nA + K) * 4 + 2 * a + b];
    } else {
      v -= Z[I] * Z[J] * Hp[((size_t)I * nA + J) * 4 + 2 * a + b];
    }
    D[(size_t)p * n + q] = v / sqrt(M[I] * M[J]);
  }
}

template <class T>
AxisPlan axis_plan(const FftPlan& fp) {
  AxisPlan p{};
  p.n = fp.n;
  p.nst = fp.nst;
  for (int i = 0; i < fp.nst && i < 16; ++i) p.rad[i] = fp.rad[i];
  p.nt = fp.threads;
  return p;
}

int grid_cap(size_t total, int cap = 65535) {
  size_t b = (total + 255) / 256;
  if (b > (size_t)cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

// Threads per transform of one axis: enough for the butterflies of every stage, a multiple of 32.
bool make_axis_plan(int n, FftPlan* plan) {
  if (n < 8 || n > 4096) return false;
  FftPlan p{};
  p.n = n;
  int m = n;
  auto push = [&](int r) { p.rad[p.nst++] = r; m /= r; };
  while (m % 4 == 0) push(4);
  while (m % 2 == 0) push(2);
  while (m % 3 == 0) push(3);
  while (m % 5 == 0) push(5);
  if (m != 1 || p.nst > 16) return false;
  int t = 1;
  for (int s = 0; s < p.nst; ++s) {
    const int r = p.rad[s];
    const int mb = (r == 2) ? 4 : (r == 3) ? 4 : (r == 4) ? 3 : 2;
    const int need = (n / r + mb - 1) / mb;
    if (need > t) t = need;
  }
  t = (t + 31) / 32 * 32;
  if (t > 512) return false;
  p.threads = t;
  *plan = p;
  return true;
}

template <class T>
acp_status spectral2d_apply(acp_ctx* ctx, const T* X, int ldx, int ncol, const T* mult, const T* V,
                            const T* shift_d, T* Y, int ldy, T* alpha_d, const int* active_d, const T* Xp, int ldp,
                            const T* beta_d, const typename Cx<T>::t* twx, const typename Cx<T>::t* twy,
                            const int* kdev, long long kstride) {
  using T2 = typename Cx<T>::t;
  if (ncol <= 0) return ACP_OK;
  {
    // the row and column passes may need more than the default 48 KB of dynamic shared memory
    std::lock_guard<std::mutex> lock(device_mutex());
    static int configured_device = -1;
    if (configured_device != ctx->device) {
      ACP_TRY(raise_smem_limit(ctx, reinterpret_cast<const void*>(rows_fwd_kernel<double>)));
      ACP_TRY(raise_smem_limit(ctx, reinterpret_cast<const void*>(rows_fwd_kernel<float>)));
      ACP_TRY(raise_smem_limit(ctx, reinterpret_cast<const void*>(cols_kernel<double>)));
      ACP_TRY(raise_smem_limit(ctx, reinterpret_cast<const void*>(cols_kernel<float>)));
      ACP_TRY(raise_smem_limit(ctx, reinterpret_cast<const void*>(rows_inv_kernel<double>)));
      ACP_TRY(raise_smem_limit(ctx, reinterpret_cast<const void*>(rows_inv_kernel<float>)));
      ACP_TRY(raise_smem_limit(ctx, reinterpret_cast<const void*>(fused2d_kernel<double>)));
      ACP_TRY(raise_smem_limit(ctx, reinterpret_cast<const void*>(fused2d_kernel<float>)));
      configured_device = ctx->device;
    }
  }
  const int nx = ctx->nx, ny = ctx->ny;
  const size_t N = (size_t)nx * ny;
  const int npairs = (ncol + 1) / 2;
  T2* Z = nullptr;
  ACP_TRY(ws(ctx, sizeof(T) == 8 ? "z2d64" : "z2d32", (size_t)npairs * N, &Z));
  PassArgs a{};
  a.nx = nx;
  a.ny = ny;
  a.ncol = ncol;
  a.px = axis_plan<T>(ctx->plan_x);
  a.py = axis_plan<T>(ctx->plan_y);
  a.active = active_d;
  a.kdev = kdev;
  a.kstride = kstride;
  const bool lanczos = Xp != nullptr;
  const int rpc = 512 / a.px.nt < 16 ? 512 / a.px.nt : 16;  // rows per CTA
  const int cpc = 512 / a.py.nt < 16 ? 512 / a.py.nt : 16;  // columns per CTA
  const dim3 grow((ny + rpc - 1) / rpc, npairs), gcol((nx + cpc - 1) / cpc, npairs);
  const double lg = std::log2((double)N);
  const size_t fused_smem = (size_t)ny * (nx + 1) * sizeof(T2);
  if (ctx->opt.fft2d_passes == 0 && fused_smem + 1024 <= ctx->smem_optin) {
    cudaEvent_t evf = prof_begin(ctx);
    ::acp::note_launch(ctx);
    fused2d_kernel<T><<<npairs, 512, fused_smem, ctx->stream>>>(a, X, ldx, twx, twy, mult, V, shift_d, Y, ldy,
                                                                alpha_d, Xp, ldp, beta_d);
    ACP_LAUNCH(ctx);
    prof_end(ctx, sizeof(T) == 8 ? "spectral" : "spectral32", evf, 2.0 * 5.0 * N * lg * npairs + 6.0 * (double)N * ncol,
             (double)sizeof(T) * N * ncol * (lanczos ? 3.0 : 2.0));
    return ACP_OK;
  }
  if (alpha_d) {
    ::acp::note_launch(ctx);
    if (sizeof(T) == 8) zero_kernel_d<<<grid_cap(ncol), 256, 0, ctx->stream>>>(ncol, reinterpret_cast<double*>(alpha_d));
    else zero_kernel_f<<<grid_cap(ncol), 256, 0, ctx->stream>>>(ncol, reinterpret_cast<float*>(alpha_d));
    ACP_LAUNCH(ctx);
  }
  cudaEvent_t ev0 = prof_begin(ctx);
  ::acp::note_launch(ctx);
  rows_fwd_kernel<T><<<grow, rpc * a.px.nt, rpc * nx * sizeof(T2), ctx->stream>>>(a, X, ldx, twx, Z);
  ACP_LAUNCH(ctx);
  ::acp::note_launch(ctx);
  cols_kernel<T><<<gcol, cpc * a.py.nt, cpc * ny * sizeof(T2), ctx->stream>>>(a, 7, mult, twy, Z, npairs);
  ACP_LAUNCH(ctx);
  ::acp::note_launch(ctx);
  rows_inv_kernel<T><<<grow, rpc * a.px.nt, rpc * nx * sizeof(T2), ctx->stream>>>(
      a, 0, twx, Z, X, ldx, V, shift_d, Y, ldy, (alpha_d || lanczos) ? alpha_d : nullptr, T(1), nullptr, nullptr,
      npairs);
  ACP_LAUNCH(ctx);
  if (lanczos) {
    ::acp::note_launch(ctx);
    lanczos2d_kernel<T><<<dim3(grid_cap(N, 64), ncol), 256, 0, ctx->stream>>>((int)N, ncol, active_d, X, ldx, Xp, ldp,
                                                                           kdev, kstride, alpha_d, beta_d, Y, ldy);
    ACP_LAUNCH(ctx);
  }
  prof_end(ctx, sizeof(T) == 8 ? "spectral" : "spectral32", ev0, 2.0 * 5.0 * N * lg * npairs + 6.0 * (double)N * ncol,
           (double)sizeof(T) * N * ncol * (lanczos ? 3.0 : 2.0));
  return ACP_OK;
}

acp_status spectral2d_apply_f64(acp_ctx* ctx, const double* X, int ldx, int ncol, const double* mult, const double* V,
                                const double* shift_d, double* Y, int ldy, double* alpha_d, const int* active_d,
                                const double* Xp, int ldp, const double* beta_d) {
  return spectral2d_apply<double>(ctx, X, ldx, ncol, mult, V, shift_d, Y, ldy, alpha_d, active_d, Xp, ldp, beta_d,
                                  ctx->d_twx, ctx->d_twy, nullptr, 0);
}

acp_status spectral2d_apply_f32(acp_ctx* ctx, const float* X, int ldx, int ncol, const float* mult, const float* V,
                                const float* shift_d, float* Y, int ldy, float* alpha_d, const int* active_d,
                                const float* Xp, int ldp, const float* beta_d, const float2* twx, const float2* twy,
                                const int* kdev, long long kstride) {
  return spectral2d_apply<float>(ctx, X, ldx, ncol, mult, V, shift_d, Y, ldy, alpha_d, active_d, Xp, ldp, beta_d, twx,
                                 twy, kdev, kstride);
}

// Perturbation potentials on the 2D grid: G, B (N x 2 nA, column 2I + a) and D2 (N x 3 nA, columns
// 3I + {xx, xy, yy}); R_d holds (x, y) per atom.  Any output may be null.
acp_status perturbations_2d(acp_ctx* ctx, int nA, const double* R_d, const double* Z_d, const double* sig_d,
                            double* G, double* B, double* D2) {
  if (nA <= 0) return ACP_OK;
  const int nx = ctx->nx, ny = ctx->ny;
  const size_t N = (size_t)nx * ny;
  double2* Zs = nullptr;
  ACP_TRY(ws(ctx, "pt2_z", 3 * (size_t)nA * N, &Zs));
  Atoms2D at{R_d, Z_d, sig_d, nA};
  PassArgs a{};
  a.nx = nx;
  a.ny = ny;
  a.ncol = 6 * nA;
  a.px = axis_plan<double>(ctx->plan_x);
  a.py = axis_plan<double>(ctx->plan_y);
  const int rpc = 512 / a.px.nt < 16 ? 512 / a.px.nt : 16;
  const int cpc = 512 / a.py.nt < 16 ? 512 / a.py.nt : 16;
  const double invA = 1.0 / (ctx->Lx * ctx->Ly);
  double* outs[3] = {G, B, D2};
  for (int kind = 0; kind < 3; ++kind) {
    if (!outs[kind]) continue;
    const int nsig = (kind == 2 ? 3 : 2) * nA;
    const dim3 grow((ny + rpc - 1) / rpc, nsig), gcol((nx + cpc - 1) / cpc, nsig);
    ::acp::note_launch(ctx);
    pert_spectra_2d<<<grid_cap(N * nsig), 256, 0, ctx->stream>>>(nx, ny, ctx->Lx, ctx->Ly, ctx->kappa, ctx->scale, at,
                                                                kind, Zs);
    ACP_LAUNCH(ctx);
    ::acp::note_launch(ctx);
    cols_kernel<double><<<gcol, cpc * a.py.nt, cpc * ny * sizeof(double2), ctx->stream>>>(a, 4, nullptr, ctx->d_twy,
                                                                                          Zs, nsig);
    ACP_LAUNCH(ctx);
    ::acp::note_launch(ctx);
    rows_inv_kernel<double><<<grow, rpc * a.px.nt, rpc * nx * sizeof(double2), ctx->stream>>>(
        a, 1, ctx->d_twx, Zs, nullptr, 0, nullptr, nullptr, nullptr, 0, nullptr, invA, outs[kind], nullptr, nsig);
    ACP_LAUNCH(ctx);
  }
  return ACP_OK;
}

// Ion-ion Hessian blocks (nA * nA * 4) of the periodic point-charge Yukawa energy; R_h on the host
// (for the smallest pair distance, which sets the Gaussian split), R_d on the device.
acp_status ion_hessian_2d(acp_ctx* ctx, int nA, const double* R_h, const double* R_d, double* Hp) {
  double dmin = 1e300;
  for (int I = 0; I < nA; ++I)
    for (int J = I + 1; J < nA; ++J) {
      double dx = std::fmod(R_h[2 * I] - R_h[2 * J], ctx->Lx), dy = std::fmod(R_h[2 * I + 1] - R_h[2 * J + 1], ctx->Ly);
      dx -= ctx->Lx * std::nearbyint(dx / ctx->Lx);
      dy -= ctx->Ly * std::nearbyint(dy / ctx->Ly);
      dmin = std::fmin(dmin, std::hypot(dx, dy));
    }
  if (!(dmin > 1e-6)) dmin = std::fmin(ctx->Lx, ctx->Ly);
  const double sg = dmin / 12.0;
  const double kmax = 6.5 / sg;
  const int Mx = (int)std::ceil(kmax * ctx->Lx / (2.0 * M_PI)), My = (int)std::ceil(kmax * ctx->Ly / (2.0 * M_PI));
  ::acp::note_launch(ctx);
  ion_pair_hessian_2d<<<nA * nA, 256, 0, ctx->stream>>>(nA, R_d, ctx->Lx, ctx->Ly, ctx->kappa, ctx->scale, sg, Mx, My,
                                                       Hp);
  ACP_LAUNCH(ctx);
  return ACP_OK;
}

acp_status assemble_2d(acp_ctx* ctx, int nA, const double* Hm, const double* dv, const double* Hp, const double* Z_d,
                       const double* M_d, double* D) {
  ::acp::note_launch(ctx);
  assemble_dmat_2d<<<grid_cap((size_t)4 * nA * nA), 256, 0, ctx->stream>>>(nA, Hm, dv, Hp, Z_d, M_d, D);
  ACP_LAUNCH(ctx);
  return ACP_OK;
}

}  // namespace acp
