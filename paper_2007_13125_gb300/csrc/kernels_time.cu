// Time-axis kernels of one WR sweep (Algorithm 1 / Algorithm 2, steps 1 and 3), the
// all-at-once residual, the CQ Toeplitz product, the right-hand side and conversions.
//
// Tiling of the time kernels: one CTA owns 2C spatial points and all N time levels.
// Point m0 + c is the real part and point m0 + C + c the imaginary part of complex
// column c, so one complex N-point FFT transforms two real time series; the half
// spectra j = 0..N/2 of both are separated afterwards with the conjugate symmetry of
// real data. Global loads and stores are coalesced over consecutive points.
#include "ff.cuh"
#include "fft.cuh"
#include "pint_internal.h"

namespace pint {

__device__ __forceinline__ ff ldff(const float* hi, const float* lo, size_t idx) {
  ff r;
  r.hi = __ldg(hi + idx);
  r.lo = __ldg(lo + idx);
  return r;
}

__device__ __forceinline__ void block_reduce_add2(double a, double b, double* out) {
  __shared__ double red[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { red[0][w] = a; red[1][w] = b; }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    a = l < nw ? red[0][l] : 0.0;
    b = l < nw ? red[1][l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (l == 0) {
      atomicAdd(out, a);
      atomicAdd(out + 1, b);
    }
  }
}

// ---------------------------------------------------------------------------
// MIXED: residual (double-float) + kappa scaling + forward DFT along time
// ---------------------------------------------------------------------------
size_t resid_fwd_smem(int N, int C) { return sizeof(float2) * ((size_t)N * C + N); }

__global__ void __launch_bounds__(kThreads) k_resid_fwd(ResidFwdArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M;
  float2* X = reinterpret_cast<float2*>(smraw);
  float2* tw = X + (size_t)N * C;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.tw[i];

  const int m0 = blockIdx.x * 2 * C;
  const int c = threadIdx.x % C;
  const int nch = blockDim.x / C;
  const int tc = threadIdx.x / C;
  const int Lc = N / nch;
  const int i0 = tc * Lc;
  const int k = a.k;
  ff cw[kMaxK + 1];
#pragma unroll
  for (int j = 0; j <= kMaxK; ++j) { cw[j].hi = a.c_hi[j]; cw[j].lo = a.c_lo[j]; }
  const ff gx = {a.gx_hi, a.gx_lo}, gy = {a.gy_hi, a.gy_lo};

  for (int half = 0; half < 2; ++half) {
    const int m = m0 + half * C + c;
    const bool valid = m < M;
    const int x = valid ? m % a.mx : 0;
    ff win[kMaxK];
#pragma unroll
    for (int j = 0; j < kMaxK; ++j) {
      const int lev = i0 - 1 - j;
      win[j].hi = 0.f; win[j].lo = 0.f;
      if (j < k && valid && lev >= 0) win[j] = ldff(a.Uhi, a.Ulo, (size_t)lev * M + m);
    }
    for (int i = i0; i < i0 + Lc; ++i) {
      float r = 0.f;
      if (valid) {
        const size_t idx = (size_t)i * M + m;
        const ff u = ldff(a.Uhi, a.Ulo, idx);
        ff_acc acc;
        acc.init(ldff(a.Fhi, a.Flo, idx));
        if (a.y) acc.sub(ff_from_double(__ldg(a.y + idx)));
        acc.fma_term(cw[0], u, -1.f);
#pragma unroll
        for (int j = 1; j <= kMaxK; ++j)
          if (j <= k) acc.fma_term(cw[j], win[j - 1], -1.f);
        if (x > 0) acc.fma_term(gx, ldff(a.Uhi, a.Ulo, idx - 1), 1.f);
        if (x < a.mx - 1) acc.fma_term(gx, ldff(a.Uhi, a.Ulo, idx + 1), 1.f);
        if (a.dim == 2) {
          if (m >= a.mx) acc.fma_term(gy, ldff(a.Uhi, a.Ulo, idx - a.mx), 1.f);
          if (m + a.mx < M) acc.fma_term(gy, ldff(a.Uhi, a.Ulo, idx + a.mx), 1.f);
        }
        r = acc.value() * __ldg(a.s + i);
#pragma unroll
        for (int j = kMaxK - 1; j > 0; --j) win[j] = win[j - 1];
        win[0] = u;
      }
      if (half == 0) X[(size_t)i * C + c].x = r;
      else X[(size_t)i * C + c].y = r;
    }
  }
  __syncthreads();
  fft_forward(X, C, C, N, tw);

  const int J = N / 2 + 1;
  for (int it = threadIdx.x; it < J * C; it += blockDim.x) {
    const int cc = it % C, j = it / C;
    const float2 Zj = X[(size_t)fft_pos(j, N) * C + cc];
    const float2 Zn = X[(size_t)fft_pos((N - j) & (N - 1), N) * C + cc];
    const float2 A = make_float2(0.5f * (Zj.x + Zn.x), 0.5f * (Zj.y - Zn.y));
    const float2 B = make_float2(0.5f * (Zj.y + Zn.y), -0.5f * (Zj.x - Zn.x));
    const int ma = m0 + cc, mb = m0 + C + cc;
    if (ma < M) a.S[(size_t)j * M + ma] = A;
    if (mb < M) a.S[(size_t)j * M + mb] = B;
  }
}

// ---------------------------------------------------------------------------
// Load a half spectrum (two real columns per complex column) into permuted order
// ---------------------------------------------------------------------------
template <typename V>
__device__ __forceinline__ void load_half_spectrum(V* X, const V* S, int N, int M, int C, int m0) {
  const int J = N / 2 + 1;
  for (int it = threadIdx.x; it < J * C; it += blockDim.x) {
    const int cc = it % C, j = it / C;
    const int ma = m0 + cc, mb = m0 + C + cc;
    V A, B;
    A.x = 0; A.y = 0; B = A;
    if (ma < M) A = S[(size_t)j * M + ma];
    if (mb < M) B = S[(size_t)j * M + mb];
    X[(size_t)fft_pos(j, N) * C + cc] = mk(A.x - B.y, A.y + B.x);                 // A + iB
    if (j > 0 && j < N / 2)
      X[(size_t)fft_pos(N - j, N) * C + cc] = mk(A.x + B.y, B.x - A.y);           // conj(A) + i conj(B)
  }
}

// ---------------------------------------------------------------------------
// MIXED: inverse DFT + unscale + U += c (double-float) + norms
// ---------------------------------------------------------------------------
size_t inv_upd_smem(int N, int C) { return sizeof(float2) * ((size_t)N * C + N); }

__global__ void __launch_bounds__(kThreads) k_inv_upd(InvUpdArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M;
  float2* X = reinterpret_cast<float2*>(smraw);
  float2* tw = X + (size_t)N * C;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.tw[i];
  const int m0 = blockIdx.x * 2 * C;
  load_half_spectrum(X, a.S, N, M, C, m0);
  __syncthreads();
  fft_inverse(X, C, C, N, tw);

  const int c = threadIdx.x % C;
  const int nch = blockDim.x / C;
  const int tc = threadIdx.x / C;
  const int Lc = N / nch;
  double sc = 0.0, su = 0.0;
  for (int half = 0; half < 2; ++half) {
    const int m = m0 + half * C + c;
    if (m >= M) continue;
    float pc = 0.f, pu = 0.f;
    for (int i = tc * Lc; i < (tc + 1) * Lc; ++i) {
      const float2 z = X[(size_t)i * C + c];
      const float cval = (half ? z.y : z.x) * __ldg(a.inv_s + i);
      const size_t idx = (size_t)i * M + m;
      ff u = {a.Uhi[idx], a.Ulo[idx]};
      u = ff_add_f(u, cval);
      a.Uhi[idx] = u.hi;
      a.Ulo[idx] = u.lo;
      pc = fmaf(cval, cval, pc);
      pu = fmaf(u.hi, u.hi, pu);
    }
    sc += pc;
    su += pu;
  }
  block_reduce_add2(sc, su, a.norms);
}

// ---------------------------------------------------------------------------
// FP64 / FP32 direct form (Algorithm 1/2 as printed): F_{m-1} -> scale -> DFT
// ---------------------------------------------------------------------------
template <typename T> size_t direct_smem(int N, int C) {
  return sizeof(typename c2<T>::t) * ((size_t)N * C + N);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_direct_fwd(DirectFwdArgs<T> a) {
  using V = typename c2<T>::t;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M;
  V* X = reinterpret_cast<V*>(smraw);
  V* tw = X + (size_t)N * C;
  const V* gtw = reinterpret_cast<const V*>(a.tw);
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = gtw[i];
  const int m0 = blockIdx.x * 2 * C;
  for (int it = threadIdx.x; it < N * C; it += blockDim.x) {
    const int cc = it % C, i = it / C;
    T val[2] = {T(0), T(0)};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = m0 + h * C + cc;
      if (m >= M) continue;
      const size_t idx = (size_t)i * M + m;
      T f = a.F[idx];
      if (a.z) {
        f += (T)a.z[idx];
      } else if (i < a.k) {
        // row n = i+1 <= k: kappa tau^-1 sum_{j=n}^{k} omega_j U^{N+n-j}
        for (int j = i + 1; j <= a.k; ++j) f += a.kw[j] * a.U[(size_t)(N + i - j) * M + m];
      }
      val[h] = f * a.s[i];
    }
    X[(size_t)i * C + cc] = mk(val[0], val[1]);
  }
  __syncthreads();
  fft_forward(X, C, C, N, tw);
  V* S = reinterpret_cast<V*>(a.S);
  const int J = N / 2 + 1;
  const T h = T(0.5);
  for (int it = threadIdx.x; it < J * C; it += blockDim.x) {
    const int cc = it % C, j = it / C;
    const V Zj = X[(size_t)fft_pos(j, N) * C + cc];
    const V Zn = X[(size_t)fft_pos((N - j) & (N - 1), N) * C + cc];
    const V A = mk(h * (Zj.x + Zn.x), h * (Zj.y - Zn.y));
    const V B = mk(h * (Zj.y + Zn.y), -h * (Zj.x - Zn.x));
    const int ma = m0 + cc, mb = m0 + C + cc;
    if (ma < M) S[(size_t)j * M + ma] = A;
    if (mb < M) S[(size_t)j * M + mb] = B;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_direct_inv(DirectInvArgs<T> a) {
  using V = typename c2<T>::t;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M;
  V* X = reinterpret_cast<V*>(smraw);
  V* tw = X + (size_t)N * C;
  const V* gtw = reinterpret_cast<const V*>(a.tw);
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = gtw[i];
  const int m0 = blockIdx.x * 2 * C;
  load_half_spectrum(X, reinterpret_cast<const V*>(a.S), N, M, C, m0);
  __syncthreads();
  fft_inverse(X, C, C, N, tw);
  double sd = 0.0, su = 0.0;
  for (int it = threadIdx.x; it < N * C; it += blockDim.x) {
    const int cc = it % C, i = it / C;
    const V z = X[(size_t)i * C + cc];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = m0 + h * C + cc;
      if (m >= M) continue;
      const size_t idx = (size_t)i * M + m;
      const T un = (h ? z.y : z.x) * a.inv_s[i];
      const double d = (double)un - (double)a.Uold[idx];
      a.Uout[idx] = un;
      sd += d * d;
      su += (double)un * (double)un;
    }
  }
  block_reduce_add2(sd, su, a.norms);
}

// ---------------------------------------------------------------------------
// CQ Toeplitz product along time: z = omega * U (zero-padded 2N-point FFTs, FP64)
// ---------------------------------------------------------------------------
size_t toep_smem(int N, int C) { return sizeof(double2) * ((size_t)2 * N * C + 2 * N); }

__global__ void __launch_bounds__(kThreads) k_toeplitz(ToepArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M, L = 2 * a.N;
  double2* X = reinterpret_cast<double2*>(smraw);
  double2* tw = X + (size_t)L * C;
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = a.tw[i];
  const int m0 = blockIdx.x * 2 * C;
  for (int it = threadIdx.x; it < L * C; it += blockDim.x) {
    const int cc = it % C, i = it / C;
    double val[2] = {0.0, 0.0};
    if (i < N) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = m0 + h * C + cc;
        if (m >= M) continue;
        const size_t idx = (size_t)i * M + m;
        if (a.ukind == 0) val[h] = a.Ud[idx];
        else if (a.ukind == 1) val[h] = (double)a.Uhi[idx] + (double)a.Ulo[idx];
        else val[h] = (double)a.Uf[idx];
      }
    }
    X[(size_t)i * C + cc] = make_double2(val[0], val[1]);
  }
  __syncthreads();
  fft_forward(X, C, C, L, tw);
  for (int it = threadIdx.x; it < L * C; it += blockDim.x) {
    const int cc = it % C, p = it / C;
    X[(size_t)p * C + cc] = cmul(X[(size_t)p * C + cc], a.what[p]);
  }
  __syncthreads();
  fft_inverse(X, C, C, L, tw);
  for (int it = threadIdx.x; it < N * C; it += blockDim.x) {
    const int cc = it % C, i = it / C;
    const double2 z = X[(size_t)(a.half * N + i) * C + cc];
    const int ma = m0 + cc, mb = m0 + C + cc;
    if (ma < M) a.out[(size_t)i * M + ma] = z.x;
    if (mb < M) a.out[(size_t)i * M + mb] = z.y;
  }
}

// ---------------------------------------------------------------------------
// Right-hand side: F_hat_n = f(t_n) + a_n (f(0) - A v) + sum_l b_{l,n} tau^l d^l f(0)
//                            + tau^-alpha sum_{j<n} omega_j v        (eq. (2.1), (2.7), (3.7), (3.12))
// ---------------------------------------------------------------------------
__global__ void k_rhs(RhsArgs a) {
  const size_t total = (size_t)a.N * a.M;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / a.M);
    const int m = (int)(t - (size_t)i * a.M);
    const double vm = a.v[m];
    double F = a.f[t] + a.beta[i] * vm;
    if (i < a.k - 1) {
      const int x = m % a.mx;
      double Av = 2.0 * a.gx * vm;
      if (x > 0) Av -= a.gx * a.v[m - 1];
      if (x < a.mx - 1) Av -= a.gx * a.v[m + 1];
      if (a.dim == 2) {
        Av += 2.0 * a.gy * vm;
        if (m >= a.mx) Av -= a.gy * a.v[m - a.mx];
        if (m + a.mx < a.M) Av -= a.gy * a.v[m + a.mx];
      }
      F += a.a[i] * (a.fd[m] - Av);
      for (int l = 1; l <= a.k - 2; ++l) F += a.bt[l][i] * a.fd[(size_t)l * a.M + m];
    }
    a.F[t] = F;
  }
}

// ---------------------------------------------------------------------------
// conversions
// ---------------------------------------------------------------------------
__global__ void k_d2ff(const double* x, float* hi, float* lo, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const ff r = ff_from_double(x[t]);
    hi[t] = r.hi;
    lo[t] = r.lo;
  }
}
__global__ void k_bcast_d2ff(const double* v, float* hi, float* lo, int N, int M) {
  const size_t total = (size_t)N * M;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const ff r = ff_from_double(v[t % M]);
    hi[t] = r.hi;
    lo[t] = r.lo;
  }
}
__global__ void k_bcast_d(const double* v, double* U, int N, int M) {
  const size_t total = (size_t)N * M;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x)
    U[t] = v[t % M];
}
__global__ void k_ff2d(const float* hi, const float* lo, double* x, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    x[t] = (double)hi[t] + (double)lo[t];
}
__global__ void k_d2f(const double* x, float* y, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    y[t] = (float)x[t];
}
__global__ void k_f2d(const float* x, double* y, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    y[t] = (double)x[t];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int grid_for(size_t n) {
  size_t b = (n + kThreads - 1) / kThreads;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b ? b : 1);
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

static int tiles(int M, int C) { return (M + 2 * C - 1) / (2 * C); }

cudaError_t launch_resid_fwd(const ResidFwdArgs& a, cudaStream_t st) {
  const size_t sm = resid_fwd_smem(a.N, a.C);
  cudaError_t e = set_smem(k_resid_fwd, sm);
  if (e != cudaSuccess) return e;
  prof_begin("resid_fwd_ff", st);
  k_resid_fwd<<<tiles(a.M, a.C), kThreads, sm, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_inv_upd(const InvUpdArgs& a, cudaStream_t st) {
  const size_t sm = inv_upd_smem(a.N, a.C);
  cudaError_t e = set_smem(k_inv_upd, sm);
  if (e != cudaSuccess) return e;
  prof_begin("inv_update_ff", st);
  k_inv_upd<<<tiles(a.M, a.C), kThreads, sm, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_direct_fwd(const DirectFwdArgs<T>& a, cudaStream_t st) {
  const size_t sm = direct_smem<T>(a.N, a.C);
  cudaError_t e = set_smem(k_direct_fwd<T>, sm);
  if (e != cudaSuccess) return e;
  prof_begin(sizeof(T) == 8 ? "direct_fwd_f64" : "direct_fwd_f32", st);
  k_direct_fwd<T><<<tiles(a.M, a.C), kThreads, sm, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_direct_inv(const DirectInvArgs<T>& a, cudaStream_t st) {
  const size_t sm = direct_smem<T>(a.N, a.C);
  cudaError_t e = set_smem(k_direct_inv<T>, sm);
  if (e != cudaSuccess) return e;
  prof_begin(sizeof(T) == 8 ? "direct_inv_f64" : "direct_inv_f32", st);
  k_direct_inv<T><<<tiles(a.M, a.C), kThreads, sm, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_toeplitz(const ToepArgs& a, cudaStream_t st) {
  const size_t sm = toep_smem(a.N, a.C);
  cudaError_t e = set_smem(k_toeplitz, sm);
  if (e != cudaSuccess) return e;
  prof_begin("toeplitz_f64", st);
  k_toeplitz<<<tiles(a.M, a.C), kThreads, sm, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_rhs(const RhsArgs& a, cudaStream_t st) {
  prof_begin("rhs_f64", st);
  k_rhs<<<grid_for((size_t)a.N * a.M), kThreads, 0, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_d2ff(const double* x, float* hi, float* lo, size_t n, cudaStream_t st) {
  prof_begin("cvt_d2ff", st);
  k_d2ff<<<grid_for(n), kThreads, 0, st>>>(x, hi, lo, n);
  prof_end(st);
  return cudaGetLastError();
}
cudaError_t launch_bcast_d2ff(const double* v, float* hi, float* lo, int N, int M, cudaStream_t st) {
  prof_begin("cvt_bcast_d2ff", st);
  k_bcast_d2ff<<<grid_for((size_t)N * M), kThreads, 0, st>>>(v, hi, lo, N, M);
  prof_end(st);
  return cudaGetLastError();
}
cudaError_t launch_bcast_d(const double* v, double* U, int N, int M, cudaStream_t st) {
  prof_begin("initial_guess", st);
  k_bcast_d<<<grid_for((size_t)N * M), kThreads, 0, st>>>(v, U, N, M);
  prof_end(st);
  return cudaGetLastError();
}
cudaError_t launch_ff2d(const float* hi, const float* lo, double* x, size_t n, cudaStream_t st) {
  prof_begin("cvt_ff2d", st);
  k_ff2d<<<grid_for(n), kThreads, 0, st>>>(hi, lo, x, n);
  prof_end(st);
  return cudaGetLastError();
}
cudaError_t launch_d2f(const double* x, float* y, size_t n, cudaStream_t st) {
  prof_begin("cvt_d2f", st);
  k_d2f<<<grid_for(n), kThreads, 0, st>>>(x, y, n);
  prof_end(st);
  return cudaGetLastError();
}
cudaError_t launch_f2d(const float* x, double* y, size_t n, cudaStream_t st) {
  prof_begin("cvt_f2d", st);
  k_f2d<<<grid_for(n), kThreads, 0, st>>>(x, y, n);
  prof_end(st);
  return cudaGetLastError();
}

template size_t direct_smem<float>(int, int);
template size_t direct_smem<double>(int, int);
template cudaError_t launch_direct_fwd<float>(const DirectFwdArgs<float>&, cudaStream_t);
template cudaError_t launch_direct_fwd<double>(const DirectFwdArgs<double>&, cudaStream_t);
template cudaError_t launch_direct_inv<float>(const DirectInvArgs<float>&, cudaStream_t);
template cudaError_t launch_direct_inv<double>(const DirectInvArgs<double>&, cudaStream_t);

}  // namespace pint
