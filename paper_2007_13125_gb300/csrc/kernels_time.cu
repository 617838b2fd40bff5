// Time-axis kernels of one WR sweep (Algorithm 1 / Algorithm 2, steps 1 and 3), the
// all-at-once residual, the CQ Toeplitz product, the right-hand side and conversions.
//
// Tiling of the time kernels: one CTA owns 2C spatial points and all N time levels.
// Point m0 + c is the real part and point m0 + C + c the imaginary part of complex
// column c, so one complex N-point FFT transforms two real time series; the half
// spectra j = 0..N/2 of both are separated afterwards with the conjugate symmetry of
// real data. Global loads and stores are coalesced over consecutive points.
// Shared memory per CTA: the [N][C] complex tile, the twiddles and the digit-reversal
// table of the FFT (fft.cuh).
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

// shared-memory carve-up of a time tile: X [N][C] (V), tw [N] (V), perm [N] (u16)
template <typename V> __host__ __device__ inline size_t time_tile_bytes(int N, int C) {
  return sizeof(V) * ((size_t)N * C + N) + sizeof(unsigned short) * (size_t)N;
}

template <typename V>
__device__ __forceinline__ void time_tile_setup(unsigned char* raw, int N, int C, const V* gtw, V*& X,
                                                V*& tw, unsigned short*& perm) {
  X = reinterpret_cast<V*>(raw);
  tw = X + (size_t)N * C;
  perm = reinterpret_cast<unsigned short*>(tw + N);
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = gtw[i];
  fft_perm_table(perm, N);
}

// Separate the spectra of the two real columns packed in complex column cc and store the
// half spectra j = 0..N/2 of points ma (real part) and mb (imaginary part).
template <typename V>
__device__ __forceinline__ void store_half_spectrum(const V* X, const unsigned short* perm, V* S, int N,
                                                    int M, int C, int logC, int m0) {
  using T = decltype(X[0].x);
  const int J = N / 2 + 1;
  const T h = T(0.5);
  for (int it = threadIdx.x; it < (J << logC); it += blockDim.x) {
    const int cc = it & (C - 1), j = it >> logC;
    const V Zj = X[(size_t)perm[j] * C + cc];
    const V Zn = X[(size_t)perm[(N - j) & (N - 1)] * C + cc];
    const V A = mk(h * (Zj.x + Zn.x), h * (Zj.y - Zn.y));      // (Z_j + conj Z_{N-j}) / 2
    const V B = mk(h * (Zj.y + Zn.y), -h * (Zj.x - Zn.x));     // (Z_j - conj Z_{N-j}) / 2i
    const int ma = m0 + cc, mb = m0 + C + cc;
    if (ma < M) S[(size_t)j * M + ma] = A;
    if (mb < M) S[(size_t)j * M + mb] = B;
  }
}

// Inverse of store_half_spectrum: Z_j = A_j + i B_j in permuted order (Hermitian symmetry
// supplies j > N/2).
template <typename V>
__device__ __forceinline__ void load_half_spectrum(V* X, const unsigned short* perm, const V* S, int N,
                                                   int M, int C, int logC, int m0) {
  const int J = N / 2 + 1;
  for (int it = threadIdx.x; it < (J << logC); it += blockDim.x) {
    const int cc = it & (C - 1), j = it >> logC;
    const int ma = m0 + cc, mb = m0 + C + cc;
    V A, B;
    A.x = 0; A.y = 0; B = A;
    if (ma < M) A = S[(size_t)j * M + ma];
    if (mb < M) B = S[(size_t)j * M + mb];
    X[(size_t)perm[j] * C + cc] = mk(A.x - B.y, A.y + B.x);                 // A + iB
    if (j > 0 && j < N / 2)
      X[(size_t)perm[N - j] * C + cc] = mk(A.x + B.y, B.x - A.y);           // conj(A) + i conj(B)
  }
}

// ---------------------------------------------------------------------------
// MIXED: residual r = F_hat - K U (double-float) + kappa scaling + forward DFT along time.
// K U = tau^-alpha sum_{j=0}^{min(n-1,k)} omega_j U^{n-j} + A_h U^n (BDF band, eq. (2.6) with
// kappa = 0), or, for CQ, the precomputed Toeplitz history y plus A_h U^n.
// ---------------------------------------------------------------------------
size_t resid_fwd_smem(int N, int C) { return time_tile_bytes<float2>(N, C); }

__global__ void __launch_bounds__(kThreads) k_resid_fwd(ResidFwdArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M, logC = a.logC;
  float2 *X, *tw;
  unsigned short* perm;
  time_tile_setup(smraw, N, C, a.tw, X, tw, perm);

  const int m0 = blockIdx.x * 2 * C;
  const int c = threadIdx.x & (C - 1);
  const int nch = blockDim.x >> logC;
  const int tc = threadIdx.x >> logC;
  const int Lc = N / nch;
  const int i0 = tc * Lc;
  const int k = a.k;
  ff cw[kMaxK + 1];
#pragma unroll
  for (int j = 0; j <= kMaxK; ++j) { cw[j].hi = a.c_hi[j]; cw[j].lo = a.c_lo[j]; }
  const ff gx = {a.gx_hi, a.gx_lo}, gy = {a.gy_hi, a.gy_lo};

  // Lane layout: a warp holds whole groups of C consecutive columns that share one time
  // chunk, so at every level the x-neighbours of a point sit in adjacent lanes (or in the
  // other half of the pair): they come from warp shuffles, and only the two tile edges
  // (points m0 - 1 and m0 + 2C) are loaded from memory. y-neighbours are plain loads.
  const int lane = threadIdx.x & 31;
  int mm[2];
  bool valid[2];
  int xx[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    mm[h] = m0 + h * C + c;
    valid[h] = mm[h] < M;
    xx[h] = valid[h] ? mm[h] % a.mx : 0;
  }
  const int src_l = c > 0 ? lane - 1 : lane + C - 1;       // left of half 1 when c == 0: half 0, col C-1
  const int src_r = c < C - 1 ? lane + 1 : lane - (C - 1); // right of half 0 when c == C-1: half 1, col 0
  ff win[2][kMaxK];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int j = 0; j < kMaxK; ++j) {
      const int lev = i0 - 1 - j;
      win[h][j].hi = 0.f;
      win[h][j].lo = 0.f;
      if (j < k && valid[h] && lev >= 0) win[h][j] = ldff(a.Uhi, a.Ulo, (size_t)lev * M + mm[h]);
    }
#pragma unroll 2
  for (int i = i0; i < i0 + Lc; ++i) {
    const float si = __ldg(a.s + i);
    const size_t row = (size_t)i * M;
    ff u[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      u[h].hi = 0.f;
      u[h].lo = 0.f;
      if (valid[h]) u[h] = ldff(a.Uhi, a.Ulo, row + mm[h]);
    }
    // x-neighbours: a shuffle delivers the *sender's* argument, so each shuffle moves one
    // fixed half and the receiver picks which result it needs.
    ff lft[2], rgt[2];
    {
      const int sl = c > 0 ? lane - 1 : lane + C - 1;
      const int sr = c < C - 1 ? lane + 1 : lane - (C - 1);
      ff s1, s2, s3, s4;
      s1.hi = __shfl_sync(0xffffffffu, u[0].hi, sl);      // c > 0: left of half 0; c == 0: left of half 1
      s1.lo = __shfl_sync(0xffffffffu, u[0].lo, sl);
      s2.hi = __shfl_sync(0xffffffffu, u[1].hi, lane - 1); // c > 0: left of half 1
      s2.lo = __shfl_sync(0xffffffffu, u[1].lo, lane - 1);
      s3.hi = __shfl_sync(0xffffffffu, u[1].hi, sr);      // c < C-1: right of half 1; c == C-1: right of half 0
      s3.lo = __shfl_sync(0xffffffffu, u[1].lo, sr);
      s4.hi = __shfl_sync(0xffffffffu, u[0].hi, lane + 1); // c < C-1: right of half 0
      s4.lo = __shfl_sync(0xffffffffu, u[0].lo, lane + 1);
      lft[0] = s1;
      lft[1] = c > 0 ? s2 : s1;
      rgt[0] = c < C - 1 ? s4 : s3;
      rgt[1] = s3;
    }
    if (c == 0 && valid[0] && xx[0] > 0) lft[0] = ldff(a.Uhi, a.Ulo, row + mm[0] - 1);
    if (c == C - 1 && valid[1] && xx[1] < a.mx - 1) rgt[1] = ldff(a.Uhi, a.Ulo, row + mm[1] + 1);
    float r[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      r[h] = 0.f;
      if (!valid[h]) continue;
      const int m = mm[h];
      const size_t idx = row + m;
      ff_acc acc;
      acc.init(ff_from_double(__ldg(a.F + idx)));
      if (a.y) acc.sub(ff_from_double(__ldg(a.y + idx)));
      acc.fma_term(cw[0], u[h], -1.f);
#pragma unroll
      for (int j = 1; j <= kMaxK; ++j)
        if (j <= k) acc.fma_term(cw[j], win[h][j - 1], -1.f);
      if (xx[h] > 0) acc.fma_term(gx, lft[h], 1.f);
      if (xx[h] < a.mx - 1) acc.fma_term(gx, rgt[h], 1.f);
      if (a.dim == 2) {
        if (m >= a.mx) acc.fma_term(gy, ldff(a.Uhi, a.Ulo, idx - a.mx), 1.f);
        if (m + a.mx < M) acc.fma_term(gy, ldff(a.Uhi, a.Ulo, idx + a.mx), 1.f);
      }
      r[h] = acc.value() * si;
#pragma unroll
      for (int j = kMaxK - 1; j > 0; --j) win[h][j] = win[h][j - 1];
      win[h][0] = u[h];
    }
    X[(size_t)i * C + c] = make_float2(r[0], r[1]);
  }
  __syncthreads();
  fft_forward(X, C, logC, N, tw);
  store_half_spectrum(X, perm, a.S, N, M, C, logC, m0);
}

// ---------------------------------------------------------------------------
// MIXED: inverse DFT + unscale + U += c (double-float) + norms
// ---------------------------------------------------------------------------
size_t inv_upd_smem(int N, int C) { return time_tile_bytes<float2>(N, C); }

__global__ void __launch_bounds__(kThreads) k_inv_upd(InvUpdArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M, logC = a.logC;
  float2 *X, *tw;
  unsigned short* perm;
  time_tile_setup(smraw, N, C, a.tw, X, tw, perm);
  const int m0 = blockIdx.x * 2 * C;
  __syncthreads();
  load_half_spectrum(X, perm, a.S, N, M, C, logC, m0);
  __syncthreads();
  fft_inverse(X, C, logC, N, tw);

  float sc = 0.f, su = 0.f;  // per-thread partial norms (FP32: the FP64 pipe is ~1/70 rate)
  for (int it = threadIdx.x; it < (N << logC); it += blockDim.x) {
    const int cc = it & (C - 1), i = it >> logC;
    const float2 z = X[(size_t)i * C + cc];
    const float is = __ldg(a.inv_s + i);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = m0 + h * C + cc;
      if (m >= M) continue;
      const float cval = (h ? z.y : z.x) * is;
      const size_t idx = (size_t)i * M + m;
      ff u = {a.Uhi[idx], a.Ulo[idx]};
      u = ff_add_f(u, cval);
      a.Uhi[idx] = u.hi;
      a.Ulo[idx] = u.lo;
      sc = fmaf(cval, cval, sc);
      su = fmaf(u.hi, u.hi, su);
    }
  }
  block_reduce_add2((double)sc, (double)su, a.norms);
}

// ---------------------------------------------------------------------------
// FP64 / FP32 direct form (Algorithm 1/2 as printed): F_{m-1} -> scale -> DFT
// ---------------------------------------------------------------------------
template <typename T> size_t direct_smem(int N, int C) { return time_tile_bytes<typename c2<T>::t>(N, C); }

template <typename T>
__global__ void __launch_bounds__(kThreads) k_direct_fwd(DirectFwdArgs<T> a) {
  using V = typename c2<T>::t;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M, logC = a.logC;
  V *X, *tw;
  unsigned short* perm;
  time_tile_setup(smraw, N, C, reinterpret_cast<const V*>(a.tw), X, tw, perm);
  const int m0 = blockIdx.x * 2 * C;
  for (int it = threadIdx.x; it < (N << logC); it += blockDim.x) {
    const int cc = it & (C - 1), i = it >> logC;
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
        // row n = i+1 <= k: kappa tau^-1 sum_{j=n}^{k} omega_j U^{N+n-j}  (eq. (2.7), reading r1)
#pragma unroll
        for (int j = 1; j <= kMaxK; ++j)
          if (j > i && j <= a.k) f += a.kw[j] * a.U[(size_t)(N + i - j) * M + m];
      }
      val[h] = f * a.s[i];
    }
    X[(size_t)i * C + cc] = mk(val[0], val[1]);
  }
  __syncthreads();
  fft_forward(X, C, logC, N, tw);
  store_half_spectrum(X, perm, reinterpret_cast<V*>(a.S), N, M, C, logC, m0);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_direct_inv(DirectInvArgs<T> a) {
  using V = typename c2<T>::t;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M, logC = a.logC;
  V *X, *tw;
  unsigned short* perm;
  time_tile_setup(smraw, N, C, reinterpret_cast<const V*>(a.tw), X, tw, perm);
  const int m0 = blockIdx.x * 2 * C;
  __syncthreads();
  load_half_spectrum(X, perm, reinterpret_cast<const V*>(a.S), N, M, C, logC, m0);
  __syncthreads();
  fft_inverse(X, C, logC, N, tw);
  double sd = 0.0, su = 0.0;
  for (int it = threadIdx.x; it < (N << logC); it += blockDim.x) {
    const int cc = it & (C - 1), i = it >> logC;
    const V z = X[(size_t)i * C + cc];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = m0 + h * C + cc;
      if (m >= M) continue;
      const size_t idx = (size_t)i * M + m;
      const T un = (h ? z.y : z.x) * a.inv_s[i];
      const T d = un - a.Uold[idx];
      a.Uout[idx] = un;
      sd += (double)(d * d);
      su += (double)(un * un);
    }
  }
  block_reduce_add2(sd, su, a.norms);
}

// ---------------------------------------------------------------------------
// CQ Toeplitz product along time: z = omega * U (zero-padded 2N-point FFTs, FP64), the
// circulant embedding of Sec. 3.2 (speedup analysis of Algorithm 2).
// ---------------------------------------------------------------------------
size_t toep_smem(int N, int C) { return time_tile_bytes<double2>(2 * N, C); }

__global__ void __launch_bounds__(kThreads) k_toeplitz(ToepArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M, L = 2 * a.N, logC = a.logC;
  double2 *X, *tw;
  unsigned short* perm;
  time_tile_setup(smraw, L, C, a.tw, X, tw, perm);
  const int m0 = blockIdx.x * 2 * C;
  for (int it = threadIdx.x; it < (L << logC); it += blockDim.x) {
    const int cc = it & (C - 1), i = it >> logC;
    double val[2] = {0.0, 0.0};
    if (i < N) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = m0 + h * C + cc;
        if (m >= M) continue;
        const size_t idx = (size_t)i * M + m;
        if (a.ukind == 0) val[h] = a.Ud[idx];
        else if (a.ukind == 1) val[h] = ff_to_double(ff{a.Uhi[idx], a.Ulo[idx]});
        else val[h] = f2d_bits(a.Uf[idx]);
      }
    }
    X[(size_t)i * C + cc] = make_double2(val[0], val[1]);
  }
  __syncthreads();
  fft_forward(X, C, logC, L, tw);
  for (int it = threadIdx.x; it < (L << logC); it += blockDim.x) {
    const int cc = it & (C - 1), p = it >> logC;
    X[(size_t)p * C + cc] = cmul(X[(size_t)p * C + cc], a.what[p]);
  }
  __syncthreads();
  fft_inverse(X, C, logC, L, tw);
  for (int it = threadIdx.x; it < (N << logC); it += blockDim.x) {
    const int cc = it & (C - 1), i = it >> logC;
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
    double F = fma(a.beta[i], vm, a.f[t]);
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
// conversions (integer bit manipulation; see ff.cuh)
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
    x[t] = ff_to_double(ff{hi[t], lo[t]});
}
__global__ void k_d2f(const double* x, float* y, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    y[t] = ff_from_double(x[t]).hi;
}
__global__ void k_f2d(const float* x, double* y, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    y[t] = f2d_bits(x[t]);
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
