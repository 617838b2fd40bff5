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
#pragma unroll 4
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
//
// The tile (2C points x all N levels) is processed in chunks of kLK levels. Each chunk is
// first staged in shared memory with asynchronous copies issued by all threads at once
// (U with kMaxK levels of history and the two x-halo points, the two y-neighbour rows, F_hat
// and y), then every thread evaluates residuals from shared memory only.
// ---------------------------------------------------------------------------
constexpr int kLK = 16;                      // levels per staged chunk

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
// Bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

struct ResidStage {
  // row-major [level][point] arrays of the staged chunk
  int W;           // 2C + 2 (U incl. x halo)
  int P2;          // 2C
  float* Uh;       // [kLK + kMaxK][W]
  float* Ul;
  float* Yh;       // [2][kLK][P2]  (row below, row above)
  float* Yl;
  double* F;       // [kLK][P2]
  float* Ych;      // [kLK][P2] (CQ history, double-float) or unused
  float* Ycl;
};

// levels per staged chunk: at least kLK, and enough that every thread has a level
__host__ __device__ inline int resid_chunk(int C) {
  const int lk = kThreads / (2 * C);
  return lk > kLK ? lk : kLK;
}

__host__ __device__ inline size_t resid_stage_bytes(int C) {
  const size_t W = 2 * (size_t)C + 2, P2 = 2 * (size_t)C, LK = resid_chunk(C);
  return 2 * sizeof(float) * (LK + kMaxK) * W + 2 * sizeof(float) * 2 * LK * P2 +
         2 * sizeof(double) * LK * P2;
}

size_t resid_fwd_smem(int N, int C) { return time_tile_bytes<float2>(N, C) + resid_stage_bytes(C) + 16; }

__global__ void __launch_bounds__(kThreads) k_resid_fwd(ResidFwdArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M, logC = a.logC, mx = a.mx;
  float2 *X, *tw;
  unsigned short* perm;
  time_tile_setup(smraw, N, C, a.tw, X, tw, perm);
  unsigned char* sp = reinterpret_cast<unsigned char*>(perm + N);
  sp = reinterpret_cast<unsigned char*>(((size_t)sp + 15) & ~(size_t)15);
  const int LKC = resid_chunk(C);  // levels per staged chunk
  ResidStage st;
  st.W = 2 * C + 2;
  st.P2 = 2 * C;
  st.F = reinterpret_cast<double*>(sp);
  st.Ych = reinterpret_cast<float*>(st.F + LKC * st.P2);
  st.Ycl = st.Ych + LKC * st.P2;
  st.Uh = st.Ycl + LKC * st.P2;
  st.Ul = st.Uh + (LKC + kMaxK) * st.W;
  st.Yh = st.Ul + (LKC + kMaxK) * st.W;
  st.Yl = st.Yh + 2 * LKC * st.P2;

  const int m0 = blockIdx.x * 2 * C;
  const int P2 = st.P2, W = st.W;
  const int k = a.k;
  ff cw[kMaxK + 1];
#pragma unroll
  for (int j = 0; j <= kMaxK; ++j) { cw[j].hi = a.c_hi[j]; cw[j].lo = a.c_lo[j]; }
  const ff gx = {a.gx_hi, a.gx_lo}, gy = {a.gy_hi, a.gy_lo};
  const bool two_d = a.dim == 2;

  // Each thread keeps one point q of the tile (2C divides the block size) and walks levels.
  const int logP2 = logC + 1;
  const int q = threadIdx.x & (P2 - 1);
  const int lstep = blockDim.x >> logP2;
  const int mq = m0 + q;
  const bool qvalid = mq < M;
  const int xq = qvalid ? mq % mx : 0;
  for (int c0 = 0; c0 < N; c0 += LKC) {
    const int LK = min(LKC, N - c0);
    // ---- stage chunk levels [c0, c0 + LK) (+ kMaxK levels of history for U) ----
    {
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
      for (int l = warp; l < LKC + kMaxK; l += nwarp) {
        const int lev = c0 - kMaxK + l;
        const bool lok = lev >= 0 && lev < N;
        const size_t grow = (size_t)(lok ? lev : 0) * M;
        for (int qq = lane; qq < W; qq += 32) {
          const int m = m0 - 1 + qq;
          float* dh = st.Uh + l * W + qq;
          float* dl = st.Ul + l * W + qq;
          if (lok && m >= 0 && m < M) {
            cp_async4(dh, a.Uhi + grow + m);
            cp_async4(dl, a.Ulo + grow + m);
          } else {
            *dh = 0.f;
            *dl = 0.f;
          }
        }
      }
    }
    for (int l = threadIdx.x >> logP2; l < LK; l += lstep) {
      const int e = (l << logP2) + q;
      const size_t g = (size_t)(c0 + l) * M + mq;
      if (qvalid) {
        cp_async8(st.F + e, a.F + g);
        if (a.yhi) {
          cp_async4(st.Ych + e, a.yhi + g);
          cp_async4(st.Ycl + e, a.ylo + g);
        }
      }
      if (two_d) {
        float* bh = st.Yh + e;
        float* bl = st.Yl + e;
        float* ah = st.Yh + LKC * P2 + e;
        float* al = st.Yl + LKC * P2 + e;
        if (qvalid && mq >= mx) { cp_async4(bh, a.Uhi + g - mx); cp_async4(bl, a.Ulo + g - mx); }
        else { *bh = 0.f; *bl = 0.f; }
        if (mq + mx < M) { cp_async4(ah, a.Uhi + g + mx); cp_async4(al, a.Ulo + g + mx); }
        else { *ah = 0.f; *al = 0.f; }
      }
    }
    cp_async_wait_all();
    __syncthreads();
    // ---- residuals of the chunk from shared memory ----
    for (int l = threadIdx.x >> logP2; l < LK; l += lstep) {
      const int e = (l << logP2) + q;
      const int i = c0 + l;
      float r = 0.f;
      if (qvalid) {
        const int ub = (l + kMaxK) * W + q + 1;  // this point in the U stage
        ff_acc acc;
        acc.init(ff_from_double(st.F[e]));
        if (a.yhi) acc.sub(ff{st.Ych[e], st.Ycl[e]});
        acc.fma_term(cw[0], ff{st.Uh[ub], st.Ul[ub]}, -1.f);
#pragma unroll
        for (int j = 1; j <= kMaxK; ++j)
          if (j <= k) acc.fma_term(cw[j], ff{st.Uh[ub - j * W], st.Ul[ub - j * W]}, -1.f);
        if (xq > 0) acc.fma_term(gx, ff{st.Uh[ub - 1], st.Ul[ub - 1]}, 1.f);
        if (xq < mx - 1) acc.fma_term(gx, ff{st.Uh[ub + 1], st.Ul[ub + 1]}, 1.f);
        if (two_d) {
          acc.fma_term(gy, ff{st.Yh[e], st.Yl[e]}, 1.f);
          acc.fma_term(gy, ff{st.Yh[LKC * P2 + e], st.Yl[LKC * P2 + e]}, 1.f);
        }
        r = acc.value() * __ldg(a.s + i);
      }
      float* xs = reinterpret_cast<float*>(X + (size_t)i * C + (q & (C - 1)));
      xs[q >= C ? 1 : 0] = r;
    }
    __syncthreads();  // the stage is reused by the next chunk
  }
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
  {
    // the update reads this tile's rows of U after the inverse FFT: start pulling them into L2
    // now. Each span is rounded out to 16-byte boundaries and clipped to the array.
    const size_t total = (size_t)N * M;
    const int p1 = min(m0 + 2 * C, M);
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) {
      const float* base = (i & 1) ? a.Ulo : a.Uhi;
      const size_t b0 = ((size_t)(i >> 1) * M + m0) & ~(size_t)3;
      size_t b1 = ((size_t)(i >> 1) * M + p1 + 3) & ~(size_t)3;
      if (b1 > (total & ~(size_t)3)) b1 = total & ~(size_t)3;
      if (b1 > b0) prefetch_l2(base + b0, (unsigned)((b1 - b0) * 4));
    }
  }
  __syncthreads();
  load_half_spectrum(X, perm, a.S, N, M, C, logC, m0);
  __syncthreads();
  fft_inverse(X, C, logC, N, tw);

  float sc = 0.f, su = 0.f;  // per-thread partial norms (FP32: the FP64 pipe is ~1/70 rate)
#pragma unroll 4
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
// MIXED CQ history y = tau^-alpha (omega * U) in double-float: the same circulant embedding
// with 2N-point FFTs whose butterflies are error-free-transformation arithmetic on the FP32
// pipes (~48-bit significand; GB300's FP64 pipe is ~70x slower than its FP32 pipes).
// ---------------------------------------------------------------------------
size_t toep_ff_smem(int N, int C) { return time_tile_bytes<ffc>(2 * N, C); }

__global__ void __launch_bounds__(kThreads) k_toeplitz_ff(ToepFFArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M, L = 2 * a.N, logC = a.logC;
  ffc* X = reinterpret_cast<ffc*>(smraw);
  ffc* tw = X + (size_t)L * C;
  unsigned short* perm = reinterpret_cast<unsigned short*>(tw + L);
  const ffc* gtw = reinterpret_cast<const ffc*>(a.tw);
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = gtw[i];
  (void)perm;
  const int m0 = blockIdx.x * 2 * C;
  for (int it = threadIdx.x; it < (L << logC); it += blockDim.x) {
    const int cc = it & (C - 1), i = it >> logC;
    ffc v = {0.f, 0.f, 0.f, 0.f};
    if (i < N) {
      const int ma = m0 + cc, mb = m0 + C + cc;
      const size_t row = (size_t)i * M;
      if (ma < M) { v.rh = a.Uhi[row + ma]; v.rl = a.Ulo[row + ma]; }
      if (mb < M) { v.ih = a.Uhi[row + mb]; v.il = a.Ulo[row + mb]; }
    }
    X[(size_t)i * C + cc] = v;
  }
  __syncthreads();
  fft_forward<kToepFFMaxLog>(X, C, logC, L, tw);
  const ffc* what = reinterpret_cast<const ffc*>(a.what);
  for (int it = threadIdx.x; it < (L << logC); it += blockDim.x) {
    const int cc = it & (C - 1), p = it >> logC;
    X[(size_t)p * C + cc] = cmul(X[(size_t)p * C + cc], what[p]);
  }
  __syncthreads();
  fft_inverse<kToepFFMaxLog>(X, C, logC, L, tw);
  for (int it = threadIdx.x; it < (N << logC); it += blockDim.x) {
    const int cc = it & (C - 1), i = it >> logC;
    const ffc z = X[(size_t)i * C + cc];
    const int ma = m0 + cc, mb = m0 + C + cc;
    const size_t row = (size_t)i * M;
    if (ma < M) { a.yhi[row + ma] = z.rh; a.ylo[row + ma] = z.rl; }
    if (mb < M) { a.yhi[row + mb] = z.ih; a.ylo[row + mb] = z.il; }
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
// convergence control inside a CUDA graph: a while-node repeats the sweep until k_converge
// clears its condition (same decision as the host loop)
// ---------------------------------------------------------------------------
__global__ void k_ctl_init(SolveCtl* c, double tol, double q_floor, int max_sweeps) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    c->tol = tol;
    c->q_floor = q_floor;
    c->prev = -1.0;
    c->upd = 0.0;
    c->max_sweeps = max_sweeps;
    c->m = 0;
    c->done = 0;
  }
}

__global__ void k_converge(const double* norms, SolveCtl* c, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double c2 = norms[0], u2 = norms[1];
  const double upd = u2 > 0.0 ? sqrt(c2 / u2) : sqrt(c2);
  const int m = c->m + 1;
  const bool done = stop_decision(m, upd, c->prev, c->tol, c->q_floor);
  c->m = m;
  c->prev = upd;
  c->upd = upd;
  c->done = done ? 1 : 0;
  cudaGraphSetConditional(h, (!done && m < c->max_sweeps) ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_ctl_init(SolveCtl* ctl, double tol, double q_floor, int max_sweeps, cudaStream_t st) {
  k_ctl_init<<<1, 32, 0, st>>>(ctl, tol, q_floor, max_sweeps);
  return cudaGetLastError();
}

cudaError_t launch_converge(const double* norms, SolveCtl* ctl, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_converge<<<1, 32, 0, st>>>(norms, ctl, h);
  return cudaGetLastError();
}

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

cudaError_t launch_toeplitz_ff(const ToepFFArgs& a, cudaStream_t st) {
  const size_t sm = toep_ff_smem(a.N, a.C);
  cudaError_t e = set_smem(k_toeplitz_ff, sm);
  if (e != cudaSuccess) return e;
  prof_begin("toeplitz_ff", st);
  k_toeplitz_ff<<<tiles(a.M, a.C), kThreads, sm, st>>>(a);
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
