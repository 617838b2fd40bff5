// Time-axis kernels of one WR sweep (Algorithm 1 / Algorithm 2, steps 1 and 3) other than the
// MIXED residual (kernels_resid.cu): the inverse transform and update, the FP64 / FP32 direct
// forms, the CQ Toeplitz product, the right-hand side, conversions and convergence control.
//
// Tiling of the time kernels: one CTA owns 2C spatial points and all N time levels.
// Point m0 + c is the real part and point m0 + C + c the imaginary part of complex
// column c, so one complex N-point FFT transforms two real time series; the half
// spectra j = 0..N/2 of both are separated afterwards with the conjugate symmetry of
// real data. Global loads and stores are coalesced over consecutive points.
// Shared memory per CTA: the [N][C] complex tile, the twiddles and the digit-reversal
// table of the FFT (fft.cuh).
#include "time_tile.cuh"

namespace pint {

// ---------------------------------------------------------------------------
// MIXED: inverse DFT + unscale + U += c (double-float) + norms
// ---------------------------------------------------------------------------
// U staging ring of the update: RING levels x 2C points, hi and lo
__host__ __device__ constexpr size_t inv_ring_bytes(int C, int ring) { return 2 * sizeof(float) * (size_t)ring * 2 * C; }
__host__ __device__ constexpr size_t inv_upd_smem_ring(int N, int C, int ring) {
  return sizeof(float2) * ((size_t)N * C + N) + sizeof(unsigned short) * (size_t)N + 16 +
         2 * sizeof(float2) * (size_t)C + 16 + inv_ring_bytes(C, ring);
}
// ring depth: as many levels (a power of two, at most 64: slots are taken modulo the depth) as fit
// next to the tile with three CTAs per SM, at least one round of kThreads / 2C levels, and no more
// than N unless one round is longer
__host__ __device__ constexpr int inv_ring_levels(int N, int C) {
  int ring = 64;
  while (ring > kThreads / (2 * C) && inv_upd_smem_ring(N, C, ring) > 72 * 1024) ring >>= 1;
  while (ring > N && ring > kThreads / (2 * C)) ring >>= 1;
  if (ring < kThreads / (2 * C)) ring = kThreads / (2 * C);
  return ring;
}
size_t inv_upd_smem(int N, int C) { return inv_upd_smem_ring(N, C, inv_ring_levels(N, C)); }

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Wait until at most n of this thread's most recent copy groups are pending (n > 7 waits as
// for 7: stricter, never weaker).
__device__ __forceinline__ void cp_async_wait_pending(int n) {
  switch (n) {
    case 0: cp_async_wait<0>(); break;
    case 1: cp_async_wait<1>(); break;
    case 2: cp_async_wait<2>(); break;
    case 3: cp_async_wait<3>(); break;
    case 4: cp_async_wait<4>(); break;
    case 5: cp_async_wait<5>(); break;
    case 6: cp_async_wait<6>(); break;
    default: cp_async_wait<7>(); break;
  }
}

// Inverse time DFT of the tile, unscaling, and U += c with the norms of c and U.
// Thread (q, r) of the update owns point q and the levels i = r (mod kThreads / 2C). Its U values
// stream through a per-thread ring of shared-memory slots filled by asynchronous copies: the
// first rounds are requested before the spectrum arrives and the FFT runs, and each consumed
// slot is refilled with the level RING further on, so the loads stay in flight behind the
// arithmetic and the stores. A thread reads only slots it filled itself (no block barrier).
// LOGN > 0: compiled for N = 2^LOGN levels and 2^LOGC columns; LOGN = 0: any shape.
// V0: the first sweep from U_0^n = v: U = v + c, v read once per point (no U stream, no ring)
template <int LOGN, int LOGC, bool V0>
__global__ void __launch_bounds__(kThreads, 4) k_inv_upd(InvUpdArgs a) {
  constexpr bool CT = LOGN > 0;
  constexpr int CT_RING = CT ? inv_ring_levels(1 << LOGN, 1 << LOGC) : 1;
  constexpr int CT_DEPTH = CT ? CT_RING / (kThreads >> (LOGC + 1)) : 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = CT ? (1 << LOGN) : a.N, M = a.M;
  const int C = CT ? (1 << LOGC) : a.C, logC = CT ? LOGC : a.logC;
  float2 *X, *tw;
  unsigned short* perm;
  const int ml = CT ? 4 : (a.maxlog == 3 ? 3 : 4);
  time_tile_setup(smraw, N, C, a.tw, X, tw, perm, ml);
  float2* B0 = reinterpret_cast<float2*>(((size_t)(perm + N) + 15) & ~(size_t)15);  // [2][C]
  // U staging ring: RING levels x 2C points of (hi, lo) pairs
  float2* ring = reinterpret_cast<float2*>(((size_t)(B0 + 2 * C) + 15) & ~(size_t)15);
  const int RING = CT ? CT_RING : a.ring, P2 = 2 * C, logP2 = logC + 1;
  const int m0 = blockIdx.x * P2;
  const int J = N / 2 + 1;
  const int q = threadIdx.x & (P2 - 1), r0 = threadIdx.x >> logP2;
  const int LPR = kThreads >> logP2;     // levels per round
  const int depth = CT ? CT_DEPTH : RING / LPR;  // rounds in flight
  const int m = m0 + q;
  const bool valid = m < M;
  __syncthreads();  // perm

  // 1. the half spectra straight into the FFT's permuted rows: A_j (real-part point) into row
  //    perm[j], B_j (imaginary-part point) into row perm[N-j]; B_0 and B_{N/2}, whose partner
  //    rows are their own, into B0
  for (int it = threadIdx.x; it < (J << logC); it += kThreads) {
    const int cc = it & (C - 1), j = it >> logC;
    const int ma = m0 + cc, mb = m0 + C + cc;
    float2* da = X + (size_t)perm[j] * C + cc;
    float2* db = (j == 0 || j == N / 2) ? B0 + (j == 0 ? 0 : C) + cc : X + (size_t)perm[N - j] * C + cc;
    if (ma < M) cp_async8(da, a.S + (size_t)j * M + ma);
    else *da = make_float2(0.f, 0.f);
    if (mb < M) cp_async8(db, a.S + (size_t)j * M + mb);
    else *db = make_float2(0.f, 0.f);
  }
  cp_async_commit();
  // 2. the first rounds of U into the ring (one group per round)
  const float2* u_src = a.U + m;
  if constexpr (!V0) {
    for (int d = 0; d < depth; ++d) {
      const int i = d * LPR + r0;  // < RING
      if (valid && i < N) cp_async8(ring + (i << logP2) + q, u_src + (size_t)i * M);
      cp_async_commit();
    }
    // 3. spectrum complete (the depth U groups committed after it may still be pending)
    if constexpr (CT) cp_async_wait<CT_DEPTH < 7 ? CT_DEPTH : 7>();
    else cp_async_wait_pending(depth);
  } else {
    cp_async_wait_all();
  }
  __syncthreads();
  for (int it = threadIdx.x; it < (J << logC); it += kThreads) {
    const int cc = it & (C - 1), j = it >> logC;
    float2* pa = X + (size_t)perm[j] * C + cc;
    const float2 A = *pa;
    if (j == 0 || j == N / 2) {
      const float2 B = B0[(j == 0 ? 0 : C) + cc];
      *pa = make_float2(A.x - B.y, A.y + B.x);
    } else {
      float2* pb = X + (size_t)perm[N - j] * C + cc;
      const float2 B = *pb;
      *pa = make_float2(A.x - B.y, A.y + B.x);   // Z_j = A_j + i B_j
      *pb = make_float2(A.x + B.y, B.x - A.y);   // Z_{N-j} = conj(A_j) + i conj(B_j)
    }
  }
  __syncthreads();
  if constexpr (CT) fft_inverse_ct<LOGN, LOGC, (1 << LOGC)>(X, tw);
  else fft_inverse_ml(X, C, logC, N, tw, ml);

  // 4. U += c, level by level through the ring
  float sc = 0.f, su = 0.f;  // per-thread partial norms (FP32: the FP64 pipe is ~1/70 rate)
  const float* Xf = reinterpret_cast<const float*>(X) + 2 * (q & (C - 1)) + (q >= C ? 1 : 0);
  float2* u_dst = a.U + m;
  if constexpr (V0) {
    const ff u0 = valid ? ff_from_double(a.v[m]) : ff{0.f, 0.f};
    for (int i = r0; i < N; i += LPR) {
      const float cval = Xf[(size_t)2 * i * C] * __ldg(a.inv_s + i);
      if (valid) {
        const ff u = ff_add_f(u0, cval);
        u_dst[(size_t)i * M] = make_float2(u.hi, u.lo);
        sc = fmaf(cval, cval, sc);
        su = fmaf(u.hi, u.hi, su);
      }
    }
    block_reduce_add2f(sc, su, a.norms);
    return;
  }
  for (int i = r0; i < N; i += LPR) {
    if constexpr (CT) cp_async_wait<(CT_DEPTH - 1 < 7 ? CT_DEPTH - 1 : 7)>();
    else cp_async_wait_pending(depth - 1);  // the group of level i is complete
    const int slot = ((i & (RING - 1)) << logP2) + q;
    const float cval = Xf[(size_t)2 * i * C] * __ldg(a.inv_s + i);
    const size_t row = (size_t)i * M;
    if (valid) {
      const float2 r = ring[slot];
      const ff u = ff_add_f(ff{r.x, r.y}, cval);
      u_dst[row] = make_float2(u.hi, u.lo);
      sc = fmaf(cval, cval, sc);
      su = fmaf(u.hi, u.hi, su);
    }
    if (valid && i + RING < N) cp_async8(ring + slot, u_src + row + (size_t)RING * M);
    cp_async_commit();
  }
  cp_async_wait_all();
  block_reduce_add2f(sc, su, a.norms);
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
      // the kappa term at point q of row i (zero outside the grid): CQ, z = kappa tau^-alpha (W' U)
      // (eq. (3.12)); BDF row n = i+1 <= k, kappa tau^-1 sum_{j=n}^{k} omega_j U^{N+n-j}, the
      // kappa-term of eq. (2.7) indexed to match B_k(kappa) of eq. (2.6) (the printed
      // sum_{j=1}^{n} omega_j U^{N-j+1} has another fixed point)
      auto kterm = [&](int q) -> T {
        if (q < 0 || q >= M) return T(0);
        if (a.z) return (T)a.z[(size_t)i * M + q];
        T c = T(0);
#pragma unroll
        for (int j = 1; j <= kMaxK; ++j)
          if (j > i && j <= a.k) c += a.kw[j] * a.U[(size_t)(N + i - j) * M + q];
        return c;
      };
      T f = a.F[idx];
      if (a.z || i < a.k) {
        // P1 elements: the time terms of the scheme act through the mass matrix M_h
        if (a.fem) f += a.h6 * (kterm(m - 1) + T(4) * kterm(m) + kterm(m + 1));
        else f += kterm(m);
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
  T sd = T(0), su = T(0);
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
      sd += d * d;
      su += un * un;
    }
  }
  if constexpr (sizeof(T) == 4) block_reduce_add2f(sd, su, a.norms);
  else block_reduce_add2(sd, su, a.norms);
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
        else if (a.ukind == 1) val[h] = ff_to_double(ff{a.Uff[idx].x, a.Uff[idx].y});
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
// pipes (~48-bit significand; GB300's FP64 pipe is ~70x slower than its FP32 pipes), in the
// lazy form (ffz: renormalised once per pass, when a value is stored).
// ---------------------------------------------------------------------------
size_t toep_ff_smem(int N, int C) { return time_tile_bytes<ffc>(2 * N, C); }

__global__ void __launch_bounds__(kThreads) k_toeplitz_ff(ToepFFArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M, L = 2 * a.N, logC = a.logC;
  ffz* X = reinterpret_cast<ffz*>(smraw);
  ffz* tw = X + (size_t)L * C;
  unsigned short* perm = reinterpret_cast<unsigned short*>(tw + L);
  const ffz* gtw = reinterpret_cast<const ffz*>(a.tw);
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = gtw[i];
  (void)perm;
  const int m0 = blockIdx.x * 2 * C;
  for (int it = threadIdx.x; it < (L << logC); it += blockDim.x) {
    const int cc = it & (C - 1), i = it >> logC;
    ffz v = {0.f, 0.f, 0.f, 0.f};
    if (i < N) {
      const int ma = m0 + cc, mb = m0 + C + cc;
      const size_t row = (size_t)i * M;
      if (ma < M) { const float2 u = a.U[row + ma]; v.rh = u.x; v.rl = u.y; }
      if (mb < M) { const float2 u = a.U[row + mb]; v.ih = u.x; v.il = u.y; }
    }
    X[(size_t)i * C + cc] = v;
  }
  __syncthreads();
  fft_forward<kToepFFMaxLog>(X, C, logC, L, tw);
  const ffz* what = reinterpret_cast<const ffz*>(a.what);
  for (int it = threadIdx.x; it < (L << logC); it += blockDim.x) {
    const int cc = it & (C - 1), p = it >> logC;
    X[(size_t)p * C + cc] = cmul(X[(size_t)p * C + cc], what[p]);
  }
  __syncthreads();
  fft_inverse<kToepFFMaxLog>(X, C, logC, L, tw);
  for (int it = threadIdx.x; it < (N << logC); it += blockDim.x) {
    const int cc = it & (C - 1), i = it >> logC;
    const ffz z = X[(size_t)i * C + cc];
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
// grid: x over points (one thread per point m), y over slices of consecutive levels
__global__ void k_rhs(RhsArgs a) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= a.M) return;
  const int per = (a.N + gridDim.y - 1) / gridDim.y;
  const int i0 = blockIdx.y * per, i1 = min(a.N, i0 + per);
  const double vm = a.v[m];
  // the beta term acts on v (FD) or on M_h v = (h/6)(v_{i-1} + 4 v_i + v_{i+1}) (P1 FEM); A v is
  // the stencil with weight gx (1/h^2 FD, 1/h for the P1 stiffness)
  double bv = vm;
  if (a.fem) {
    const int x = m % a.mx;
    bv = 4.0 * vm;
    if (x > 0) bv += a.v[m - 1];
    if (x < a.mx - 1) bv += a.v[m + 1];
    bv *= a.mass6;
  }
  double Av = 0.0;
  if (i0 < a.k - 1) {
    // the stencil; on periodic axes the neighbours wrap around
    const int x = m % a.mx;
    const bool per = a.periodic != 0;
    Av = 2.0 * a.gx * vm;
    if (x > 0) Av -= a.gx * a.v[m - 1];
    else if (per) Av -= a.gx * a.v[m + a.mx - 1];
    if (x < a.mx - 1) Av -= a.gx * a.v[m + 1];
    else if (per) Av -= a.gx * a.v[m + 1 - a.mx];
    if (a.dim >= 2) {
      // y neighbours inside the (x, y) plane of the point
      const int mxy = a.mx * a.my;
      const int mp = a.dim == 3 ? m % mxy : m, Mp = a.dim == 3 ? mxy : a.M;
      Av += 2.0 * a.gy * vm;
      if (mp >= a.mx) Av -= a.gy * a.v[m - a.mx];
      else if (per) Av -= a.gy * a.v[m - a.mx + a.M];
      if (mp + a.mx < Mp) Av -= a.gy * a.v[m + a.mx];
      else if (per) Av -= a.gy * a.v[m + a.mx - a.M];
      if (a.dim == 3) {
        Av += 2.0 * a.gz * vm;
        if (m >= mxy) Av -= a.gz * a.v[m - mxy];
        if (m + mxy < a.M) Av -= a.gz * a.v[m + mxy];
      }
    }
  }
  constexpr int B = 4;
  for (int ib = i0; ib < i1; ib += B) {
    double f[B];
#pragma unroll
    for (int b = 0; b < B; ++b) f[b] = ib + b < i1 ? a.f[(size_t)(ib + b) * a.M + m] : 0.0;
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int i = ib + b;
      if (i >= i1) break;
      // (beta_n = 0 beyond the first k levels of BDF-k: no FP64 arithmetic there, the FP64
      // pipe runs at ~1/70 of the FP32 rate; the test is on the bit pattern, an integer compare)
      const double bn = a.beta[i];
      double F = __double_as_longlong(bn) != 0 ? fma(bn, bv, f[b]) : f[b];
      if (i < a.k - 1) {
        F += a.a[i] * (a.fd[m] - Av);
        for (int l = 1; l <= a.k - 2; ++l) F += a.bt[l][i] * a.fd[(size_t)l * a.M + m];
      }
      a.F[(size_t)i * a.M + m] = F;
    }
  }
}

// ---------------------------------------------------------------------------
// conversions (integer bit manipulation; see ff.cuh)
// ---------------------------------------------------------------------------
__global__ void k_d2ff(const double* __restrict__ x, float2* __restrict__ y, size_t n) {
  constexpr int B = 4;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t0 < n; t0 += B * stride) {
    double v[B];
#pragma unroll
    for (int b = 0; b < B; ++b) v[b] = t0 + b * stride < n ? x[t0 + b * stride] : 0.0;
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const size_t t = t0 + b * stride;
      if (t < n) {
        const ff r = ff_from_double(v[b]);
        y[t] = make_float2(r.hi, r.lo);
      }
    }
  }
}
// grid: x over points, y over slices of levels; U^n = v for every level n
__global__ void k_bcast_d2ff(const double* v, float2* U, int N, int M) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int per = (N + gridDim.y - 1) / gridDim.y;
  const int i0 = blockIdx.y * per, i1 = min(N, i0 + per);
  const ff r = ff_from_double(v[m]);
  for (int i = i0; i < i1; ++i) U[(size_t)i * M + m] = make_float2(r.hi, r.lo);
}
__global__ void k_bcast_d(const double* v, double* U, int N, int M) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int per = (N + gridDim.y - 1) / gridDim.y;
  const int i0 = blockIdx.y * per, i1 = min(N, i0 + per);
  const double vm = v[m];
  for (int i = i0; i < i1; ++i) U[(size_t)i * M + m] = vm;
}
__global__ void k_ff2d(const float2* __restrict__ y, double* __restrict__ x, size_t n) {
  constexpr int B = 4;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t0 < n; t0 += B * stride) {
    float2 h[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const size_t t = t0 + b * stride;
      h[b] = t < n ? y[t] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int b = 0; b < B; ++b)
      if (t0 + b * stride < n) x[t0 + b * stride] = ff_to_double(ff{h[b].x, h[b].y});
  }
}
__global__ void k_d2f(const double* __restrict__ x, float* __restrict__ y, size_t n) {
  constexpr int B = 4;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t0 < n; t0 += B * stride) {
    double v[B];
#pragma unroll
    for (int b = 0; b < B; ++b) v[b] = t0 + b * stride < n ? x[t0 + b * stride] : 0.0;
#pragma unroll
    for (int b = 0; b < B; ++b)
      if (t0 + b * stride < n) y[t0 + b * stride] = ff_from_double(v[b]).hi;
  }
}
__global__ void k_f2d(const float* __restrict__ x, double* __restrict__ y, size_t n) {
  constexpr int B = 4;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t0 < n; t0 += B * stride) {
    float v[B];
#pragma unroll
    for (int b = 0; b < B; ++b) v[b] = t0 + b * stride < n ? x[t0 + b * stride] : 0.f;
#pragma unroll
    for (int b = 0; b < B; ++b)
      if (t0 + b * stride < n) y[t0 + b * stride] = f2d_bits(v[b]);
  }
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
    c->err = 0;
  }
}

__global__ void k_converge(const double* norms, SolveCtl* c, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double c2 = norms[0], u2 = norms[1];
  const double upd = u2 > 0.0 ? sqrt(c2 / u2) : sqrt(c2);
  const int m = c->m + 1;
  const bool done = c->err == 0 && stop_decision(m, upd, c->prev, c->tol, c->q_floor);
  c->m = m;
  c->prev = upd;
  c->upd = upd;
  c->done = done ? 1 : 0;
  cudaGraphSetConditional(h, (!done && m < c->max_sweeps && c->err == 0) ? 1u : 0u);
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

// points along x (one thread each), slices of levels along y: about 8 CTAs per SM in total
static dim3 grid_pts(int M, int N) {
  const int bx = (M + kThreads - 1) / kThreads;
  int by = (152 * 8 + bx - 1) / bx;
  if (by > N) by = N;
  if (by < 1) by = 1;
  return dim3((unsigned)bx, (unsigned)by, 1);
}

static int grid_for(size_t n) {
  size_t b = (n + kThreads - 1) / kThreads;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b ? b : 1);
}





template <int LOGN, int LOGC> static cudaError_t launch_inv_k(const InvUpdArgs& a, cudaStream_t st) {
  const size_t sm = inv_upd_smem(a.N, a.C);
  InvUpdArgs b = a;
  b.ring = inv_ring_levels(a.N, a.C);
  if (a.v) {
    cudaError_t e = set_smem(k_inv_upd<LOGN, LOGC, true>, sm);
    if (e != cudaSuccess) return e;
    prof_begin("inv_update_v0_ff", st);
    k_inv_upd<LOGN, LOGC, true><<<tiles(a.M, a.C), kThreads, sm, st>>>(b);
  } else {
    cudaError_t e = set_smem(k_inv_upd<LOGN, LOGC, false>, sm);
    if (e != cudaSuccess) return e;
    prof_begin("inv_update_ff", st);
    k_inv_upd<LOGN, LOGC, false><<<tiles(a.M, a.C), kThreads, sm, st>>>(b);
  }
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_inv_upd(const InvUpdArgs& a, cudaStream_t st) {
  // compiled shapes: the tile widths the plan picks for large grids at these N
  if (a.N == 128 && a.C == 16) return launch_inv_k<7, 4>(a, st);
  if (a.N == 256 && a.C == 16) return launch_inv_k<8, 4>(a, st);
  if (a.N == 512 && a.C == 16) return launch_inv_k<9, 4>(a, st);
  if (a.N == 1024 && a.C == 8) return launch_inv_k<10, 3>(a, st);
  if (a.N == 2048 && a.C == 4) return launch_inv_k<11, 2>(a, st);
  if (a.N == 4096 && a.C == 2) return launch_inv_k<12, 1>(a, st);
  return launch_inv_k<0, 0>(a, st);
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
  prof_begin(a.head ? "rhs_head_f64" : "rhs_f64", st);
  k_rhs<<<grid_pts(a.M, a.N), kThreads, 0, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_d2ff(const double* x, float2* y, size_t n, cudaStream_t st) {
  prof_begin("cvt_d2ff", st);
  k_d2ff<<<grid_for(n), kThreads, 0, st>>>(x, y, n);
  prof_end(st);
  return cudaGetLastError();
}
cudaError_t launch_bcast_d2ff(const double* v, float2* U, int N, int M, cudaStream_t st) {
  prof_begin("cvt_bcast_d2ff", st);
  k_bcast_d2ff<<<grid_pts(M, N), kThreads, 0, st>>>(v, U, N, M);
  prof_end(st);
  return cudaGetLastError();
}
cudaError_t launch_bcast_d(const double* v, double* U, int N, int M, cudaStream_t st) {
  prof_begin("initial_guess", st);
  k_bcast_d<<<grid_pts(M, N), kThreads, 0, st>>>(v, U, N, M);
  prof_end(st);
  return cudaGetLastError();
}
cudaError_t launch_ff2d(const float2* y, double* x, size_t n, cudaStream_t st) {
  prof_begin("cvt_ff2d", st);
  k_ff2d<<<grid_for(n), kThreads, 0, st>>>(y, x, n);
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
