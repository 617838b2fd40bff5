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
// One thread owns one point of the tile and marches through a block of N/G consecutive levels
// (G level groups per CTA). The k previous levels of its U stay in registers, so each level
// reads U, its y neighbours, F_hat (and y) once, straight from global memory with coalesced
// loads issued one level ahead (four CTAs per SM hide the rest of the latency); x neighbours
// come from the adjacent lanes by warp shuffles (global loads only at warp edges). The
// residuals go into the shared-memory tile, which is then transformed along time.
//
// The stencil coefficients 1/hx^2, 1/hy^2 are powers of two (mx + 1, my + 1 are), so the four
// neighbour terms are two exact double-float sums scaled exactly; only the BDF weights and the
// stencil centre need error-free products.
// ---------------------------------------------------------------------------

// level groups of a residual tile: up to kThreads / 2C, each with at least 4 levels
__host__ __device__ inline int resid_groups(int N, int C) {
  int g = kThreads / (2 * C);
  while (g > 1 && N / g < 4) g >>= 1;
  return g;
}

size_t resid_fwd_smem(int N, int C) { return time_tile_bytes<float2>(N, C) + 16; }

// one level of one point as loaded from global memory
struct ResidLevel {
  float uh, ul;    // U
  float wh, wl;    // west neighbour (only where no lane holds it)
  float eh, el;    // east neighbour (idem)
  float sh, sl;    // south neighbour (m - mx)
  float nh, nl;    // north neighbour (m + mx)
  float bh, bl;    // 3D: bottom neighbour (m - mx my)
  float th, tl;    // 3D: top neighbour (m + mx my)
  float yh, yl;    // CQ history
  float ywh, ywl;  // P1 FEM + CQ: west / east neighbours of the history (warp edges)
  float yeh, yel;
  double f;        // F_hat
  float s;         // kappa^{i/N}
};

// FEM = P1 finite elements (1D): the time terms act on V = M_h U, the history registers hold V,
// and the stiffness K_h U = (1/h)(2 U_i - U_{i-1} - U_{i+1}) replaces the FD stencil.
// PER = periodic axes: the stencil's neighbours wrap around (compile-time, so that Dirichlet
// instances keep constant neighbour offsets).
template <int K, bool CQ, int DIM, bool FEM, bool PER>
__global__ void __launch_bounds__(kThreads, 4) k_resid_fwd(ResidFwdArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M, logC = a.logC, mx = a.mx;
  float2 *X, *tw;
  unsigned short* perm;
  time_tile_setup(smraw, N, C, a.tw, X, tw, perm);

  const int P2 = 2 * C, logP2 = logC + 1;
  const int G = resid_groups(N, C), NL = N / G;
  const int q = threadIdx.x & (P2 - 1), g = threadIdx.x >> logP2;
  const int lane = threadIdx.x & 31;
  const int m = blockIdx.x * P2 + q;
  const bool valid = g < G && m < M;
  constexpr bool two_d = DIM >= 2, three_d = DIM == 3, cq = CQ;
  const int mxy = mx * a.my;  // z-neighbour distance (3D)
  const int xq = m % mx;
  // neighbour offsets (wrapping around on periodic axes) and which neighbours exist
  constexpr bool per = PER;
  const int dW = (!per || xq > 0) ? -1 : mx - 1, dE = (!per || xq < mx - 1) ? 1 : 1 - mx;
  const int dS = (!per || m >= mx) ? -mx : M - mx, dN = (!per || m + mx < M) ? mx : mx - M;
  const bool hasW = valid && (xq > 0 || per), hasE = valid && (xq < mx - 1 || per);
  // y neighbours stay inside the (x, y) plane of the point (3D: planes of mx * my points)
  const int mp = three_d ? m % mxy : m, Mp = three_d ? mxy : M;
  const bool hasS = valid && two_d && (mp >= mx || per), hasN = valid && two_d && (mp + mx < Mp || per);
  const bool hasB = valid && three_d && m >= mxy, hasT = valid && three_d && m + mxy < M;
  // x neighbours by shuffle when a warp holds 32 consecutive points of one level; a lane loads
  // its neighbour itself at warp edges and where a periodic row wraps
  const bool shfl = P2 >= 32;
  const bool ldW = hasW && (!shfl || lane == 0 || (per && xq == 0));
  const bool ldE = hasE && (!shfl || lane == 31 || (per && xq == mx - 1));
  float* Xf = reinterpret_cast<float*>(X) + 2 * (q & (C - 1)) + (q >= C ? 1 : 0);

  auto load = [&](int i) {
    ResidLevel v;
    const size_t idx = (size_t)i * M + m;
    v.uh = valid ? a.Uhi[idx] : 0.f;
    v.ul = valid ? a.Ulo[idx] : 0.f;
    v.wh = ldW ? a.Uhi[idx + dW] : 0.f;
    v.wl = ldW ? a.Ulo[idx + dW] : 0.f;
    v.eh = ldE ? a.Uhi[idx + dE] : 0.f;
    v.el = ldE ? a.Ulo[idx + dE] : 0.f;
    if (two_d) {
      v.sh = hasS ? a.Uhi[idx + dS] : 0.f;
      v.sl = hasS ? a.Ulo[idx + dS] : 0.f;
      v.nh = hasN ? a.Uhi[idx + dN] : 0.f;
      v.nl = hasN ? a.Ulo[idx + dN] : 0.f;
    } else {
      v.sh = v.sl = v.nh = v.nl = 0.f;
    }
    if (three_d) {
      v.bh = hasB ? a.Uhi[idx - mxy] : 0.f;
      v.bl = hasB ? a.Ulo[idx - mxy] : 0.f;
      v.th = hasT ? a.Uhi[idx + mxy] : 0.f;
      v.tl = hasT ? a.Ulo[idx + mxy] : 0.f;
    } else {
      v.bh = v.bl = v.th = v.tl = 0.f;
    }
    if (cq) {
      v.yh = valid ? a.yhi[idx] : 0.f;
      v.yl = valid ? a.ylo[idx] : 0.f;
    } else {
      v.yh = 0.f;
      v.yl = 0.f;
    }
    if (FEM && cq) {
      v.ywh = ldW ? a.yhi[idx + dW] : 0.f;
      v.ywl = ldW ? a.ylo[idx + dW] : 0.f;
      v.yeh = ldE ? a.yhi[idx + dE] : 0.f;
      v.yel = ldE ? a.ylo[idx + dE] : 0.f;
    } else {
      v.ywh = v.ywl = v.yeh = v.yel = 0.f;
    }
    v.f = valid ? a.F[idx] : 0.0;
    v.s = __ldg(a.s + i);
    return v;
  };

  // x neighbours of a per-point double-float value: adjacent lanes, or the values this lane
  // loaded itself (warp edges, periodic wrap); zero beyond a Dirichlet boundary. (shfl is
  // uniform over the CTA and then every warp is fully inside one level group.)
  auto neighbours = [&](float ch, float cl, float ewh, float ewl, float eeh, float eel, float& wh, float& wl,
                        float& eh, float& el) {
    wh = ewh; wl = ewl; eh = eeh; el = eel;
    if (shfl) {
      const float uwh = __shfl_up_sync(0xffffffffu, ch, 1), uwl = __shfl_up_sync(0xffffffffu, cl, 1);
      const float ueh = __shfl_down_sync(0xffffffffu, ch, 1), uel = __shfl_down_sync(0xffffffffu, cl, 1);
      if (!ldW) { wh = uwh; wl = uwl; }
      if (!ldE) { eh = ueh; el = uel; }
    }
    if (!hasW) { wh = 0.f; wl = 0.f; }
    if (!hasE) { eh = 0.f; el = 0.f; }
  };
  // one row of the P1 mass matrix, (h/6)(u_{i-1} + 4 u_i + u_{i+1}), in double-float
  auto mass = [&](float ch, float cl, float wh, float wl, float eh, float el) {
    float b1, e1, b2, e2;
    two_sum(wh, eh, b1, e1);
    two_sum(b1, 4.f * ch, b2, e2);
    const float lo = e1 + e2 + ((wl + el) + 4.f * cl);
    return ff_mul(ff{b2, lo}, ff{a.m_hi, a.m_lo});
  };

  if (g < G) {
    const int i0 = g * NL, i1 = i0 + NL;
    // the K levels before i0 (zero before level 0): U, or M_h U for P1 elements
    ff h[K > 0 ? K : 1];
#pragma unroll
    for (int t = 0; t < K; ++t) {
      const int lev = i0 - 1 - t;
      const size_t idx = (size_t)(lev >= 0 ? lev : 0) * M + m;
      h[t].hi = (valid && lev >= 0) ? a.Uhi[idx] : 0.f;
      h[t].lo = (valid && lev >= 0) ? a.Ulo[idx] : 0.f;
      if constexpr (FEM) {
        float wh, wl, eh, el;
        neighbours(h[t].hi, h[t].lo, (ldW && lev >= 0) ? a.Uhi[idx + dW] : 0.f,
                   (ldW && lev >= 0) ? a.Ulo[idx + dW] : 0.f, (ldE && lev >= 0) ? a.Uhi[idx + dE] : 0.f,
                   (ldE && lev >= 0) ? a.Ulo[idx + dE] : 0.f, wh, wl, eh, el);
        h[t] = mass(h[t].hi, h[t].lo, wh, wl, eh, el);
      }
    }
    const float gx = a.gx_hi, gy = a.gy_hi, gz = a.gz_hi;
    // reaction term w c_i U_i^n (1D, the linearised operator of Algorithm 3): one coefficient per point
    const bool react = DIM == 1 && a.react != nullptr;
    const ff rc = (react && valid) ? ff_from_double(a.react[m]) : ff{0.f, 0.f};
    ResidLevel nx = load(i0);
#pragma unroll 2
    for (int i = i0; i < i1; ++i) {
      const ResidLevel c = nx;
      if (i + 1 < i1) nx = load(i + 1);

      float wh, wl, eh, el;
      neighbours(c.uh, c.ul, c.wh, c.wl, c.eh, c.el, wh, wl, eh, el);

      ff_acc A;
      A.init(ff_split_trunc(c.f));
      ff cur;  // what the history keeps of this level
      if constexpr (FEM) {
        // F_hat - M_h (tau^-alpha sum_j omega_j U^{n-j}) - K_h U^n
        cur = mass(c.uh, c.ul, wh, wl, eh, el);
        if constexpr (CQ) {
          float ywh, ywl, yeh, yel;
          neighbours(c.yh, c.yl, c.ywh, c.ywl, c.yeh, c.yel, ywh, ywl, yeh, yel);
          A.sub(mass(c.yh, c.yl, ywh, ywl, yeh, yel));
        } else {
          A.fma_term(ff{a.c_hi[0], a.c_lo[0]}, cur, -1.f);
        }
#pragma unroll
        for (int t = 1; t <= K; ++t) A.fma_term(ff{a.c_hi[t], a.c_lo[t]}, h[t - 1], -1.f);
        // stiffness centre 2/h and neighbours 1/h: powers of two, exact
        A.add_hi(-2.f * gx * c.uh);
        A.sl = fmaf(-2.f * gx, c.ul, A.sl);
        float bx, ex;
        two_sum(wh, eh, bx, ex);
        A.add_hi(gx * bx);
        A.sl += gx * (ex + (wl + el));
      } else {
        cur = ff{c.uh, c.ul};
        // stencil centre, BDF history (and CQ history): error-free products
        if constexpr (CQ) A.sub(ff{c.yh, c.yl});
        A.fma_term(ff{a.c_hi[0], a.c_lo[0]}, cur, -1.f);
#pragma unroll
        for (int t = 1; t <= K; ++t) A.fma_term(ff{a.c_hi[t], a.c_lo[t]}, h[t - 1], -1.f);
        // neighbours: exact sums, exact power-of-two scaling
        float bx, ex;
        two_sum(wh, eh, bx, ex);
        A.add_hi(gx * bx);
        float lo = gx * (ex + (wl + el));
        if constexpr (DIM >= 2) {
          float by, ey;
          two_sum(c.sh, c.nh, by, ey);
          A.add_hi(gy * by);
          lo = fmaf(gy, ey + (c.sl + c.nl), lo);
        }
        if constexpr (DIM == 3) {
          float bz, ez;
          two_sum(c.bh, c.th, bz, ez);
          A.add_hi(gz * bz);
          lo = fmaf(gz, ez + (c.bl + c.tl), lo);
        }
        A.sl += lo;
      }
      if constexpr (DIM == 1) {
        if (react) A.fma_term(rc, ff{c.uh, c.ul}, -1.f);
      }
      Xf[(size_t)2 * i * C] = valid ? A.value() * c.s : 0.f;

#pragma unroll
      for (int t = K - 1; t > 0; --t) h[t] = h[t - 1];
      if (K > 0) h[0] = cur;
    }
  }
  __syncthreads();
  // compiled transform shapes for the tile widths the plan picks at these N (uniform branch)
  if (N == 256 && C == 16) fft_forward_ct<8, 4, 16>(X, tw);
  else if (N == 512 && C == 16) fft_forward_ct<9, 4, 16>(X, tw);
  else if (N == 1024 && C == 8) fft_forward_ct<10, 3, 8>(X, tw);
  else fft_forward(X, C, logC, N, tw);
  store_half_spectrum(X, perm, a.S, N, M, C, logC, (int)blockIdx.x * P2);
}

// ---------------------------------------------------------------------------
// MIXED: inverse DFT + unscale + U += c (double-float) + norms
// ---------------------------------------------------------------------------
// U staging ring of the update: RING levels x 2C points, hi and lo
__host__ __device__ constexpr size_t inv_ring_bytes(int C, int ring) { return 2 * sizeof(float) * (size_t)ring * 2 * C; }
__host__ __device__ constexpr size_t inv_upd_smem_ring(int N, int C, int ring) {
  return sizeof(float2) * ((size_t)N * C + N) + sizeof(unsigned short) * (size_t)N + 16 +
         2 * sizeof(float2) * (size_t)C + 16 + inv_ring_bytes(C, ring);
}
// ring depth: as many levels (a power of two, at most 64) as fit next to the tile with three
// CTAs per SM, at least one round of kThreads / 2C levels and at most N
__host__ __device__ constexpr int inv_ring_levels(int N, int C) {
  int ring = 64;
  while (ring > kThreads / (2 * C) && inv_upd_smem_ring(N, C, ring) > 72 * 1024) ring >>= 1;
  if (ring > N) ring = N;
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
__global__ void __launch_bounds__(kThreads, 3) k_inv_upd(InvUpdArgs a) {
  constexpr bool CT = LOGN > 0;
  constexpr int CT_RING = CT ? inv_ring_levels(1 << LOGN, 1 << LOGC) : 1;
  constexpr int CT_DEPTH = CT ? CT_RING / (kThreads >> (LOGC + 1)) : 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = CT ? (1 << LOGN) : a.N, M = a.M;
  const int C = CT ? (1 << LOGC) : a.C, logC = CT ? LOGC : a.logC;
  float2 *X, *tw;
  unsigned short* perm;
  time_tile_setup(smraw, N, C, a.tw, X, tw, perm);
  float2* B0 = reinterpret_cast<float2*>(((size_t)(perm + N) + 15) & ~(size_t)15);  // [2][C]
  float* ring_h = reinterpret_cast<float*>(((size_t)(B0 + 2 * C) + 15) & ~(size_t)15);
  const int RING = CT ? CT_RING : a.ring, P2 = 2 * C, logP2 = logC + 1;
  float* ring_l = ring_h + (size_t)RING * P2;
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
  const float* uh_src = a.Uhi + m;
  const float* ul_src = a.Ulo + m;
  if constexpr (!V0) {
    for (int d = 0; d < depth; ++d) {
      const int i = d * LPR + r0;  // < RING
      if (valid && i < N) {
        cp_async4(ring_h + (i << logP2) + q, uh_src + (size_t)i * M);
        cp_async4(ring_l + (i << logP2) + q, ul_src + (size_t)i * M);
      }
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
  else fft_inverse(X, C, logC, N, tw);

  // 4. U += c, level by level through the ring
  float sc = 0.f, su = 0.f;  // per-thread partial norms (FP32: the FP64 pipe is ~1/70 rate)
  const float* Xf = reinterpret_cast<const float*>(X) + 2 * (q & (C - 1)) + (q >= C ? 1 : 0);
  float* uh_dst = a.Uhi + m;
  float* ul_dst = a.Ulo + m;
  if constexpr (V0) {
    const ff u0 = valid ? ff_from_double(a.v[m]) : ff{0.f, 0.f};
    for (int i = r0; i < N; i += LPR) {
      const float cval = Xf[(size_t)2 * i * C] * __ldg(a.inv_s + i);
      if (valid) {
        const ff u = ff_add_f(u0, cval);
        uh_dst[(size_t)i * M] = u.hi;
        ul_dst[(size_t)i * M] = u.lo;
        sc = fmaf(cval, cval, sc);
        su = fmaf(u.hi, u.hi, su);
      }
    }
    block_reduce_add2((double)sc, (double)su, a.norms);
    return;
  }
  for (int i = r0; i < N; i += LPR) {
    if constexpr (CT) cp_async_wait<(CT_DEPTH - 1 < 7 ? CT_DEPTH - 1 : 7)>();
    else cp_async_wait_pending(depth - 1);  // the group of level i is complete
    const int slot = ((i & (RING - 1)) << logP2) + q;
    const float cval = Xf[(size_t)2 * i * C] * __ldg(a.inv_s + i);
    const size_t row = (size_t)i * M;
    if (valid) {
      const ff u = ff_add_f(ff{ring_h[slot], ring_l[slot]}, cval);
      uh_dst[row] = u.hi;
      ul_dst[row] = u.lo;
      sc = fmaf(cval, cval, sc);
      su = fmaf(u.hi, u.hi, su);
    }
    if (valid && i + RING < N) {
      cp_async4(ring_h + slot, uh_src + row + (size_t)RING * M);
      cp_async4(ring_l + slot, ul_src + row + (size_t)RING * M);
    }
    cp_async_commit();
  }
  cp_async_wait_all();
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
      double F = fma(a.beta[i], bv, f[b]);
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
__global__ void k_d2ff(const double* __restrict__ x, float* __restrict__ hi, float* __restrict__ lo, size_t n) {
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
        hi[t] = r.hi;
        lo[t] = r.lo;
      }
    }
  }
}
// grid: x over points, y over slices of levels; U^n = v for every level n
__global__ void k_bcast_d2ff(const double* v, float* hi, float* lo, int N, int M) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int per = (N + gridDim.y - 1) / gridDim.y;
  const int i0 = blockIdx.y * per, i1 = min(N, i0 + per);
  const ff r = ff_from_double(v[m]);
  for (int i = i0; i < i1; ++i) {
    hi[(size_t)i * M + m] = r.hi;
    lo[(size_t)i * M + m] = r.lo;
  }
}
__global__ void k_bcast_d(const double* v, double* U, int N, int M) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int per = (N + gridDim.y - 1) / gridDim.y;
  const int i0 = blockIdx.y * per, i1 = min(N, i0 + per);
  const double vm = v[m];
  for (int i = i0; i < i1; ++i) U[(size_t)i * M + m] = vm;
}
__global__ void k_ff2d(const float* __restrict__ hi, const float* __restrict__ lo, double* __restrict__ x, size_t n) {
  constexpr int B = 4;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t0 < n; t0 += B * stride) {
    float h[B], l[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const size_t t = t0 + b * stride;
      h[b] = t < n ? hi[t] : 0.f;
      l[b] = t < n ? lo[t] : 0.f;
    }
#pragma unroll
    for (int b = 0; b < B; ++b)
      if (t0 + b * stride < n) x[t0 + b * stride] = ff_to_double(ff{h[b], l[b]});
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

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

static int tiles(int M, int C) { return (M + 2 * C - 1) / (2 * C); }

// ---------------------------------------------------------------------------
// MIXED, first sweep from the initial guess U_0^n = v of every level (Theorem 2.7). Then
// K U_0 = tau^-alpha (sum_{j<n} omega_j) M v + A v = beta_n M v + A v for BDF and CQ alike, so
//   r_0^n = F_hat_n - beta_n M v - A v   (- w c v with a reaction term),
// with A v (and M v) formed once per point: no U is read, no history is formed, and the kernel
// reads F_hat and writes the half spectrum like k_resid_fwd (same tile, same transform).
// ---------------------------------------------------------------------------
template <int DIM, bool FEM, bool PER>
__global__ void __launch_bounds__(kThreads, 4) k_resid_v0(ResidFwdArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M, logC = a.logC, mx = a.mx;
  float2 *X, *tw;
  unsigned short* perm;
  time_tile_setup(smraw, N, C, a.tw, X, tw, perm);
  const int P2 = 2 * C, logP2 = logC + 1;
  const int G = resid_groups(N, C), NL = N / G;
  const int q = threadIdx.x & (P2 - 1), g = threadIdx.x >> logP2;
  const int m = blockIdx.x * P2 + q;
  const bool valid = g < G && m < M;
  constexpr bool two_d = DIM >= 2, three_d = DIM == 3, per = PER;
  const int mxy = mx * a.my;
  const int xq = m % mx;
  const int dW = (!per || xq > 0) ? -1 : mx - 1, dE = (!per || xq < mx - 1) ? 1 : 1 - mx;
  const int dS = (!per || m >= mx) ? -mx : M - mx, dN = (!per || m + mx < M) ? mx : mx - M;
  const bool hasW = valid && (xq > 0 || per), hasE = valid && (xq < mx - 1 || per);
  const int mp = three_d ? m % mxy : m, Mp = three_d ? mxy : M;
  const bool hasS = valid && two_d && (mp >= mx || per), hasN = valid && two_d && (mp + mx < Mp || per);
  const bool hasB = valid && three_d && m >= mxy, hasT = valid && three_d && m + mxy < M;
  float* Xf = reinterpret_cast<float*>(X) + 2 * (q & (C - 1)) + (q >= C ? 1 : 0);

  // A v (and M v for P1) at this point, in double-float
  const ff vc = valid ? ff_from_double(a.v[m]) : ff{0.f, 0.f};
  const ff vw = hasW ? ff_from_double(a.v[m + dW]) : ff{0.f, 0.f};
  const ff ve = hasE ? ff_from_double(a.v[m + dE]) : ff{0.f, 0.f};
  const float gx = a.gx_hi;
  ff_acc Av;
  Av.init(ff{0.f, 0.f});
  // centre: 2 gx + 2 gy + 2 gz (FD), 2/h (P1 stiffness) -- exact multiples of powers of two
  {
    float b0, e0;
    two_sum(vw.hi, ve.hi, b0, e0);
    Av.add_hi(2.f * gx * vc.hi);
    Av.sl = fmaf(2.f * gx, vc.lo, Av.sl);
    Av.add_hi(-gx * b0);
    Av.sl -= gx * (e0 + (vw.lo + ve.lo));
  }
  if constexpr (DIM >= 2) {
    const float gy = a.gy_hi;
    const ff vs = hasS ? ff_from_double(a.v[m + dS]) : ff{0.f, 0.f};
    const ff vn = hasN ? ff_from_double(a.v[m + dN]) : ff{0.f, 0.f};
    float b1, e1;
    two_sum(vs.hi, vn.hi, b1, e1);
    Av.add_hi(2.f * gy * vc.hi);
    Av.sl = fmaf(2.f * gy, vc.lo, Av.sl);
    Av.add_hi(-gy * b1);
    Av.sl -= gy * (e1 + (vs.lo + vn.lo));
  }
  if constexpr (DIM == 3) {
    const float gz = a.gz_hi;
    const ff vb = hasB ? ff_from_double(a.v[m - mxy]) : ff{0.f, 0.f};
    const ff vt = hasT ? ff_from_double(a.v[m + mxy]) : ff{0.f, 0.f};
    float b2, e2;
    two_sum(vb.hi, vt.hi, b2, e2);
    Av.add_hi(2.f * gz * vc.hi);
    Av.sl = fmaf(2.f * gz, vc.lo, Av.sl);
    Av.add_hi(-gz * b2);
    Av.sl -= gz * (e2 + (vb.lo + vt.lo));
  }
  if (DIM == 1 && a.react && valid) Av.fma_term(ff_from_double(a.react[m]), vc, 1.f);
  const ff Avn = Av.normalized();
  ff Mv = vc;
  if constexpr (FEM) {
    // (h/6)(v_{i-1} + 4 v_i + v_{i+1}) in double-float
    float b1, e1, b2, e2;
    two_sum(vw.hi, ve.hi, b1, e1);
    two_sum(b1, 4.f * vc.hi, b2, e2);
    const float lo = e1 + e2 + ((vw.lo + ve.lo) + 4.f * vc.lo);
    Mv = ff_mul(ff{b2, lo}, ff{a.m_hi, a.m_lo});
  }

  if (g < G) {
    // F_hat in batches of 8 independent loads per thread (the only stream of this kernel)
    const int i0 = g * NL, i1 = i0 + NL;
    const double* Fp = a.F + m;
    for (int b = i0; b < i1; b += 8) {
      double f[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) f[t] = (valid && b + t < i1) ? Fp[(size_t)(b + t) * M] : 0.0;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int i = b + t;
        if (i < i1) {
          ff_acc A;
          A.init(ff_split_trunc(f[t]));
          const float2 bt = __ldg(a.beta_ff + i);
          A.fma_term(ff{bt.x, bt.y}, Mv, -1.f);
          A.sub(Avn);
          Xf[(size_t)2 * i * C] = valid ? A.value() * __ldg(a.s + i) : 0.f;
        }
      }
    }
  }
  __syncthreads();
  if (N == 256 && C == 16) fft_forward_ct<8, 4, 16>(X, tw);
  else if (N == 512 && C == 16) fft_forward_ct<9, 4, 16>(X, tw);
  else if (N == 1024 && C == 8) fft_forward_ct<10, 3, 8>(X, tw);
  else fft_forward(X, C, logC, N, tw);
  store_half_spectrum(X, perm, a.S, N, M, C, logC, (int)blockIdx.x * P2);
}

template <int K, bool CQ, int DIM, bool FEM, bool PER>
static cudaError_t launch_resid_k(const ResidFwdArgs& a, size_t sm, cudaStream_t st) {
  cudaError_t e = set_smem(k_resid_fwd<K, CQ, DIM, FEM, PER>, sm);
  if (e != cudaSuccess) return e;
  prof_begin("resid_fwd_ff", st);
  k_resid_fwd<K, CQ, DIM, FEM, PER><<<tiles(a.M, a.C), kThreads, sm, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

template <int DIM, bool FEM, bool PER>
static cudaError_t launch_resid_d(const ResidFwdArgs& a, size_t sm, cudaStream_t st) {
  if (a.yhi) return a.k == 0 ? launch_resid_k<0, true, DIM, FEM, PER>(a, sm, st) : cudaErrorInvalidValue;
  switch (a.k) {
    case 1: return launch_resid_k<1, false, DIM, FEM, PER>(a, sm, st);
    case 2: return launch_resid_k<2, false, DIM, FEM, PER>(a, sm, st);
    case 3: return launch_resid_k<3, false, DIM, FEM, PER>(a, sm, st);
    case 4: return launch_resid_k<4, false, DIM, FEM, PER>(a, sm, st);
    case 5: return launch_resid_k<5, false, DIM, FEM, PER>(a, sm, st);
    case 6: return launch_resid_k<6, false, DIM, FEM, PER>(a, sm, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_resid_fwd(const ResidFwdArgs& a, cudaStream_t st) {
  // the neighbour terms assume exact power-of-two stencil coefficients
  if (a.gx_lo != 0.f || a.gy_lo != 0.f) return cudaErrorInvalidValue;
  const size_t sm = resid_fwd_smem(a.N, a.C);
  if (a.fem) return a.dim == 1 && !a.periodic ? launch_resid_d<1, true, false>(a, sm, st) : cudaErrorInvalidValue;
  if (a.periodic) {
    if (a.dim == 3) return cudaErrorInvalidValue;
    return a.dim == 2 ? launch_resid_d<2, false, true>(a, sm, st) : launch_resid_d<1, false, true>(a, sm, st);
  }
  if (a.dim == 3) return launch_resid_d<3, false, false>(a, sm, st);
  return a.dim == 2 ? launch_resid_d<2, false, false>(a, sm, st) : launch_resid_d<1, false, false>(a, sm, st);
}

template <int DIM, bool FEM, bool PER>
static cudaError_t launch_v0_k(const ResidFwdArgs& a, size_t sm, cudaStream_t st) {
  cudaError_t e = set_smem(k_resid_v0<DIM, FEM, PER>, sm);
  if (e != cudaSuccess) return e;
  prof_begin("resid_v0_ff", st);
  k_resid_v0<DIM, FEM, PER><<<tiles(a.M, a.C), kThreads, sm, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_resid_v0(const ResidFwdArgs& a, cudaStream_t st) {
  if (a.gx_lo != 0.f || a.gy_lo != 0.f || !a.v || !a.beta_ff) return cudaErrorInvalidValue;
  const size_t sm = resid_fwd_smem(a.N, a.C);
  if (a.fem) return a.dim == 1 && !a.periodic ? launch_v0_k<1, true, false>(a, sm, st) : cudaErrorInvalidValue;
  if (a.periodic) {
    if (a.dim == 3) return cudaErrorInvalidValue;
    return a.dim == 2 ? launch_v0_k<2, false, true>(a, sm, st) : launch_v0_k<1, false, true>(a, sm, st);
  }
  if (a.dim == 3) return launch_v0_k<3, false, false>(a, sm, st);
  return a.dim == 2 ? launch_v0_k<2, false, false>(a, sm, st) : launch_v0_k<1, false, false>(a, sm, st);
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
  prof_begin("rhs_f64", st);
  k_rhs<<<grid_pts(a.M, a.N), kThreads, 0, st>>>(a);
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
  k_bcast_d2ff<<<grid_pts(M, N), kThreads, 0, st>>>(v, hi, lo, N, M);
  prof_end(st);
  return cudaGetLastError();
}
cudaError_t launch_bcast_d(const double* v, double* U, int N, int M, cudaStream_t st) {
  prof_begin("initial_guess", st);
  k_bcast_d<<<grid_pts(M, N), kThreads, 0, st>>>(v, U, N, M);
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
