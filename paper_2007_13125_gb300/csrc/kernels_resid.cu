// The all-at-once residual kernels of the MIXED sweep (Algorithm 1 / 2 with the residual-correction
// form): k_resid_fwd (F_hat - K U in double-float, kappa scaling, forward time DFT) and k_resid_v0
// (the same for the first sweep from U_0^n = v). Time tiles as in kernels_time.cu (time_tile.cuh).
#include "time_tile.cuh"

namespace pint {

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

// level groups of a residual tile: up to kThreads / 2C, each with at least 4 levels, and a divisor
// of N (N = 2^a 5^b: a power of two up to 2^a)
__host__ __device__ inline int resid_groups(int N, int C) {
  int g = kThreads / (2 * C);
  while (g > 1 && (N / g < 4 || N % g != 0)) g >>= 1;
  return g;
}

// A += g b with the product's rounding error kept: exact by itself when g is a power of two (the
// stencil weights of grids with m + 1 = 2^a), otherwise the error (one fma) joins the low part.
// `exact` is uniform over the launch.
__device__ __forceinline__ void add_prod(ff_acc& A, float g, float b, bool exact) {
  const float p = g * b;
  A.add_hi(p);
  if (!exact) A.sl += fmaf(g, b, -p);
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
// CTF: the tile shape (N, C) is one of the compiled transforms; otherwise the runtime-shape one.
// Keeping the two apart keeps the compiled instances within 64 registers without spill code.
__host__ __device__ inline bool compiled_time_fft(int N, int C) { return compiled_time_fft_shape(N, C); }
template <bool CTF>
__device__ __forceinline__ void resid_time_fft(float2* X, int C, int logC, int N, const float2* tw, int maxlog) {
  if constexpr (CTF) {
    if (N == 128) fft_forward_ct<7, 4, 16>(X, tw);
    else if (N == 256) fft_forward_ct<8, 4, 16>(X, tw);
    else if (N == 512) fft_forward_ct<9, 4, 16>(X, tw);
    else fft_forward_ct<10, 3, 8>(X, tw);
  } else {
    fft_forward_ml(X, C, logC, N, tw, maxlog);
  }
}
// radix bound of the tile's transform: the compiled shapes use radix <= 16
template <bool CTF> __device__ __forceinline__ int resid_maxlog(const ResidFwdArgs& a) {
  return CTF ? 4 : (a.maxlog == 3 ? 3 : 4);
}

template <int K, bool CQ, int DIM, bool FEM, bool PER, bool CTF>
__global__ void __launch_bounds__(kThreads, 4) k_resid_fwd(ResidFwdArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M, logC = a.logC, mx = a.mx;
  float2 *X, *tw;
  unsigned short* perm;
  const int ml = resid_maxlog<CTF>(a);
  time_tile_setup(smraw, N, C, a.tw, X, tw, perm, ml);

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
    const float2 z2 = make_float2(0.f, 0.f);
    const float2 u = valid ? a.U[idx] : z2;
    const float2 uw = ldW ? a.U[idx + dW] : z2;
    const float2 ue = ldE ? a.U[idx + dE] : z2;
    v.uh = u.x; v.ul = u.y;
    v.wh = uw.x; v.wl = uw.y;
    v.eh = ue.x; v.el = ue.y;
    if (two_d) {
      const float2 us = hasS ? a.U[idx + dS] : z2;
      const float2 un = hasN ? a.U[idx + dN] : z2;
      v.sh = us.x; v.sl = us.y;
      v.nh = un.x; v.nl = un.y;
    } else {
      v.sh = v.sl = v.nh = v.nl = 0.f;
    }
    if (three_d) {
      const float2 ub = hasB ? a.U[idx - mxy] : z2;
      const float2 ut = hasT ? a.U[idx + mxy] : z2;
      v.bh = ub.x; v.bl = ub.y;
      v.th = ut.x; v.tl = ut.y;
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
    const double* Fb = i < a.kc ? a.Fh : a.F;  // F_hat's first levels, then f (= F_hat there)
    v.f = valid ? Fb[idx] : 0.0;
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
      const float2 z2 = make_float2(0.f, 0.f);
      const float2 u = (valid && lev >= 0) ? a.U[idx] : z2;
      h[t].hi = u.x;
      h[t].lo = u.y;
      if constexpr (FEM) {
        float wh, wl, eh, el;
        const float2 uw = (ldW && lev >= 0) ? a.U[idx + dW] : z2;
        const float2 ue = (ldE && lev >= 0) ? a.U[idx + dE] : z2;
        neighbours(h[t].hi, h[t].lo, uw.x, uw.y, ue.x, ue.y, wh, wl, eh, el);
        h[t] = mass(h[t].hi, h[t].lo, wh, wl, eh, el);
      }
    }
    const float gx = a.gx_hi, gy = a.gy_hi, gz = a.gz_hi;
    const bool gexact = a.g_pow2 != 0;
    // reaction term w c_i U_i^n (1D, the linearised operator of Algorithm 3): one coefficient per point
    const bool react = DIM == 1 && a.react != nullptr;
    const ff rc = (react && valid) ? ff_from_double(a.react[m]) : ff{0.f, 0.f};
    ResidLevel nx = load(i0);
    // (3D: no unrolling, which keeps the two extra neighbour streams within 64 registers)
#pragma unroll (DIM == 3 ? 1 : 2)
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
        add_prod(A, -2.f * gx, c.uh, gexact);
        A.sl = fmaf(-2.f * gx, c.ul, A.sl);
        float bx, ex;
        two_sum(wh, eh, bx, ex);
        add_prod(A, gx, bx, gexact);
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
        add_prod(A, gx, bx, gexact);
        float lo = gx * (ex + (wl + el));
        if constexpr (DIM >= 2) {
          float by, ey;
          two_sum(c.sh, c.nh, by, ey);
          add_prod(A, gy, by, gexact);
          lo = fmaf(gy, ey + (c.sl + c.nl), lo);
        }
        if constexpr (DIM == 3) {
          float bz, ez;
          two_sum(c.bh, c.th, bz, ez);
          add_prod(A, gz, bz, gexact);
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
  resid_time_fft<CTF>(X, C, logC, N, tw, ml);
  store_half_spectrum(X, perm, a.S, N, M, C, logC, (int)blockIdx.x * P2);
}

// ---------------------------------------------------------------------------
// MIXED, first sweep from the initial guess U_0^n = v of every level (Theorem 2.7). Then
// K U_0 = tau^-alpha (sum_{j<n} omega_j) M v + A v = beta_n M v + A v for BDF and CQ alike, so
//   r_0^n = F_hat_n - beta_n M v - A v   (- w c v with a reaction term),
// with A v (and M v) formed once per point: no U is read, no history is formed, and the kernel
// reads F_hat and writes the half spectrum like k_resid_fwd (same tile, same transform).
// ---------------------------------------------------------------------------
template <int DIM, bool FEM, bool PER, bool CTF>
__global__ void __launch_bounds__(kThreads, 4) k_resid_v0(ResidFwdArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = a.N, C = a.C, M = a.M, logC = a.logC, mx = a.mx;
  float2 *X, *tw;
  unsigned short* perm;
  const int ml = resid_maxlog<CTF>(a);
  time_tile_setup(smraw, N, C, a.tw, X, tw, perm, ml);
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
  const bool gexact = a.g_pow2 != 0;
  ff_acc Av;
  Av.init(ff{0.f, 0.f});
  // centre: 2 gx + 2 gy + 2 gz (FD), 2/h (P1 stiffness) -- exact multiples of powers of two
  {
    float b0, e0;
    two_sum(vw.hi, ve.hi, b0, e0);
    add_prod(Av, 2.f * gx, vc.hi, gexact);
    Av.sl = fmaf(2.f * gx, vc.lo, Av.sl);
    add_prod(Av, -gx, b0, gexact);
    Av.sl -= gx * (e0 + (vw.lo + ve.lo));
  }
  if constexpr (DIM >= 2) {
    const float gy = a.gy_hi;
    const ff vs = hasS ? ff_from_double(a.v[m + dS]) : ff{0.f, 0.f};
    const ff vn = hasN ? ff_from_double(a.v[m + dN]) : ff{0.f, 0.f};
    float b1, e1;
    two_sum(vs.hi, vn.hi, b1, e1);
    add_prod(Av, 2.f * gy, vc.hi, gexact);
    Av.sl = fmaf(2.f * gy, vc.lo, Av.sl);
    add_prod(Av, -gy, b1, gexact);
    Av.sl -= gy * (e1 + (vs.lo + vn.lo));
  }
  if constexpr (DIM == 3) {
    const float gz = a.gz_hi;
    const ff vb = hasB ? ff_from_double(a.v[m - mxy]) : ff{0.f, 0.f};
    const ff vt = hasT ? ff_from_double(a.v[m + mxy]) : ff{0.f, 0.f};
    float b2, e2;
    two_sum(vb.hi, vt.hi, b2, e2);
    add_prod(Av, 2.f * gz, vc.hi, gexact);
    Av.sl = fmaf(2.f * gz, vc.lo, Av.sl);
    add_prod(Av, -gz, b2, gexact);
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
      for (int t = 0; t < 8; ++t) {
        // F_hat's first levels from their own block, then f (= F_hat there)
        const double* Fb = b + t < a.kc ? a.Fh + m : Fp;
        f[t] = (valid && b + t < i1) ? Fb[(size_t)(b + t) * M] : 0.0;
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int i = b + t;
        if (i < i1) {
          ff_acc A;
          A.init(ff_split_trunc(f[t]));
          const float2 bt = __ldg(a.beta_ff + i);
          // (warp-uniform: beta_n = 0 beyond the first k levels of BDF-k)
          if (bt.x != 0.f) A.fma_term(ff{bt.x, bt.y}, Mv, -1.f);
          A.sub(Avn);
          Xf[(size_t)2 * i * C] = valid ? A.value() * __ldg(a.s + i) : 0.f;
        }
      }
    }
  }
  __syncthreads();
  resid_time_fft<CTF>(X, C, logC, N, tw, ml);
  store_half_spectrum(X, perm, a.S, N, M, C, logC, (int)blockIdx.x * P2);
}

template <int K, bool CQ, int DIM, bool FEM, bool PER, bool CTF>
static cudaError_t launch_resid_kc(const ResidFwdArgs& a, size_t sm, cudaStream_t st) {
  cudaError_t e = set_smem(k_resid_fwd<K, CQ, DIM, FEM, PER, CTF>, sm);
  if (e != cudaSuccess) return e;
  prof_begin("resid_fwd_ff", st);
  k_resid_fwd<K, CQ, DIM, FEM, PER, CTF><<<tiles(a.M, a.C), kThreads, sm, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

template <int K, bool CQ, int DIM, bool FEM, bool PER>
static cudaError_t launch_resid_k(const ResidFwdArgs& a, size_t sm, cudaStream_t st) {
  return compiled_time_fft(a.N, a.C) ? launch_resid_kc<K, CQ, DIM, FEM, PER, true>(a, sm, st)
                                     : launch_resid_kc<K, CQ, DIM, FEM, PER, false>(a, sm, st);
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

template <int DIM, bool FEM, bool PER, bool CTF>
static cudaError_t launch_v0_kc(const ResidFwdArgs& a, size_t sm, cudaStream_t st) {
  cudaError_t e = set_smem(k_resid_v0<DIM, FEM, PER, CTF>, sm);
  if (e != cudaSuccess) return e;
  prof_begin("resid_v0_ff", st);
  k_resid_v0<DIM, FEM, PER, CTF><<<tiles(a.M, a.C), kThreads, sm, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

template <int DIM, bool FEM, bool PER>
static cudaError_t launch_v0_k(const ResidFwdArgs& a, size_t sm, cudaStream_t st) {
  return compiled_time_fft(a.N, a.C) ? launch_v0_kc<DIM, FEM, PER, true>(a, sm, st)
                                     : launch_v0_kc<DIM, FEM, PER, false>(a, sm, st);
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

}  // namespace pint
