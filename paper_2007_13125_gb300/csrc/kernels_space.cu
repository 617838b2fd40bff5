// Spatial part of the sweep (Algorithm 1/2, step 2): the N/2+1 shifted systems
// (sigma_j + A_h) q_j = h_j, sigma_j = g_j tau^-alpha, with A_h the finite-difference
// Dirichlet Laplacian. A_h is diagonalised exactly by the discrete sine transform
// DST-I, D_{pi} = sin(pi p i / (n+1)), with eigenvalues (4/h^2) sin^2(p pi h / 2).
//
// k_axis -- a sine transform of a (complex) line x_1..x_n through its odd extension of
// length L = 2(n+1): the forward FFT of [0, x, 0, -reverse(x)] is -2i D x at frequencies
// 1..n and keeps the odd symmetry. Dividing that spectrum by a symmetric factor keeps it
// odd, and the inverse FFT of an odd spectrum Z is 2i D Z. So a shifted solve along one
// axis is: odd-extend, forward FFT, divide, inverse FFT -- in place, in shared memory,
// with no permutation (the inverse consumes the forward transform's permuted order).
// Line layouts: mode 0 -- lines are contiguous rows of n elements (x direction, or the
// whole 1D grid); mode 1 -- lines run across rows with stride P (y direction in 2D),
// consecutive lines are consecutive x-modes so loads stay coalesced.
//
// k_tri -- the y direction as a tridiagonal solve (after the x sine transform every line
// (j, p) is a constant-coefficient system): thread per line, data staged in shared memory.
//
// k_trivar_factor / k_trivar_solve -- 1D shifted systems whose diagonal varies along x (a
// reaction term, the linearised operator of Algorithm 3): no transform diagonalises them, so
// each frequency's tridiagonal system is solved by Gaussian elimination without pivoting, the
// substitutions as parallel scans of affine maps (the
// systems are diagonally dominant up to the reaction term: sigma_j lies in the sector where the
// BDF / CQ symbols live, and A_h + w diag(c) is positive definite for the reactions of interest).
#include "ff.cuh"
#include "fft.cuh"
#include "pint_internal.h"

namespace pint {

// Tile layout: element (row, line) of a C-line tile at X[row * (C + 1) + line]. With C = 16 (the
// usual width) a warp touches 16 lines of two rows in the FFT passes, or 32 consecutive rows of
// one line when it moves a contiguous line between global and shared memory; the +1 pitch keeps
// both patterns free of bank conflicts. Rows read in the FFT's digit-reversed order are first
// brought into natural order through registers (lanes along lines), for the same reason.
template <typename T> constexpr int axis_regs() { return sizeof(T) == 4 ? 16 : 8; }
// (the mass-eigenvalue table is carved only for P1 FEM lines: has_mu)
// (rows: tile rows, L for the generic instance, odd_rows<LOGL>() for the compiled shapes)
template <typename T> size_t axis_smem(int n, int C, bool has_mu, int rows) {
  const size_t L = 2 * (size_t)(n + 1);
  return sizeof(typename c2<T>::t) * ((size_t)rows * (C + 1) + L + C) + (has_mu ? 2 : 1) * sizeof(T) * (size_t)(n + 1) +
         sizeof(unsigned short) * L + 2 * sizeof(int) * C + 64;
}

__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// The divide of op 1 for the compiled shapes, fused with the last forward and the first inverse
// FFT pass: both work on groups of R = 2^LR consecutive rows without twiddles, so each thread takes
// one group of one line through forward DFT-R, division, inverse DFT-R in registers (one shared-
// memory round trip instead of three). Row base + q of the permuted spectrum holds frequency
// ct_freq(base) + q L / R; frequencies f and L - f share the divisor, 0 and n + 1 are zero. Only
// the odd_rows<LOGL>() rows of the spectrum that are formed are visited.
template <typename T, int LOGL, int LOGC, typename V>
__device__ __forceinline__ void axis_divide_fused(V* X, const V* dcol, const T* lam, const T* mu, bool has_mu,
                                                  T scale, int cols) {
  constexpr int NP = ct_npass(LOGL, 4), LR = ct_logradix(LOGL, NP - 1, 4);
  constexpr int R = 1 << LR, C = 1 << LOGC, LD = C + 1, L = 1 << LOGL, n = L / 2 - 1;
  constexpr int ITEMS = (odd_rows<LOGL>() >> LR) << LOGC;
  const T zero = T(0);
  for (int it = threadIdx.x; it < ITEMS; it += blockDim.x) {
    const int c = it & (C - 1);
    const int base = (it >> LOGC) << LR;
    V* p = X + base * LD + c;
    V x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = p[r * LD];
    dft_reg<R, -1>(x);
    const V dc = dcol[c];
    const bool ok = c < cols;
    const int f0 = ct_freq<LOGL>(base);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      int f = f0 + q * (L / R);
      if (f > n + 1) f = L - f;
      if (!ok || f == 0 || f == n + 1) {
        x[q] = mk(zero, zero);
      } else {
        // scale * (sigma_j mu_f + lambda_other + lambda_f), mu_f = 1 for finite differences
        const T mp = has_mu ? mu[f - 1] : T(1);
        const T dx = (dc.x * mp + lam[f - 1]) * scale, dy = dc.y * mp * scale;
        const T inv = rcp(dx * dx + dy * dy);
        x[q] = cmulc(x[q], mk(dx * inv, dy * inv));  // x / d = x conj(d) / |d|^2
      }
    }
    dft_reg<R, 1>(x);
#pragma unroll
    for (int r = 0; r < R; ++r) p[r * LD] = x[r];
  }
}

// (L = 512, radix 8 everywhere: 64 registers and a 50 KB tile, so four CTAs fit on an SM; the
// radix-16 shapes need about 80 registers.)
// LOGL > 0: compiled for lines of L = 2^LOGL extended points in tiles of 2^LOGC lines (the
// shapes of the usual grids), transformed as odd sequences (only rows 0..L/2 of the extension are
// stored, and only the odd_rows<LOGL>() rows of the spectrum that are not mirrors of others are
// formed); LOGL = 0: any shape, taken from the arguments, with the full odd extension.
template <typename T, int LOGL, int LOGC>
__global__ void __launch_bounds__(kThreads, LOGL == 9 ? 4 : 3) k_axis(AxisArgs<T> a) {
  using V = typename c2<T>::t;
  constexpr int KR = axis_regs<T>();  // register slots per thread for the reordering
  constexpr int KB = 8;               // global loads in flight per thread
  constexpr bool CT = LOGL > 0;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n = CT ? (1 << (LOGL - 1)) - 1 : a.n;
  const int C = CT ? (1 << LOGC) : a.C, logC = CT ? LOGC : a.logC, ld = CT ? (1 << LOGC) + 1 : a.ld;
  const int L = 2 * (n + 1);
  constexpr int XROWS = odd_rows<(CT ? LOGL : 7)>();
  V* X = reinterpret_cast<V*>(smraw);
  V* tw = X + (size_t)(CT ? XROWS : L) * ld;
  V* dcol = tw + L;                                      // line -> sigma_j + lambda_other (op 1)
  T* lam = reinterpret_cast<T*>(dcol + C);               // lambda along this axis (op 1)
  T* mu = lam + n + 1;                                   // P1 mass eigenvalues (op 1, FEM)
  unsigned short* perm = reinterpret_cast<unsigned short*>(a.mu_axis ? mu + n + 1 : mu);
  int* lj = reinterpret_cast<int*>(perm + L + (L & 1));  // line -> j
  int* lp = lj + C;                                      // line -> position within its slice
  const V* gtw = reinterpret_cast<const V*>(a.tw);
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = gtw[i];
  if constexpr (CT) {
    // (op 1 finds frequencies arithmetically)
    if (a.op == 0)
      for (int j = threadIdx.x; j < L; j += blockDim.x) perm[j] = (unsigned short)odd_pos<(CT ? LOGL : 7)>(j);
  } else {
    fft_perm_table(perm, L);
  }
  V* S = reinterpret_cast<V*>(a.S);
  const int line0 = blockIdx.x * C;
  const int per = a.mode == 0 ? a.lines_per_j : a.P;
  for (int cc = threadIdx.x; cc < C; cc += blockDim.x) {
    const int line = line0 + cc;
    lj[cc] = line / per;
    lp[cc] = line - lj[cc] * per;
  }
  __syncthreads();
  const T zero = T(0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  // rows 1..n of the tile back to the lines (op 1's result)
  auto store_lines = [&]() {
    if (a.mode == 0) {
      for (int cc = warp; cc < C; cc += nwarp) {
        const int line = line0 + cc;
        if (line >= a.lines) continue;
        for (int i = lane; i < n; i += 32) S[(size_t)line * n + i] = X[(size_t)(i + 1) * ld + cc];
      }
    } else {
      for (int it = threadIdx.x; it < (n << logC); it += blockDim.x) {
        const int cc = it & (C - 1), i = it >> logC;
        if (line0 + cc < a.lines) S[((size_t)lj[cc] * n + i) * a.P + lp[cc]] = X[(size_t)(i + 1) * ld + cc];
      }
    }
  };

  // ---- load with odd extension (KB independent loads per thread before the stores) ----
  if (a.mode == 0) {
    for (int cc = warp; cc < C; cc += nwarp) {
      const int line = line0 + cc;
      const bool ok = line < a.lines;
      const V* src = S + (size_t)(ok ? line : 0) * n;
      for (int i0 = 0; i0 < n; i0 += 32 * KB) {
        V v[KB];
#pragma unroll
        for (int t = 0; t < KB; ++t) {
          const int i = i0 + lane + 32 * t;
          v[t] = (ok && i < n) ? src[i] : mk(zero, zero);
        }
#pragma unroll
        for (int t = 0; t < KB; ++t) {
          const int i = i0 + lane + 32 * t;
          if (i < n) {
            X[(size_t)(i + 1) * ld + cc] = v[t];
            if constexpr (!CT) X[(size_t)(L - 1 - i) * ld + cc] = mk(-v[t].x, -v[t].y);
          }
        }
      }
    }
  } else {
    const int tot = n << logC;
    for (int it0 = threadIdx.x; it0 < tot; it0 += KB * blockDim.x) {
      V v[KB];
#pragma unroll
      for (int t = 0; t < KB; ++t) {
        const int it = it0 + t * blockDim.x;
        const int cc = it & (C - 1), i = it >> logC;
        v[t] = (it < tot && line0 + cc < a.lines) ? S[((size_t)lj[cc] * n + i) * a.P + lp[cc]] : mk(zero, zero);
      }
#pragma unroll
      for (int t = 0; t < KB; ++t) {
        const int it = it0 + t * blockDim.x;
        if (it < tot) {
          const int cc = it & (C - 1), i = it >> logC;
          X[(size_t)(i + 1) * ld + cc] = v[t];
          if constexpr (!CT) X[(size_t)(L - 1 - i) * ld + cc] = mk(-v[t].x, -v[t].y);
        }
      }
    }
  }
  for (int cc = threadIdx.x; cc < C; cc += blockDim.x) {
    X[cc] = mk(zero, zero);
    X[(size_t)(n + 1) * ld + cc] = mk(zero, zero);
  }
  if (a.op == 1) {
    // per-line part of the divisor and the eigenvalues along this axis
    const V* sigma = reinterpret_cast<const V*>(a.sigma);
    for (int cc = threadIdx.x; cc < C; cc += blockDim.x) {
      V d = mk(zero, zero);
      if (line0 + cc < a.lines) {
        d = sigma[lj[cc]];
        if (a.lam_other) d.x += a.lam_other[lp[cc]];
      }
      dcol[cc] = d;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      lam[i] = a.lam_axis[i];
      if (a.mu_axis) mu[i] = a.mu_axis[i];
    }
  }
  __syncthreads();
  if constexpr (CT) {
    constexpr int LD = (1 << LOGC) + 1, NP = ct_npass(LOGL, 4), LR0 = ct_logradix(LOGL, 0, 4);
    constexpr int LRL = ct_logradix(LOGL, NP - 1, 4);
    odd_forward_pass0<LOGL, LOGC, LD, kThreads>(X, tw);
    __syncthreads();
    odd_forward_rec<1, NP - 1, LOGL, LOGL - LR0, LOGC, LD, XROWS>(X, tw);
    if (a.op == 1) {
      axis_divide_fused<T, LOGL, LOGC>(X, dcol, lam, mu, a.mu_axis != nullptr, a.scale, a.lines - line0);
      __syncthreads();
      odd_inverse_rec<NP - 2, LOGL, LRL, LOGC, LD, XROWS>(X, tw);
      odd_inverse_pass0<LOGL, LOGC, LD, kThreads>(X, tw);
      __syncthreads();
      store_lines();
      return;
    }
    odd_forward_rec<NP - 1, NP, LOGL, LRL, LOGC, LD, XROWS>(X, tw);
  } else {
    fft_forward(X, ld, logC, L, tw);
  }

  if (a.op == 0) {
    // D-transform only: -2i D x at frequencies 1..n, stored in natural order. A perm entry is the
    // row of a frequency; for the compiled shapes bit 15 marks a row holding the negated value.
    auto fetch = [&](unsigned short e, int cc) {
      if constexpr (CT) {
        const V v = X[(size_t)(e & 0x7fff) * ld + cc];
        return (e & 0x8000) ? mk(-v.x, -v.y) : v;
      } else {
        return X[(size_t)e * ld + cc];
      }
    };
    const int tot = n << logC;
    if (tot <= KR * (int)blockDim.x) {
      // frequency p sits in row perm[p]: move rows perm[1..n] to rows 1..n through registers
      V v[KR];
#pragma unroll
      for (int t = 0; t < KR; ++t) {
        const int it = threadIdx.x + t * blockDim.x;
        if (it < tot) v[t] = fetch(perm[1 + (it >> logC)], it & (C - 1));
      }
      __syncthreads();
#pragma unroll
      for (int t = 0; t < KR; ++t) {
        const int it = threadIdx.x + t * blockDim.x;
        if (it < tot) X[(size_t)(1 + (it >> logC)) * ld + (it & (C - 1))] = v[t];
      }
      __syncthreads();
      if (a.mode == 0) {
        for (int cc = warp; cc < C; cc += nwarp) {
          const int line = line0 + cc;
          if (line >= a.lines) continue;
          for (int i = lane; i < n; i += 32) S[(size_t)line * n + i] = X[(size_t)(i + 1) * ld + cc];
        }
      } else {
        for (int it = threadIdx.x; it < tot; it += blockDim.x) {
          const int cc = it & (C - 1), i = it >> logC;
          if (line0 + cc < a.lines) S[((size_t)lj[cc] * n + i) * a.P + lp[cc]] = X[(size_t)(i + 1) * ld + cc];
        }
      }
    } else if (a.mode == 0) {
      for (int cc = warp; cc < C; cc += nwarp) {
        const int line = line0 + cc;
        if (line >= a.lines) continue;
        for (int i = lane; i < n; i += 32) S[(size_t)line * n + i] = fetch(perm[i + 1], cc);
      }
    } else {
      for (int it = threadIdx.x; it < tot; it += blockDim.x) {
        const int cc = it & (C - 1), i = it >> logC;
        if (line0 + cc < a.lines)
          S[((size_t)lj[cc] * n + i) * a.P + lp[cc]] = fetch(perm[i + 1], cc);
      }
    }
    return;
  }

  // ---- divide by scale * (sigma_j + lambda_other + lambda_p) at frequencies p and L-p ----
  // (both rows share the divisor; frequencies 0 and n+1 are zero for an odd sequence)
  if constexpr (!CT) {
  for (int it = threadIdx.x; it < ((n + 2) << logC); it += blockDim.x) {
    const int cc = it & (C - 1), p = it >> logC;
    const size_t pos = (size_t)perm[p] * ld + cc;
    if (p == 0 || p == n + 1 || line0 + cc >= a.lines) {
      X[pos] = mk(zero, zero);
      if (p != 0 && p != n + 1) X[(size_t)perm[L - p] * ld + cc] = mk(zero, zero);
      continue;
    }
    // sigma_j mu_p + lambda_p (mu_p = 1 for finite differences)
    V d = dcol[cc];
    const T mp = a.mu_axis ? mu[p - 1] : T(1);
    d.x = d.x * mp + lam[p - 1];
    d.y *= mp;
    d.x *= a.scale;
    d.y *= a.scale;
    const T inv = rcp(d.x * d.x + d.y * d.y);
    const V q = mk(d.x * inv, d.y * inv);
    const size_t pos2 = (size_t)perm[L - p] * ld + cc;
    X[pos] = cmulc(X[pos], q);   // X / d = X conj(d) / |d|^2
    X[pos2] = cmulc(X[pos2], q);
  }
  __syncthreads();
  fft_inverse(X, ld, logC, L, tw);
  store_lines();
  }
}

template <typename T, int LOGL, int LOGC>
static cudaError_t launch_axis_k(const AxisArgs<T>& a, cudaStream_t st) {
  const size_t sm = axis_smem<T>(a.n, a.C, a.mu_axis != nullptr, LOGL > 0 ? odd_rows<(LOGL > 0 ? LOGL : 7)>()
                                                                          : 2 * (a.n + 1));
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_axis<T, LOGL, LOGC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  const int blocks = (a.lines + a.C - 1) / a.C;
  const char* name = a.op == 0 ? (sizeof(T) == 8 ? "dst_f64" : "dst_f32")
                               : (sizeof(T) == 8 ? "axis_solve_f64" : "axis_solve_f32");
  prof_begin(name, st);
  k_axis<T, LOGL, LOGC><<<blocks, kThreads, sm, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_axis(const AxisArgs<T>& a, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    // compiled shapes: n = 2^q - 1 with the tile widths the plan picks for them
    const int L = 2 * (a.n + 1);
    if (a.ld == a.C + 1) {
      if (L == 128 && a.C == 16) return launch_axis_k<T, 7, 4>(a, st);
      if (L == 256 && a.C == 16) return launch_axis_k<T, 8, 4>(a, st);
      if (L == 512 && a.C == 16) return launch_axis_k<T, 9, 4>(a, st);
      if (L == 1024 && a.C == 8) return launch_axis_k<T, 10, 3>(a, st);
      if (L == 2048 && a.C == 4) return launch_axis_k<T, 11, 2>(a, st);
      if (L == 4096 && a.C == 2) return launch_axis_k<T, 12, 1>(a, st);
    }
  }
  return launch_axis_k<T, 0, 0>(a, st);
}

// ---------------------------------------------------------------------------
// Periodic axis (the remark of Sec. 2.2: with periodic boundary conditions the spatial systems are
// diagonalised by the FFT itself). Lines of n points, n a power of two, x_i = i/n; the circulant
// Laplacian (1/h^2)[-1 2 -1] has eigenvalues lambda_p = (4/h^2) sin^2(pi p/n) on e^{2 pi i p x}.
// op 0: forward FFT of each line, spectrum stored in natural order;
// op 1: forward FFT, divide by scale * (sigma_j + lambda_other + lambda_p), inverse FFT;
// op 2: inverse FFT of a natural-order spectrum (unnormalised; the 1/(nx ny) sits in op 1's scale).
// Same tile layout as k_axis (C lines, row pitch C + 1).
// ---------------------------------------------------------------------------
template <typename T> size_t axis_per_smem(int n, int C, int ld) {
  return sizeof(typename c2<T>::t) * ((size_t)n * ld + n + C) + sizeof(T) * (size_t)n +
         sizeof(unsigned short) * (size_t)n + 2 * sizeof(int) * C + 64;
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 3) k_axis_per(AxisArgs<T> a) {
  using V = typename c2<T>::t;
  constexpr int KR = axis_regs<T>();
  constexpr int KB = 8;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n = a.n, C = a.C, logC = a.logC, ld = a.ld, L = a.n;
  V* X = reinterpret_cast<V*>(smraw);
  V* tw = X + (size_t)L * ld;
  V* dcol = tw + L;
  T* lam = reinterpret_cast<T*>(dcol + C);
  unsigned short* perm = reinterpret_cast<unsigned short*>(lam + n);
  int* lj = reinterpret_cast<int*>(perm + L + (L & 1));
  int* lp = lj + C;
  const V* gtw = reinterpret_cast<const V*>(a.tw);
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = gtw[i];
  fft_perm_table(perm, L);
  V* S = reinterpret_cast<V*>(a.S);
  const int line0 = blockIdx.x * C;
  const int per = a.mode == 0 ? a.lines_per_j : a.P;
  for (int cc = threadIdx.x; cc < C; cc += blockDim.x) {
    const int line = line0 + cc;
    lj[cc] = line / per;
    lp[cc] = line - lj[cc] * per;
  }
  __syncthreads();
  const T zero = T(0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const int tot = n << logC;
  auto gidx = [&](int cc, int i) -> size_t {  // element i of tile line cc in S
    return a.mode == 0 ? (size_t)(line0 + cc) * n + i : ((size_t)lj[cc] * n + i) * a.P + lp[cc];
  };
  // op 2 on a tile too large for the register reordering: load straight into digit-reversed rows
  const bool direct_perm = a.op == 2 && tot > KR * (int)blockDim.x;
  auto row_of = [&](int i) { return direct_perm ? (int)perm[i] : i; };

  // ---- load rows 0..n-1 in natural order (KB loads in flight per thread) ----
  if (a.mode == 0) {
    for (int cc = warp; cc < C; cc += nwarp) {
      const bool ok = line0 + cc < a.lines;
      for (int i0 = 0; i0 < n; i0 += 32 * KB) {
        V v[KB];
#pragma unroll
        for (int t = 0; t < KB; ++t) {
          const int i = i0 + lane + 32 * t;
          v[t] = (ok && i < n) ? S[gidx(cc, i)] : mk(zero, zero);
        }
#pragma unroll
        for (int t = 0; t < KB; ++t) {
          const int i = i0 + lane + 32 * t;
          if (i < n) X[(size_t)row_of(i) * ld + cc] = v[t];
        }
      }
    }
  } else {
    for (int it0 = threadIdx.x; it0 < tot; it0 += KB * blockDim.x) {
      V v[KB];
#pragma unroll
      for (int t = 0; t < KB; ++t) {
        const int it = it0 + t * blockDim.x;
        const int cc = it & (C - 1), i = it >> logC;
        v[t] = (it < tot && line0 + cc < a.lines) ? S[gidx(cc, i)] : mk(zero, zero);
      }
#pragma unroll
      for (int t = 0; t < KB; ++t) {
        const int it = it0 + t * blockDim.x;
        if (it < tot) X[(size_t)row_of(it >> logC) * ld + (it & (C - 1))] = v[t];
      }
    }
  }
  if (a.op == 1) {
    const V* sigma = reinterpret_cast<const V*>(a.sigma);
    for (int cc = threadIdx.x; cc < C; cc += blockDim.x) {
      V d = mk(zero, zero);
      if (line0 + cc < a.lines) {
        d = sigma[lj[cc]];
        if (a.lam_other) d.x += a.lam_other[lp[cc]];
      }
      dcol[cc] = d;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = a.lam_axis[i];
  }
  __syncthreads();

  // move row r to row map(r) through registers (lanes along lines: no bank conflicts);
  // to_perm: natural -> digit-reversed (before an inverse), else digit-reversed -> natural
  auto reorder = [&](bool to_perm) {
    if (tot <= KR * (int)blockDim.x) {
      V v[KR];
#pragma unroll
      for (int t = 0; t < KR; ++t) {
        const int it = threadIdx.x + t * blockDim.x;
        const int r = it >> logC;
        if (it < tot) v[t] = X[(size_t)(to_perm ? r : perm[r]) * ld + (it & (C - 1))];
      }
      __syncthreads();
#pragma unroll
      for (int t = 0; t < KR; ++t) {
        const int it = threadIdx.x + t * blockDim.x;
        const int r = it >> logC;
        if (it < tot) X[(size_t)(to_perm ? perm[r] : r) * ld + (it & (C - 1))] = v[t];
      }
      __syncthreads();
      return true;
    }
    return false;
  };

  // forward transform (rows end digit-reversed), or for op 2 the natural-order spectrum moved to
  // the digit-reversed rows the inverse transform consumes
  if (a.op != 2) fft_forward(X, ld, logC, L, tw);
  else if (!direct_perm) reorder(true);
  if (a.op == 1) {
    for (int it = threadIdx.x; it < tot; it += blockDim.x) {
      const int cc = it & (C - 1), p = it >> logC;
      const size_t pos = (size_t)perm[p] * ld + cc;
      if (line0 + cc >= a.lines) { X[pos] = mk(zero, zero); continue; }
      V d = dcol[cc];
      d.x += lam[p];
      d.x *= a.scale;
      d.y *= a.scale;
      const T inv = rcp(d.x * d.x + d.y * d.y);
      X[pos] = cmulc(X[pos], mk(d.x * inv, d.y * inv));   // X / d
    }
    __syncthreads();
  }
  if (a.op == 0) {
    if (!reorder(false)) {
      // no room to reorder through registers: store through perm
      for (int it = threadIdx.x; it < tot; it += blockDim.x) {
        const int cc = it & (C - 1), i = it >> logC;
        if (line0 + cc < a.lines) S[gidx(cc, i)] = X[(size_t)perm[i] * ld + cc];
      }
      return;
    }
  } else {
    fft_inverse(X, ld, logC, L, tw);
  }
  // ---- store rows 0..n-1 (natural order) ----
  if (a.mode == 0) {
    for (int cc = warp; cc < C; cc += nwarp) {
      if (line0 + cc >= a.lines) continue;
      for (int i = lane; i < n; i += 32) S[gidx(cc, i)] = X[(size_t)i * ld + cc];
    }
  } else {
    for (int it = threadIdx.x; it < tot; it += blockDim.x) {
      const int cc = it & (C - 1), i = it >> logC;
      if (line0 + cc < a.lines) S[gidx(cc, i)] = X[(size_t)i * ld + cc];
    }
  }
}

template <typename T> cudaError_t launch_axis_per(const AxisArgs<T>& a, cudaStream_t st) {
  const size_t sm = axis_per_smem<T>(a.n, a.C, a.ld);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_axis_per<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  const int blocks = (a.lines + a.C - 1) / a.C;
  const char* name = a.op == 1 ? (sizeof(T) == 8 ? "axis_solve_per_f64" : "axis_solve_per_f32")
                               : (sizeof(T) == 8 ? "fft_per_f64" : "fft_per_f32");
  prof_begin(name, st);
  k_axis_per<T><<<blocks, kThreads, sm, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tridiagonal y-solve: d q_y - g (q_{y-1} + q_{y+1}) = b_y, d = sigma_j + lambda_p^x + 2g.
// With r + 1/r = d/g, |r| < 1 (r = 1 + e/2 - sqrt(e + e^2/4), e = (sigma_j + lambda_p^x)/g,
// evaluated without cancellation), the matrix is
//   T = (g/r)(I - rZ)(I - rZ^T) + g r e_0 e_0^T      (Z the down-shift),
// so T^-1 b = x0 - zeta * (g r x0_0) / (1 + g r zeta_0) with x0 = B^-1 b from two first-order
// recurrences with the constant factor r, and zeta = B^-1 e_0 in closed form:
//   zeta_i = (r^{i+1} - r^{2n-i+1}) / (g (1 - r^2)).
// Pass 1 (forward) also accumulates x0_0 = sum_i r^i w_i, so the correction is known before
// the backward pass; pass 3 applies it while storing.
// ---------------------------------------------------------------------------
size_t tri_smem(int n, int C) { return sizeof(float2) * (size_t)n * C + 2 * sizeof(int) * C; }

__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {  // a*b + c
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 csqrtf_(float2 z) {
  const float m = hypotf(z.x, z.y);
  const float re = sqrtf(fmaxf(0.5f * (m + z.x), 0.f));
  float im = sqrtf(fmaxf(0.5f * (m - z.x), 0.f));
  if (z.y < 0.f) im = -im;
  return make_float2(re, im);
}
__device__ __forceinline__ float2 cdiv(float2 a, float2 b) {
  const float inv = __frcp_rn(b.x * b.x + b.y * b.y);
  return make_float2((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}

__global__ void __launch_bounds__(kThreads) k_tri(TriArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n = a.n, C = a.C, logC = a.logC;
  float2* X = reinterpret_cast<float2*>(smraw);  // [n][C]
  int* lj = reinterpret_cast<int*>(X + (size_t)n * C);
  int* lp = lj + C;
  const int line0 = blockIdx.x * C;
  for (int cc = threadIdx.x; cc < C; cc += blockDim.x) {
    const int line = line0 + cc;
    lj[cc] = line / a.P;
    lp[cc] = line - lj[cc] * a.P;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < (n << logC); it += blockDim.x) {
    const int cc = it & (C - 1), i = it >> logC;
    float2 v = make_float2(0.f, 0.f);
    if (line0 + cc < a.lines) v = a.S[((size_t)lj[cc] * n + i) * a.P + lp[cc]];
    X[(size_t)i * C + cc] = v;
  }
  __syncthreads();
  for (int cc = threadIdx.x; cc < C; cc += blockDim.x) {
    if (line0 + cc >= a.lines) continue;
    const float g = a.g;
    const float2 sg = a.sigma[lj[cc]];
    const float ig = 1.f / g;
    const float2 e = make_float2((sg.x + a.lam_x[lp[cc]]) * ig, sg.y * ig);
    // r = 1 + e/2 - sqrt(e (1 + e/4)), the root of r + 1/r = 2 + e inside the unit disk
    const float2 q = make_float2(e.x * (1.f + 0.25f * e.x) - 0.25f * e.y * e.y,
                                 e.y * (1.f + 0.25f * e.x) + 0.25f * e.x * e.y);
    const float2 sq = csqrtf_(q);
    float2 r = make_float2(1.f + 0.5f * e.x - sq.x, 0.5f * e.y - sq.y);
    if (r.x * r.x + r.y * r.y > 1.f) r = make_float2(1.f + 0.5f * e.x + sq.x, 0.5f * e.y + sq.y);
    // pass 1: w_i = b_i + r w_{i-1}; x0_0 = sum_i r^i w_i
    float2 w = make_float2(0.f, 0.f), acc = make_float2(0.f, 0.f), rp = make_float2(1.f, 0.f);
    for (int i = 0; i < n; ++i) {
      w = cfma(r, w, X[(size_t)i * C + cc]);
      X[(size_t)i * C + cc] = w;
      acc = cfma(rp, w, acc);
      rp = cfma(rp, r, make_float2(0.f, 0.f));
    }
    // pass 2: x0_i = w_i + r x0_{i+1}   (B^-1 b = (r/g) x0)
    float2 x = make_float2(0.f, 0.f);
    for (int i = n - 1; i >= 0; --i) {
      x = cfma(r, x, X[(size_t)i * C + cc]);
      X[(size_t)i * C + cc] = x;
    }
    // correction: gamma = g r X0_0 / (1 + g r zeta_0), X0 = (r/g) x0
    const float2 r2 = cfma(r, r, make_float2(0.f, 0.f));
    const float2 one_m_r2 = make_float2(1.f - r2.x, -r2.y);
    // r^{2n}
    float2 r2n = make_float2(1.f, 0.f), b = r2;
    for (int t = n; t > 0; t >>= 1) {
      if (t & 1) r2n = cfma(r2n, b, make_float2(0.f, 0.f));
      b = cfma(b, b, make_float2(0.f, 0.f));
    }
    // g r zeta_0 = r^2 (1 - r^{2n}) / (1 - r^2)
    const float2 grz0 = cdiv(cfma(r2, make_float2(-r2n.x, -r2n.y), r2), one_m_r2);
    const float2 X00 = cfma(r, acc, make_float2(0.f, 0.f));          // r x0_0
    // gamma * zeta_i = [g r X0_0 / (1 + g r zeta_0)] * (r^{i+1} - r^{2n-i+1}) / (g (1 - r^2))
    //                = (r/g) K (r^{i+1} - r^{2n+1-i}),  K = r x0_0 / ((1 + g r zeta_0)(1 - r^2))
    const float2 den = cfma(make_float2(1.f + grz0.x, grz0.y), one_m_r2, make_float2(0.f, 0.f));
    const float2 K = cdiv(X00, den);
    // pass 3: q_i = scale * (r/g) (x0_i - K' (r^{i+1} - r^{2n+1-i})),  K' = K (in x0 units)
    const float2 rg = make_float2(r.x * ig * a.scale, r.y * ig * a.scale);
    float2 A = r;                                                         // r^{i+1}
    float2 E = cfma(r2n, r, make_float2(0.f, 0.f));                      // r^{2n+1-i}, i = 0
    const float2 ir = cdiv(make_float2(1.f, 0.f), r);
    const size_t col = (size_t)lj[cc] * n * a.P + lp[cc];
    for (int i = 0; i < n; ++i) {
      const float2 z = make_float2(A.x - E.x, A.y - E.y);
      const float2 x0 = X[(size_t)i * C + cc];
      const float2 xi = cfma(make_float2(-K.x, -K.y), z, x0);
      a.S[col + (size_t)i * a.P] = cfma(rg, xi, make_float2(0.f, 0.f));
      A = cfma(A, r, make_float2(0.f, 0.f));
      E = cfma(E, ir, make_float2(0.f, 0.f));
    }
  }
}

cudaError_t launch_tri(const TriArgs& a, cudaStream_t st) {
  const size_t sm = tri_smem(a.n, a.C);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_tri, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  const int blocks = (a.lines + a.C - 1) / a.C;
  prof_begin("tri_y_f32", st);
  k_tri<<<blocks, kThreads, sm, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// k_pcr -- the same constant-coefficient tridiagonal systems along y by parallel cyclic reduction:
// parallel within a system, for batches of few systems (small grids and few frequencies), where
// one thread per system leaves the GPU idle. Divided by g, row i is
//   a_i q_{i-1} + b_i q_i + c_i q_{i+1} = d_i,  a_i = -1 (i > 0), c_i = -1 (i < n-1), b_i = 2 + e,
// e = (s_j + lambda_p^x) / g. A reduction step of stride s eliminates q_{i-s} and q_{i+s} with rows
// i - s and i + s (k1 = a_i / b_{i-s}, k2 = c_i / b_{i+s}):
//   a_i' = -a_{i-s} k1,  c_i' = -c_{i+s} k2,  b_i' = b_i - c_{i-s} k1 - a_{i+s} k2,
//   d_i' = d_i - d_{i-s} k1 - d_{i+s} k2,
// rows outside 0..n-1 acting as the identity (a = c = d = 0, b = 1). After the steps s = 1, 2, 4, ...
// < n every row is decoupled: q_i = d_i / b_i. No pivoting: the rows are those of sigma_j + A_h
// restricted to one sine mode in x, nonsingular for every frequency.
// Lines of at most 32 rows: one warp per line, one row per lane, neighbours by warp shuffles. Longer
// lines (up to 1024 rows): the whole CTA on one line, E rows per thread (row tid + 256 e), neighbours
// through one shared-memory copy of the coefficients (read, barrier, write, barrier per step).
// Lines are staged through a [n][C] tile for coalesced loads and stores, as in k_tri.
// ---------------------------------------------------------------------------
struct PcrRow { float2 a, b, c, d; };

__device__ __forceinline__ float2 crcp_mul(float2 a, float2 b) {  // a / b
  const float inv = __frcp_rn(b.x * b.x + b.y * b.y);
  return make_float2((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) { return cfma(a, b, make_float2(0.f, 0.f)); }
__device__ __forceinline__ float2 csubf(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ PcrRow pcr_step(const PcrRow& r, const PcrRow& m, const PcrRow& p) {
  const float2 k1 = crcp_mul(r.a, m.b), k2 = crcp_mul(r.c, p.b);
  PcrRow o;
  o.a = cmulf(make_float2(-m.a.x, -m.a.y), k1);
  o.c = cmulf(make_float2(-p.c.x, -p.c.y), k2);
  o.b = csubf(csubf(r.b, cmulf(m.c, k1)), cmulf(p.a, k2));
  o.d = csubf(csubf(r.d, cmulf(m.d, k1)), cmulf(p.d, k2));
  return o;
}

__device__ __forceinline__ PcrRow pcr_identity() {
  PcrRow r;
  r.a = r.c = r.d = make_float2(0.f, 0.f);
  r.b = make_float2(1.f, 0.f);
  return r;
}

__device__ __forceinline__ float2 shfl_up2(float2 v, int s) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, s), __shfl_up_sync(0xffffffffu, v.y, s));
}
__device__ __forceinline__ float2 shfl_down2(float2 v, int s) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, s), __shfl_down_sync(0xffffffffu, v.y, s));
}

size_t pcr_smem(int n, int C) {
  const int E = n <= 32 ? 0 : (n + kThreads - 1) / kThreads;
  return sizeof(float2) * (size_t)n * C + 2 * sizeof(int) * C + sizeof(PcrRow) * (size_t)kThreads * E;
}

template <int E>
__global__ void __launch_bounds__(kThreads) k_pcr(TriArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n = a.n, C = a.C, logC = a.logC;
  float2* X = reinterpret_cast<float2*>(smraw);   // [n][C]
  int* lj = reinterpret_cast<int*>(X + (size_t)n * C);
  int* lp = lj + C;
  PcrRow* R = reinterpret_cast<PcrRow*>(lp + C);   // E > 0: [kThreads * E] rows of the current line
  const int line0 = blockIdx.x * C;
  for (int cc = threadIdx.x; cc < C; cc += blockDim.x) {
    const int line = line0 + cc;
    lj[cc] = line / a.P;
    lp[cc] = line - lj[cc] * a.P;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < (n << logC); it += blockDim.x) {
    const int cc = it & (C - 1), i = it >> logC;
    float2 v = make_float2(0.f, 0.f);
    if (line0 + cc < a.lines) v = a.S[((size_t)lj[cc] * n + i) * a.P + lp[cc]];
    X[(size_t)i * C + cc] = v;
  }
  __syncthreads();
  const float ig = 1.f / a.g;
  if constexpr (E == 0) {
    // one warp per line, row = lane
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    for (int cc = warp; cc < C; cc += nwarp) {
      if (line0 + cc >= a.lines) break;  // warp-uniform
      const float2 sg = a.sigma[lj[cc]];
      const float2 b0 = make_float2(2.f + (sg.x + a.lam_x[lp[cc]]) * ig, sg.y * ig);
      PcrRow r = pcr_identity();
      if (lane < n) {
        r.a = make_float2(lane > 0 ? -1.f : 0.f, 0.f);
        r.c = make_float2(lane < n - 1 ? -1.f : 0.f, 0.f);
        r.b = b0;
        r.d = X[(size_t)lane * C + cc];
      }
      for (int st = 1; st < n; st <<= 1) {
        PcrRow m, p;
        m.a = shfl_up2(r.a, st); m.b = shfl_up2(r.b, st); m.c = shfl_up2(r.c, st); m.d = shfl_up2(r.d, st);
        p.a = shfl_down2(r.a, st); p.b = shfl_down2(r.b, st); p.c = shfl_down2(r.c, st); p.d = shfl_down2(r.d, st);
        if (lane < st) m = pcr_identity();
        if (lane + st >= 32) p = pcr_identity();
        r = pcr_step(r, m, p);
      }
      if (lane < n) {
        const float2 q = crcp_mul(r.d, r.b);
        const float f = ig * a.scale;
        X[(size_t)lane * C + cc] = make_float2(q.x * f, q.y * f);
      }
    }
  } else {
    const int NR = kThreads * E;  // rows of the buffer; rows >= n are the identity
    for (int cc = 0; cc < C; ++cc) {
      if (line0 + cc >= a.lines) break;
      const float2 sg = a.sigma[lj[cc]];
      const float2 b0 = make_float2(2.f + (sg.x + a.lam_x[lp[cc]]) * ig, sg.y * ig);
      PcrRow r[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int i = threadIdx.x + kThreads * e;
        r[e] = pcr_identity();
        if (i < n) {
          r[e].a = make_float2(i > 0 ? -1.f : 0.f, 0.f);
          r[e].c = make_float2(i < n - 1 ? -1.f : 0.f, 0.f);
          r[e].b = b0;
          r[e].d = X[(size_t)i * C + cc];
        }
        R[i] = r[e];
      }
      __syncthreads();
      for (int st = 1; st < n; st <<= 1) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = threadIdx.x + kThreads * e;
          const PcrRow m = i - st >= 0 ? R[i - st] : pcr_identity();
          const PcrRow p = i + st < NR ? R[i + st] : pcr_identity();
          r[e] = pcr_step(r[e], m, p);
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) R[threadIdx.x + kThreads * e] = r[e];
        __syncthreads();
      }
      const float f = ig * a.scale;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int i = threadIdx.x + kThreads * e;
        if (i < n) {
          const float2 q = crcp_mul(r[e].d, r[e].b);
          X[(size_t)i * C + cc] = make_float2(q.x * f, q.y * f);
        }
      }
      // (the next line rewrites R only after the barrier that ends its first row set-up)
      __syncthreads();
    }
  }
  __syncthreads();
  for (int it = threadIdx.x; it < (n << logC); it += blockDim.x) {
    const int cc = it & (C - 1), i = it >> logC;
    if (line0 + cc < a.lines) a.S[((size_t)lj[cc] * n + i) * a.P + lp[cc]] = X[(size_t)i * C + cc];
  }
}

cudaError_t launch_pcr(const TriArgs& a, cudaStream_t st) {
  const size_t sm = pcr_smem(a.n, a.C);
  const int blocks = (a.lines + a.C - 1) / a.C;
  auto go = [&](auto kern) -> cudaError_t {
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    prof_begin("pcr_y_f32", st);
    kern<<<blocks, kThreads, sm, st>>>(a);
    prof_end(st);
    return cudaGetLastError();
  };
  if (a.n <= 32) return go(k_pcr<0>);
  if (a.n <= kThreads) return go(k_pcr<1>);
  if (a.n <= 2 * kThreads) return go(k_pcr<2>);
  if (a.n <= 4 * kThreads) return go(k_pcr<4>);
  return cudaErrorInvalidValue;
}

// ---- variable-coefficient tridiagonal systems ----
template <typename T> struct cx_ops;
template <> struct cx_ops<float> {
  using V = float2;
  static __device__ __forceinline__ V mul(V a, V b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
  }
  static __device__ __forceinline__ V fma_(V a, V b, V c) {  // a * b + c
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
  }
  static __device__ __forceinline__ V inv(V a) {
    const float d = __frcp_rn(fmaf(a.x, a.x, a.y * a.y));
    return make_float2(a.x * d, -a.y * d);
  }
  static __device__ __forceinline__ V mk(float x, float y) { return make_float2(x, y); }
  static __device__ __forceinline__ V shfl_up(V v, int d) {
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
  }
  static __device__ __forceinline__ V shfl_down(V v, int d) {
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
  }
};
template <> struct cx_ops<double> {
  using V = double2;
  static __device__ __forceinline__ V mul(V a, V b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
  }
  static __device__ __forceinline__ V fma_(V a, V b, V c) {
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
  }
  static __device__ __forceinline__ V inv(V a) {
    const double d = 1.0 / fma(a.x, a.x, a.y * a.y);
    return make_double2(a.x * d, -a.y * d);
  }
  static __device__ __forceinline__ V mk(double x, double y) { return make_double2(x, y); }
  static __device__ __forceinline__ V shfl_up(V v, int d) {
    return make_double2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
  }
  static __device__ __forceinline__ V shfl_down(V v, int d) {
    return make_double2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
  }
};

// LU factors of each frequency's system, in FP64, stored in T ([J][n]): pivot_i = b_i - o c'_{i-1},
// c'_i = o / pivot_i, b_i = sigma_j m_d + k_d + r_i, o = sigma_j m_o + k_o. The low frequencies
// give systems close to the (singular-looking) Laplacian, where this recurrence is only neutrally
// stable and FP32 rounding would accumulate along the line, hence FP64. The recurrence is a
// Moebius map of c'_{i-1}: with c' = u / v, (u_i, v_i) = M_i (u_{i-1}, v_{i-1}),
// M_i = [[0, o], [-o, b_i]], (u_{-1}, v_{-1}) = (0, 1). One CTA per frequency: each thread
// multiplies the matrices of its PER rows, a scan of the products (rescaled by powers of two,
// which leaves the ratio u / v unchanged) gives c' entering each chunk, and the thread then runs
// the recurrence over its rows.
struct cm2 { double2 a, b, c, d; };  // [[a, b], [c, d]]
__device__ __forceinline__ double2 zmul(double2 x, double2 y) {
  return make_double2(fma(x.x, y.x, -x.y * y.y), fma(x.x, y.y, x.y * y.x));
}
__device__ __forceinline__ double2 zfma(double2 x, double2 y, double2 z) {
  return make_double2(fma(x.x, y.x, fma(-x.y, y.y, z.x)), fma(x.x, y.y, fma(x.y, y.x, z.y)));
}
__device__ __forceinline__ cm2 cm_mul(const cm2& X, const cm2& Y) {  // X Y
  cm2 R;
  R.a = zfma(X.a, Y.a, zmul(X.b, Y.c));
  R.b = zfma(X.a, Y.b, zmul(X.b, Y.d));
  R.c = zfma(X.c, Y.a, zmul(X.d, Y.c));
  R.d = zfma(X.c, Y.b, zmul(X.d, Y.d));
  return R;
}
__device__ __forceinline__ cm2 cm_rescale(cm2 X) {  // divide by a power of two near the largest entry
  const double m = fmax(fmax(fmax(fabs(X.a.x), fabs(X.a.y)), fmax(fabs(X.b.x), fabs(X.b.y))),
                        fmax(fmax(fabs(X.c.x), fabs(X.c.y)), fmax(fabs(X.d.x), fabs(X.d.y))));
  if (!(m > 0.0)) return X;
  int e;
  frexp(m, &e);
  const double s = ldexp(1.0, -e);
  X.a.x *= s; X.a.y *= s; X.b.x *= s; X.b.y *= s; X.c.x *= s; X.c.y *= s; X.d.x *= s; X.d.y *= s;
  return X;
}
__device__ __forceinline__ cm2 cm_shfl_up(const cm2& X, int d) {
  cm2 R;
  R.a = make_double2(__shfl_up_sync(0xffffffffu, X.a.x, d), __shfl_up_sync(0xffffffffu, X.a.y, d));
  R.b = make_double2(__shfl_up_sync(0xffffffffu, X.b.x, d), __shfl_up_sync(0xffffffffu, X.b.y, d));
  R.c = make_double2(__shfl_up_sync(0xffffffffu, X.c.x, d), __shfl_up_sync(0xffffffffu, X.c.y, d));
  R.d = make_double2(__shfl_up_sync(0xffffffffu, X.d.x, d), __shfl_up_sync(0xffffffffu, X.d.y, d));
  return R;
}

template <typename T, int PER>
__global__ void __launch_bounds__(256) k_trivar_factor(TriVarArgs<T> a) {
  using V = typename c2<T>::t;
  __shared__ cm2 tot[8];
  const int j = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int n = a.n, i0 = t * PER;
  const V sg = reinterpret_cast<const V*>(a.sigma)[j];
  const double2 o = make_double2((double)sg.x * a.mo + a.ko, (double)sg.y * a.mo);
  const double2 mo_ = make_double2(-o.x, -o.y);
  const double bx = (double)sg.x * a.md + a.kd, by = (double)sg.y * a.md;
  const double2 z0 = make_double2(0.0, 0.0), one = make_double2(1.0, 0.0);
  // product of this chunk's matrices, later rows on the left
  cm2 P{one, z0, z0, one};
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = i0 + q;
    if (i < n) {
      const double2 bi = make_double2(bx + a.r[i], by);
      // [[0, o], [-o, b_i]] P
      cm2 R;
      R.a = zmul(o, P.c);
      R.b = zmul(o, P.d);
      R.c = zfma(mo_, P.a, zmul(bi, P.c));
      R.d = zfma(mo_, P.b, zmul(bi, P.d));
      P = R;
    }
  }
  P = cm_rescale(P);
  // inclusive warp scan: P <- P (lower lanes' product)
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const cm2 U = cm_shfl_up(P, d);
    if (lane >= d) P = cm_rescale(cm_mul(P, U));
  }
  if (lane == 31) tot[w] = P;
  __syncthreads();
  // (u, v) entering the chunk: the warps below, then the lanes below, applied to (0, 1)
  double2 u = z0, v = one;
  for (int q = 0; q < w; ++q) {
    const cm2& X = tot[q];
    const double2 nu = zfma(X.a, u, zmul(X.b, v)), nv = zfma(X.c, u, zmul(X.d, v));
    u = nu; v = nv;
  }
  {
    const cm2 E = cm_shfl_up(P, 1);
    if (lane > 0) {
      const double2 nu = zfma(E.a, u, zmul(E.b, v)), nv = zfma(E.c, u, zmul(E.d, v));
      u = nu; v = nv;
    }
  }
  // c'_{i0-1} = u / v, then the recurrence over the chunk
  double2 c;
  {
    const double dd = 1.0 / fma(v.x, v.x, v.y * v.y);
    c = zmul(u, make_double2(v.x * dd, -v.y * dd));
  }
  V* ip = reinterpret_cast<V*>(a.ip) + (size_t)j * n;
  V* cp = reinterpret_cast<V*>(a.cp) + (size_t)j * n;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = i0 + q;
    if (i < n) {
      const double2 piv = zfma(mo_, c, make_double2(bx + a.r[i], by));
      const double dd = 1.0 / fma(piv.x, piv.x, piv.y * piv.y);
      const double2 iq = make_double2(piv.x * dd, -piv.y * dd);
      c = zmul(o, iq);
      ip[i].x = (T)iq.x; ip[i].y = (T)iq.y;
      cp[i].x = (T)c.x; cp[i].y = (T)c.y;
    }
  }
}

// One CTA per frequency j. Both substitutions are first-order affine recurrences,
//   forward  y_i = A_i y_{i-1} + B_i,   A_i = -o / pivot_i,  B_i = b_i / pivot_i,
//   backward q_i = -c'_i q_{i+1} + y_i,
// evaluated as parallel scans of the affine maps x -> A x + B under composition: each thread
// composes the maps of its PER consecutive rows (registers), a warp scan with shuffles and a scan
// of the 8 warp totals give each thread the value entering its chunk, and the thread then runs its
// rows. |A_i| < 1 for the diagonally dominant systems, so the composed products stay bounded.
template <typename T, int PER>
__global__ void __launch_bounds__(256) k_trivar_solve(TriVarArgs<T> a) {
  using V = typename c2<T>::t;
  using O = cx_ops<T>;
  __shared__ V tA[8], tB[8];
  const int j = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int n = a.n;
  const V sg = reinterpret_cast<const V*>(a.sigma)[j];
  const V mo = O::mk((T)(-((double)sg.x * a.mo + a.ko)), (T)(-((double)sg.y * a.mo)));  // -o
  V* row = reinterpret_cast<V*>(a.S) + (size_t)j * n;
  const V* ip = reinterpret_cast<const V*>(a.ip) + (size_t)j * n;
  const V* cp = reinterpret_cast<const V*>(a.cp) + (size_t)j * n;
  const V one = O::mk(1, 0), zero = O::mk(0, 0);
  const int i0 = t * PER;
  V b[PER], p[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = i0 + q;
    b[q] = i < n ? row[i] : zero;
    p[q] = i < n ? ip[i] : zero;   // beyond n: A = B = 0 (a constant map to 0, never used)
  }
  // ---- forward: compose this chunk's maps (rows in increasing order) ----
  V cA = one, cB = zero;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    if (i0 + q < n) {
      const V Ai = O::mul(mo, p[q]), Bi = O::mul(b[q], p[q]);
      cB = O::fma_(Ai, cB, Bi);
      cA = O::mul(Ai, cA);
    }
  }
  // inclusive warp scan: (cA, cB) <- mine o lower lanes'
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const V uA = O::shfl_up(cA, d), uB = O::shfl_up(cB, d);
    if (lane >= d) {
      cB = O::fma_(cA, uB, cB);
      cA = O::mul(cA, uA);
    }
  }
  if (lane == 31) { tA[w] = cA; tB[w] = cB; }
  __syncthreads();
  // value entering the chunk: (inclusive scan of the lanes below) applied to the warps below
  V x = zero;  // y_{-1} = 0
  for (int q = 0; q < w; ++q) x = O::fma_(tA[q], x, tB[q]);
  {
    const V eA = O::shfl_up(cA, 1), eB = O::shfl_up(cB, 1);
    if (lane > 0) x = O::fma_(eA, x, eB);
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    if (i0 + q < n) {
      x = O::fma_(O::mul(mo, p[q]), x, O::mul(b[q], p[q]));
      b[q] = x;  // y_i
    }
  }
  __syncthreads();  // the warp totals are reused below
  // ---- backward: q_i = -c'_i q_{i+1} + y_i, chunks composed from the top ----
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = i0 + q;
    p[q] = i < n ? cp[i] : zero;
    p[q] = O::mk(-p[q].x, -p[q].y);
  }
  cA = one;
  cB = zero;
#pragma unroll
  for (int q = PER - 1; q >= 0; --q) {
    if (i0 + q < n) {
      cB = O::fma_(p[q], cB, b[q]);
      cA = O::mul(p[q], cA);
    }
  }
  // inclusive suffix scan over lanes: (cA, cB) <- mine o higher lanes'
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const V uA = O::shfl_down(cA, d), uB = O::shfl_down(cB, d);
    if (lane + d < 32) {
      cB = O::fma_(cA, uB, cB);
      cA = O::mul(cA, uA);
    }
  }
  if (lane == 0) { tA[w] = cA; tB[w] = cB; }
  __syncthreads();
  x = zero;  // q_n = 0
  for (int q = (int)(blockDim.x >> 5) - 1; q > w; --q) x = O::fma_(tA[q], x, tB[q]);
  {
    const V eA = O::shfl_down(cA, 1), eB = O::shfl_down(cB, 1);
    if (lane < 31) x = O::fma_(eA, x, eB);
  }
#pragma unroll
  for (int q = PER - 1; q >= 0; --q) {
    if (i0 + q < n) {
      x = O::fma_(p[q], x, b[q]);
      row[i0 + q] = x;
    }
  }
}

// The same factorisation for factors stored in FP32 (MIXED / FP32 plans), in double-float
// arithmetic on the FP32 pipes (~48-bit significands: the accuracy the low frequencies need,
// without the FP64 pipe, which runs at a small fraction of the FP32 rate). Same scan structure.
struct cmf { ffc a, b, c, d; };  // [[a, b], [c, d]]
__device__ __forceinline__ ffc cfma_ff(ffc x, ffc y, ffc z) { return cadd(cmul(x, y), z); }
__device__ __forceinline__ cmf cmf_mul(const cmf& X, const cmf& Y) {  // X Y
  cmf R;
  R.a = cfma_ff(X.a, Y.a, cmul(X.b, Y.c));
  R.b = cfma_ff(X.a, Y.b, cmul(X.b, Y.d));
  R.c = cfma_ff(X.c, Y.a, cmul(X.d, Y.c));
  R.d = cfma_ff(X.c, Y.b, cmul(X.d, Y.d));
  return R;
}
__device__ __forceinline__ ffc ffc_scale(ffc x, float s) { return ffc{x.rh * s, x.rl * s, x.ih * s, x.il * s}; }
__device__ __forceinline__ cmf cmf_rescale(cmf X) {  // divide by a power of two near the largest entry
  const float m = fmaxf(fmaxf(fmaxf(fabsf(X.a.rh), fabsf(X.a.ih)), fmaxf(fabsf(X.b.rh), fabsf(X.b.ih))),
                        fmaxf(fmaxf(fabsf(X.c.rh), fabsf(X.c.ih)), fmaxf(fabsf(X.d.rh), fabsf(X.d.ih))));
  if (!(m > 0.f)) return X;
  int e;
  frexpf(m, &e);
  const float s = ldexpf(1.f, -e);
  X.a = ffc_scale(X.a, s); X.b = ffc_scale(X.b, s); X.c = ffc_scale(X.c, s); X.d = ffc_scale(X.d, s);
  return X;
}
__device__ __forceinline__ ffc ffc_shfl_up(ffc x, int d) {
  return ffc{__shfl_up_sync(0xffffffffu, x.rh, d), __shfl_up_sync(0xffffffffu, x.rl, d),
             __shfl_up_sync(0xffffffffu, x.ih, d), __shfl_up_sync(0xffffffffu, x.il, d)};
}
__device__ __forceinline__ cmf cmf_shfl_up(const cmf& X, int d) {
  return cmf{ffc_shfl_up(X.a, d), ffc_shfl_up(X.b, d), ffc_shfl_up(X.c, d), ffc_shfl_up(X.d, d)};
}
// 1 / d for a double-float d > 0: FP32 reciprocal refined by one Newton step (error ~2^-46)
__device__ __forceinline__ ff ff_recip(ff d) {
  const float q = __frcp_rn(d.hi);
  const ff e = ff_add(ff{1.f, 0.f}, ff_mul(d, ff{-q, 0.f}));  // 1 - d q
  return ff_add(ff{q, 0.f}, ff_mul(ff{q, 0.f}, e));
}
__device__ __forceinline__ ffc ffc_inv(ffc z) {  // conj(z) / |z|^2
  const ff re = ffc_re(z), im = ffc_im(z);
  const ff n = ff_add(ff_mul(re, re), ff_mul(im, im));
  const ff r = ff_recip(n);
  return ffc_make(ff_mul(re, r), ff_mul(ff{-im.hi, -im.lo}, r));
}

template <int PER>
__global__ void __launch_bounds__(256) k_trivar_factor_ff(TriVarArgs<float> a) {
  __shared__ cmf tot[8];
  const int j = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int n = a.n, i0 = t * PER;
  const float2 sg = reinterpret_cast<const float2*>(a.sigma)[j];
  const ff sx{sg.x, 0.f}, sy{sg.y, 0.f};
  const ff md = ff_from_double(a.md), mo = ff_from_double(a.mo), kd = ff_from_double(a.kd),
           ko = ff_from_double(a.ko);
  const ffc o = ffc_make(ff_add(ff_mul(sx, mo), ko), ff_mul(sy, mo));   // sigma_j m_o + k_o
  const ffc mo_ = ffc{-o.rh, -o.rl, -o.ih, -o.il};
  const ff bx = ff_add(ff_mul(sx, md), kd), by = ff_mul(sy, md);        // sigma_j m_d + k_d
  const ffc z0{0.f, 0.f, 0.f, 0.f}, one{1.f, 0.f, 0.f, 0.f};
  cmf P{one, z0, z0, one};
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = i0 + q;
    if (i < n) {
      const ffc bi = ffc_make(ff_add(bx, ff_from_double(a.r[i])), by);
      cmf R;
      R.a = cmul(o, P.c);
      R.b = cmul(o, P.d);
      R.c = cfma_ff(mo_, P.a, cmul(bi, P.c));
      R.d = cfma_ff(mo_, P.b, cmul(bi, P.d));
      P = R;
      if ((q & 1) == 1) P = cmf_rescale(P);  // keep the FP32 exponent range
    }
  }
  P = cmf_rescale(P);
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const cmf U = cmf_shfl_up(P, d);
    if (lane >= d) P = cmf_rescale(cmf_mul(P, U));
  }
  if (lane == 31) tot[w] = P;
  __syncthreads();
  ffc u = z0, v = one;
  for (int q = 0; q < w; ++q) {
    const cmf& X = tot[q];
    const ffc nu = cfma_ff(X.a, u, cmul(X.b, v)), nv = cfma_ff(X.c, u, cmul(X.d, v));
    const float s = ldexpf(1.f, -ilogbf(fmaxf(fmaxf(fabsf(nu.rh), fabsf(nu.ih)), fmaxf(fabsf(nv.rh), fabsf(nv.ih))) + 1e-30f));
    u = ffc_scale(nu, s); v = ffc_scale(nv, s);
  }
  {
    const cmf E = cmf_shfl_up(P, 1);
    if (lane > 0) {
      const ffc nu = cfma_ff(E.a, u, cmul(E.b, v)), nv = cfma_ff(E.c, u, cmul(E.d, v));
      u = nu; v = nv;
    }
  }
  ffc c = cmul(u, ffc_inv(v));  // c'_{i0-1}
  float2* ip = reinterpret_cast<float2*>(a.ip) + (size_t)j * n;
  float2* cp = reinterpret_cast<float2*>(a.cp) + (size_t)j * n;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = i0 + q;
    if (i < n) {
      const ffc piv = cfma_ff(mo_, c, ffc_make(ff_add(bx, ff_from_double(a.r[i])), by));
      const ffc iq = ffc_inv(piv);
      c = cmul(o, iq);
      ip[i] = make_float2(__fadd_rn(iq.rh, iq.rl), __fadd_rn(iq.ih, iq.il));
      cp[i] = make_float2(__fadd_rn(c.rh, c.rl), __fadd_rn(c.ih, c.il));
    }
  }
}

template <typename T> cudaError_t launch_trivar_factor(const TriVarArgs<T>& a, cudaStream_t st) {
  if (a.n < 1 || a.n > 8 * 256) return cudaErrorInvalidValue;
  prof_begin("trivar_factor", st);
  if constexpr (sizeof(T) == 4) {
    if (a.n <= 256) k_trivar_factor_ff<1><<<a.J, 256, 0, st>>>(a);
    else if (a.n <= 512) k_trivar_factor_ff<2><<<a.J, 256, 0, st>>>(a);
    else if (a.n <= 1024) k_trivar_factor_ff<4><<<a.J, 256, 0, st>>>(a);
    else k_trivar_factor_ff<8><<<a.J, 256, 0, st>>>(a);
  } else {
    if (a.n <= 256) k_trivar_factor<T, 1><<<a.J, 256, 0, st>>>(a);
    else if (a.n <= 512) k_trivar_factor<T, 2><<<a.J, 256, 0, st>>>(a);
    else if (a.n <= 1024) k_trivar_factor<T, 4><<<a.J, 256, 0, st>>>(a);
    else k_trivar_factor<T, 8><<<a.J, 256, 0, st>>>(a);
  }
  prof_end(st);
  return cudaGetLastError();
}
template <typename T> cudaError_t launch_trivar_solve(const TriVarArgs<T>& a, cudaStream_t st) {
  if (a.n < 1 || a.n > 8 * 256) return cudaErrorInvalidValue;
  prof_begin(sizeof(T) == 4 ? "trivar_solve_f32" : "trivar_solve_f64", st);
  // rows per thread: the smallest of 1, 2, 4, 8 that covers the line with 256 threads
  if (a.n <= 256) k_trivar_solve<T, 1><<<a.J, 256, 0, st>>>(a);
  else if (a.n <= 512) k_trivar_solve<T, 2><<<a.J, 256, 0, st>>>(a);
  else if (a.n <= 1024) k_trivar_solve<T, 4><<<a.J, 256, 0, st>>>(a);
  else k_trivar_solve<T, 8><<<a.J, 256, 0, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

template size_t axis_smem<float>(int, int, bool, int);
template size_t axis_smem<double>(int, int, bool, int);
template cudaError_t launch_axis<float>(const AxisArgs<float>&, cudaStream_t);
template cudaError_t launch_axis<double>(const AxisArgs<double>&, cudaStream_t);
template cudaError_t launch_axis_per<float>(const AxisArgs<float>&, cudaStream_t);
template cudaError_t launch_axis_per<double>(const AxisArgs<double>&, cudaStream_t);
template cudaError_t launch_trivar_factor<float>(const TriVarArgs<float>&, cudaStream_t);
template cudaError_t launch_trivar_factor<double>(const TriVarArgs<double>&, cudaStream_t);
template cudaError_t launch_trivar_solve<float>(const TriVarArgs<float>&, cudaStream_t);
template cudaError_t launch_trivar_solve<double>(const TriVarArgs<double>&, cudaStream_t);

}  // namespace pint
