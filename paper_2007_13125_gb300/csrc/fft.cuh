// Shared-memory FFT over many columns, used for every transform of the sweep:
// the kappa-scaled DFT along time (Algorithm 1/2, steps 1 and 3), the sine transforms
// along x / y that diagonalise the finite-difference Laplacian, and the zero-padded
// 2N-point FFTs of the CQ Toeplitz products (Sec. 3.2, speedup analysis of Algorithm 2).
//
// Layout: element (n, c) of a tile of L points x C columns lives at X[n * ld + c]
// (column index fastest, so a warp touches consecutive columns: conflict-free banks).
//
// Algorithm: in-place mixed-radix decimation in frequency. L = R_1 R_2 ... R_s with each
// R_i in {2, 4, 8, 16}; pass i splits every block of length Ls into R_i interleaved
// sub-sequences (stride Ls/R_i), does an R_i-point DFT in registers, multiplies by the
// twiddles W_Ls^{n2 q}, and writes back in place. After all passes, position
//   p = sum_i q_i L/(R_1..R_i)   holds frequency   j = sum_i q_i R_1..R_{i-1}
// (a mixed-radix digit reversal; fft_pos() maps j -> p). The inverse transform applies
// the conjugate-transposed passes in reverse order: it takes a spectrum stored in that
// permuted order and returns L times the inverse DFT in natural order, so a forward /
// pointwise-multiply / inverse sequence needs no permutation at all.
#pragma once
#include <cuda_runtime.h>

#include "ff.cuh"

namespace pint {

template <typename T> struct c2;
template <> struct c2<float> { using t = float2; };
template <> struct c2<double> { using t = double2; };

__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { V r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { V r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
  V r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}

// cos(2 pi m / 16), m = 0..15
__host__ __device__ constexpr double cos16(int m) {
  return m == 0 ? 1.0 : m == 1 ? 0.92387953251128674 : m == 2 ? 0.70710678118654757
       : m == 3 ? 0.38268343236508984 : m == 4 ? 0.0 : m == 5 ? -0.38268343236508984
       : m == 6 ? -0.70710678118654757 : m == 7 ? -0.92387953251128674 : m == 8 ? -1.0
       : m == 9 ? -0.92387953251128674 : m == 10 ? -0.70710678118654757
       : m == 11 ? -0.38268343236508984 : m == 12 ? 0.0 : m == 13 ? 0.38268343236508984
       : m == 14 ? 0.70710678118654757 : 0.92387953251128674;
}
__host__ __device__ constexpr double sin16(int m) { return cos16((m + 12) & 15); }

// v * exp(DIR * 2 pi i M / 16), DIR = -1 (forward) or +1, M a compile-time constant
template <int M, int DIR, typename V>
__device__ __forceinline__ V twid16(V v) {
  using T = decltype(v.x);
  if constexpr (M == 0) {
    return v;
  } else if constexpr (M == 4) {
    return DIR < 0 ? mk(v.y, -v.x) : mk(-v.y, v.x);
  } else {
    constexpr T c = (T)cos16(M);
    constexpr T s = (T)(DIR * sin16(M));
    return mk(v.x * c - v.y * s, v.x * s + v.y * c);
  }
}

// The same rotation for a double-float complex value (ffc, ff.cuh), constants split into
// hi + lo floats at compile time.
template <int M, int DIR>
__device__ __forceinline__ ffc twid16(ffc v) {
  if constexpr (M == 0) {
    return v;
  } else if constexpr (M == 4) {
    return DIR < 0 ? ffc{v.ih, v.il, -v.rh, -v.rl} : ffc{-v.ih, -v.il, v.rh, v.rl};
  } else {
    constexpr double c = cos16(M), s = DIR * sin16(M);
    constexpr float ch = (float)c, sh = (float)s;
    constexpr float cl = (float)(c - (double)ch), sl = (float)(s - (double)sh);
    return cmul(v, ffc{ch, cl, sh, sl});
  }
}

__host__ __device__ constexpr int ilog2c(int r) { return r <= 1 ? 0 : 1 + ilog2c(r >> 1); }
__host__ __device__ constexpr int brev(int i, int bits) {
  return bits == 0 ? 0 : ((i & 1) << (bits - 1)) | brev(i >> 1, bits - 1);
}

// Butterflies of one radix-2 decimation-in-time stage of span LEN, block start I, offset J.
// Template recursion keeps every array index a compile-time constant (registers only).
template <int LEN, int I, int J, int R, int DIR, typename V>
__device__ __forceinline__ void dit_bfly(V (&y)[R]) {
  if constexpr (I < R) {
    if constexpr (J < LEN / 2) {
      const V u = y[I + J];
      const V t = twid16<J * (16 / LEN), DIR>(y[I + J + LEN / 2]);
      y[I + J] = cadd(u, t);
      y[I + J + LEN / 2] = csub(u, t);
      dit_bfly<LEN, I, J + 1, R, DIR>(y);
    } else {
      dit_bfly<LEN, I + LEN, 0, R, DIR>(y);
    }
  }
}

template <int LEN, int R, int DIR, typename V>
__device__ __forceinline__ void dit_stage(V (&y)[R]) {
  dit_bfly<LEN, 0, 0, R, DIR>(y);
  if constexpr (LEN < R) dit_stage<LEN * 2, R, DIR>(y);
}

template <int I, int R, typename V>
__device__ __forceinline__ void brev_copy(V (&y)[R], const V (&x)[R]) {
  if constexpr (I < R) {
    constexpr int J = brev(I, ilog2c(R));
    y[J] = x[I];
    brev_copy<I + 1, R>(y, x);
  }
}

// y_q = sum_r x_r exp(DIR 2 pi i r q / R), natural order in and out; R <= 16.
template <int R, int DIR, typename V>
__device__ __forceinline__ void dft_reg(V (&x)[R]) {
  V y[R];
  brev_copy<0, R>(y, x);
  if constexpr (R > 1) dit_stage<2, R, DIR>(y);
#pragma unroll
  for (int i = 0; i < R; ++i) x[i] = y[i];
}

// Radix schedule: np = ceil(log2 L / MAXLOG) passes with the bits spread evenly (first passes
// take the extra bit), each radix at most 2^MAXLOG (16 by default; smaller for wide element
// types to bound registers).
__host__ __device__ inline int fft_npass(int L, int maxlog = 4) {
  const int e = ilog2c(L);
  return (e + maxlog - 1) / maxlog;
}
__host__ __device__ inline int fft_logradix(int L, int pass, int maxlog = 4) {
  const int e = ilog2c(L);
  const int np = (e + maxlog - 1) / maxlog;
  return e / np + (pass < e % np ? 1 : 0);
}
__host__ __device__ inline int fft_radix(int L, int pass, int maxlog = 4) { return 1 << fft_logradix(L, pass, maxlog); }

// position of frequency j in the output of the forward transform
__host__ __device__ inline int fft_pos(int j, int L, int maxlog = 4) {
  const int np = fft_npass(L, maxlog);
  int p = 0, logLs = ilog2c(L);
  for (int i = 0; i < np; ++i) {
    const int lr = fft_logradix(L, i, maxlog);
    const int q = j & ((1 << lr) - 1);
    j >>= lr;
    logLs -= lr;
    p += q << logLs;
  }
  return p;
}

// fill perm[j] = fft_pos(j, L), j < L (cooperatively, by the whole block)
__device__ __forceinline__ void fft_perm_table(unsigned short* perm, int L, int maxlog = 4) {
  for (int j = threadIdx.x; j < L; j += blockDim.x) perm[j] = (unsigned short)fft_pos(j, L, maxlog);
}

// One pass of radix R = 2^LR at sub-length Ls = 2^logLs on a tile of C = 2^logC columns.
// DIR < 0: forward (gather natural stride, DFT, twiddle, scatter). DIR > 0: its conjugate
// transpose. All index arithmetic is shifts and masks.
template <int LR, int DIR, typename V>
__device__ __forceinline__ void fft_pass(V* X, int ld, int logC, int logL, int logLs, const V* tw) {
  constexpr int R = 1 << LR;
  const int logS = logLs - LR;
  const int Smask = (1 << logS) - 1;
  const int items = 1 << (logL - LR + logC);
  const int tshift = logL - logLs;  // W_Ls^e = W_L^{e << tshift}
  const int Lmask = (1 << logL) - 1;
  const int Cmask = (1 << logC) - 1;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int c = it & Cmask;
    const int g = it >> logC;
    const int n2 = g & Smask;
    const int base = ((g >> logS) << logLs) + n2;
    V x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = X[(base + (r << logS)) * ld + c];
    if (DIR < 0) {
      dft_reg<R, -1>(x);
#pragma unroll
      for (int q = 1; q < R; ++q) x[q] = cmul(x[q], tw[((n2 * q) << tshift) & Lmask]);
    } else {
#pragma unroll
      for (int q = 1; q < R; ++q) x[q] = cmulc(x[q], tw[((n2 * q) << tshift) & Lmask]);
      dft_reg<R, 1>(x);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) X[(base + (r << logS)) * ld + c] = x[r];
  }
}

template <int DIR, int MAXLOG, typename V>
__device__ __forceinline__ void fft_pass_dispatch(int lr, V* X, int ld, int logC, int logL, int logLs,
                                                  const V* tw) {
  switch (lr) {
    case 1: fft_pass<1, DIR>(X, ld, logC, logL, logLs, tw); break;
    case 2: fft_pass<2, DIR>(X, ld, logC, logL, logLs, tw); break;
    default:
      if constexpr (MAXLOG >= 4) {
        if (lr == 4) { fft_pass<4, DIR>(X, ld, logC, logL, logLs, tw); break; }
      }
      fft_pass<3, DIR>(X, ld, logC, logL, logLs, tw);
      break;
  }
}

// Forward: natural order in, permuted (fft_pos(., ., MAXLOG)) order out; exp(-2 pi i n j / L).
// tw[m] = exp(-2 pi i m / L), m < L, must be visible to all threads. C = 2^logC columns.
template <int MAXLOG = 4, typename V>
__device__ void fft_forward(V* X, int ld, int logC, int L, const V* tw) {
  const int logL = ilog2c(L);
  const int np = fft_npass(L, MAXLOG);
  int logLs = logL;
  for (int i = 0; i < np; ++i) {
    const int lr = fft_logradix(L, i, MAXLOG);
    fft_pass_dispatch<-1, MAXLOG>(lr, X, ld, logC, logL, logLs, tw);
    logLs -= lr;
    __syncthreads();
  }
}

// Inverse: permuted order in, natural order out, unnormalised: x_n = sum_j X_j exp(+2 pi i n j / L).
template <int MAXLOG = 4, typename V>
__device__ void fft_inverse(V* X, int ld, int logC, int L, const V* tw) {
  const int logL = ilog2c(L);
  const int np = fft_npass(L, MAXLOG);
  int logLs = 0;
  for (int i = np - 1; i >= 0; --i) {
    const int lr = fft_logradix(L, i, MAXLOG);
    logLs += lr;
    fft_pass_dispatch<1, MAXLOG>(lr, X, ld, logC, logL, logLs, tw);
    __syncthreads();
  }
}

// ---- compile-time variant: L = 2^LOGL, C = 2^LOGC columns, pitch LD, all known to the
// compiler, so every shared-memory address is a base register plus an immediate and the
// twiddle indices need no masks. Same radix schedule (and output order) as above.
__host__ __device__ constexpr int ct_npass(int logL, int maxlog) { return (logL + maxlog - 1) / maxlog; }
__host__ __device__ constexpr int ct_logradix(int logL, int pass, int maxlog) {
  return logL / ct_npass(logL, maxlog) + (pass < logL % ct_npass(logL, maxlog) ? 1 : 0);
}

template <int LR, int DIR, int LOGL, int LOGLS, int LOGC, int LD, typename V>
__device__ __forceinline__ void fft_pass_ct(V* X, const V* tw) {
  constexpr int R = 1 << LR, LOGS = LOGLS - LR, S = 1 << LOGS, C = 1 << LOGC;
  constexpr int ITEMS = 1 << (LOGL - LR + LOGC);
  constexpr int TSHIFT = LOGL - LOGLS;  // W_Ls^e = W_L^{e << TSHIFT}
  for (int it = threadIdx.x; it < ITEMS; it += blockDim.x) {
    const int c = it & (C - 1);
    const int g = it >> LOGC;
    const int n2 = g & (S - 1);
    const int base = ((g >> LOGS) << LOGLS) + n2;
    V* p = X + base * LD + c;
    V x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = p[r * S * LD];
    if constexpr (DIR < 0) {
      dft_reg<R, -1>(x);
      if constexpr (S > 1) {
        const V* w = tw + (n2 << TSHIFT);
#pragma unroll
        for (int q = 1; q < R; ++q) x[q] = cmul(x[q], w[(q - 1) * (n2 << TSHIFT)]);
      }
    } else {
      if constexpr (S > 1) {
        const V* w = tw + (n2 << TSHIFT);
#pragma unroll
        for (int q = 1; q < R; ++q) x[q] = cmulc(x[q], w[(q - 1) * (n2 << TSHIFT)]);
      }
      dft_reg<R, 1>(x);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) p[r * S * LD] = x[r];
  }
}

template <int P, int NP, int LOGL, int LOGLS, int LOGC, int LD, int MAXLOG, typename V>
__device__ __forceinline__ void fft_forward_ct_rec(V* X, const V* tw) {
  if constexpr (P < NP) {
    constexpr int LR = ct_logradix(LOGL, P, MAXLOG);
    fft_pass_ct<LR, -1, LOGL, LOGLS, LOGC, LD>(X, tw);
    __syncthreads();
    fft_forward_ct_rec<P + 1, NP, LOGL, LOGLS - LR, LOGC, LD, MAXLOG>(X, tw);
  }
}

template <int P, int LOGL, int LOGLS, int LOGC, int LD, int MAXLOG, typename V>
__device__ __forceinline__ void fft_inverse_ct_rec(V* X, const V* tw) {
  if constexpr (P >= 0) {
    constexpr int LR = ct_logradix(LOGL, P, MAXLOG);
    fft_pass_ct<LR, 1, LOGL, LOGLS + LR, LOGC, LD>(X, tw);
    __syncthreads();
    fft_inverse_ct_rec<P - 1, LOGL, LOGLS + LR, LOGC, LD, MAXLOG>(X, tw);
  }
}

// Same contracts as fft_forward / fft_inverse.
template <int LOGL, int LOGC, int LD, int MAXLOG = 4, typename V>
__device__ void fft_forward_ct(V* X, const V* tw) {
  fft_forward_ct_rec<0, ct_npass(LOGL, MAXLOG), LOGL, LOGL, LOGC, LD, MAXLOG>(X, tw);
}
template <int LOGL, int LOGC, int LD, int MAXLOG = 4, typename V>
__device__ void fft_inverse_ct(V* X, const V* tw) {
  fft_inverse_ct_rec<ct_npass(LOGL, MAXLOG) - 1, LOGL, 0, LOGC, LD, MAXLOG>(X, tw);
}

}  // namespace pint
