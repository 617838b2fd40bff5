// Shared-memory FFT over many columns, used for every transform of the sweep:
// the kappa-scaled DFT along time (Algorithm 1/2, steps 1 and 3), the sine transforms
// along x / y that diagonalise the finite-difference Laplacian, and the zero-padded
// 2N-point FFTs of the CQ Toeplitz products (Sec. 3.2, speedup analysis of Algorithm 2).
//
// Layout: element (n, c) of a tile of L points x C columns lives at X[n * ld + c]
// (column index fastest, so a warp touches consecutive columns: conflict-free banks).
//
// Algorithm: in-place mixed-radix decimation in frequency. L = R_1 R_2 ... R_s with each
// R_i in {2, 4, 8, 16} (L a power of two), or, for L = 2^a 5^b, b passes of radix 5 first and
// then the power-of-two passes of 2^a (index arithmetic by division instead of shifts; the
// paper's own sizes, N = 100 and 999 interior nodes, are of that form); pass i splits every
// block of length Ls into R_i interleaved
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
template <typename V> __device__ __forceinline__ V cneg(V a) { V r; r.x = -a.x; r.y = -a.y; return r; }
template <typename V> __device__ __forceinline__ V czero() { V r; r.x = 0; r.y = 0; return r; }
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

// ... and for the lazy double-float complex type (ffz, ff.cuh)
template <int M, int DIR>
__device__ __forceinline__ ffz twid16(ffz v) {
  if constexpr (M == 0) {
    return v;
  } else if constexpr (M == 4) {
    return DIR < 0 ? ffz{v.ih, v.il, -v.rh, -v.rl} : ffz{-v.ih, -v.il, v.rh, v.rl};
  } else {
    constexpr double c = cos16(M), s = DIR * sin16(M);
    constexpr float ch = (float)c, sh = (float)s;
    constexpr float cl = (float)(c - (double)ch), sl = (float)(s - (double)sh);
    return cmul(v, ffz{ch, cl, sh, sl});
  }
}

// value as a pass stores it: unchanged, except for types that renormalise there (ffz)
template <typename V> __device__ __forceinline__ V fft_store(V v) { return v; }

__host__ __device__ constexpr int ilog2c(int r) { return r <= 1 ? 0 : 1 + ilog2c(r >> 1); }
// the same for values known only at run time (ilog2c recurses when its argument is not a constant)
__host__ __device__ inline int ilog2r(int r) {
#ifdef __CUDA_ARCH__
  return r <= 1 ? 0 : 31 - __clz(r);
#else
  int e = 0;
  while (r > 1) { r >>= 1; ++e; }
  return e;
#endif
}
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
  const int e = ilog2r(L);
  return (e + maxlog - 1) / maxlog;
}
__host__ __device__ inline int fft_logradix(int L, int pass, int maxlog = 4) {
  const int e = ilog2r(L);
  const int np = (e + maxlog - 1) / maxlog;
  return e / np + (pass < e % np ? 1 : 0);
}
__host__ __device__ inline int fft_radix(int L, int pass, int maxlog = 4) { return 1 << fft_logradix(L, pass, maxlog); }

// ---- lengths L = 2^a 5^b that are not powers of two ----
__host__ __device__ inline bool fft_is_pow2(int L) { return L > 0 && (L & (L - 1)) == 0; }
// b (the power of 5 in L)
__host__ __device__ inline int fft_fives(int L) {
  int b = 0;
  while (L > 1 && L % 5 == 0) { L /= 5; ++b; }
  return b;
}
// passes of the mixed schedule: b radix-5 passes, then the schedule above for 2^a
__host__ __device__ inline int fft_mr_npass(int L, int maxlog) {
  const int b = fft_fives(L);
  int P = L;
  for (int i = 0; i < b; ++i) P /= 5;
  return b + (P > 1 ? fft_npass(P, maxlog) : 0);
}
__host__ __device__ inline int fft_mr_radix(int L, int pass, int maxlog) {
  const int b = fft_fives(L);
  if (pass < b) return 5;
  int P = L;
  for (int i = 0; i < b; ++i) P /= 5;
  return fft_radix(P, pass - b, maxlog);
}
// True if L = 2^a 5^b, the lengths the transforms accept.
__host__ __device__ inline bool fft_len_ok(int L) {
  if (L < 1) return false;
  while (L % 5 == 0) L /= 5;
  return fft_is_pow2(L);
}
__host__ __device__ inline int fft_pos_mr(int j, int L, int maxlog) {
  const int np = fft_mr_npass(L, maxlog);
  int p = 0, Ls = L;
  for (int i = 0; i < np; ++i) {
    const int R = fft_mr_radix(L, i, maxlog);
    const int q = j % R;
    j /= R;
    Ls /= R;
    p += q * Ls;
  }
  return p;
}

// position of frequency j in the output of the forward transform
__host__ __device__ inline int fft_pos(int j, int L, int maxlog = 4) {
  if (!fft_is_pow2(L)) return fft_pos_mr(j, L, maxlog);
  const int e = ilog2r(L), np = (e + maxlog - 1) / maxlog, base = e / np, extra = e - base * np;
  int p = 0, logLs = e;
  for (int i = 0; i < np; ++i) {
    const int lr = base + (i < extra ? 1 : 0);
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
    for (int r = 0; r < R; ++r) X[(base + (r << logS)) * ld + c] = fft_store(x[r]);
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

// 5-point DFT. Constants: cos(2 pi/5) = (sqrt5 - 1)/4, cos(4 pi/5) = -(sqrt5 + 1)/4,
// sin(2 pi/5) = sqrt((5 + sqrt5)/8), sin(4 pi/5) = sqrt((5 - sqrt5)/8). With t1 = x1 + x4,
// t2 = x2 + x3, t3 = x1 - x4, t4 = x2 - x3 and w = exp(DIR 2 pi i/5):
//   y0 = x0 + t1 + t2,
//   y1 = a1 + DIR i b1,  y4 = a1 - DIR i b1,  a1 = x0 + c1 t1 + c2 t2,  b1 = s1 t3 + s2 t4,
//   y2 = a2 + DIR i b2,  y3 = a2 - DIR i b2,  a2 = x0 + c2 t1 + c1 t2,  b2 = s2 t3 - s1 t4.
constexpr double kCos1of5 = 0.30901699437494742, kCos2of5 = -0.80901699437494742;
constexpr double kSin1of5 = 0.95105651629515357, kSin2of5 = 0.58778525229247313;
__device__ __forceinline__ float2 rscale(float2 v, double c) { const float f = (float)c; return mk(v.x * f, v.y * f); }
__device__ __forceinline__ double2 rscale(double2 v, double c) { return mk(v.x * c, v.y * c); }
__device__ __forceinline__ ffc rscale(ffc v, double c) {
  const float h = (float)c, l = (float)(c - (double)h);
  return cmul(v, ffc{h, l, 0.f, 0.f});
}
__device__ __forceinline__ ffz rscale(ffz v, double c) {
  const float h = (float)c, l = (float)(c - (double)h);
  return cmul(v, ffz{h, l, 0.f, 0.f});
}
// v * (DIR i)
template <int DIR> __device__ __forceinline__ float2 rot_i(float2 v) { return DIR < 0 ? mk(v.y, -v.x) : mk(-v.y, v.x); }
template <int DIR> __device__ __forceinline__ double2 rot_i(double2 v) { return DIR < 0 ? mk(v.y, -v.x) : mk(-v.y, v.x); }
template <int DIR> __device__ __forceinline__ ffc rot_i(ffc v) {
  return DIR < 0 ? ffc{v.ih, v.il, -v.rh, -v.rl} : ffc{-v.ih, -v.il, v.rh, v.rl};
}
template <int DIR> __device__ __forceinline__ ffz rot_i(ffz v) {
  return DIR < 0 ? ffz{v.ih, v.il, -v.rh, -v.rl} : ffz{-v.ih, -v.il, v.rh, v.rl};
}
template <int DIR, typename V>
__device__ __forceinline__ void dft5(V (&x)[5]) {
  const V t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]);
  const V t3 = csub(x[1], x[4]), t4 = csub(x[2], x[3]);
  const V a1 = cadd(x[0], cadd(rscale(t1, kCos1of5), rscale(t2, kCos2of5)));
  const V a2 = cadd(x[0], cadd(rscale(t1, kCos2of5), rscale(t2, kCos1of5)));
  const V b1 = rot_i<DIR>(cadd(rscale(t3, kSin1of5), rscale(t4, kSin2of5)));
  const V b2 = rot_i<DIR>(csub(rscale(t3, kSin2of5), rscale(t4, kSin1of5)));
  x[0] = cadd(x[0], cadd(t1, t2));
  x[1] = cadd(a1, b1);
  x[4] = csub(a1, b1);
  x[2] = cadd(a2, b2);
  x[3] = csub(a2, b2);
}
template <int R, int DIR, typename V>
__device__ __forceinline__ void dft_any(V (&x)[R]) {
  if constexpr (R == 5) dft5<DIR>(x);
  else dft_reg<R, DIR>(x);
}

// One pass of radix R (5 or a power of two) at sub-length Ls of a length L = 2^a 5^b: the same
// gather / DFT / twiddle / scatter as fft_pass, with the stride S = Ls / R and the block index
// found by division. Twiddle index n2 q L / Ls < L.
template <int R, int DIR, typename V>
__device__ __forceinline__ void fft_pass_mr(V* X, int ld, int logC, int L, int Ls, const V* tw) {
  const int S = Ls / R;
  const int items = (L / R) << logC;
  const int tstep = L / Ls;
  const int Cmask = (1 << logC) - 1;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int c = it & Cmask;
    const int g = it >> logC;
    const int blk = g / S, n2 = g - blk * S;
    const int base = blk * Ls + n2;
    V x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = X[(base + r * S) * ld + c];
    if (DIR < 0) {
      dft_any<R, -1>(x);
#pragma unroll
      for (int q = 1; q < R; ++q) x[q] = cmul(x[q], tw[n2 * q * tstep]);
    } else {
#pragma unroll
      for (int q = 1; q < R; ++q) x[q] = cmulc(x[q], tw[n2 * q * tstep]);
      dft_any<R, 1>(x);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) X[(base + r * S) * ld + c] = fft_store(x[r]);
  }
}

template <int DIR, int MAXLOG, typename V>
__device__ __forceinline__ void fft_pass_mr_dispatch(int R, V* X, int ld, int logC, int L, int Ls, const V* tw) {
  switch (R) {
    case 5: fft_pass_mr<5, DIR>(X, ld, logC, L, Ls, tw); break;
    case 2: fft_pass_mr<2, DIR>(X, ld, logC, L, Ls, tw); break;
    case 4: fft_pass_mr<4, DIR>(X, ld, logC, L, Ls, tw); break;
    default:
      if constexpr (MAXLOG >= 4) {
        if (R == 16) { fft_pass_mr<16, DIR>(X, ld, logC, L, Ls, tw); break; }
      }
      fft_pass_mr<8, DIR>(X, ld, logC, L, Ls, tw);
      break;
  }
}

template <int MAXLOG, typename V>
__device__ __noinline__ void fft_forward_mr(V* X, int ld, int logC, int L, const V* tw) {
  const int np = fft_mr_npass(L, MAXLOG);
  int Ls = L;
  for (int i = 0; i < np; ++i) {
    const int R = fft_mr_radix(L, i, MAXLOG);
    fft_pass_mr_dispatch<-1, MAXLOG>(R, X, ld, logC, L, Ls, tw);
    Ls /= R;
    __syncthreads();
  }
}

template <int MAXLOG, typename V>
__device__ __noinline__ void fft_inverse_mr(V* X, int ld, int logC, int L, const V* tw) {
  const int np = fft_mr_npass(L, MAXLOG);
  int Ls = 1;
  for (int i = np - 1; i >= 0; --i) {
    const int R = fft_mr_radix(L, i, MAXLOG);
    Ls *= R;
    fft_pass_mr_dispatch<1, MAXLOG>(R, X, ld, logC, L, Ls, tw);
    __syncthreads();
  }
}

// Forward: natural order in, permuted (fft_pos(., ., MAXLOG)) order out; exp(-2 pi i n j / L).
// tw[m] = exp(-2 pi i m / L), m < L, must be visible to all threads. C = 2^logC columns.
template <int MAXLOG = 4, typename V>
__device__ void fft_forward(V* X, int ld, int logC, int L, const V* tw) {
  if (!fft_is_pow2(L)) {
    fft_forward_mr<MAXLOG>(X, ld, logC, L, tw);
    return;
  }
  const int logL = ilog2r(L);
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
  if (!fft_is_pow2(L)) {
    fft_inverse_mr<MAXLOG>(X, ld, logC, L, tw);
    return;
  }
  const int logL = ilog2r(L);
  const int np = fft_npass(L, MAXLOG);
  int logLs = 0;
  for (int i = np - 1; i >= 0; --i) {
    const int lr = fft_logradix(L, i, MAXLOG);
    logLs += lr;
    fft_pass_dispatch<1, MAXLOG>(lr, X, ld, logC, logL, logLs, tw);
    __syncthreads();
  }
}

// The runtime-shape transforms with the radix bound chosen at run time (maxlog 3: radix <= 8,
// otherwise radix <= 16); the position table of the same schedule is fft_perm_table(perm, L, maxlog).
template <typename V, typename TW>
__device__ __forceinline__ void fft_forward_ml(V* X, int ld, int logC, int L, const TW tw, int maxlog) {
  if (maxlog == 3) fft_forward<3>(X, ld, logC, L, tw);
  else fft_forward<4>(X, ld, logC, L, tw);
}
template <typename V, typename TW>
__device__ __forceinline__ void fft_inverse_ml(V* X, int ld, int logC, int L, const TW tw, int maxlog) {
  if (maxlog == 3) fft_inverse<3>(X, ld, logC, L, tw);
  else fft_inverse<4>(X, ld, logC, L, tw);
}

// ---- compile-time variant: L = 2^LOGL, C = 2^LOGC columns, pitch LD, all known to the
// compiler, so every shared-memory address is a base register plus an immediate and the
// twiddle indices need no masks. Same radix schedule (and output order) as above.
__host__ __device__ constexpr int ct_npass(int logL, int maxlog) { return (logL + maxlog - 1) / maxlog; }
__host__ __device__ constexpr int ct_logradix(int logL, int pass, int maxlog) {
  return logL / ct_npass(logL, maxlog) + (pass < logL % ct_npass(logL, maxlog) ? 1 : 0);
}

// NITEMS > 0 restricts the pass to its first NITEMS (group, column) items, i.e. to the leading
// rows NITEMS / C * R of the tile (whole blocks of sub-length 2^LOGLS).
template <int LR, int DIR, int LOGL, int LOGLS, int LOGC, int LD, int NITEMS = 0, typename V>
__device__ __forceinline__ void fft_pass_ct(V* X, const V* tw) {
  constexpr int R = 1 << LR, LOGS = LOGLS - LR, S = 1 << LOGS, C = 1 << LOGC;
  constexpr int ITEMS = NITEMS > 0 ? NITEMS : 1 << (LOGL - LR + LOGC);
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

// ---- transforms of odd sequences, x_{L-i} = -x_i (the odd extension behind the sine transform),
// compiled shapes, radix schedule MAXLOG = 4. The spectrum of an odd sequence is odd, Y_{L-j} = -Y_j,
// and the first forward pass (radix R = 2^LR0, stride S = L/R) sends frequency j to block j mod R
// (rows (j mod R) S .. + S - 1), so blocks q > R/2 are the negated mirrors of blocks R - q and are
// never formed: the tile holds ODD_ROWS = (R/2 + 1) S rows instead of L, and every pass after the
// first runs on those rows only.
//   odd_forward_pass0: rows 0..L/2 hold x_0..x_{L/2} (x_0 = x_{L/2} = 0) on entry; on exit blocks
//     0..R/2 hold what the full first pass writes there. Items pair n2 = t with S - t (t = 0 pairs
//     0 with S/2): between them they read exactly the rows they write, so the pass is in place.
//   odd_inverse_pass0: the inverse's last pass from blocks 0..R/2, using for q > R/2
//     z_q(n2) = -W_S^{n2} z_{R-q}(S - n2) (z_q the inverse sub-transforms of the blocks, W_S =
//     exp(-2 pi i / S)); writes x_n at rows n < L/2.
//   Where the pairs would leave threads of an NT-thread block idle (S C <= NT), each n2 is an item
//   of its own instead: one item per thread, all loads, a barrier, then the stores.
// Frequency j (j mod R <= R/2) sits at row fft_pos(j); odd_pos gives the row and sign of any j.
template <int LOGL> __host__ __device__ constexpr int odd_rows() {
  return ((1 << (ct_logradix(LOGL, 0, 4) - 1)) + 1) << (LOGL - ct_logradix(LOGL, 0, 4));
}

template <int LOGL, int LOGC, int LD, int NT, typename V>
__device__ __forceinline__ void odd_forward_pass0(V* X, const V* tw) {
  constexpr int LR = ct_logradix(LOGL, 0, 4), R = 1 << LR, H = R / 2, S = 1 << (LOGL - LR), C = 1 << LOGC;
  if constexpr ((S << LOGC) <= NT) {
    const int it = threadIdx.x, c = it & (C - 1), n2 = it >> LOGC;
    const bool act = it < (S << LOGC);
    V* col = X + c;
    V a[R];
    if (act) {
#pragma unroll
      for (int u = 0; u < H; ++u) a[u] = col[(n2 + S * u) * LD];
#pragma unroll
      for (int s = 1; s <= H; ++s) a[R - s] = cneg(col[(S * s - n2) * LD]);
    }
    __syncthreads();
    if (act) {
      dft_reg<R, -1>(a);
#pragma unroll
      for (int q = 0; q <= H; ++q) col[(n2 + S * q) * LD] = q ? cmul(a[q], tw[n2 * q]) : a[q];
    }
    return;
  }
  constexpr int ITEMS = (S / 2) << LOGC;
  for (int it = threadIdx.x; it < ITEMS; it += blockDim.x) {
    const int c = it & (C - 1), t = it >> LOGC;
    V* col = X + c;
    V a[R], b[R];
    int na, nb;
    if (t == 0) {
      na = 0;
      nb = S / 2;
      a[0] = czero<V>();
      a[H] = czero<V>();
#pragma unroll
      for (int u = 1; u < H; ++u) {
        const V v = col[(S * u) * LD];
        a[u] = v;
        a[R - u] = cneg(v);
      }
#pragma unroll
      for (int u = 0; u < H; ++u) {
        const V v = col[(S / 2 + S * u) * LD];
        b[u] = v;
        b[R - 1 - u] = cneg(v);
      }
    } else {
      na = t;
      nb = S - t;
#pragma unroll
      for (int u = 0; u < H; ++u) {
        const V d = col[(t + S * u) * LD];
        a[u] = d;
        b[R - 1 - u] = cneg(d);
      }
#pragma unroll
      for (int s = 1; s <= H; ++s) {
        const V e = col[(S * s - t) * LD];
        a[R - s] = cneg(e);
        b[s - 1] = e;
      }
    }
    dft_reg<R, -1>(a);
#pragma unroll
    for (int q = 0; q <= H; ++q) col[(na + S * q) * LD] = q ? cmul(a[q], tw[na * q]) : a[q];
    dft_reg<R, -1>(b);
#pragma unroll
    for (int q = 0; q <= H; ++q) col[(nb + S * q) * LD] = q ? cmul(b[q], tw[nb * q]) : b[q];
  }
}

template <int LOGL, int LOGC, int LD, int NT, typename V>
__device__ __forceinline__ void odd_inverse_pass0(V* X, const V* tw) {
  constexpr int LR = ct_logradix(LOGL, 0, 4), R = 1 << LR, H = R / 2, S = 1 << (LOGL - LR), C = 1 << LOGC;
  if constexpr ((S << LOGC) <= NT) {
    const int it = threadIdx.x, c = it & (C - 1), n2 = it >> LOGC, m2 = (S - n2) & (S - 1);
    const bool act = it < (S << LOGC);
    V* col = X + c;
    V z[H + 1], zm[H];
    if (act) {
#pragma unroll
      for (int q = 0; q <= H; ++q) z[q] = col[(S * q + n2) * LD];
#pragma unroll
      for (int q = 1; q < H; ++q) zm[q] = col[(S * q + m2) * LD];
    }
    __syncthreads();
    if (act) {
      V y[R];
      y[0] = z[0];
#pragma unroll
      for (int q = 1; q <= H; ++q) y[q] = cmulc(z[q], tw[n2 * q]);
#pragma unroll
      for (int q = 1; q < H; ++q) y[R - q] = cneg(cmul(zm[q], tw[n2 * q]));
      dft_reg<R, 1>(y);
#pragma unroll
      for (int r = 0; r < H; ++r) col[(n2 + S * r) * LD] = y[r];
    }
    return;
  }
  constexpr int ITEMS = (S / 2) << LOGC;
  for (int it = threadIdx.x; it < ITEMS; it += blockDim.x) {
    const int c = it & (C - 1), t = it >> LOGC;
    V* col = X + c;
    const int na = t == 0 ? 0 : t, nb = t == 0 ? S / 2 : S - t;
    V za[H + 1], zb[H + 1];
#pragma unroll
    for (int q = 0; q <= H; ++q) {
      za[q] = col[(S * q + na) * LD];
      zb[q] = col[(S * q + nb) * LD];
    }
    // n2 = na: its mirror S - na is na itself when t = 0, else nb
    {
      V y[R];
      y[0] = za[0];
#pragma unroll
      for (int q = 1; q <= H; ++q) y[q] = cmulc(za[q], tw[na * q]);
#pragma unroll
      for (int q = 1; q < H; ++q) y[R - q] = cneg(cmul(t == 0 ? za[q] : zb[q], tw[na * q]));
      dft_reg<R, 1>(y);
#pragma unroll
      for (int r = 0; r < H; ++r) col[(na + S * r) * LD] = y[r];
    }
    {
      V y[R];
      y[0] = zb[0];
#pragma unroll
      for (int q = 1; q <= H; ++q) y[q] = cmulc(zb[q], tw[nb * q]);
#pragma unroll
      for (int q = 1; q < H; ++q) y[R - q] = cneg(cmul(t == 0 ? zb[q] : za[q], tw[nb * q]));
      dft_reg<R, 1>(y);
#pragma unroll
      for (int r = 0; r < H; ++r) col[(nb + S * r) * LD] = y[r];
    }
  }
}

// forward passes P..NP-1 (inverse passes P..1) on the leading ROWS rows; __syncthreads after each
template <int P, int NP, int LOGL, int LOGLS, int LOGC, int LD, int ROWS, typename V>
__device__ __forceinline__ void odd_forward_rec(V* X, const V* tw) {
  if constexpr (P < NP) {
    constexpr int LR = ct_logradix(LOGL, P, 4);
    fft_pass_ct<LR, -1, LOGL, LOGLS, LOGC, LD, (ROWS >> LR) << LOGC>(X, tw);
    __syncthreads();
    odd_forward_rec<P + 1, NP, LOGL, LOGLS - LR, LOGC, LD, ROWS>(X, tw);
  }
}
template <int P, int LOGL, int LOGLS, int LOGC, int LD, int ROWS, typename V>
__device__ __forceinline__ void odd_inverse_rec(V* X, const V* tw) {
  if constexpr (P >= 1) {
    constexpr int LR = ct_logradix(LOGL, P, 4);
    fft_pass_ct<LR, 1, LOGL, LOGLS + LR, LOGC, LD, (ROWS >> LR) << LOGC>(X, tw);
    __syncthreads();
    odd_inverse_rec<P - 1, LOGL, LOGLS + LR, LOGC, LD, ROWS>(X, tw);
  }
}

// row of frequency j in the odd-sequence spectrum, with bit 15 set where the row holds -Y_j
template <int LOGL>
__device__ __forceinline__ int odd_pos(int j) {
  constexpr int R = 1 << ct_logradix(LOGL, 0, 4), L = 1 << LOGL;
  return (j & (R - 1)) > R / 2 ? (fft_pos(L - j, L) | 0x8000) : fft_pos(j, L);
}

// ct_freq maps a row of the permuted spectrum to its frequency (the inverse of fft_pos for the
// compiled shapes).
template <int LOGL, int MAXLOG = 4>
__device__ __forceinline__ int ct_freq(int pos) {
  constexpr int NP = ct_npass(LOGL, MAXLOG);
  int j = 0, shift = 0, logLs = LOGL;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    const int lr = ct_logradix(LOGL, i, MAXLOG);
    logLs -= lr;
    j += ((pos >> logLs) & ((1 << lr) - 1)) << shift;
    shift += lr;
  }
  return j;
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
