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

// v * exp(DIR * 2 pi i m / 16), DIR = -1 (forward) or +1
template <int DIR, typename V>
__device__ __forceinline__ V twid16(V v, int m) {
  using T = decltype(v.x);
  if (m == 0) return v;
  if (m == 4) return DIR < 0 ? mk(v.y, -v.x) : mk(-v.y, v.x);
  const T c = (T)cos16(m);
  const T s = (T)(DIR * sin16(m));
  return mk(v.x * c - v.y * s, v.x * s + v.y * c);
}

__host__ __device__ constexpr int ilog2c(int r) { return r <= 1 ? 0 : 1 + ilog2c(r >> 1); }
__host__ __device__ constexpr int brev(int i, int bits) {
  return bits == 0 ? 0 : ((i & 1) << (bits - 1)) | brev(i >> 1, bits - 1);
}

// One radix-2 decimation-in-time stage of butterfly span LEN over a register array;
// recursion on LEN keeps every index a compile-time constant (the array stays in registers).
template <int LEN, int R, int DIR, typename V>
__device__ __forceinline__ void dit_stage(V (&y)[R]) {
#pragma unroll
  for (int i = 0; i < R; i += LEN) {
#pragma unroll
    for (int j = 0; j < LEN / 2; ++j) {
      V u = y[i + j];
      V t = twid16<DIR>(y[i + j + LEN / 2], j * (16 / LEN));
      y[i + j] = cadd(u, t);
      y[i + j + LEN / 2] = csub(u, t);
    }
  }
  if constexpr (LEN < R) dit_stage<LEN * 2, R, DIR>(y);
}

// y_q = sum_r x_r exp(DIR 2 pi i r q / R), natural order in and out; R <= 16.
template <int R, int DIR, typename V>
__device__ __forceinline__ void dft_reg(V (&x)[R]) {
  constexpr int B = ilog2c(R);
  V y[R];
#pragma unroll
  for (int i = 0; i < R; ++i) y[brev(i, B)] = x[i];
  if constexpr (R > 1) dit_stage<2, R, DIR>(y);
#pragma unroll
  for (int i = 0; i < R; ++i) x[i] = y[i];
}

// Radix schedule: the remainder radix first, then 16s.
__host__ __device__ inline int fft_npass(int L) {
  int e = ilog2c(L);
  return e / 4 + ((e % 4) ? 1 : 0);
}
__host__ __device__ inline int fft_radix(int L, int pass) {
  int e = ilog2c(L);
  int rem = e % 4;
  if (rem && pass == 0) return 1 << rem;
  return 16;
}

// position of frequency j in the output of the forward transform
__host__ __device__ inline int fft_pos(int j, int L) {
  int np = fft_npass(L);
  int p = 0, Ls = L;
  for (int i = 0; i < np; ++i) {
    int R = fft_radix(L, i);
    int q = j % R;
    j /= R;
    Ls /= R;
    p += q * Ls;
  }
  return p;
}

// One pass of radix R at sub-length Ls. DIR < 0: forward (gather natural stride,
// DFT, twiddle, scatter). DIR > 0: its conjugate transpose.
template <int R, int DIR, typename V>
__device__ __forceinline__ void fft_pass(V* X, int ld, int C, int L, int Ls, const V* tw) {
  const int S = Ls / R;
  const int items = (L / R) * C;
  const int tstep = L / Ls;  // W_Ls^e = W_L^{e * tstep}
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int c = it % C;
    const int g = it / C;
    const int b = g / S;
    const int n2 = g - b * S;
    const int base = b * Ls + n2;
    V x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = X[(base + r * S) * ld + c];
    if (DIR < 0) {
      dft_reg<R, -1>(x);
#pragma unroll
      for (int q = 1; q < R; ++q) x[q] = cmul(x[q], tw[(n2 * q * tstep) & (L - 1)]);
    } else {
#pragma unroll
      for (int q = 1; q < R; ++q) x[q] = cmulc(x[q], tw[(n2 * q * tstep) & (L - 1)]);
      dft_reg<R, 1>(x);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) X[(base + r * S) * ld + c] = x[r];
  }
}

template <int DIR, typename V>
__device__ __forceinline__ void fft_pass_dispatch(int R, V* X, int ld, int C, int L, int Ls, const V* tw) {
  switch (R) {
    case 2: fft_pass<2, DIR>(X, ld, C, L, Ls, tw); break;
    case 4: fft_pass<4, DIR>(X, ld, C, L, Ls, tw); break;
    case 8: fft_pass<8, DIR>(X, ld, C, L, Ls, tw); break;
    default: fft_pass<16, DIR>(X, ld, C, L, Ls, tw); break;
  }
}

// Forward: natural order in, permuted (fft_pos) order out; exp(-2 pi i n j / L).
// tw[m] = exp(-2 pi i m / L), m < L, must be visible to all threads.
template <typename V>
__device__ void fft_forward(V* X, int ld, int C, int L, const V* tw) {
  const int np = fft_npass(L);
  int Ls = L;
  for (int i = 0; i < np; ++i) {
    const int R = fft_radix(L, i);
    fft_pass_dispatch<-1>(R, X, ld, C, L, Ls, tw);
    Ls /= R;
    __syncthreads();
  }
}

// Inverse: permuted order in, natural order out, unnormalised: x_n = sum_j X_j exp(+2 pi i n j / L).
template <typename V>
__device__ void fft_inverse(V* X, int ld, int C, int L, const V* tw) {
  const int np = fft_npass(L);
  int Ls = 1;
  for (int i = np - 1; i >= 0; --i) {
    const int R = fft_radix(L, i);
    Ls *= R;
    fft_pass_dispatch<1>(R, X, ld, C, L, Ls, tw);
    __syncthreads();
  }
}

}  // namespace pint
