// Spatial part of the sweep (Algorithm 1/2, step 2): the N/2+1 shifted systems
// (sigma_j + A_h) q_j = h_j, sigma_j = g_j tau^-alpha, with A_h the finite-difference
// Dirichlet Laplacian. A_h is diagonalised exactly by the discrete sine transform
// DST-I, D_{pi} = sin(pi p i / (n+1)), with eigenvalues (4/h^2) sin^2(p pi h / 2).
//
// A sine transform of a (complex) line x_1..x_n is taken through its odd extension of
// length L = 2(n+1): the forward FFT of [0, x, 0, -reverse(x)] is -2i D x at frequencies
// 1..n and keeps the odd symmetry. Dividing that spectrum by a symmetric factor keeps it
// odd, and the inverse FFT of an odd spectrum Z is 2i D Z. So a shifted solve along one
// axis is: odd-extend, forward FFT, divide, inverse FFT -- in place, in shared memory,
// with no permutation (the inverse consumes the forward transform's permuted order).
//
// Line layouts: mode 0 -- lines are contiguous rows of n elements (x direction, or the
// whole 1D grid); mode 1 -- lines run across rows with stride P (y direction in 2D),
// consecutive lines are consecutive x-modes so loads stay coalesced.
#include "fft.cuh"
#include "pint_internal.h"

namespace pint {

template <typename T> size_t axis_smem(int n, int C) {
  const size_t L = 2 * (size_t)(n + 1);
  return sizeof(typename c2<T>::t) * (L * (C + 1) + L);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_axis(AxisArgs<T> a) {
  using V = typename c2<T>::t;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n = a.n, C = a.C, ld = a.ld, L = 2 * (a.n + 1);
  V* X = reinterpret_cast<V*>(smraw);
  V* tw = X + (size_t)L * ld;
  const V* gtw = reinterpret_cast<const V*>(a.tw);
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = gtw[i];
  V* S = reinterpret_cast<V*>(a.S);
  const int line0 = blockIdx.x * C;
  const T zero = T(0);

  // ---- load with odd extension ----
  if (a.mode == 0) {
    for (int it = threadIdx.x; it < n * C; it += blockDim.x) {
      const int cc = it / n, i = it - cc * n;
      const int line = line0 + cc;
      V v = mk(zero, zero);
      if (line < a.lines) v = S[(size_t)line * n + i];
      X[(size_t)(i + 1) * ld + cc] = v;
      X[(size_t)(L - 1 - i) * ld + cc] = mk(-v.x, -v.y);
    }
  } else {
    for (int it = threadIdx.x; it < n * C; it += blockDim.x) {
      const int cc = it % C, i = it / C;
      const int line = line0 + cc;
      V v = mk(zero, zero);
      if (line < a.lines) {
        const int j = line / a.P, p = line - j * a.P;
        v = S[((size_t)j * n + i) * a.P + p];
      }
      X[(size_t)(i + 1) * ld + cc] = v;
      X[(size_t)(L - 1 - i) * ld + cc] = mk(-v.x, -v.y);
    }
  }
  for (int cc = threadIdx.x; cc < C; cc += blockDim.x) {
    X[cc] = mk(zero, zero);
    X[(size_t)(n + 1) * ld + cc] = mk(zero, zero);
  }
  __syncthreads();
  fft_forward(X, ld, C, L, tw);

  if (a.op == 0) {
    // D-transform only: -2i D x at frequencies 1..n, stored in natural order
    if (a.mode == 0) {
      for (int it = threadIdx.x; it < n * C; it += blockDim.x) {
        const int cc = it / n, i = it - cc * n;
        const int line = line0 + cc;
        if (line < a.lines) S[(size_t)line * n + i] = X[(size_t)fft_pos(i + 1, L) * ld + cc];
      }
    } else {
      for (int it = threadIdx.x; it < n * C; it += blockDim.x) {
        const int cc = it % C, i = it / C;
        const int line = line0 + cc;
        if (line < a.lines) {
          const int j = line / a.P, p = line - j * a.P;
          S[((size_t)j * n + i) * a.P + p] = X[(size_t)fft_pos(i + 1, L) * ld + cc];
        }
      }
    }
    return;
  }

  // ---- divide by scale * (sigma_j + lambda_other + lambda_p) at frequencies p and L-p ----
  const V* sigma = reinterpret_cast<const V*>(a.sigma);
  for (int it = threadIdx.x; it < L * C; it += blockDim.x) {
    const int cc = it % C, fq = it / C;
    const int line = line0 + cc;
    const int p = fq <= n + 1 ? fq : L - fq;
    const size_t pos = (size_t)fft_pos(fq, L) * ld + cc;
    if (p == 0 || p == n + 1 || line >= a.lines) {
      X[pos] = mk(zero, zero);
      continue;
    }
    int j, po = 0;
    if (a.mode == 0) {
      j = line / a.lines_per_j;
    } else {
      j = line / a.P;
      po = line - j * a.P;
    }
    V d = sigma[j];
    d.x += a.lam_axis[p - 1];
    if (a.lam_other) d.x += a.lam_other[po];
    d.x *= a.scale;
    d.y *= a.scale;
    const T inv = T(1) / (d.x * d.x + d.y * d.y);
    X[pos] = cmulc(X[pos], mk(d.x * inv, d.y * inv));   // X / d = X conj(d) / |d|^2
  }
  __syncthreads();
  fft_inverse(X, ld, C, L, tw);

  if (a.mode == 0) {
    for (int it = threadIdx.x; it < n * C; it += blockDim.x) {
      const int cc = it / n, i = it - cc * n;
      const int line = line0 + cc;
      if (line < a.lines) S[(size_t)line * n + i] = X[(size_t)(i + 1) * ld + cc];
    }
  } else {
    for (int it = threadIdx.x; it < n * C; it += blockDim.x) {
      const int cc = it % C, i = it / C;
      const int line = line0 + cc;
      if (line < a.lines) {
        const int j = line / a.P, p = line - j * a.P;
        S[((size_t)j * n + i) * a.P + p] = X[(size_t)(i + 1) * ld + cc];
      }
    }
  }
}

template <typename T> cudaError_t launch_axis(const AxisArgs<T>& a, cudaStream_t st) {
  const size_t sm = axis_smem<T>(a.n, a.C);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_axis<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  const int blocks = (a.lines + a.C - 1) / a.C;
  const char* name = a.op == 0 ? (sizeof(T) == 8 ? "dst_f64" : "dst_f32")
                               : (sizeof(T) == 8 ? "axis_solve_f64" : "axis_solve_f32");
  prof_begin(name, st);
  k_axis<T><<<blocks, kThreads, sm, st>>>(a);
  prof_end(st);
  return cudaGetLastError();
}

template size_t axis_smem<float>(int, int);
template size_t axis_smem<double>(int, int);
template cudaError_t launch_axis<float>(const AxisArgs<float>&, cudaStream_t);
template cudaError_t launch_axis<double>(const AxisArgs<double>&, cudaStream_t);

}  // namespace pint
