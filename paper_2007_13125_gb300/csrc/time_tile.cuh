// Shared pieces of the time-axis kernels (kernels_time.cu, kernels_resid.cu): the time tile
// (one CTA owns 2C spatial points and all N levels; point m0 + c is the real part and m0 + C + c
// the imaginary part of complex column c), its shared-memory carve-up, the separation of the two
// packed half spectra, block reductions and launch helpers.
#pragma once
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

// out[0] += sum of a, out[1] += sum of b over the block. The float version adds in FP32 within
// the block and converts once per block (FP64 instructions run at ~1/70 of the FP32 rate here);
// it serves the stopping test's norms, where a relative error of 1e-5 is immaterial.
__device__ __forceinline__ void block_reduce_add2f(float a, float b, double* out) {
  __shared__ float redf[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { redf[0][w] = a; redf[1][w] = b; }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    a = l < nw ? redf[0][l] : 0.f;
    b = l < nw ? redf[1][l] : 0.f;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (l == 0) {
      atomicAdd(out, (double)a);
      atomicAdd(out + 1, (double)b);
    }
  }
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

// (maxlog: the radix bound of the transform the tile will use, for its position table)
template <typename V>
__device__ __forceinline__ void time_tile_setup(unsigned char* raw, int N, int C, const V* gtw, V*& X,
                                                V*& tw, unsigned short*& perm, int maxlog = 4) {
  X = reinterpret_cast<V*>(raw);
  tw = X + (size_t)N * C;
  perm = reinterpret_cast<unsigned short*>(tw + N);
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = gtw[i];
  fft_perm_table(perm, N, maxlog);
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
    const V Zn = X[(size_t)perm[j == 0 ? 0 : N - j] * C + cc];
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


template <typename K> inline cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

inline int tiles(int M, int C) { return (M + 2 * C - 1) / (2 * C); }

}  // namespace pint
