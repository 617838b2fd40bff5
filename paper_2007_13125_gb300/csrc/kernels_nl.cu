// Kernels of the semilinear extension (Sec. 4.3, Algorithm 3): D_t^alpha u + A u + g(u) = f with
// a cubic g(u) = c_0 + c_1 u + c_2 u^2 + c_3 u^3, in all-at-once form K U + w g(U) = F_hat (w the
// reaction weight of a row: 1 for finite differences, h for P1 elements with nodal quadrature).
//
// One outer step of Algorithm 3 linearises at the time average of the current iterate,
//   Ubar = (1/N) sum_n U^n,  D = g'(Ubar),
// and solves (K + I (x) w D) W = F_hat - K U - w g(U) by WR from W_0 = 0. With V = U + W that is
// the linear problem (K + I (x) w D) V = F_hat - w g(U) + w D U started from V_0 = U, which the
// plan's WR solve handles once w D is installed as its reaction term. These kernels form Ubar
// and w D, the right-hand side of that problem, and the norms of the outer update; all FP64.
#include "pint_internal.h"

namespace pint {

__device__ __forceinline__ double poly_g(const NlPoly& g, double u) {
  return fma(fma(fma(g.c[3], u, g.c[2]), u, g.c[1]), u, g.c[0]);
}
__device__ __forceinline__ double poly_dg(const NlPoly& g, double u) {
  return fma(fma(3.0 * g.c[3], u, 2.0 * g.c[2]), u, g.c[1]);
}

// r_i = w g'(Ubar_i). A CTA owns 32 points; its 8 warps sum interleaved levels of them and the
// partial sums are added in a fixed order (deterministic).
__global__ void __launch_bounds__(256) k_nl_linearise(const double* __restrict__ U, int N, int M, NlPoly g,
                                                      double w, double* __restrict__ r) {
  __shared__ double part[8][33];
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (i < M) {
#pragma unroll 4
    for (int n = grp; n < N; n += 8) s += U[(size_t)n * M + i];
  }
  part[grp][lane] = s;
  __syncthreads();
  if (grp == 0 && i < M) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += part[q][lane];
    r[i] = w * poly_dg(g, t / N);
  }
}

// Fout = F - w g(U) + r U (r = w D), U0 = U; grid (points, levels)
__global__ void __launch_bounds__(256) k_nl_rhs(const double* __restrict__ F, const double* __restrict__ U,
                                                const double* __restrict__ r, NlPoly g, double w, int M,
                                                double* __restrict__ Fout, double* __restrict__ U0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const size_t idx = (size_t)blockIdx.y * M + i;
  const double u = U[idx];
  Fout[idx] = fma(r[i], u, F[idx] - w * poly_g(g, u));
  U0[idx] = u;
}

// norms[0] += sum (U - U0)^2, norms[1] += sum U^2
__global__ void __launch_bounds__(256) k_nl_norms(const double* __restrict__ U, const double* __restrict__ U0,
                                                  size_t NM, double* norms) {
  __shared__ double red[2][8];
  double a = 0.0, b = 0.0;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < NM; idx += (size_t)gridDim.x * blockDim.x) {
    const double u = U[idx], d = u - U0[idx];
    a = fma(d, d, a);
    b = fma(u, u, b);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  if (lane == 0) { red[0][wq] = a; red[1][wq] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { sa += red[0][q]; sb += red[1][q]; }
    atomicAdd(norms, sa);
    atomicAdd(norms + 1, sb);
  }
}

// The derivative rows of the source with the lower-order terms moved into row 0: out = fd with
// f(0) replaced by f(0) - w g(v) - r v (r = w c a reaction coefficient, or null), so that the
// a_n term of the corrected source reads a_n (f(0) - A v - w c v - w g(v)).
__global__ void __launch_bounds__(256) k_nl_fd0(const double* __restrict__ fd, const double* __restrict__ v,
                                                NlPoly g, double w, const double* __restrict__ r, int M,
                                                double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const size_t idx = (size_t)blockIdx.y * M + i;
  double x = fd[idx];
  if (blockIdx.y == 0) {
    x -= w * poly_g(g, v[i]);
    if (r) x -= r[i] * v[i];
  }
  out[idx] = x;
}

// Right-hand side of a time window after the first (BDF-k, alpha = 1): level n (0-based) of
// F = f minus the BDF terms reaching into the previous window Up [Np][M]:
//   F_n = f_n - sum_{j=n+1}^{k} c_j (M Up)_{Np + n - j},   c_j = omega_j / tau,
// with M the identity, or the P1 mass matrix (h/6)[1 4 1] (fem). Grid (points, levels).
__global__ void __launch_bounds__(256) k_window_rhs(const double* __restrict__ f, const double* __restrict__ Up,
                                                    double* __restrict__ F, int Np, int M, int k, WinCoef c, int fem,
                                                    double m6) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int n = blockIdx.y;
  double x = f[(size_t)n * M + i];
  for (int j = n + 1; j <= k; ++j) {
    const double* row = Up + (size_t)(Np + n - j) * M;
    double u = row[i];
    if (fem) u = m6 * (4.0 * u + (i > 0 ? row[i - 1] : 0.0) + (i + 1 < M ? row[i + 1] : 0.0));
    x -= c.c[j] * u;
  }
  F[(size_t)n * M + i] = x;
}

// out = w c
__global__ void __launch_bounds__(256) k_scale(const double* __restrict__ c, double w, int M, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) out[i] = w * c[i];
}

cudaError_t launch_nl_linearise(const double* U, int N, int M, const NlPoly& g, double w, double* r,
                                cudaStream_t st) {
  prof_begin("nl_linearise", st);
  k_nl_linearise<<<(M + 31) / 32, 256, 0, st>>>(U, N, M, g, w, r);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_nl_rhs(const double* F, const double* U, const double* r, const NlPoly& g, double w, int N,
                          int M, double* Fout, double* U0, cudaStream_t st) {
  prof_begin("nl_rhs", st);
  k_nl_rhs<<<dim3((M + 255) / 256, N), 256, 0, st>>>(F, U, r, g, w, M, Fout, U0);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_nl_norms(const double* U, const double* U0, size_t NM, double* norms, cudaStream_t st) {
  const size_t want = (NM + 255) / 256;
  const int blocks = (int)(want < 4 * 152 ? (want > 0 ? want : 1) : 4 * 152);
  prof_begin("nl_norms", st);
  k_nl_norms<<<blocks, 256, 0, st>>>(U, U0, NM, norms);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_nl_fd0(const double* fd, const double* v, const NlPoly& g, double w, const double* r, int rows,
                          int M, double* out, cudaStream_t st) {
  k_nl_fd0<<<dim3((M + 255) / 256, rows), 256, 0, st>>>(fd, v, g, w, r, M, out);
  return cudaGetLastError();
}

cudaError_t launch_window_rhs(const double* f, const double* Up, double* F, int N, int Np, int M, int k,
                              const WinCoef& c, int fem, double m6, cudaStream_t st) {
  prof_begin("window_rhs", st);
  k_window_rhs<<<dim3((M + 255) / 256, N), 256, 0, st>>>(f, Up, F, Np, M, k, c, fem, m6);
  prof_end(st);
  return cudaGetLastError();
}

cudaError_t launch_scale(const double* c, double w, int M, double* out, cudaStream_t st) {
  k_scale<<<(M + 255) / 256, 256, 0, st>>>(c, w, M, out);
  return cudaGetLastError();
}

}  // namespace pint
