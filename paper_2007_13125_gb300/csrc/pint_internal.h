// Internal declarations shared by the kernel translation units and the host plan code.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <string>

namespace pint {

constexpr int kThreads = 256;   // threads per CTA of every tile kernel
constexpr int kMaxK = 6;

// ---- time-axis kernels (kernels_time.cu) ----

// MIXED: r = F_hat - K U in double-float, times kappa^{i/N}, real -> half-complex DFT.
// Time-tile shapes (N, tile width) with a compiled time FFT: the residual kernels' and the update
// kernel's (the launchers pick those instances; every other shape runs the runtime-shape transform).
__host__ __device__ inline bool compiled_time_fft_shape(int N, int C) {
  return (N == 128 && C == 16) || (N == 256 && C == 16) || (N == 512 && C == 16) || (N == 1024 && C == 8);
}
__host__ __device__ inline bool compiled_update_shape(int N, int C) {
  return compiled_time_fft_shape(N, C) || (N == 2048 && C == 4) || (N == 4096 && C == 2);
}

struct ResidFwdArgs {
  const float2* U;                         // iterate U [N][M] (double-float pairs: hi, lo)
  const double* F;                         // F_hat [N][M] (FP64, split to double-float on load), or f
  const double* Fh;                        // with f: F_hat on levels < kc ([kc][M]; beyond them
  int kc;                                  // F_hat = f exactly: BDF-k), else null
  const float* yhi; const float* ylo;      // CQ: tau^-alpha (L_omega U) [N][M] double-float, else null
  float2* S;                               // half spectrum [(N/2+1)][M]
  const float* s;                          // kappa^{i/N}, i < N
  const float2* tw;                        // exp(-2 pi i m / N), m < N
  int N, M, mx, dim, k, C, logC;
  float c_hi[kMaxK + 1], c_lo[kMaxK + 1];  // c_0 (FD: incl. stencil centre), c_j = omega_j tau^-alpha
  float gx_hi, gx_lo, gy_hi, gy_lo;        // off-diagonal Laplacian weights: 1/h^2 (FD), 1/h (P1)
  float gz_hi, gz_lo;                      // 3D: 1/hz^2
  int my;                                  // points along y (3D: the z neighbours are mx * my apart)
  int fem;                                 // P1 FEM (1D): time terms act on M_h U, centre 2/h
  float m_hi, m_lo;                        // P1 FEM: h/6 (mass matrix off-diagonal)
  int periodic;                            // periodic boundary conditions: neighbours wrap around
  int g_pow2;                              // gx, gy, gz all powers of two (their products are exact)
  int maxlog;                              // runtime-shape time FFT: radix <= 2^maxlog (3 or 4; 0: 4)
  const double* react;                     // 1D: [M] weighted reaction coefficient w c_i; the
                                           // residual loses w c_i U_i^n (null: no reaction term)
  // first sweep from U_0^n = v (k_resid_v0): r_0^n = F_hat_n - beta_n M v - A v
  const double* v;                         // [M] (FP64)
  const float2* beta_ff;                   // [N] tau^-alpha sum_{j<n} omega_j, n = 1..N (double-float)
};

// MIXED: inverse DFT, times 1/(N kappa^{i/N}), U += c (double-float), norms.
struct InvUpdArgs {
  const float2* S; float2* U;             // U [N][M] double-float pairs (hi, lo)
  const float* inv_s; const float2* tw;
  int N, M, C, logC;
  double* norms;                           // [0] += sum c^2, [1] += sum U^2
  int ring;                                // levels in the U staging ring (set by the launcher)
  int maxlog;                              // runtime-shape time FFT: radix <= 2^maxlog (3 or 4; 0: 4)
  const double* v;                         // first sweep from U_0^n = v: U = v + c ([M]), else null
};

// FP64 / FP32: F_{m-1} = F_hat + (P - K) U_{m-1}, times kappa^{i/N}, DFT.
template <typename T> struct DirectFwdArgs {
  const T* F; const T* U;                  // F_hat, U_{m-1} [N][M]
  const double* z;                         // CQ: kappa tau^-alpha (W' U) [N][M], else null
  void* S;                                 // half spectrum of T2
  const T* s; const void* tw;
  int N, M, C, logC, k;
  T kw[kMaxK + 1];                         // kappa tau^-alpha omega_j (BDF corner)
  int fem;                                 // P1 elements (1D): the kappa terms act through M_h
  T h6;                                    // h / 6 (M_h = (h/6) tridiag(1, 4, 1))
};

template <typename T> struct DirectInvArgs {
  const void* S; const T* Uold; T* Uout;
  const T* inv_s; const void* tw;
  int N, M, C, logC;
  double* norms;                           // [0] += sum (Unew-Uold)^2, [1] += sum Unew^2
};

// CQ Toeplitz product z = omega * U (linear convolution along time, 2N-point FFTs).
struct ToepArgs {
  const double* Ud; const float2* Uff; const float* Uf;
  int ukind;                               // 0 double, 1 double-float, 2 float
  double* out;                             // [N][M]
  const double2* what;                     // FFT_{2N}(omega, zero padded), permuted, pre-scaled
  const double2* tw;                       // exp(-2 pi i m / 2N)
  int N, M, C, logC, half;                 // half 0: z_0..z_{N-1}; 1: z_N..z_{2N-1}
};

// MIXED CQ: the same product in double-float arithmetic on the FP32 pipes.
struct ToepFFArgs {
  const float2* U;                         // U [N][M] (double-float pairs)
  float* yhi; float* ylo;                  // tau^-alpha (L_omega U) [N][M] (double-float)
  const void* what;                        // ffc [2N]: FFT_{2N}(omega), radix-8 permuted order, * tau^-alpha / 2N
  const void* tw;                          // ffc [2N]: exp(-2 pi i m / 2N)
  int N, M, C, logC;
};

// right-hand side F_hat (FP64)
struct RhsArgs {
  const double* v; const double* f; const double* fd; double* F;
  const double* beta;                      // tau^-alpha sum_{j<n} omega_j, n = 1..N
  int N, M, mx, dim, k;
  double gx, gy, gz;
  int my;                                  // 3D: z neighbours are mx * my apart
  double a[kMaxK];                         // a_n, n = 1..k-1
  double bt[kMaxK][kMaxK];                 // b_{l,n} tau^l
  int fem;                                 // P1 FEM: A v -> K_h v, v -> M_h v in the beta term
  double mass6;                            // h/6
  int periodic;                            // periodic boundary conditions: neighbours wrap around
  int head;                                // the first N levels of a longer F_hat only (profiling label)
};

// ---- spatial kernels (kernels_space.cu) ----
// Sine transform / shifted solve along one axis of the half spectrum.
template <typename T> struct AxisArgs {
  void* S;                                 // T2 spectrum
  int n;                                   // points along the axis (interior)
  int lines;                               // number of lines
  int mode;                                // 0: lines contiguous (stride 1); 1: stride P
  int P;                                   // mode 1: lines per j-slice (= mx), stride
  int op;                                  // 0: transform only; 1: transform, divide, transform
  const void* sigma;                       // T2 [N/2+1] (op 1)
  const T* lam_axis;                       // [n] eigenvalues along this axis (op 1)
  const T* lam_other;                      // mode 1: [P] eigenvalues of the other axis
  const T* mu_axis;                        // P1 FEM: [n] mass eigenvalues along this axis (divisor
                                           // sigma_j mu_p + lam_p), else null
  T scale;                                 // op 1 divisor scale
  int lines_per_j;                         // op 1: j = line / lines_per_j
  const void* tw;                          // exp(-2 pi i m / L), L = 2(n+1)
  int C, logC, ld;
};

// Sine transform along x of lines of 255 points as tensor-core products (kernels_dst_tc.cu): the
// output of AxisArgs op 0 (Y_k = -2i sum_x X_x sin(pi k x / 256)), in place on `lines`
// consecutive lines of 255 complex values.
struct DstTcArgs {
  float2* S;                               // the lines (in place)
  const void* tab;                         // matrix image, dst_tc_table_bytes(n) (16-byte aligned)
  int n;                                   // points per line: 255 or 127 (dst_tc_line_ok)
  int lines;
  // 1: lines stored one after another ([lines][n]); > 1 (n = 127 only): point i of line
  // l = q * stride + x at S[(q * n + i) * stride + x], i.e. planes of n rows of `stride` points, a
  // line per column (lines = planes * stride)
  int stride;
  int* err;                                // set to 1 if a bounded wait of the kernel gave up
  // strided lines with sigma set: the solve of AxisArgs op 1 instead of the transform -- forward
  // transform, divide line (q, x) at frequency k by scale (sigma[q] + lam_other[x] +
  // lam_axis[k - 1]), transform back (+2i)
  const float2* sigma;
  const float* lam_other;
  const float* lam_axis;
  float scale;
};
inline bool dst_tc_line_ok(int n) { return n == 255 || n == 127; }
size_t dst_tc_table_bytes(int n);
void dst_tc_table(int n, unsigned short* img);  // host: fills the image (dst_tc_table_bytes(n) / 2 halves)
cudaError_t launch_dst_tc(const DstTcArgs& a, cudaStream_t st);

// Toeplitz tridiagonal solve along y (2D, after the x sine transform): for each line (j, p),
// (s_j + lambda_p^x + 2 g) q_y - g (q_{y-1} + q_{y+1}) = b_y, g = 1/h_y^2, through the
// factorisation T = (g/r)(I - r Z)(I - r Z^T) + g r e_0 e_0^T, r + 1/r = d/g, |r| < 1.
struct TriArgs {
  float2* S;                               // spectrum [(N/2+1)][my][mx] (in place)
  int n;                                   // my
  int P;                                   // mx (lines per j-slice)
  int lines;                               // (N/2+1) * mx
  const float2* sigma;                     // [N/2+1]
  const float* lam_x;                      // [mx]
  float g;                                 // 1/h_y^2
  float scale;                             // result multiplied by this (folds DST-x normalisation)
  int C, logC;
};

// 1D shifted systems with a space-varying reaction term (the linearised operator of Algorithm 3,
// Sec. 4.3): for each frequency j the tridiagonal system
//   (sigma_j m_d + k_d + r_i) q_i + (sigma_j m_o + k_o) (q_{i-1} + q_{i+1}) = b_i,  i = 0..n-1,
// with (m_d, m_o) the mass row ((1, 0) for finite differences, (4h/6, h/6) for P1 elements),
// (k_d, k_o) the stiffness row and r = w c the weighted reaction coefficient. The factor kernel
// computes the LU factors (in FP64, stored in T) once per reaction coefficient; the solve kernel runs the two
// substitutions in T on the half spectrum in place. Factors are stored [J][n] (a frequency's
// factors contiguous).
template <typename T> struct TriVarArgs {
  void* S;                                 // T2 spectrum [J][n] (in place; solve only)
  void* ip;                                // T2 [J][n]: 1 / pivot_i
  void* cp;                                // T2 [J][n]: (sigma_j m_o + k_o) / pivot_i
  const void* sigma;                       // T2 [J]: g_j tau^-alpha
  const double* r;                         // [n]: w c_i (factor only)
  int n, J;
  double md, mo, kd, ko;
};

size_t resid_fwd_smem(int N, int C);
size_t inv_upd_smem(int N, int C);
template <typename T> size_t direct_smem(int N, int C);
size_t toep_smem(int N, int C);
template <typename T> size_t axis_smem(int n, int C, bool has_mu, int rows);

cudaError_t launch_resid_fwd(const ResidFwdArgs& a, cudaStream_t st);
// first sweep from U_0^n = v (a.v, a.beta set): no U read, no history
cudaError_t launch_resid_v0(const ResidFwdArgs& a, cudaStream_t st);
cudaError_t launch_inv_upd(const InvUpdArgs& a, cudaStream_t st);
template <typename T> cudaError_t launch_direct_fwd(const DirectFwdArgs<T>& a, cudaStream_t st);
template <typename T> cudaError_t launch_direct_inv(const DirectInvArgs<T>& a, cudaStream_t st);
cudaError_t launch_toeplitz(const ToepArgs& a, cudaStream_t st);
cudaError_t launch_toeplitz_ff(const ToepFFArgs& a, cudaStream_t st);
size_t toep_ff_smem(int N, int C);
constexpr int kToepFFMaxLog = 3;           // radix <= 8 for the double-float FFT (register budget)
cudaError_t launch_rhs(const RhsArgs& a, cudaStream_t st);
template <typename T> cudaError_t launch_axis(const AxisArgs<T>& a, cudaStream_t st);
// periodic lines (complex FFT of n points): op 0 forward, 1 shifted solve, 2 inverse
template <typename T> cudaError_t launch_axis_per(const AxisArgs<T>& a, cudaStream_t st);
cudaError_t launch_tri(const TriArgs& a, cudaStream_t st);
// the same systems by parallel cyclic reduction (n <= 1024 rows)
cudaError_t launch_pcr(const TriArgs& a, cudaStream_t st);
template <typename T> cudaError_t launch_trivar_factor(const TriVarArgs<T>& a, cudaStream_t st);
template <typename T> cudaError_t launch_trivar_solve(const TriVarArgs<T>& a, cudaStream_t st);
size_t tri_smem(int n, int C);

// conversions
cudaError_t launch_d2ff(const double* x, float2* y, size_t n, cudaStream_t st);
cudaError_t launch_ff2d(const float2* y, double* x, size_t n, cudaStream_t st);
cudaError_t launch_d2f(const double* x, float* y, size_t n, cudaStream_t st);
cudaError_t launch_f2d(const float* x, double* y, size_t n, cudaStream_t st);
cudaError_t launch_bcast_d(const double* v, double* U, int N, int M, cudaStream_t st);
cudaError_t launch_bcast_d2ff(const double* v, float2* U, int N, int M, cudaStream_t st);

// ---- semilinear extension (kernels_nl.cu) ----
struct NlPoly { double c[4]; };          // g(u) = c[0] + c[1] u + c[2] u^2 + c[3] u^3
// r_i = w g'(Ubar_i), Ubar the time average of U [N][M]
cudaError_t launch_nl_linearise(const double* U, int N, int M, const NlPoly& g, double w, double* r,
                                cudaStream_t st);
// Fout = F - w g(U) + r U, U0 = U ([N][M])
cudaError_t launch_nl_rhs(const double* F, const double* U, const double* r, const NlPoly& g, double w, int N,
                          int M, double* Fout, double* U0, cudaStream_t st);
// norms[0] += ||U - U0||^2, norms[1] += ||U||^2
cudaError_t launch_nl_norms(const double* U, const double* U0, size_t NM, double* norms, cudaStream_t st);
// out [rows][M] = fd with row 0 minus w g(v) and minus r v (r: [M] or null)
cudaError_t launch_nl_fd0(const double* fd, const double* v, const NlPoly& g, double w, const double* r, int rows,
                          int M, double* out, cudaStream_t st);
// out = w c ([M])
cudaError_t launch_scale(const double* c, double w, int M, double* out, cudaStream_t st);
// time windows (BDF-k): F = f minus the BDF terms on the previous window's levels Up [Np][M]
struct WinCoef { double c[kMaxK + 1]; };  // omega_j / tau
cudaError_t launch_window_rhs(const double* f, const double* Up, double* F, int N, int Np, int M, int k,
                              const WinCoef& c, int fem, double m6, cudaStream_t st);

// ---- convergence control (shared by the host loop and the graph's device-side check) ----
struct SolveCtl {
  double tol, q_floor, prev, upd;
  int max_sweeps, m, done;
  int err;  // nonzero: a bounded device-side wait gave up; the solve stops and reports PINT_ECUDA
};

// Whole MIXED solve of a small 1D problem in one CTA (kernels_small.cu): finite differences,
// Dirichlet, BDF-k, no reaction term; tables as for the multi-kernel sweep (float).
constexpr int kSmallThreads = 512;
struct SmallArgs {
  const double* F;        // F_hat [N][M]
  double* U;              // in: the guess (when v is null); out: the solution
  const double* v;        // non-null: start from U_0^n = v
  const float2* tw_t;     // [N] time twiddles
  const float* s;         // [N] kappa^{n/N}
  const float* inv_s;     // [N] kappa^{-n/N} / N
  const float2* sigma;    // [N/2+1] g_j tau^-alpha
  const float* lam;       // [M] eigenvalues of the stencil on the sine modes
  const float2* tw_x;     // [L] twiddles of the odd extension, L = 2(M+1)
  float c_hi[kMaxK + 1], c_lo[kMaxK + 1];  // c_0 = omega_0 / tau + 2/h^2, c_j = omega_j / tau
  float gx;               // 1/h^2 (a power of two)
  int k, N, M, Ct, logCt, L, Cs, logCs;    // Ct = (M+1)/2 time-tile columns, Cs lines per batch
  double tol, q_floor;
  int max_sweeps;
  SolveCtl* ctl;          // written at the end: sweeps, last update, done
};
size_t small_smem(int N, int M, int Ct, int L, int Cs);
cudaError_t launch_small_solve(const SmallArgs& a, cudaStream_t st);

// Stop after sweep m? upd = ||U_m - U_{m-1}|| / ||U_m||, prev = upd_{m-1}. For m >= 2 the
// contraction is estimated as q = max(upd / prev, q_floor) (q_floor: rounding floor of the inner
// solves) and the error as upd q / (1 - q).
__host__ __device__ inline bool stop_decision(int m, double upd, double prev, double tol, double q_floor) {
  if (m == 1) return upd <= 0.01 * tol;
  const double q = prev > 0.0 ? upd / prev : 0.0;
  const double qh = q > q_floor ? q : q_floor;
  if (qh < 1.0) return upd * qh / (1.0 - qh) <= tol;
  return upd <= tol;
}

cudaError_t launch_ctl_init(SolveCtl* ctl, double tol, double q_floor, int max_sweeps, cudaStream_t st);
cudaError_t launch_converge(const double* norms, SolveCtl* ctl, cudaGraphConditionalHandle h, cudaStream_t st);

// Thread-local message returned by pint_last_error().
// Every allocation of the library goes through these (device: cudaMalloc / cudaFree, pinned host:
// cudaMallocHost / cudaFreeHost), so that the failure-path hook pint_debug_fail_allocation can make
// any of them fail and pint_device_bytes_held can count what is held. lib_free takes the size that
// lib_malloc was given.
cudaError_t lib_malloc(void** p, size_t bytes);
void lib_free(void* p, size_t bytes);
cudaError_t lib_malloc_host(void** p, size_t bytes);
void lib_free_host(void* p);
// The failure-path hook for allocations that are not cudaMalloc calls (sub-allocations from a
// server's budget): true if this allocation is to fail.
bool inject_alloc_failure();

void set_last_error(const char* msg);
inline void set_last_error(const std::string& msg) { set_last_error(msg.c_str()); }

// Kernel timing hooks (per-kernel CUDA events when profiling is on).
void prof_begin(const char* name, cudaStream_t st);
void prof_end(cudaStream_t st);

}  // namespace pint
