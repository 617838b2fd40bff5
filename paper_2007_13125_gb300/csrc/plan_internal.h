// The plan object and the internal entry points shared by the C-ABI translation units
// (plan.cu: plans, sweeps and solves; server.cu: the serving loop).
#pragma once
#include <cuda_runtime.h>

#include <complex>
#include <vector>

#include "../../include/pint.h"
#include "pint_internal.h"

namespace pint {

template <typename T> struct DevTables {
  void* tw_time = nullptr;   // V[N]
  T* s = nullptr;            // [N]
  T* inv_s = nullptr;        // [N]
  void* sigma = nullptr;     // V[N/2+1]
  void* tw_x = nullptr;      // V[2(mx+1)]
  void* tw_y = nullptr;      // V[2(my+1)]
  T* lam_x = nullptr;        // [mx]
  T* lam_y = nullptr;        // [my]
  void* tw_z = nullptr;      // V[2(mz+1)] (3D)
  T* lam_z = nullptr;        // [mz] (3D)
  T* lam_xy = nullptr;       // [my][mx] lambda_x + lambda_y per z line (3D)
  T* mu_x = nullptr;         // [mx] mass-matrix eigenvalues (P1 FEM only)
};

// Source of a plan's device memory: cudaMalloc by default, or a sub-allocator (the server's
// budgeted arena). alloc returns nullptr on failure.
struct HostStage;
// frees the staging of pint_solve_host (host_io.cu); called by plan destruction
void host_stage_free(pint_plan p);

struct DevAllocator {
  virtual void* alloc(size_t bytes) = 0;
  virtual void release(void* p) = 0;
  // small pinned host buffers (convergence state read back by the host)
  virtual void* host_alloc(size_t bytes) {
    void* p = nullptr;
    return lib_malloc_host(&p, bytes) == cudaSuccess ? p : nullptr;
  }
  virtual void host_release(void* p) { lib_free_host(p); }
  virtual ~DevAllocator() {}
};

// Cached executable graph of one whole solve (prologue, while-loop of sweeps, epilogue).
// One instantiated whole-solve graph and the arguments it was built for.
struct SolveGraph {
  cudaGraphExec_t exec = nullptr;
  const double* F = nullptr;
  const double* Fc = nullptr;       // F is f, F_hat's first kc levels in Fc (null: F is F_hat)
  double* U = nullptr;
  const double* v = nullptr;        // solve from U_0^n = v (null: from the content of U)
  double tol = 0.0;
  int max_sweeps = 0;
  bool react = false;               // captured with the reaction term's spatial solve
  unsigned long long last_use = 0;
};
// Graphs cached per plan (least recently used replaced): callers that alternate between a few
// buffer sets, e.g. to overlap host transfers with solves, reuse their graphs.
constexpr int kSolveGraphs = 4;

}  // namespace pint

struct pint_plan_s {
  int k; double alpha, kappa, tau; int N;
  int dim, mx, my, mz, M;
  pint_precision prec;
  pint_eig_variant eig;
  bool cq;
  bool fem;                         // P1 finite elements (1D): mass matrix in the time terms
  bool periodic;                    // periodic boundary conditions (FFT in space)
  std::vector<double> omega;
  double a[5];
  double b[4][5];
  std::vector<std::complex<double>> g;
  double gx, gy, gz;
  // device
  pint::DevAllocator* alloc = nullptr;   // null: cudaMalloc / cudaFree
  std::vector<void*> allocs;
  std::vector<size_t> alloc_sizes;
  pint::HostStage* hstage = nullptr;      // staging of pint_solve_host (host_io.cu), on first use
  size_t bytes = 0;
  pint::DevTables<float> tf;
  pint::DevTables<double> td;
  double* beta = nullptr;           // [N]
  float2* beta_ff = nullptr;        // [N] beta as double-float (MIXED first sweep from v)
  double2* tw_2n = nullptr;         // [2N]
  double2* what_lo = nullptr;       // [2N] permuted, * tau^-alpha / 2N
  double2* what_up = nullptr;       // [2N] permuted, * kappa tau^-alpha / 2N
  float4* what_ff = nullptr;        // MIXED CQ: [2N] double-float complex, radix-8 permuted, * tau^-alpha / 2N
  float4* tw_ff = nullptr;          // MIXED CQ: [2N] double-float complex exp(-2 pi i m / 2N)
  float2* Uff = nullptr;            // MIXED: U as double-float pairs (hi, lo) [N][M]
  double* fcorr = nullptr;          // MIXED BDF: F_hat's first kc levels [kc][M] (pint_solve_fv)
  int kc = 0;
  double* Fws = nullptr;            // pint_solve_fv without the fused form: F_hat [N][M] (on first use)
  int xdst = 1;                     // x sine transforms of FP32 inner solves: 1 odd-sequence FFT,
                                    // 2 tensor-core products (mx = 255 or 127)
  unsigned short* dst_tab = nullptr;  // xdst 2: the sine-matrix image (FP16 hi / lo)
  int ydst = 1;                     // y sine transforms of 3D FP32 inner solves: 1 odd-sequence FFT,
                                    // 2 tensor-core products (lines of 127 points, strided)
  unsigned short* dst_tab_y = nullptr;  // ydst / zsolve 2: the 127-point sine-matrix image
  int zsolve = 1;                   // z solve of 3D FP32 inner solves: 1 odd-sequence FFT (k_axis op 1),
                                    // 2 two tensor-core passes around the divide (mz = 127)
  float *Uhi = nullptr, *Fhi = nullptr;  // FP32: U, F_hat
  void* S = nullptr;                // spectrum
  double* z = nullptr;              // CQ Toeplitz output [N][M]
  double* norms = nullptr;          // device [2]
  double* h_norms = nullptr;        // pinned host [2]
  pint::SolveCtl* ctl = nullptr;    // device convergence state
  pint::SolveCtl* h_ctl = nullptr;  // pinned host copy written by the graph's epilogue
  cudaStream_t cap = nullptr;       // stream used to capture graphs
  pint::SolveGraph sg[pint::kSolveGraphs];
  unsigned long long sg_clock = 0;
  // tiles
  int Ct, Cr, Ci, Ctd, Cz, Cx, Cy, Czl, Ctri;  // columns per CTA: time (float), residual, update, time (T),
                                             // toeplitz, x, y, z lines, tri
  int ysolve;                       // 2D y direction: 1 sine transform, 2 tridiagonal, 4 PCR
  int rml = 4, uml = 4;             // radix bound (log2) of the runtime-shape time FFTs of the
                                    // MIXED residual and update kernels (tuned: 3 or 4)
  double q_floor;                   // predicted floor of the per-sweep contraction (inner precision)
  // reaction term (1D, Dirichlet): the spatial operator A + w diag(c) of the linear solves
  // (pint_set_reaction; the linearised operator of Algorithm 3)
  bool react_on = false;
  // small 1D problems: the whole MIXED solve in one CTA (kernels_small.cu); time-tile columns and
  // spatial lines per batch of that kernel
  bool small = false;
  int small_Ct = 0, small_Cs = 0;
  double* react = nullptr;          // [M] w c_i
  void* tri_ip = nullptr;           // [N/2+1][M] T2: inverse pivots of the shifted systems
  void* tri_cp = nullptr;           // [N/2+1][M] T2: eliminated super-diagonal
  // Algorithm 3 workspaces (allocated on first use)
  double* nl_F = nullptr;           // [N][M] right-hand side of the linearised problem
  double* nl_U0 = nullptr;          // [N][M] previous outer iterate
  double* nl_fd = nullptr;          // [k-1][M] derivative rows with f(0) - w g(v)
  double* nl_norms = nullptr;       // device [2]
  double* nl_h = nullptr;           // pinned host [2]
};

namespace pint {

// Plan creation with an explicit device-memory source (null: cudaMalloc).
pint_status plan_create_internal(const pint_plan_desc* d, DevAllocator* A, pint_plan* out);
// Free a plan's memory without synchronising the device (its work must have completed).
void plan_release(pint_plan p);
// Device bytes a plan for this description will hold (workspaces and tables).
size_t plan_bytes_estimate(const pint_plan_desc* d);
// Enqueue one whole solve on `st` as a single graph launch (building or reusing the cached graph);
// the graph ends with a copy of the convergence state into pinned host memory.
pint_status solve_enqueue(pint_plan p, const double* F, double* U, double tol, int max_sweeps, cudaStream_t st,
                          const double* v = nullptr, const double* Fc = nullptr);
// Result of the last enqueued solve (valid once its stream work has completed).
void solve_result(pint_plan p, int* sweeps, double* upd, bool* converged);
bool solve_wait_gave_up(pint_plan p);
// The fused right-hand side (MIXED BDF plans without a reaction term, not the one-CTA solve): a
// solve from f with F_hat's first kc levels formed into the plan's block (form_rhs_corr) and
// passed to solve_enqueue as Fc.
bool fused_rhs_ok(pint_plan p);
bool profiling_on();  // pint_set_profiling is on (sweeps launched one by one, no graphs)
pint_status form_rhs_corr(pint_plan p, const double* v, const double* f, const double* fderiv, cudaStream_t st);  // the last solve's device-side wait gave up (after it completed)
// Add one solve (prologue, while-loop, epilogue, or the one-CTA solve) of plan p to graph g.
// v: start from U_0^n = v (MIXED: the first sweep in the prologue; otherwise v is broadcast into U).
// dep (optional): a node the solve's first node must follow; *last (optional): its final node.
pint_status add_solve_nodes(pint_plan p, cudaGraph_t g, const double* F, double* U, double tol, int max_sweeps,
                            const double* v, cudaGraphNode_t dep = nullptr, cudaGraphNode_t* last = nullptr,
                            const double* Fc = nullptr);

}  // namespace pint
