/*
 * pint.h -- C ABI of the GB300 parallel-in-time solver for BDF-k (k = 1..6) diffusion and
 * CQ-BDF-k subdiffusion, after Wu & Zhou, "A parallel-in-time algorithm for high-order BDF
 * methods for diffusion and subdiffusion equations" (arXiv 2007.13125).
 *
 * Problem (Sec. 1, eq. (1.1) and eq. (1.4)):  D_t^alpha u + A u = f on (0, T], u(0) = v, with
 * D_t^alpha the first derivative (alpha = 1) or the Caputo derivative (0 < alpha < 1), and A the
 * finite-difference Dirichlet Laplacian on the unit interval (dim = 1), square (dim = 2) or cube
 * (dim = 3): interior points only, h_x = 1/(mx+1), h_y = 1/(my+1), h_z = 1/(mz+1), 3/5/7-point
 * stencil. pint_plan_desc also selects periodic boundaries (the remark of Sec. 2.2) and P1 finite
 * elements in 1D (the discretisation of Sec. 4), and a semilinear term g(u) is handled by
 * Algorithm 3 (pint_nl_solve).
 *
 * Discretisation: uniform steps t_n = n tau, n = 1..N; corrected BDF-k (Sec. 2.1, eq. (2.1)) or
 * corrected CQ-BDF-k (Sec. 3.1, eq. (3.7)) with the starting-step constants of Table 1. The
 * sequential scheme is the all-at-once system K U = F_hat (eq. (2.6)/(3.11) with kappa = 0).
 *
 * Parallel-in-time solve: the waveform-relaxation iteration (eq. (2.5) / eq. (3.10)) replaces
 * the history by kappa-periodic data; each sweep solves P_kappa U_m = F_{m-1} with the
 * kappa-circulant matrix B_k(kappa) = S D S^-1, S = Lambda(kappa) V (Lemma 2.3 / Lemma 3.3):
 * a kappa^{n/N}-scaled DFT along time, N independent shifted spatial solves
 * (g_j tau^-alpha + A) q_j = h_j, g_j the eigenvalues of B_k(kappa), and the inverse DFT and
 * scaling (Algorithm 1 / Algorithm 2). The exact time-stepping solution is the fixed point.
 *
 * Data layout (all solver arrays): FP64, row-major [N][M], row n-1 holds time level t_n, and a
 * row is the grid flattened as (z * my + y) * mx + x (x fastest), M = mx * my * mz (my = 1 in 1D,
 * mz = 1 below 3D).
 *
 * Memory: every array argument marked "device" is a device pointer owned by the caller (for
 * example torch.Tensor.data_ptr() of a CUDA tensor) that must stay valid until the stream work
 * of the call has completed. A plan owns its device workspaces and constant tables.
 * `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *
 * Errors: every call returns a pint_status and never aborts, throws or traps. A failing call
 * leaves a message retrievable with pint_last_error() (thread-local). Invalid arguments return
 * PINT_EINVAL before anything is enqueued. A plan is not thread-safe; use one per host thread.
 *
 * Supported sizes: N a power of two, 8 <= N <= 4096 (CQ: N <= 2048); mx + 1, my + 1, mz + 1
 * powers of two, 3 <= mx, my, mz <= 2047 (the sine transforms run as FFTs of length 2(m+1));
 * periodic axes take m points, m a power of two, 8 <= m <= 4096.
 */
#ifndef PINT_H
#define PINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pint_plan_s* pint_plan;

typedef enum {
  PINT_OK = 0,
  PINT_EINVAL = 1,     /* invalid argument or unsupported size */
  PINT_ENOMEM = 2,     /* device or host allocation failed */
  PINT_ECUDA = 3,      /* a CUDA runtime call failed (message in pint_last_error) */
  PINT_ENOTCONV = 4,   /* pint_solve reached max_sweeps above tol */
  PINT_ETIMEOUT = 5,   /* bounded wait expired (serving API) */
  PINT_EAGAIN = 6,     /* result not ready yet (serving API) */
  PINT_EBUDGET = 7,    /* request larger than the serving memory budget */
  PINT_ENOTFOUND = 8   /* unknown ticket (serving API) */
} pint_status;

/* Arithmetic of a sweep.
 * PINT_FP64:  Algorithm 1/2 as printed, every step in FP64 (direct form F_{m-1} of eq. (2.7) /
 *             eq. (3.12), FP64 DFTs and spatial solves).
 * PINT_MIXED: residual-correction form U_m = U_{m-1} + P~^-1 (F_hat - K U_{m-1}), algebraically the
 *             same iteration; the residual in double-float (~48-bit) arithmetic, the kappa-scaled
 *             DFT and the shifted solves (P~^-1) in FP32 complex, the iterate kept in double-float.
 * PINT_FP32:  Algorithm 1/2 entirely in FP32 (reports the single-precision floor). */
typedef enum { PINT_FP64 = 0, PINT_MIXED = 1, PINT_FP32 = 2 } pint_precision;

/* Eigenvalues used for the CQ kappa-circulant (identical for alpha = 1):
 * TRUNC_DFT:   g_j = sum_{l<N} kappa^{l/N} omega_l e^{-2 pi i j l/N}, the spectrum of B_k(kappa) as
 *              printed in eq. (3.11) (weights omega_0..omega_{N-1}).
 * CLOSED_FORM: g_j = delta_k(kappa^{1/N} e^{-2 pi i j/N})^alpha (principal branch). */
typedef enum { PINT_EIG_TRUNC_DFT = 0, PINT_EIG_CLOSED_FORM = 1 } pint_eig_variant;
/* CLOSED_FORM with alpha < 1 is accepted only with PINT_MIXED: the residual-correction form has
 * the sequential solution as its fixed point for any preconditioner, whereas the printed direct
 * form's kappa-term (eq. (3.12)) belongs to the truncated matrix (PINT_EINVAL otherwise). */

/* Spatial discretisation of the Dirichlet Laplacian on the unit interval / square, interior
 * nodes only, h = 1/(m+1) per axis:
 * FD:     finite differences, A_h = the 3-/5-point stencil (1/h^2) [-1 2 -1] per axis.
 * FEM_P1: piecewise-linear Galerkin finite elements on the uniform mesh (Sec. 4, the space
 *         discretisation of the paper's 1D tests): the time derivative acts through the mass
 *         matrix M_h = (h/6) tridiag(1, 4, 1) and the Laplacian is the stiffness matrix
 *         K_h = (1/h) tridiag(-1, 2, -1); unknowns are nodal values. 1D and PINT_MIXED only.
 * PERIODIC: finite differences with periodic boundary conditions (the remark of Sec. 2.2: the
 *         spatial systems are then diagonalised by the FFT): m points per axis, x_i = i/m,
 *         h = 1/m, m a power of two in [8, 4096] (mx, and my in 2D); the 3-/5-point stencil
 *         wraps around. Every precision. */
typedef enum { PINT_SPACE_FD = 0, PINT_SPACE_FEM_P1 = 1, PINT_SPACE_PERIODIC = 2 } pint_space;

typedef struct {
  int dim;  /* 1, 2 or 3 (3: finite differences with Dirichlet boundaries) */
  int mx;   /* interior points along x */
  int my;   /* interior points along y (ignored, taken as 1, when dim == 1) */
  int mz;   /* interior points along z (ignored, taken as 1, when dim < 3) */
} pint_grid;

typedef struct {
  int k;                  /* BDF order 1..6 */
  double alpha;           /* 1 (diffusion) or 0 < alpha < 1 (subdiffusion) */
  double kappa;           /* WR relaxation parameter, 0 < kappa < 1 */
  double tau;             /* time step T/N > 0 */
  int N;                  /* time levels */
  pint_grid grid;
  pint_precision precision;
  pint_eig_variant eig;
  int ysolve;             /* 2D y-direction solver of the shifted systems: 0 or 1 = sine transform
                             (default), 2 = tridiagonal by a thread-per-line recurrence (for
                             batches of many lines), 4 = tridiagonal by parallel cyclic reduction
                             (parallel within a line: one warp per line up to 32 rows, the whole
                             CTA on a line up to 1024 rows, for batches of few lines; my <= 1024,
                             else 1), 3 = whichever of 1, 2 and 4 runs fastest on this GPU, timed
                             at plan creation (cached per shape). 2 and 4 apply to FP32 inner
                             solves only (FP64 uses 1). The sine transform is the default: its
                             FP32 inner solves are more accurate (the tridiagonal recurrences
                             amplify rounding with the condition of the line systems), which
                             saves a sweep at tol 1e-8 on a 255 x 255, N = 256 heat problem */
  int space;              /* pint_space (0 = FD, the default when the struct is zeroed) */
  int xdst;               /* x-direction sine transforms of the FP32 inner solves (Algorithm 1 / 2,
                             step 2; 2D and 3D finite differences, Dirichlet): 1 = odd-sequence FFT;
                             2 = a dense product with the sine matrix on the tensor cores (tcgen05;
                             FP16 operands split in two, three products per term, the accuracy of
                             the FP32 FFT) where the lines have 255 or 127 points, else 1;
                             3 = whichever of 1 and 2 runs faster, timed at plan creation (cached
                             per shape); 0 (default) = 2 when the lines have 255 points and there
                             are at least 16384 of them ((N/2 + 1) my mz), or 127 points and at
                             least 8192 of them, else 1. PINT_FP64 plans use 1. The tensor-core
                             form holds 128 KB (255 points) or 64 KB (127 points) of tables on the
                             device. The y-direction transforms of 3D grids with my = 127 follow
                             the same switch (tensor cores for 2, and for 0 and 3 from 8192 lines
                             (N/2 + 1) mx mz; 64 KB more of tables; pint_plan_tuning out[8]); the
                             z solves of 3D grids with mz = 127 take two tensor-core passes
                             around the divide for 2 only (slower than the FFT form on the
                             grids measured; the same table; out[9]). */
} pint_plan_desc;

/* Build a plan: FP64 constant tables (BDF / CQ weights omega_j of eq. (2.2) / eq. (3.2) --
 * CQ weights by the power-series recursion for delta_k^alpha --, the Table 1 constants, the
 * time scales kappa^{n/N}, the eigenvalues g_j of Lemma 2.3 / 3.3, the sine-transform
 * eigenvalues, FFT twiddles) on the host, one upload, and the device workspaces.
 * Returns PINT_EINVAL for k outside 1..6, alpha outside (0,1], kappa outside (0,1), tau <= 0,
 * or unsupported N / mx / my; PINT_ENOMEM / PINT_ECUDA on device failure. *out is set only on
 * success. Synchronous. Tile widths of the time kernels: as many points per CTA as shared memory
 * allows, narrowed so that the points still give two CTAs per SM; when that narrowing applies to a
 * PINT_MIXED problem of at least 2^18 space-time unknowns, the residual, update and CQ-history
 * kernels are timed at every admissible width on the new plan's workspaces and each keeps its
 * fastest width (a few milliseconds; cached per problem shape for the process). */
pint_status pint_plan_create(int k, double alpha, double kappa, double tau, int N,
                             const pint_grid* grid, pint_precision precision, pint_plan* out);
pint_status pint_plan_create_desc(const pint_plan_desc* desc, pint_plan* out);

/* Free a plan and its device memory (synchronises the device first). NULL is accepted. */
pint_status pint_plan_destroy(pint_plan plan);

/* Bytes of device memory the plan holds (tables + workspaces); 0 for NULL. */
size_t pint_plan_workspace_bytes(pint_plan plan);

/* Right-hand side of the all-at-once system (eq. (2.7) / eq. (3.12) without the kappa term):
 *   F_hat_n = f(t_n) + a_n^(k) (f(0) - A v) + sum_{l=1}^{k-2} b_{l,n}^(k) tau^l d_t^l f(0)
 *             + tau^-alpha sum_{j=0}^{n-1} omega_j v,        n = 1..N.
 * v      [M]      device, initial value on the grid
 * f      [N][M]   device, f(t_n) on the grid
 * fderiv [k-1][M] device, row l = d_t^l f(0) (row 0 = f(0)); may be NULL when k = 1
 * Fhat   [N][M]   device, output (FP64)
 * With PINT_SPACE_FEM_P1 the same formula holds in weak form: v holds the nodal values of v_h,
 * f and fderiv hold load vectors ((f(t_n), phi_i) and (d_t^l f(0), phi_i)), A v becomes K_h v
 * and the last term tau^-alpha sum_j omega_j M_h v.
 * With a reaction term installed (pint_set_reaction) the starting correction uses the operator
 * with it: a_n^(k) (f(0) - A v - w c v).
 * Enqueued on `stream`; asynchronous. */
pint_status pint_form_rhs(pint_plan plan, const double* v, const double* f, const double* fderiv,
                          double* Fhat, void* stream);

/* Time windows (BDF-k, alpha = 1; the remark closing Sec. 4.3): a horizon of W N levels solved as
 * W windows of N levels with this plan, each window restarted from the previous one. K is lower
 * triangular with k sub-diagonal blocks in time, so window w >= 2 is the all-at-once system
 * K U = F_hat of this plan with
 *   F_hat_n = f(t_n) - tau^-1 sum_{j=n}^{k} omega_j U_prev^{N+n-j}   (n = 1..k),   f(t_n)   (n > k),
 * U_prev the previous window's solution (P1 elements: M_h U_prev), and the windows together are
 * the sequential solution of the whole horizon. The first window is formed by pint_form_rhs /
 * pint_nl_form_rhs; a natural initial guess for window w is its predecessor's last level
 * (pint_initial_guess with v = U_prev + (N-1) M). The semilinear term is pointwise in time, so
 * pint_nl_solve runs per window unchanged (its linearisation point follows the window).
 * f [N][M] device: f(t_n) (or load vectors) at the window's levels; U_prev [N][M] device;
 * Fhat [N][M] device output. PINT_EINVAL for alpha < 1 (the CQ history would reach every earlier
 * window) or while a reaction term is installed. Asynchronous on `stream`. */
pint_status pint_form_rhs_window(pint_plan plan, const double* f, const double* U_prev, double* Fhat,
                                 void* stream);

/* Initial guess U_0^n = v for n = 1..N (the starting iterate of Theorem 2.7).
 * v [M] device; U [N][M] device, output. Asynchronous on `stream`. */
pint_status pint_initial_guess(pint_plan plan, const double* v, double* U, void* stream);

/* One WR sweep U_next = P_kappa^-1 (F_hat + (P_kappa - K) U_prev) (Algorithm 1 / 2, one iteration
 * of eq. (2.5) / eq. (3.10); in PINT_MIXED the same iterate in residual-correction form).
 * Fhat, U_prev, U_next [N][M] device; U_next may equal U_prev.
 * upd_rel: optional host pointer; when non-NULL the call waits for the stream and stores
 * ||U_next - U_prev||_2 / ||U_next||_2 (space-time l2). */
pint_status pint_wr_sweep(pint_plan plan, const double* Fhat, const double* U_prev, double* U_next,
                          double* upd_rel, void* stream);

/* Iterate sweeps from the initial guess in U until converged (Theorem 2.7 uses U_0^n = v).
 * After sweep m, upd_m = ||U_m - U_{m-1}|| / ||U_m||. For m >= 2 the contraction is estimated as
 * q = max(upd_m / upd_{m-1}, q_floor), q_floor = eps * (lambda_max + max_j |g_j| tau^-alpha) /
 * min_j |g_j tau^-alpha + lambda_min| / kappa the rounding floor of the inner solves (eps = 2^-24
 * for MIXED/FP32, 2^-53 for FP64), and the error estimate is upd_m q / (1 - q). Stops when that
 * estimate is <= tol (or upd_1 <= tol/100), or, if q >= 1, when upd_m <= tol. Returns
 * PINT_ENOTCONV after max_sweeps otherwise (U then holds the last iterate).
 * Fhat [N][M] device input; U [N][M] device, in: initial guess, out: solution.
 * sweeps_out, upd_rel_out: optional host pointers. The whole solve is one CUDA-graph launch (a
 * while-node repeats the sweep until a device-side check of the fused norms stops it); the graph
 * is built on first use of an (Fhat, U, tol, max_sweeps) combination and reused for it (a plan
 * keeps the four most recently used, so alternating buffer sets do not rebuild). The call waits
 * for `stream` once. With per-kernel profiling on, sweeps are launched one by one instead.
 * Small 1D problems (MIXED, finite differences, Dirichlet, BDF-k, N * M <= 4096) run the whole
 * solve, every sweep and the same stopping rule (evaluated in FP32), as one kernel in one CTA,
 * in either mode (the profile then lists "small_solve_ff"). */
pint_status pint_solve(pint_plan plan, const double* Fhat, double* U, double tol, int max_sweeps,
                       int* sweeps_out, double* upd_rel_out, void* stream);

/* Resume a preempted solve (checkpoint / restart). U [N][M] device holds the iterate U_m left by an
 * earlier solve of the same problem after sweeps_done sweeps -- for example what pint_solve or
 * pint_solve_v left in U when it returned PINT_ENOTCONV at max_sweeps = m, saved by the caller and
 * written back, possibly into another plan with the same description or in another process -- and
 * upd_last that solve's last relative update (its upd_rel_out). The WR iteration is a stationary
 * fixed-point iteration (eq. (2.5) / eq. (3.10)), so any iterate is a valid restart point; with the
 * stopping rule's history restored (the sweep count and the last update) the resumed solve takes
 * the same sweeps and the same stopping decision as a solve that was not interrupted (PINT_FP64:
 * bit-identical iterates; PINT_MIXED: the FP64 iterate re-split into double-float differs from the
 * uninterrupted one by its last bits). max_sweeps bounds the total count (done + new); sweeps_out
 * reports the total. Sweeps are launched one by one from the host (no graph); the call waits for
 * `stream`. PINT_EINVAL unless 0 <= sweeps_done <= max_sweeps and upd_last >= 0. */
pint_status pint_solve_resume(pint_plan plan, const double* Fhat, double* U, int sweeps_done, double upd_last,
                              double tol, int max_sweeps, int* sweeps_out, double* upd_rel_out, void* stream);

/* pint_solve from the initial guess U_0^n = v of Theorem 2.7 (every level equal to the initial
 * value), without materialising it: for that iterate K U_0 = beta_n M v + A v with
 * beta_n = tau^-alpha sum_{j<n} omega_j (BDF and CQ alike), so the first residual is
 * F_hat_n - beta_n M v - A v, formed in one pass over F_hat with no read of U (and, for CQ, no
 * history product), and the first update writes U_1 = v + c. The iterates and the stopping rule
 * are those of pint_initial_guess followed by pint_solve. v [M] device (FP64); U [N][M] device,
 * output only (its input content is not read). PINT_MIXED runs the first sweep this way; the
 * FP64 and FP32 paths broadcast v into U inside the solve's graph. */
pint_status pint_solve_v(pint_plan plan, const double* Fhat, const double* v, double* U, double tol,
                         int max_sweeps, int* sweeps_out, double* upd_rel_out, void* stream);

/* pint_form_rhs followed by pint_solve_v, from the problem data (v, f, the derivatives of f at 0,
 * laid out as for pint_form_rhs; device FP64) to U (device, output only), with the same iterates,
 * stopping rule, results and errors. For PINT_MIXED BDF plans (alpha = 1, no reaction term) F_hat
 * is not materialised: F_hat_n = f(t_n) exactly beyond the first k levels (the starting
 * corrections of eq. (2.7) act on levels n <= k - 1 and beta_n = 0 from level k + 1 on), so the
 * residual kernels read the first k levels of F_hat from a k x M block of the plan (formed by the
 * right-hand-side kernel) and f for the others; the results are those of the unfused path. Other
 * plans form F_hat into a plan workspace of N M doubles, allocated on the first call (PINT_ENOMEM
 * if it cannot be) and freed with the plan. Waits for `stream`. */
pint_status pint_solve_fv(pint_plan plan, const double* v, const double* f, const double* fderiv, double* U,
                          double tol, int max_sweeps, int* sweeps_out, double* upd_rel_out, void* stream);

/* pint_solve_v enqueued without waiting (as pint_solve_async; result by pint_solve_result). */
pint_status pint_solve_v_async(pint_plan plan, const double* Fhat, const double* v, double* U, double tol,
                               int max_sweeps, void* stream);

/* The whole solve of pint_solve (one graph launch) enqueued on `stream` without waiting, so that
 * host transfers or other work can be queued behind it. The plan's workspaces stay in use until
 * the stream has completed the solve: later calls on the same plan must be ordered after it
 * (same stream, or an event). Fhat, U, tol, max_sweeps as in pint_solve. PINT_EINVAL while
 * per-kernel profiling is on (that mode launches sweeps from the host). */
pint_status pint_solve_async(pint_plan plan, const double* Fhat, double* U, double tol, int max_sweeps,
                             void* stream);

/* End-to-end solve through host buffers: copies v [M], f [N][M] and fderiv [k-1][M] (NULL when
 * k = 1) from host memory into device buffers the plan owns, forms F_hat (pint_form_rhs), solves
 * from U_0^n = v (pint_solve_v, tol and max_sweeps as there) and copies the solution into the host
 * array U_out [N][M]; everything is enqueued without waiting. The device work runs on `stream`;
 * the copies run on two streams of the plan, and the plan keeps two sets of staging buffers, so
 * consecutive calls overlap their transfers with the neighbouring solves (the inputs of call i+1
 * are copied in, and the solution of call i-1 is copied out, while call i solves).
 * pint_solve_host_join makes a stream wait for every copy-out issued so far: once that stream has
 * completed, every U_out is filled; pint_solve_result then reports the last solve. Host arrays must
 * stay valid, and the inputs unchanged, until then; page-locked host memory (cudaHostAlloc) makes
 * the copies asynchronous, pageable memory works with the driver's staging. The staging buffers
 * (two sets of v, f, d^l f(0) and U, and one F_hat: 5 N M + 2 k M doubles) are allocated on the
 * first call (PINT_ENOMEM if they cannot be) and freed with the plan. A plan runs one call at a
 * time per stream ordering: calls on different streams must not overlap. */
pint_status pint_solve_host(pint_plan plan, const double* v, const double* f, const double* fderiv,
                            double* U_out, double tol, int max_sweeps, void* stream);
pint_status pint_solve_host_join(pint_plan plan, void* stream);

/* The plan's tuned choices: out[0] residual tile width (points / 2 per CTA), out[1] update tile
 * width, out[2] CQ-history tile width, out[3] y-direction solver (1 sine transform, 2 recurrence,
 * 4 parallel cyclic reduction), out[4] / out[5] largest FFT radix of the residual / update time
 * transforms (16 for the compiled shapes; 8 or 16 as timed for runtime shapes; 0 when not MIXED),
 * out[6] 1 if the whole solve runs as one CTA, out[7] x sine transform of the FP32 inner solves
 * (1 odd-sequence FFT, 2 tensor-core products), out[8] y sine transform of 3D plans (the same
 * codes), out[9] z solve of 3D plans (1 odd-sequence FFTs around the divide, 2 two tensor-core
 * passes around it). Fills min(n, 10) entries and returns 10 (-1 for a NULL plan or out).
 * Host-only. */
int pint_plan_tuning(pint_plan plan, int* out, int n);

/* Outcome of the plan's most recent graph-launched solve: sweeps, final relative update, and
 * PINT_OK if it met tol, PINT_ENOTCONV if it stopped at max_sweeps. Valid once the stream has
 * completed that solve; the next solve on the plan overwrites it. */
pint_status pint_solve_result(pint_plan plan, int* sweeps_out, double* upd_rel_out);

/* Solve n independent problems with one graph launch. Each plan's whole solve (prologue, a
 * while-loop of sweeps with the device-side convergence check, epilogue) becomes an independent
 * branch of one CUDA graph, so problems of different sizes, orders and alpha run concurrently on
 * the GPU and each stops on its own. plans: n distinct plans; Fhat[i], U[i]: device arrays of
 * plans[i] as in pint_solve; sweeps_out, upd_out: optional host arrays of length n. Waits for the
 * stream once. Returns PINT_ENOTCONV if any problem reached max_sweeps above tol. */
pint_status pint_batch_solve(pint_plan* plans, int n, const double* const* Fhat, double* const* U,
                             double tol, int max_sweeps, int* sweeps_out, double* upd_out, void* stream);

/* pint_batch_solve with every problem started from U_0^n = v[i] as in pint_solve_v (v[i]: [M]
 * device arrays of plans[i]; U[i] output only). */
pint_status pint_batch_solve_v(pint_plan* plans, int n, const double* const* Fhat, const double* const* v,
                               double* const* U, double tol, int max_sweeps, int* sweeps_out, double* upd_out,
                               void* stream);

/* ---- reaction terms and semilinear problems (Sec. 4.3, Algorithm 3) ----
 * 1D plans with Dirichlet boundaries (PINT_SPACE_FD in every precision, PINT_SPACE_FEM_P1 with
 * PINT_MIXED); other plans return PINT_EINVAL. A reaction coefficient enters each row with the
 * weight w = 1 (finite differences) or w = h (P1 elements: (c U_h, phi_i) and (g(U_h), phi_i) by
 * nodal quadrature, h c_i U_i and h g(U_i)). */

/* Install a space-varying reaction term in the plan's linear solves: A becomes A + w diag(c), so
 * pint_wr_sweep, pint_solve, pint_solve_async and pint_batch_solve then solve
 * (D_tau^alpha + A + w diag(c)) U = F_hat. c [M] device, FP64, copied before the call's stream
 * work ends (the caller may reuse it afterwards); NULL removes the term. With the term present the
 * shifted systems sigma_j M + A + w diag(c) of Algorithm 1 / 2 step 2 are no longer diagonalised by
 * the sine transform: each frequency's tridiagonal system is solved by Gaussian elimination with
 * LU factors computed here (FP64 arithmetic, stored in the plan's inner precision); sweeps then use
 * the forward / backward substitutions. The elimination does not pivot: it is meant for
 * A + w diag(c) positive definite (c > -lambda_min(A) / w suffices), the case of the linearised
 * operators of Algorithm 3. Enqueued on `stream`. */
pint_status pint_set_reaction(pint_plan plan, const double* c, void* stream);

/* Cubic nonlinearity g(u) = c[0] + c[1] u + c[2] u^2 + c[3] u^3 of the semilinear problem
 * D_t^alpha u + A u + g(u) = f (eq. (4.3)); the Allen-Cahn term of Example 4 is
 * c = {0, -1/eps^2, 0, 1/eps^2}. */
typedef struct { double c[4]; } pint_poly;

/* F_hat of the semilinear scheme (eq. (4.4)): pint_form_rhs with the starting correction
 * a_n^(k) (f(0) - A v - w g(v)) in place of a_n^(k) (f(0) - A v); arguments as there. The scheme
 * is then the all-at-once system K U + w g(U) = F_hat. PINT_EINVAL while a reaction term is
 * installed. Asynchronous on `stream`. */
pint_status pint_nl_form_rhs(pint_plan plan, const pint_poly* g, const double* v, const double* f,
                             const double* fderiv, double* Fhat, void* stream);

#define PINT_NL_MAX_STEPS 64
typedef struct {
  int steps;                        /* outer (Newton) steps taken */
  int sweeps[PINT_NL_MAX_STEPS];    /* inner WR sweeps of each outer step */
  double upd[PINT_NL_MAX_STEPS];    /* ||U_l - U_{l-1}|| / ||U_l|| (space-time l2) of each step */
} pint_nl_info;

/* Algorithm 3 (modified Newton iteration, eqs. (4.6)-(4.7)): from the iterate in U (Algorithm 3
 * starts from U_0^n = v: pint_initial_guess), step l = 1, 2, ...
 *   Ubar = (1/N) sum_n U_{l-1}^n,  D = g'(Ubar)  (one spatial field for all levels),
 *   solve (K + I (x) w D) W = F_hat - K U_{l-1} - w g(U_{l-1}) by the WR iteration from W_0 = 0,
 *   U_l = U_{l-1} + W,
 * where the inner solve is pint_solve of the plan with the reaction term w D installed (its
 * stopping rule and tolerance `tol`, at most max_sweeps sweeps; one graph launch) applied to
 * V = U_{l-1} + W. The linearised term carries +g'(Ubar), the sign of Newton's linearisation
 * (eqs. (4.6)-(4.7) print -g'(Ubar); only + reproduces the contraction of Table 4). The outer
 * loop stops on upd_l = ||U_l - U_{l-1}|| / ||U_l||: at l = 1 or 2 when upd_l <= newton_tol / 100
 * (the ratio upd_2 / upd_1 reflects the distance of the starting iterate, not the contraction of
 * later steps, so it is not used on its own); from l = 3 when upd_l q / (1 - q) <= newton_tol with
 * q the larger of upd_l / upd_{l-1} and upd_{l-1} / upd_{l-2}.
 * Fhat [N][M] device (pint_nl_form_rhs); U [N][M] device, in: initial
 * iterate, out: U_l. info: optional host pointer. The solve installs w D in the plan's reaction
 * slot and removes it before returning; PINT_EINVAL if a reaction term is already installed.
 * Waits for `stream` once per outer step. Returns PINT_ENOTCONV
 * if max_steps (<= PINT_NL_MAX_STEPS) outer steps did not meet newton_tol or an inner solve
 * stopped at max_sweeps (U then holds the last iterate). */
pint_status pint_nl_solve(pint_plan plan, const pint_poly* g, const double* Fhat, double* U, double newton_tol,
                          int max_steps, double tol, int max_sweeps, pint_nl_info* info, void* stream);

/* ---- serving: continuous batching of independent solves ----
 * A server owns a device-memory budget (reserved once at creation and sub-allocated, so admission
 * never calls cudaMalloc), up to max_active concurrent solves (one stream each) and a worker
 * thread. Requests are admitted in arrival order while a slot is free and the budget holds their
 * plan, F_hat, U, f and v; each admitted request runs as one graph launch (F_hat, U_0 = v, the
 * whole WR solve with its device-side convergence loop), so requests admitted while others run
 * overlap on the GPU. The iterate stays on the device until pint_poll copies it out and releases
 * the request's memory: a finished solution is held on the device (counted against the budget)
 * until it is polled, except that when held solutions keep a queued request out, the oldest is
 * moved to host memory first. The server is thread-safe; plans are internal to it. */
typedef struct pint_server_s* pint_server;
typedef struct {
  pint_plan_desc desc;  /* problem and precision (precision PINT_MIXED or PINT_FP64 recommended) */
  double tol;           /* stopping tolerance as in pint_solve */
  int max_sweeps;
  int inputs_on_device; /* 0: v, f, fderiv are host arrays, copied by pint_submit; 1: they are
                           device arrays owned by the caller, read when the request is admitted,
                           and must stay valid until the request has been polled */
} pint_request;
typedef struct {
  int status;           /* PINT_OK, PINT_ENOTCONV, PINT_EBUDGET (larger than the budget), ... */
  int sweeps;
  double upd_rel;       /* last relative update */
  double t_submit, t_start, t_done;  /* seconds since server creation: submitted, admitted, solved */
} pint_solve_info;

/* hbm_budget_bytes >= 1 MiB is reserved now (PINT_ENOMEM if it cannot be); max_active in 1..256. */
pint_status pint_server_create(size_t hbm_budget_bytes, int max_active, pint_server* out);
/* Finishes admitted work, frees everything (unpolled results are dropped). NULL is accepted. */
pint_status pint_server_destroy(pint_server s);
/* v [M], f [N][M], fderiv [k-1][M] (NULL when k = 1): host arrays copied before returning, or
 * device arrays (req->inputs_on_device = 1) that are read while the request runs (from its
 * admission until it is done; PINT_MIXED BDF requests read f during the solve). */
pint_status pint_submit(pint_server s, const pint_request* req, const double* v, const double* f,
                        const double* fderiv, uint64_t* ticket);
/* Wait up to timeout_us for the result: PINT_EAGAIN (timeout_us == 0) or PINT_ETIMEOUT if not
 * done yet (the request stays live); otherwise the request's status, with U copied into the host
 * array U_out [N][M] (may be NULL) and the request retired. PINT_ENOTFOUND for an unknown ticket.
 * info (optional) receives the status, sweeps and timestamps. */
pint_status pint_poll(pint_server s, uint64_t ticket, int timeout_us, double* U_out, pint_solve_info* info);
/* out[8]: completed, active, queued, device bytes in use, DOF solved, sweeps, seconds since
 * creation, peak device bytes in use. */
pint_status pint_server_stats(pint_server s, double* out);

/* ---- a solve that allocates no device memory ----
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory when they run: code under a device-memory budget fixed up front,
 * plugins whose host runtime owns every allocation, or real-time loops where a cudaMalloc
 * (which may synchronise the device) is not acceptable. Such callers cannot build a plan.
 *
 * Q = P_kappa^{-1} R for the 1D heat problem (alpha = 1, FP64, finite differences): scale level
 * n by kappa^{n/N}, transform along time, solve the N/2 + 1 complex-shifted 1D systems by the
 * sine transform, transform back and undo the scaling -- the same kernels as a PINT_FP64 plan,
 * i.e. the result of pint_wr_sweep with U_prev = 0 and Fhat = R.
 * R, Q: [N][mx] FP64 arrays of the current device owned by the caller; Q may not overlap R
 * (PINT_EINVAL for host pointers, arrays of another device, or overlapping arrays; the sizes of
 * the arrays cannot be checked from raw pointers: each must hold N * mx doubles).
 * Limits: N a power of two in [8, 1024] with N > k; mx + 1 a power of two, 3 <= mx <= 1023;
 * (N/2 + 1) * mx <= 262144. Larger sizes return PINT_EINVAL (message in pint_last_error).
 * Memory: the intermediate spectrum and the constant tables live in one static device array of
 * about 4.2 MiB that is part of the library: every GPU that loads the library holds it until
 * the process exits. No cudaMalloc, cudaFree or other allocating routine is called.
 * Set-up: the first call made on a device looks up that array's device address for the
 * current device (a synchronous driver query), so make that first call before any stream
 * capture. The address is kept per device together with the ID of the context it was found in;
 * after a cudaDeviceReset the next call (again the first in the new context, so again before
 * any capture) looks it up anew. The array is shared by every call and keeps the last call's
 * contents (the parts that must start at zero are cleared by each call): calls whose GPU work
 * overlaps -- on different streams or from different host threads -- race on it; serialise
 * them. */
pint_status pint_kappa_solve_noalloc(int k, double kappa, double tau, int N, int mx, const double* R,
                                     double* Q, void* stream);

/* ---- host-only queries (no GPU needed) ---- */

/* omega_0..omega_{n-1}: BDF-k weights (alpha = 1, zero past k; eq. (2.2)) or the CQ weights,
 * coefficients of delta_k(xi)^alpha (eq. (3.2)), by the power-series recursion
 * q_0 = p_0^alpha, q_m = (1/(m p_0)) sum_{i=1}^{min(m,k)} ((alpha+1) i - m) p_i q_{m-i}. */
pint_status pint_time_weights(int k, double alpha, int n, double* omega);

/* Table 1 constants: a[n-1] = a_n^(k) (n = 1..5), b[(l-1)*5 + (n-1)] = b_{l,n}^(k) (l = 1..4);
 * zero where the table has no entry. b_{3,1}^(5) is returned as -1/720 (the printed +1/720
 * contradicts the order conditions that define the table). */
pint_status pint_correction_coefficients(int k, double* a, double* b);

/* Eigenvalues g_j, j = 0..N-1, of B_k(kappa) for the chosen variant (Lemma 2.3 / 3.3), FP64. */
pint_status pint_circulant_eigenvalues(int k, double alpha, double kappa, int N, pint_eig_variant eig,
                                       double* re, double* im);

/* ---- diagnostics ---- */
const char* pint_last_error(void);
const char* pint_status_string(pint_status s);
const char* pint_version(void);

/* Device memory, in bytes, that the library holds right now through cudaMalloc: the workspaces of
 * live plans and the budgets of live servers (the static array of pint_kappa_solve_noalloc is not
 * counted). Every creation that fails gives back what it took, so the figure returns to its earlier
 * value once the plans and servers created since are destroyed or failed. */
long long pint_device_bytes_held(void);

/* Failure-path hook for tests: the n-th next memory allocation the library attempts (n = 0: the
 * very next one; a cudaMalloc, a cudaMallocHost, or a sub-allocation from a server's budget) fails
 * as if the memory were exhausted, taking the same error path and clean-up as a real failure
 * (PINT_ENOMEM from plan creation and server creation; a request whose memory cannot be taken while
 * nothing else runs finishes with PINT_EBUDGET). n < 0 disarms it. Process-wide; returns the
 * previous setting. Nothing is faulted on the GPU. */
int pint_debug_fail_allocation(int n);

/* Per-kernel timing with CUDA events recorded around every launch on its stream (off by
 * default). pint_kernel_stats waits for the recorded events, then fills up to `max` entries
 * (names are static strings) and returns the number of distinct kernels; reset != 0 clears. */
pint_status pint_set_profiling(int enable);
int pint_kernel_stats(int max, const char** names, int* launches, double* total_ms, int reset);

#ifdef __cplusplus
}
#endif
#endif /* PINT_H */
