// Host side of the C ABI: plan construction (FP64 constant tables), workspaces, the sweep
// and solve drivers, host-only queries, error reporting and per-kernel timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pint.h"
#include "fft.cuh"
#include "pint_internal.h"
#include "plan_internal.h"

using cd = std::complex<double>;

namespace pint {

// ---------------------------------------------------------------------------
// error state
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static pint_status fail(pint_status s, const std::string& msg) {
  g_err = msg;
  return s;
}
void set_last_error(const char* msg) { g_err = msg; }

static pint_status cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  // the error is reported through the status; clear the runtime's per-thread error so that a
  // recoverable one (e.g. an over-sized launch request) does not surface in the caller's next
  // unrelated CUDA call (a sticky error stays regardless)
  (void)cudaGetLastError();
  return PINT_ECUDA;
}
#define PINT_CUDA(call)                                        \
  do {                                                         \
    cudaError_t _e = (call);                                   \
    if (_e != cudaSuccess) return cuda_fail(_e, #call);        \
  } while (0)

// ---------------------------------------------------------------------------
// allocations: the failure-path hook and the count of device bytes held
// ---------------------------------------------------------------------------
static std::atomic<int> g_fail_countdown{-1};   // < 0: off; 0: the next allocation fails
static std::atomic<long long> g_device_bytes{0};

bool inject_alloc_failure() {
  int v = g_fail_countdown.load();
  while (v >= 0) {
    if (g_fail_countdown.compare_exchange_weak(v, v - 1)) return v == 0;
  }
  return false;
}

cudaError_t lib_malloc(void** p, size_t bytes) {
  *p = nullptr;
  if (inject_alloc_failure()) return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_device_bytes += (long long)bytes;
  else (void)cudaGetLastError();
  return e;
}

void lib_free(void* p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  g_device_bytes -= (long long)bytes;
}

cudaError_t lib_malloc_host(void** p, size_t bytes) {
  *p = nullptr;
  if (inject_alloc_failure()) return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMallocHost(p, bytes);
  if (e != cudaSuccess) (void)cudaGetLastError();
  return e;
}

void lib_free_host(void* p) {
  if (p) cudaFreeHost(p);
}

// ---------------------------------------------------------------------------
// per-kernel timing
// ---------------------------------------------------------------------------
struct ProfRec { const char* name; cudaEvent_t a, b; };
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof_recs;
static std::vector<cudaEvent_t> g_prof_pool;
static thread_local ProfRec g_prof_open = {nullptr, nullptr, nullptr};

static cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void prof_begin(const char* name, cudaStream_t st) {
  if (!g_prof_on) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_open.name = name;
  g_prof_open.a = prof_event();
  g_prof_open.b = prof_event();
  cudaEventRecord(g_prof_open.a, st);
}
void prof_end(cudaStream_t st) {
  if (!g_prof_on || !g_prof_open.name) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEventRecord(g_prof_open.b, st);
  g_prof_recs.push_back(g_prof_open);
  g_prof_open.name = nullptr;
}

// ---------------------------------------------------------------------------
// FP64 host math: weights, Table 1, eigenvalues
// ---------------------------------------------------------------------------
static void bdf_poly(int k, double* w) {  // omega_0..omega_k of sum_l (1 - z)^l / l
  for (int j = 0; j <= k; ++j) w[j] = 0.0;
  for (int l = 1; l <= k; ++l) {
    double binom = 1.0;  // C(l, j)
    for (int j = 0; j <= l; ++j) {
      w[j] += ((j & 1) ? -binom : binom) / l;
      binom = binom * (l - j) / (j + 1);
    }
  }
}

static void time_weights(int k, double alpha, int n, double* out) {
  double p[kMaxK + 1];
  bdf_poly(k, p);
  if (alpha == 1.0) {
    for (int i = 0; i < n; ++i) out[i] = i <= k ? p[i] : 0.0;
    return;
  }
  if (n <= 0) return;
  out[0] = std::pow(p[0], alpha);
  for (int m = 1; m < n; ++m) {
    double s = 0.0;
    const int top = std::min(m, k);
    for (int i = 1; i <= top; ++i) s += ((alpha + 1.0) * i - m) * p[i] * out[m - i];
    out[m] = s / (m * p[0]);
  }
}

// Table 1 (Sec. 2.1), b_{3,1}^(5) = -1/720.
static void table1(int k, double* a, double (*b)[5]) {
  static const double A[7][5] = {
      {0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}, {1.0 / 2, 0, 0, 0, 0},
      {11.0 / 12, -5.0 / 12, 0, 0, 0},
      {31.0 / 24, -7.0 / 6, 3.0 / 8, 0, 0},
      {1181.0 / 720, -177.0 / 80, 341.0 / 240, -251.0 / 720, 0},
      {2837.0 / 1440, -2543.0 / 720, 17.0 / 5, -1201.0 / 720, 95.0 / 288}};
  static const double B[7][4][5] = {
      {}, {}, {},
      {{1.0 / 12, 0, 0, 0, 0}},
      {{1.0 / 6, -1.0 / 12, 0, 0, 0}, {0, 0, 0, 0, 0}},
      {{59.0 / 240, -29.0 / 120, 19.0 / 240, 0, 0}, {1.0 / 240, -1.0 / 240, 0, 0, 0},
       {-1.0 / 720, 0, 0, 0, 0}},
      {{77.0 / 240, -7.0 / 15, 73.0 / 240, -3.0 / 40, 0}, {1.0 / 96, -1.0 / 60, 1.0 / 160, 0, 0},
       {-1.0 / 360, 1.0 / 720, 0, 0, 0}, {0, 0, 0, 0, 0}}};
  for (int n = 0; n < 5; ++n) a[n] = A[k][n];
  for (int l = 0; l < 4; ++l)
    for (int n = 0; n < 5; ++n) b[l][n] = B[k][l][n];
}

// delta_k(z) = sum_l s^l / l with s = 1 - z supplied directly (no cancellation near z = 1)
static cd delta_from_s(int k, cd s) {
  cd out = 0.0, p = 1.0;
  for (int l = 1; l <= k; ++l) {
    p *= s;
    out += p / double(l);
  }
  return out;
}

// exp(-2 pi i m / L) with the angle reduced exactly
static cd unit_root(long m, long L) {
  m %= L;
  if (m < 0) m += L;
  const double x = 2.0 * double(m) / double(L);  // angle = pi x
  double s, c;
  sincospi(x, &s, &c);
  return cd(c, -s);
}

static void host_fft(std::vector<cd>& a, bool inverse) {  // natural order, radix-2 (any length: direct sum)
  const size_t n = a.size();
  if (n & (n - 1)) {
    // a length 2^a 5^b: the plain DFT, every angle reduced exactly (O(n^2), plan time only)
    std::vector<cd> out(n);
    for (size_t j = 0; j < n; ++j) {
      cd acc(0.0, 0.0);
      for (size_t l = 0; l < n; ++l) {
        cd w = unit_root((long)((j * l) % n), (long)n);
        if (inverse) w = std::conj(w);
        acc += a[l] * w;
      }
      out[j] = acc;
    }
    a.swap(out);
    return;
  }
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= n; len <<= 1) {
    for (size_t i = 0; i < n; i += len)
      for (size_t j = 0; j < len / 2; ++j) {
        cd w = unit_root((long)j, (long)len);
        if (inverse) w = std::conj(w);
        cd u = a[i + j], t = a[i + j + len / 2] * w;
        a[i + j] = u + t;
        a[i + j + len / 2] = u - t;
      }
  }
}

static void eigenvalues(int k, double alpha, double kappa, int N, pint_eig_variant eig,
                        const std::vector<double>& omega, std::vector<cd>& g) {
  g.assign(N, cd(0.0, 0.0));
  const double lk = std::log(kappa) / N;
  if (alpha == 1.0 || eig == PINT_EIG_CLOSED_FORM) {
    // g_j = delta_k(kappa^{1/N} e^{-2 pi i j / N})^alpha, 1 - z = -expm1(ln kappa / N - 2 pi i j / N)
    const double r = std::exp(lk);           // kappa^{1/N}
    const double om = -std::expm1(lk);       // 1 - kappa^{1/N}
    for (int j = 0; j < N; ++j) {
      // z = r e^{-i t}, t = 2 pi j / N;  1 - z = (1 - r) + r (1 - e^{-i t}),
      // 1 - e^{-i t} = 2 sin^2(t/2) + i sin t: both parts free of cancellation
      double sn, cs, sh, ch;
      sincospi(2.0 * double(j) / double(N), &sn, &cs);
      sincospi(double(j) / double(N), &sh, &ch);
      const cd one_minus_e(2.0 * sh * sh, sn);
      const cd s = om + r * one_minus_e;
      cd d = delta_from_s(k, s);
      if (alpha != 1.0) d = std::exp(alpha * std::log(d));
      g[j] = d;
    }
    return;
  }
  // truncated kappa-circulant of eq. (3.11): DFT of c_l = kappa^{l/N} omega_l, l < N
  std::vector<cd> c(N);
  for (int l = 0; l < N; ++l) c[l] = std::exp(lk * l) * omega[l];
  host_fft(c, false);
  g = c;
}

}  // namespace pint

using namespace pint;

namespace {
// The last batch graph, reused while the same plans, arrays, tol and max_sweeps come back.
struct BatchCache {
  std::mutex mu;
  std::vector<const void*> key;
  double tol = 0.0;
  int max_sweeps = 0;
  cudaGraphExec_t exec = nullptr;
} g_batch;
}  // namespace

#define PINT_CUDA_B(call)                                      \
  do {                                                         \
    cudaError_t _e = (call);                                   \
    if (_e != cudaSuccess) return bail(cuda_fail(_e, #call));  \
  } while (0)

namespace {

bool pow2(long x) { return x > 0 && (x & (x - 1)) == 0; }

template <typename X> pint_status dalloc(pint_plan p, X** ptr, size_t count) {
  void* q = nullptr;
  if (p->alloc) {
    q = p->alloc->alloc(count * sizeof(X));
    if (!q) return fail(PINT_ENOMEM, "device memory budget exhausted");
  } else {
    cudaError_t e = lib_malloc(&q, count * sizeof(X));
    if (e != cudaSuccess) return fail(PINT_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  p->allocs.push_back(q);
  p->alloc_sizes.push_back(count * sizeof(X));
  p->bytes += count * sizeof(X);
  *ptr = reinterpret_cast<X*>(q);
  return PINT_OK;
}

template <typename X> pint_status upload(pint_plan p, X** ptr, const std::vector<X>& host) {
  pint_status s = dalloc(p, ptr, host.size());
  if (s != PINT_OK) return s;
  PINT_CUDA(cudaMemcpy(*ptr, host.data(), host.size() * sizeof(X), cudaMemcpyHostToDevice));
  return PINT_OK;
}

int pick_cols(size_t per_col_bytes, size_t budget, int cmax, int cmin) {
  int C = cmax;
  while (C > cmin && per_col_bytes * C > budget) C >>= 1;
  return C;
}

template <typename T>
pint_status build_tables(pint_plan p, DevTables<T>& t) {
  using V = typename c2<T>::t;
  const int N = p->N;
  auto tw_of = [](int L) {
    std::vector<V> w(L);
    for (int m = 0; m < L; ++m) {
      cd r = unit_root(m, L);
      w[m].x = (T)r.real();
      w[m].y = (T)r.imag();
    }
    return w;
  };
  std::vector<V> tw = tw_of(N);
  pint_status s;
  V* dtw;
  if ((s = upload(p, &dtw, tw)) != PINT_OK) return s;
  t.tw_time = dtw;
  std::vector<T> sc(N), isc(N);
  const double lk = std::log(p->kappa) / N;
  for (int i = 0; i < N; ++i) {
    sc[i] = (T)std::exp(lk * i);
    isc[i] = (T)(std::exp(-lk * i) / N);
  }
  if ((s = upload(p, &t.s, sc)) != PINT_OK) return s;
  if ((s = upload(p, &t.inv_s, isc)) != PINT_OK) return s;
  std::vector<V> sig(N / 2 + 1);
  const double ta = std::pow(p->tau, -p->alpha);
  for (int j = 0; j <= N / 2; ++j) {
    sig[j].x = (T)(p->g[j].real() * ta);
    sig[j].y = (T)(p->g[j].imag() * ta);
  }
  V* dsig;
  if ((s = upload(p, &dsig, sig)) != PINT_OK) return s;
  t.sigma = dsig;
  // eigenvalues of the discrete Laplacian on sin(q pi x): (4/h^2) sin^2(q pi h/2) (FD stencil),
  // (4/h) sin^2(q pi h/2) (P1 stiffness); P1 mass: (h/3)(2 + cos(q pi h))
  const bool fem = p->fem;
  auto lam_of = [fem](int m) {
    std::vector<T> l(m);
    const double h = 1.0 / (m + 1);
    for (int q = 1; q <= m; ++q) {
      double sn, cs;
      sincospi(0.5 * q * h, &sn, &cs);
      l[q - 1] = (T)((fem ? 4.0 / h : 4.0 / (h * h)) * sn * sn);
    }
    return l;
  };
  auto mu_of = [](int m) {
    std::vector<T> u(m);
    const double h = 1.0 / (m + 1);
    for (int q = 1; q <= m; ++q) {
      double sn, cs;
      sincospi((double)q * h, &sn, &cs);
      u[q - 1] = (T)(h / 3.0 * (2.0 + cs));
    }
    return u;
  };
  // periodic axis of m points: eigenvalues (4 m^2) sin^2(pi q/m), q = 0..m-1, m-point twiddles
  auto lam_per = [](int m) {
    std::vector<T> l(m);
    for (int q = 0; q < m; ++q) {
      double sn, cs;
      sincospi((double)q / m, &sn, &cs);
      l[q] = (T)(4.0 * m * (double)m * sn * sn);
    }
    return l;
  };
  const bool per = p->periodic;
  std::vector<V> twx = tw_of(per ? p->mx : 2 * (p->mx + 1));
  V* dtwx;
  if ((s = upload(p, &dtwx, twx)) != PINT_OK) return s;
  t.tw_x = dtwx;
  if ((s = upload(p, &t.lam_x, per ? lam_per(p->mx) : lam_of(p->mx))) != PINT_OK) return s;
  if (fem && (s = upload(p, &t.mu_x, mu_of(p->mx))) != PINT_OK) return s;
  if (p->dim >= 2) {
    std::vector<V> twy = tw_of(per ? p->my : 2 * (p->my + 1));
    V* dtwy;
    if ((s = upload(p, &dtwy, twy)) != PINT_OK) return s;
    t.tw_y = dtwy;
    if ((s = upload(p, &t.lam_y, per ? lam_per(p->my) : lam_of(p->my))) != PINT_OK) return s;
  }
  if (p->dim == 3) {
    std::vector<V> twz = tw_of(2 * (p->mz + 1));
    V* dtwz;
    if ((s = upload(p, &dtwz, twz)) != PINT_OK) return s;
    t.tw_z = dtwz;
    if ((s = upload(p, &t.lam_z, lam_of(p->mz))) != PINT_OK) return s;
    // z lines are indexed by the (x, y) mode pair: lambda_x + lambda_y per line
    const std::vector<T> lx = lam_of(p->mx), ly = lam_of(p->my);
    std::vector<T> lxy((size_t)p->mx * p->my);
    for (int y = 0; y < p->my; ++y)
      for (int x = 0; x < p->mx; ++x) lxy[(size_t)y * p->mx + x] = lx[x] + ly[y];
    if ((s = upload(p, &t.lam_xy, lxy)) != PINT_OK) return s;
  }
  return PINT_OK;
}

pint_status validate(int k, double alpha, double kappa, double tau, int N, const pint_grid* g, int space) {
  if (!g) return fail(PINT_EINVAL, "grid is NULL");
  if (k < 1 || k > kMaxK) return fail(PINT_EINVAL, "k must be in 1..6");
  if (!(alpha > 0.0 && alpha <= 1.0)) return fail(PINT_EINVAL, "alpha must be in (0, 1]");
  if (!(kappa > 0.0 && kappa < 1.0)) return fail(PINT_EINVAL, "kappa must be in (0, 1)");
  if (!(tau > 0.0) || !std::isfinite(tau)) return fail(PINT_EINVAL, "tau must be positive");
  if (g->dim < 1 || g->dim > 3) return fail(PINT_EINVAL, "grid.dim must be 1, 2 or 3");
  // lengths of the FFTs: powers of two everywhere; 2^a 5^b (a >= 1) for Dirichlet finite differences
  // and P1 elements in 1D and 2D (the paper's N = 100 and h = 1/1000 are of that form)
  const bool mixed_ok = g->dim <= 2 && space != PINT_SPACE_PERIODIC;
  auto len_ok = [mixed_ok](long L) { return pow2(L) || (mixed_ok && fft_len_ok((int)L) && L % 2 == 0); };
  if (!len_ok(N) || N < 8 || N > 4096)
    return fail(PINT_EINVAL, "N must be in [8, 4096], a power of two (or 2^a 5^b, a >= 1, for Dirichlet 1D/2D grids)");
  if (alpha != 1.0 && N > 2048) return fail(PINT_EINVAL, "CQ (alpha < 1) supports N <= 2048");
  if (N <= k) return fail(PINT_EINVAL, "N must exceed k");
  if (g->dim == 3 && space != PINT_SPACE_FD) return fail(PINT_EINVAL, "3D grids are supported with finite differences");
  if (space == PINT_SPACE_PERIODIC) {
    if (!pow2(g->mx) || g->mx < 8 || g->mx > 4096) return fail(PINT_EINVAL, "periodic: mx must be a power of two in [8, 4096]");
    if (g->dim == 2 && (!pow2(g->my) || g->my < 8 || g->my > 4096))
      return fail(PINT_EINVAL, "periodic: my must be a power of two in [8, 4096]");
    return PINT_OK;
  }
  if (!len_ok(g->mx + 1) || g->mx < 3 || g->mx > 2047)
    return fail(PINT_EINVAL, "mx + 1 must be a power of two (or 2^a 5^b in 1D/2D), 3 <= mx <= 2047");
  if (g->dim >= 2 && (!len_ok(g->my + 1) || g->my < 3 || g->my > 2047))
    return fail(PINT_EINVAL, "my + 1 must be a power of two (or 2^a 5^b in 2D), 3 <= my <= 2047");
  if (g->dim == 3 && (!pow2(g->mz + 1) || g->mz < 3 || g->mz > 2047))
    return fail(PINT_EINVAL, "mz + 1 must be a power of two, 3 <= mz <= 2047");
  return PINT_OK;
}

void destroy_plan(pint_plan p) {
  if (!p) return;
  host_stage_free(p);
  for (SolveGraph& c : p->sg)
    if (c.exec) cudaGraphExecDestroy(c.exec);
  if (p->cap) cudaStreamDestroy(p->cap);
  for (size_t i = 0; i < p->allocs.size(); ++i) {
    if (p->alloc) p->alloc->release(p->allocs[i]);
    else lib_free(p->allocs[i], p->alloc_sizes[i]);
  }
  if (p->alloc) {
    if (p->h_norms) p->alloc->host_release(p->h_norms);
    if (p->h_ctl) p->alloc->host_release(p->h_ctl);
    if (p->nl_h) p->alloc->host_release(p->nl_h);
  } else {
    if (p->h_norms) lib_free_host(p->h_norms);
    if (p->h_ctl) lib_free_host(p->h_ctl);
    if (p->nl_h) lib_free_host(p->nl_h);
  }
  delete p;
}

}  // namespace

namespace {
pint_status autotune_ysolve(pint_plan p);
pint_status autotune_xdst(pint_plan p);
// the tensor-core x sine transform serves lines of 255 or 127 points of FP32 inner solves (2D /
// 3D, Dirichlet finite differences)
bool dst_tc_applies(pint_plan p) {
  return dst_tc_line_ok(p->mx) && (p->dim == 2 || p->dim == 3) && !p->periodic && !p->fem && p->prec != PINT_FP64;
}
// ... and the y sine transforms of 3D grids with lines of 127 points (strided: the columns of
// the (j, z) planes)
bool dst_tc_y_applies(pint_plan p) {
  return p->dim == 3 && p->my == 127 && !p->periodic && !p->fem && p->prec != PINT_FP64;
}
// ... and the z solves of 3D grids with lines of 127 points (mz = 127)
bool dst_tc_z_applies(pint_plan p) {
  return p->dim == 3 && p->mz == 127 && !p->periodic && !p->fem && p->prec != PINT_FP64;
}
// the matrix image of a line length (255 or 127), built once per process
const std::vector<unsigned short>& dst_tc_image(int n) {
  static std::once_flag once[2];
  static std::vector<unsigned short> img[2];
  const int which = n == 255 ? 0 : 1;
  std::call_once(once[which], [which] {
    const int len = which == 0 ? 255 : 127;
    img[which].resize(dst_tc_table_bytes(len) / 2);
    dst_tc_table(len, img[which].data());
  });
  return img[which];
}
pint_status tune_time_tiles(pint_plan p, int cmax_t, int cmax_z);
pint_status tune_radix(pint_plan p);
}

extern "C" pint_status pint_plan_create_desc(const pint_plan_desc* d, pint_plan* out) {
  return plan_create_internal(d, nullptr, out);
}

pint_status pint::plan_create_internal(const pint_plan_desc* d, DevAllocator* A, pint_plan* out) {
  if (!d || !out) return fail(PINT_EINVAL, "NULL argument");
  pint_status s = validate(d->k, d->alpha, d->kappa, d->tau, d->N, &d->grid, d->space);
  if (s != PINT_OK) return s;
  if (d->precision < PINT_FP64 || d->precision > PINT_FP32) return fail(PINT_EINVAL, "bad precision");
  if (d->eig != PINT_EIG_TRUNC_DFT && d->eig != PINT_EIG_CLOSED_FORM) return fail(PINT_EINVAL, "bad eig variant");
  if (d->eig == PINT_EIG_CLOSED_FORM && d->alpha != 1.0 && d->precision != PINT_MIXED)
    return fail(PINT_EINVAL, "CLOSED_FORM eigenvalues with alpha < 1 need the residual form (PINT_MIXED)");
  if (d->ysolve < 0 || d->ysolve > 4) return fail(PINT_EINVAL, "bad ysolve variant");
  if (d->xdst < 0 || d->xdst > 3) return fail(PINT_EINVAL, "bad xdst variant");
  if (d->space != PINT_SPACE_FD && d->space != PINT_SPACE_FEM_P1 && d->space != PINT_SPACE_PERIODIC)
    return fail(PINT_EINVAL, "bad space discretisation");
  if (d->space == PINT_SPACE_FEM_P1 && d->grid.dim != 1)
    return fail(PINT_EINVAL, "P1 finite elements are supported in 1D");
  pint_plan p = new pint_plan_s();
  p->alloc = A;
  p->k = d->k; p->alpha = d->alpha; p->kappa = d->kappa; p->tau = d->tau; p->N = d->N;
  p->dim = d->grid.dim; p->mx = d->grid.mx; p->my = d->grid.dim >= 2 ? d->grid.my : 1;
  p->mz = d->grid.dim == 3 ? d->grid.mz : 1;
  p->M = p->mx * p->my * p->mz;
  p->prec = d->precision; p->eig = d->eig;
  p->cq = d->alpha != 1.0;
  p->fem = d->space == PINT_SPACE_FEM_P1;
  p->periodic = d->space == PINT_SPACE_PERIODIC;
  const int N = p->N, M = p->M;
  p->omega.resize(N);
  time_weights(p->k, p->alpha, N, p->omega.data());
  table1(p->k, p->a, p->b);
  eigenvalues(p->k, p->alpha, p->kappa, N, p->eig, p->omega, p->g);
  // mesh widths: 1/(m+1) for Dirichlet nodes, 1/m on a periodic axis
  const double hx = p->periodic ? 1.0 / p->mx : 1.0 / (p->mx + 1);
  const double hy = p->periodic ? 1.0 / p->my : 1.0 / (p->my + 1);
  // off-diagonal weight of the discrete Laplacian: 1/h^2 (FD stencil), 1/h (P1 stiffness)
  // (as the integers 1/h and 1/h^2, below 2^24: exact in FP32 as well)
  const double ix = p->periodic ? p->mx : p->mx + 1, iy = p->periodic ? p->my : p->my + 1;
  p->gx = p->fem ? ix : ix * ix;
  p->gy = p->dim >= 2 ? iy * iy : 0.0;
  p->gz = p->dim == 3 ? (double)(p->mz + 1) * (p->mz + 1) : 0.0;

  auto bail = [&](pint_status st) { destroy_plan(p); return st; };

  // tables
  if (p->prec == PINT_FP64) {
    if ((s = build_tables(p, p->td)) != PINT_OK) return bail(s);
  } else {
    if ((s = build_tables(p, p->tf)) != PINT_OK) return bail(s);
  }
  const double ta = std::pow(p->tau, -p->alpha);
  std::vector<double> beta(N);
  double cs = 0.0;
  for (int i = 0; i < N; ++i) {
    cs += p->omega[i];
    // BDF-k (alpha = 1): sum_{j<=i} omega_j = delta_k(1) = 0 exactly once i >= k
    beta[i] = (p->alpha == 1.0 && i >= p->k) ? 0.0 : ta * cs;
  }
  if ((s = upload(p, &p->beta, beta)) != PINT_OK) return bail(s);
  if (p->prec == PINT_MIXED) {
    std::vector<float2> bff(N);
    for (int i = 0; i < N; ++i) {
      bff[i].x = (float)beta[i];
      bff[i].y = (float)(beta[i] - (double)bff[i].x);
    }
    if ((s = upload(p, &p->beta_ff, bff)) != PINT_OK) return bail(s);
  }
  if (p->cq) {
    const int L = 2 * N;
    std::vector<double2> tw(L);
    for (int m = 0; m < L; ++m) {
      cd r = unit_root(m, L);
      tw[m] = make_double2(r.real(), r.imag());
    }
    if ((s = upload(p, &p->tw_2n, tw)) != PINT_OK) return bail(s);
    std::vector<cd> w(L, cd(0.0, 0.0));
    for (int i = 0; i < N; ++i) w[i] = p->omega[i];
    host_fft(w, false);
    std::vector<double2> lo(L), up(L);
    for (int j = 0; j < L; ++j) {
      const int pos = fft_pos(j, L);
      const cd vlo = w[j] * (ta / L), vup = w[j] * (p->kappa * ta / L);
      lo[pos] = make_double2(vlo.real(), vlo.imag());
      up[pos] = make_double2(vup.real(), vup.imag());
    }
    if ((s = upload(p, &p->what_lo, lo)) != PINT_OK) return bail(s);
    if ((s = upload(p, &p->what_up, up)) != PINT_OK) return bail(s);
    if (p->prec == PINT_MIXED) {
      // double-float tables for the MIXED history product (FFT radix <= 8 ordering)
      auto split = [](double x, float& h, float& l) {
        h = (float)x;
        l = (float)(x - (double)h);
      };
      std::vector<float4> wff(L), tff(L);
      for (int j = 0; j < L; ++j) {
        const int pos = fft_pos(j, L, kToepFFMaxLog);
        const cd vlo = w[j] * (ta / L);
        float4 q;
        split(vlo.real(), q.x, q.y);
        split(vlo.imag(), q.z, q.w);
        wff[pos] = q;
        const cd r = unit_root(j, L);
        split(r.real(), q.x, q.y);
        split(r.imag(), q.z, q.w);
        tff[j] = q;
      }
      if ((s = upload(p, &p->what_ff, wff)) != PINT_OK) return bail(s);
      if ((s = upload(p, &p->tw_ff, tff)) != PINT_OK) return bail(s);
    }
    if ((s = dalloc(p, &p->z, (size_t)N * M)) != PINT_OK) return bail(s);
  }
  // workspaces
  const size_t NM = (size_t)N * M, JM = (size_t)(N / 2 + 1) * M;
  if (p->prec == PINT_MIXED) {
    if ((s = dalloc(p, &p->Uff, NM)) != PINT_OK) return bail(s);
    if (p->alpha == 1.0) {
      // BDF-k: F_hat = f exactly beyond the first k levels (the corrections act on levels < k - 1
      // and beta_n = 0 from level k on), so a solve from f needs F_hat itself on k levels only
      p->kc = p->k < N ? p->k : N;
      if ((s = dalloc(p, &p->fcorr, (size_t)p->kc * M)) != PINT_OK) return bail(s);
    }
  } else if (p->prec == PINT_FP32) {
    if ((s = dalloc(p, &p->Uhi, NM)) != PINT_OK) return bail(s);
    if ((s = dalloc(p, &p->Fhi, NM)) != PINT_OK) return bail(s);
  }
  {
    const size_t esz = p->prec == PINT_FP64 ? sizeof(double2) : sizeof(float2);
    unsigned char* S;
    if ((s = dalloc(p, &S, JM * esz)) != PINT_OK) return bail(s);
    p->S = S;
  }
  if ((s = dalloc(p, &p->norms, 2)) != PINT_OK) return bail(s);
  if ((s = dalloc(p, &p->ctl, 1)) != PINT_OK) return bail(s);
  if (p->alloc) {
    p->h_norms = (double*)p->alloc->host_alloc(2 * sizeof(double));
    p->h_ctl = (SolveCtl*)p->alloc->host_alloc(sizeof(SolveCtl));
    if (!p->h_norms || !p->h_ctl) return bail(fail(PINT_ENOMEM, "pinned host buffer"));
  } else {
    void* hn = nullptr;
    void* hc = nullptr;
    if (lib_malloc_host(&hn, 2 * sizeof(double)) != cudaSuccess) return bail(fail(PINT_ENOMEM, "cudaMallocHost"));
    p->h_norms = (double*)hn;
    if (lib_malloc_host(&hc, sizeof(SolveCtl)) != cudaSuccess) return bail(fail(PINT_ENOMEM, "cudaMallocHost"));
    p->h_ctl = (SolveCtl*)hc;
  }
  PINT_CUDA_B(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));

  // tile widths (columns per CTA): limited by ~96 KB of shared memory, and narrow enough that
  // the M points of a problem still give two CTAs per SM (small M: many narrow tiles rather
  // than a few wide ones)
  const size_t budget = 96 * 1024;
  int occ = 1;
  while (occ < 32 && (size_t)M / (size_t)(4 * occ) >= 2 * 152) occ *= 2;
  p->Ct = std::min(pick_cols((size_t)N * sizeof(float2), budget, 32, 1), occ);
  p->Cr = std::min(p->Ct, 16);
  p->Ci = p->Cr;
  p->Ctd = std::min(pick_cols((size_t)N * (p->prec == PINT_FP64 ? sizeof(double2) : sizeof(float2)), budget, 32, 1), occ);
  p->Cz = std::min(pick_cols((size_t)2 * N * sizeof(double2), 160 * 1024, 16, 1), occ);
  const size_t ve = p->prec == PINT_FP64 ? sizeof(double2) : sizeof(float2);
  // sine-transform tiles: up to 64 KB of extended lines (16 lines of 512 FP32 complex points),
  // three CTAs per SM
  p->Cx = pick_cols((size_t)2 * (p->mx + 1) * ve, 64 * 1024, 16, 1);
  p->Cy = pick_cols((size_t)2 * (p->my + 1) * ve, 64 * 1024, 16, 1);
  if (p->periodic) {
    // periodic lines of m points; m * C within the registers of the in-tile reordering
    const size_t rlim = (p->prec == PINT_FP64 ? 8 : 16) * (size_t)kThreads;
    auto pc = [&](int m) {
      int C = pick_cols((size_t)m * ve, 64 * 1024, 16, 1);
      while (C > 1 && (size_t)m * C > rlim) C >>= 1;
      return C;
    };
    p->Cx = pc(p->mx);
    p->Cy = pc(p->my);
  }
  p->Czl = pick_cols((size_t)2 * (p->mz + 1) * ve, 64 * 1024, 16, 1);
  p->Ctri = pick_cols((size_t)p->my * sizeof(float2), 72 * 1024, 32, 1);
  PINT_CUDA_B(cudaMemset(p->S, 0, JM * (p->prec == PINT_FP64 ? sizeof(double2) : sizeof(float2))));
  PINT_CUDA_B(cudaMemset(p->ctl, 0, sizeof(SolveCtl)));
  p->xdst = 1;
  // default (0): the tensor-core transform where it applies and there are enough lines to fill
  // the GPU: at least 16384 lines of 255 points (~3.4 tiles of 32 per SM) or 8192 lines of 127
  // points (~0.8 tiles of 64 per SM). Measured per launch: below 4096 lines both FFT forms are
  // ahead (their four CTAs per SM start faster than the tensor-core pipeline fills), from 4096 to
  // 16384 lines of 255 points the two are within 4%, and from 8192 lines of 127 points on the
  // tensor cores win (1.2x there, 1.8x at 130K lines in 2D, 2x in 3D)
  const long long xlines = (long long)(N / 2 + 1) * p->my * p->mz;
  const bool tc_default = d->xdst == 0 && xlines >= (p->mx == 255 ? 16384 : 8192);
  if (dst_tc_applies(p) && (d->xdst >= 2 || tc_default)) {
    if ((s = upload(p, &p->dst_tab, dst_tc_image(p->mx))) != PINT_OK) return bail(s);
    p->xdst = 2;
    if (d->xdst == 3 && (s = autotune_xdst(p)) != PINT_OK) return bail(s);
  }
  // the y transforms of 3D grids (my = 127) on the tensor cores under the same switch: 2 always,
  // 0 and 3 from 8192 lines ((N/2 + 1) mx mz), 1 never
  p->ydst = 1;
  const long long ylines = (long long)(N / 2 + 1) * p->mx * p->mz;
  if (dst_tc_y_applies(p) && d->xdst != 1 && (d->xdst == 2 || ylines >= 8192)) {
    if ((s = upload(p, &p->dst_tab_y, dst_tc_image(127))) != PINT_OK) return bail(s);
    p->ydst = 2;
  }
  // the z solves (mz = 127) on the tensor cores only when asked for (xdst = 2): two passes per tile
  // around the divide measured slower than the FFT form on a 127^3, N = 128 grid (1283 against
  // 1181 us per launch); one image for y and z
  p->zsolve = 1;
  if (dst_tc_z_applies(p) && d->xdst == 2) {
    if (!p->dst_tab_y && (s = upload(p, &p->dst_tab_y, dst_tc_image(127))) != PINT_OK) return bail(s);
    p->zsolve = 2;
  }
  p->ysolve = 1;
  if (p->dim == 2 && p->prec != PINT_FP64 && !p->periodic) {
    if (d->ysolve == 2) p->ysolve = 2;
    else if (d->ysolve == 4 && p->my <= 1024) p->ysolve = 4;
    else if (d->ysolve == 3 && (s = autotune_ysolve(p)) != PINT_OK) return bail(s);
  }
  {
    // Inner-solve accuracy bounds the per-sweep contraction from below: rounding of size
    // eps * ||r|| in the transforms is amplified by the spread of the shifted spectrum
    // (max over min of |g_j tau^-alpha + lambda|) and by the kappa^{-1} unscaling.
    const double hx = 1.0 / (p->mx + 1), hy = 1.0 / (p->my + 1);
    double lmin = 4.0 / (hx * hx) * std::pow(std::sin(M_PI * hx / 2), 2);
    double lmax = 4.0 / (hx * hx);
    if (p->fem) {
      // generalized eigenvalues (stiffness over mass) of the P1 pencil, q = 1 and q = mx
      lmin = 12.0 / (hx * hx) * std::pow(std::sin(M_PI * hx / 2), 2) / (2.0 + std::cos(M_PI * hx));
      lmax = 12.0 / (hx * hx) * std::pow(std::sin(M_PI * hx * p->mx / 2), 2) / (2.0 + std::cos(M_PI * hx * p->mx));
    }
    if (p->dim >= 2) {
      lmin += 4.0 / (hy * hy) * std::pow(std::sin(M_PI * hy / 2), 2);
      lmax += 4.0 / (hy * hy);
    }
    if (p->dim == 3) {
      const double hz = 1.0 / (p->mz + 1);
      lmin += 4.0 / (hz * hz) * std::pow(std::sin(M_PI * hz / 2), 2);
      lmax += 4.0 / (hz * hz);
    }
    if (p->periodic) {
      // circulant Laplacian: the constant mode has eigenvalue 0, the largest is 4/h^2 per axis
      lmin = 0.0;
      lmax = 4.0 * p->mx * (double)p->mx + (p->dim == 2 ? 4.0 * p->my * (double)p->my : 0.0);
    }
    const double ta = std::pow(p->tau, -p->alpha);
    double smax = 0.0, dmin = 1e300;
    for (int j = 0; j <= N / 2; ++j) {
      const cd sg = p->g[j] * ta;
      smax = std::max(smax, std::abs(sg));
      dmin = std::min(dmin, std::abs(sg + lmin));
    }
    const double eps = p->prec == PINT_FP64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
    p->q_floor = std::min(0.5, eps * (lmax + smax) / dmin / p->kappa);
    if (p->periodic) {
      // the constant mode (lambda = 0) is not damped in time: its WR contraction is
      // kappa / (1 - kappa) (the k = 1 closed form kappa r^N / (1 - kappa r^N) at r = 1), a rate
      // the observed update ratios of the first sweeps can underestimate
      p->q_floor = std::max(p->q_floor, std::min(0.99, p->kappa / (1.0 - p->kappa)));
    }
  }
  {
    // Few points (the occupancy rule narrowed the time tiles below what shared memory allows):
    // the best width depends on the kernel (threads per FFT pass against CTAs per SM), so time
    // each MIXED time kernel at the admissible widths and keep the fastest (plans created through
    // the public entry points; server plans keep the rule).
    const int cmax_t = std::min(pick_cols((size_t)N * sizeof(float2), budget, 32, 1), 16);
    const int cmax_z = pick_cols((size_t)2 * N * sizeof(double2), 160 * 1024, 16, 1);
    // (below 2^18 space-time unknowns launch latency dominates and the timings carry no signal)
    if (!A && p->prec == PINT_MIXED && occ < cmax_t && (size_t)N * M >= ((size_t)1 << 18) &&
        (s = tune_time_tiles(p, cmax_t, cmax_z)) != PINT_OK)
      return bail(s);
    // the radix schedule of time FFTs without a compiled shape (at the widths now fixed)
    if (!A && p->prec == PINT_MIXED && (size_t)N * M >= ((size_t)1 << 18) &&
        (!compiled_time_fft_shape(N, p->Cr) || !compiled_update_shape(N, p->Ci)) &&
        (s = tune_radix(p)) != PINT_OK)
      return bail(s);
  }
  {
    // Small 1D problems (finite differences, Dirichlet, BDF-k, MIXED): the whole solve in one CTA
    // whose iterate and tiles fit in shared memory; launch and memory latency dominate the
    // multi-kernel sweep there. One SM's issue rate bounds the one-CTA solve, so it is kept to
    // problems of up to 4096 space-time unknowns (the 1D heat problem of 63 points and 64
    // levels: 0.108 -> 0.082 ms per step).
    // (Cs lines per batch of the spatial step: a power of two dividing N/2, at most 64)
    const int Ct = (p->mx + 1) / 2, L = 2 * (p->mx + 1);
    int Cs = std::min(N / 2, 64);
    if (p->prec == PINT_MIXED && p->dim == 1 && !p->fem && !p->periodic && !p->cq && Ct >= 2 &&
        (size_t)N * M <= 4096 && pow2(N) && pow2(p->mx + 1)) {
      for (; Cs >= 4; Cs /= 2) {
        if (small_smem(N, M, Ct, L, Cs) <= 200 * 1024) {
          p->small = true;
          p->small_Ct = Ct;
          p->small_Cs = Cs;
          break;
        }
      }
    }
  }
  *out = p;
  return PINT_OK;
}

extern "C" pint_status pint_plan_create(int k, double alpha, double kappa, double tau, int N,
                                        const pint_grid* grid, pint_precision precision, pint_plan* out) {
  if (!grid) return fail(PINT_EINVAL, "grid is NULL");
  pint_plan_desc d{};
  d.k = k; d.alpha = alpha; d.kappa = kappa; d.tau = tau; d.N = N; d.grid = *grid;
  d.precision = precision; d.eig = PINT_EIG_TRUNC_DFT; d.ysolve = 0;
  return pint_plan_create_desc(&d, out);
}

extern "C" pint_status pint_plan_destroy(pint_plan p) {
  if (!p) return PINT_OK;
  {
    std::lock_guard<std::mutex> lk(g_batch.mu);
    if (g_batch.exec && std::find(g_batch.key.begin(), g_batch.key.end(), (const void*)p) != g_batch.key.end()) {
      cudaGraphExecDestroy(g_batch.exec);
      g_batch.exec = nullptr;
      g_batch.key.clear();
    }
  }
  cudaDeviceSynchronize();
  destroy_plan(p);
  return PINT_OK;
}

extern "C" size_t pint_plan_workspace_bytes(pint_plan p) { return p ? p->bytes : 0; }

namespace {
pint_status nl_alloc_fd(pint_plan p);
double react_weight(pint_plan p);
// F_hat with the starting correction a_n (f(0) - A v - w c v - w g(v)): the reaction term when one
// is installed, the nonlinearity when g is given (the rows of fderiv are then copied with f(0)
// replaced first)
// head_levels > 0: Fhat receives the first head_levels levels of F_hat only (pitch M)
pint_status form_rhs(pint_plan p, const double* v, const double* f, const double* fderiv, double* Fhat,
                     cudaStream_t st, const NlPoly* g, int head_levels = 0) {
  if (!p || !v || !f || !Fhat) return fail(PINT_EINVAL, "NULL argument");
  if (p->k >= 2 && !fderiv) return fail(PINT_EINVAL, "fderiv is required for k >= 2");
  if (p->k >= 2 && (g || p->react_on)) {
    pint_status s = nl_alloc_fd(p);
    if (s != PINT_OK) return s;
    NlPoly zero{};
    cudaError_t e = launch_nl_fd0(fderiv, v, g ? *g : zero, react_weight(p), p->react_on ? p->react : nullptr,
                                  p->k - 1, p->M, p->nl_fd, st);
    if (e != cudaSuccess) return cuda_fail(e, "source correction kernel");
    fderiv = p->nl_fd;
  }
  RhsArgs a{};
  a.v = v; a.f = f; a.fd = fderiv; a.F = Fhat; a.beta = p->beta;
  a.N = p->N; a.M = p->M; a.mx = p->mx; a.dim = p->dim; a.k = p->k;
  a.gx = p->gx; a.gy = p->gy; a.gz = p->gz; a.my = p->my;
  a.fem = p->fem ? 1 : 0;
  a.mass6 = 1.0 / (6.0 * (p->mx + 1));  // h/6
  a.periodic = p->periodic ? 1 : 0;
  for (int n = 0; n < kMaxK - 1; ++n) {
    a.a[n] = n < 5 ? p->a[n] : 0.0;
    for (int l = 1; l <= 4; ++l) a.bt[l][n] = p->b[l - 1][n] * std::pow(p->tau, l);
  }
  if (head_levels > 0) {
    a.N = head_levels;
    a.head = 1;
  }
  cudaError_t e = launch_rhs(a, st);
  if (e != cudaSuccess) return cuda_fail(e, "rhs kernel");
  return PINT_OK;
}
}  // namespace

extern "C" pint_status pint_form_rhs(pint_plan p, const double* v, const double* f, const double* fderiv,
                                     double* Fhat, void* stream) {
  return form_rhs(p, v, f, fderiv, Fhat, (cudaStream_t)stream, nullptr);
}

extern "C" pint_status pint_form_rhs_window(pint_plan p, const double* f, const double* U_prev, double* Fhat,
                                            void* stream) {
  if (!p || !f || !U_prev || !Fhat) return fail(PINT_EINVAL, "NULL argument");
  if (p->cq) return fail(PINT_EINVAL, "time windows need alpha = 1 (the CQ history reaches every earlier window)");
  if (p->react_on) return fail(PINT_EINVAL, "a reaction term is installed (pint_set_reaction(plan, NULL) removes it)");
  WinCoef c{};
  for (int j = 0; j <= p->k; ++j) c.c[j] = p->omega[j] / p->tau;
  cudaError_t e = launch_window_rhs(f, U_prev, Fhat, p->N, p->N, p->M, p->k, c, p->fem ? 1 : 0,
                                    1.0 / (6.0 * (p->mx + 1)), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "window rhs kernel");
  return PINT_OK;
}

extern "C" pint_status pint_initial_guess(pint_plan p, const double* v, double* U, void* stream) {
  if (!p || !v || !U) return fail(PINT_EINVAL, "NULL argument");
  cudaError_t e = launch_bcast_d(v, U, p->N, p->M, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "initial guess kernel");
  return PINT_OK;
}

namespace {

void split_ff(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

template <typename T> bool ysolve_tri(pint_plan p) { return sizeof(T) == 4 && (p->ysolve == 2 || p->ysolve == 4); }

// x sine transform (AxisArgs op 0) of `lines` lines: the odd-sequence FFT, or for FP32 lines of
// 255 or 127 points on a plan that selected it, the tensor-core products
template <typename T> cudaError_t xform_x(pint_plan p, const AxisArgs<T>& ax, cudaStream_t st) {
  if (sizeof(T) == 4 && p->xdst == 2) {
    DstTcArgs g{};
    g.S = reinterpret_cast<float2*>(ax.S);
    g.tab = p->dst_tab;
    g.n = p->mx;
    g.lines = ax.lines;
    g.stride = 1;
    g.err = &p->ctl->err;
    return launch_dst_tc(g, st);
  }
  return launch_axis(ax, st);
}

// z solve (AxisArgs op 1, strided) of 3D grids: the odd-sequence FFTs around the divide, or for
// FP32 lines of 127 points on a plan that selected it, two tensor-core passes around it
template <typename T> cudaError_t solve_z3(pint_plan p, const AxisArgs<T>& az, cudaStream_t st) {
  if (sizeof(T) == 4 && p->zsolve == 2) {
    DstTcArgs g{};
    g.S = reinterpret_cast<float2*>(az.S);
    g.tab = p->dst_tab_y;
    g.n = 127;
    g.lines = az.lines;
    g.stride = az.P;
    g.err = &p->ctl->err;
    g.sigma = reinterpret_cast<const float2*>(az.sigma);
    g.lam_other = reinterpret_cast<const float*>(az.lam_other);
    g.lam_axis = reinterpret_cast<const float*>(az.lam_axis);
    g.scale = (float)az.scale;
    return launch_dst_tc(g, st);
  }
  return launch_axis(az, st);
}

// y sine transform (AxisArgs op 0, strided) of 3D grids: the odd-sequence FFT, or for FP32 lines of
// 127 points on a plan that selected it, the tensor-core products
template <typename T> cudaError_t xform_y3(pint_plan p, const AxisArgs<T>& ay, cudaStream_t st) {
  if (sizeof(T) == 4 && p->ydst == 2) {
    DstTcArgs g{};
    g.S = reinterpret_cast<float2*>(ay.S);
    g.tab = p->dst_tab_y;
    g.n = 127;
    g.lines = ay.lines;
    g.stride = ay.P;
    g.err = &p->ctl->err;
    return launch_dst_tc(g, st);
  }
  return launch_axis(ay, st);
}

// spatial step on the half spectrum for T (float: MIXED/FP32, double: FP64)
// mass and stiffness rows (diagonal, off-diagonal) of a 1D plan: finite differences (1, 0) and
// (2/h^2, -1/h^2); P1 elements (4h/6, h/6) and (2/h, -1/h)
void row_coefficients(pint_plan p, double& md, double& mo, double& kd, double& ko) {
  const double h = 1.0 / (p->mx + 1);
  md = p->fem ? 4.0 * h / 6.0 : 1.0;
  mo = p->fem ? h / 6.0 : 0.0;
  kd = 2.0 * p->gx;
  ko = -p->gx;
}

template <typename T>
cudaError_t spatial(pint_plan p, const DevTables<T>& t, cudaStream_t st) {
  const int J = p->N / 2 + 1;
  if (p->react_on) {
    // 1D with a reaction term: each frequency's tridiagonal system by its stored LU factors
    TriVarArgs<T> a{};
    a.S = p->S; a.ip = p->tri_ip; a.cp = p->tri_cp; a.sigma = t.sigma; a.n = p->mx; a.J = J;
    row_coefficients(p, a.md, a.mo, a.kd, a.ko);
    return launch_trivar_solve<T>(a, st);
  }
  if (p->periodic) {
    // FFT diagonalisation: 1D one fused solve; 2D forward FFT along x, fused solve along y,
    // inverse FFT along x (the 1/(mx my) normalisation in the solve's divisor)
    AxisArgs<T> a{};
    a.S = p->S; a.sigma = t.sigma;
    // row pitch C + 1 keeps multi-line tiles free of bank conflicts; a one-line tile needs none
    auto pitch = [](int C) { return C > 1 ? C + 1 : 1; };
    if (p->dim == 1) {
      a.n = p->mx; a.lines = J; a.mode = 0; a.P = 1; a.op = 1; a.lines_per_j = 1;
      a.lam_axis = t.lam_x; a.scale = (T)p->mx; a.tw = t.tw_x;
      a.C = p->Cx; a.logC = ilog2c(p->Cx); a.ld = pitch(p->Cx);
      return launch_axis_per(a, st);
    }
    AxisArgs<T> ax{};
    ax.S = p->S; ax.n = p->mx; ax.lines = J * p->my; ax.mode = 0; ax.P = 1; ax.op = 0;
    ax.lines_per_j = p->my; ax.tw = t.tw_x; ax.C = p->Cx; ax.logC = ilog2c(p->Cx); ax.ld = pitch(p->Cx);
    cudaError_t e = launch_axis_per(ax, st);
    if (e != cudaSuccess) return e;
    a.n = p->my; a.lines = J * p->mx; a.mode = 1; a.P = p->mx; a.op = 1; a.lines_per_j = p->mx;
    a.lam_axis = t.lam_y; a.lam_other = t.lam_x; a.scale = (T)((double)p->mx * p->my);
    a.tw = t.tw_y; a.C = p->Cy; a.logC = ilog2c(p->Cy); a.ld = pitch(p->Cy);
    if ((e = launch_axis_per(a, st)) != cudaSuccess) return e;
    ax.op = 2;
    return launch_axis_per(ax, st);
  }
  if (p->dim == 3) {
    // sine transforms along x and y, the shifted solve along z, the transforms back: five passes
    // over the half spectrum. Each transform without divide applies -2i D; two of them give
    // -2 (m+1) per axis, hence the z solve's divisor scale 8 (mx+1)(my+1)(mz+1).
    AxisArgs<T> ax{};
    ax.S = p->S; ax.n = p->mx; ax.lines = J * p->mz * p->my; ax.mode = 0; ax.P = 1; ax.op = 0;
    ax.lines_per_j = p->my * p->mz; ax.tw = t.tw_x; ax.C = p->Cx; ax.logC = ilog2c(p->Cx); ax.ld = p->Cx + 1;
    AxisArgs<T> ay{};  // y lines of every (j, z) plane: stride mx
    ay.S = p->S; ay.n = p->my; ay.lines = J * p->mz * p->mx; ay.mode = 1; ay.P = p->mx; ay.op = 0;
    ay.lines_per_j = p->mx; ay.tw = t.tw_y; ay.C = p->Cy; ay.logC = ilog2c(p->Cy); ay.ld = p->Cy + 1;
    AxisArgs<T> az{};  // z lines of every j: stride mx my, one line per (x, y) mode
    az.S = p->S; az.n = p->mz; az.lines = J * p->mx * p->my; az.mode = 1; az.P = p->mx * p->my; az.op = 1;
    az.sigma = t.sigma; az.lam_axis = t.lam_z; az.lam_other = t.lam_xy;
    az.scale = (T)(8.0 * (p->mx + 1) * (double)(p->my + 1) * (double)(p->mz + 1));
    az.lines_per_j = p->mx * p->my; az.tw = t.tw_z; az.C = p->Czl; az.logC = ilog2c(p->Czl); az.ld = p->Czl + 1;
    cudaError_t e;
    if ((e = xform_x(p, ax, st)) != cudaSuccess) return e;
    if ((e = xform_y3(p, ay, st)) != cudaSuccess) return e;
    if ((e = solve_z3(p, az, st)) != cudaSuccess) return e;
    if ((e = xform_y3(p, ay, st)) != cudaSuccess) return e;
    return xform_x(p, ax, st);
  }
  if (p->dim == 1) {
    AxisArgs<T> a{};
    a.S = p->S; a.n = p->mx; a.lines = J; a.mode = 0; a.P = 1; a.op = 1;
    a.sigma = t.sigma; a.lam_axis = t.lam_x; a.lam_other = nullptr; a.mu_axis = t.mu_x;
    a.scale = (T)(2.0 * (p->mx + 1)); a.lines_per_j = 1; a.tw = t.tw_x;
    a.C = p->Cx; a.logC = ilog2c(p->Cx); a.ld = p->Cx + 1;
    return launch_axis(a, st);
  }
  AxisArgs<T> ax{};
  ax.S = p->S; ax.n = p->mx; ax.lines = J * p->my; ax.mode = 0; ax.P = 1; ax.op = 0;
  ax.lines_per_j = p->my; ax.tw = t.tw_x; ax.C = p->Cx; ax.logC = ilog2c(p->Cx); ax.ld = p->Cx + 1;
  cudaError_t e = xform_x(p, ax, st);
  if (e != cudaSuccess) return e;
  if (ysolve_tri<T>(p)) {
    TriArgs tr{};
    tr.S = reinterpret_cast<float2*>(p->S); tr.n = p->my; tr.P = p->mx; tr.lines = J * p->mx;
    tr.sigma = reinterpret_cast<const float2*>(t.sigma); tr.lam_x = reinterpret_cast<const float*>(t.lam_x);
    tr.g = (float)p->gy; tr.scale = (float)(-0.5 / (p->mx + 1));
    tr.C = p->Ctri; tr.logC = ilog2c(p->Ctri);
    e = p->ysolve == 4 ? launch_pcr(tr, st) : launch_tri(tr, st);
  } else {
    AxisArgs<T> ay{};
    ay.S = p->S; ay.n = p->my; ay.lines = J * p->mx; ay.mode = 1; ay.P = p->mx; ay.op = 1;
    ay.sigma = t.sigma; ay.lam_axis = t.lam_y; ay.lam_other = t.lam_x;
    ay.scale = (T)(-4.0 * (p->mx + 1) * (double)(p->my + 1)); ay.lines_per_j = p->mx;
    ay.tw = t.tw_y; ay.C = p->Cy; ay.logC = ilog2c(p->Cy); ay.ld = p->Cy + 1;
    e = launch_axis(ay, st);
  }
  if (e != cudaSuccess) return e;
  return xform_x(p, ax, st);
}

// Time the x sine transforms (odd-sequence FFT, tensor-core products) on this plan's workspace and
// keep the faster; cached per (N, my, mz, dim) for the process.
pint_status autotune_xdst(pint_plan p) {
  static std::mutex mu;
  static std::vector<std::pair<long long, int>> cache;
  const long long key = ((((long long)p->N * 4096 + p->mx) * 4096 + p->my) * 4096 + p->mz) * 4 + p->dim;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& kv : cache)
      if (kv.first == key) { p->xdst = kv.second; return PINT_OK; }
  }
  cudaStream_t st;
  PINT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  AxisArgs<float> ax{};
  ax.S = p->S; ax.n = p->mx; ax.lines = (p->N / 2 + 1) * p->my * p->mz; ax.mode = 0; ax.P = 1; ax.op = 0;
  ax.lines_per_j = p->my * p->mz; ax.tw = p->tf.tw_x; ax.C = p->Cx; ax.logC = ilog2c(p->Cx); ax.ld = p->Cx + 1;
  float best = 1e30f;
  int bestv = 1;
  const bool prof = g_prof_on;
  g_prof_on = false;
  for (int v : {1, 2}) {
    p->xdst = v;
    cudaError_t e = xform_x<float>(p, ax, st);
    cudaEventRecord(e0, st);
    for (int r = 0; r < 4 && e == cudaSuccess; ++r) e = xform_x<float>(p, ax, st);
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      g_prof_on = prof;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      cudaStreamDestroy(st);
      return cuda_fail(e, "x sine transform tuning");
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; bestv = v; }
  }
  g_prof_on = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  p->xdst = bestv;
  // the timing ran on the zeroed workspace; the device error flag must still be clear
  int err = 0;
  PINT_CUDA(cudaMemcpy(&err, &p->ctl->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) return fail(PINT_ECUDA, "x sine transform tuning: a device-side wait gave up");
  std::lock_guard<std::mutex> lk(mu);
  cache.emplace_back(key, bestv);
  return PINT_OK;
}

// Time the y-direction solvers (sine transform, thread-per-line recurrence, parallel cyclic
// reduction) on this plan's workspace and keep the fastest; the choice is cached per
// (N, mx, my, precision) for the process.
pint_status autotune_ysolve(pint_plan p) {
  static std::mutex mu;
  static std::vector<std::pair<long long, int>> cache;
  const long long key = (((long long)p->N * 4096 + p->mx) * 4096 + p->my) * 4 + (int)p->prec;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& kv : cache)
      if (kv.first == key) { p->ysolve = kv.second; return PINT_OK; }
  }
  cudaStream_t st;
  PINT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bestv = 1;
  const bool prof = g_prof_on;
  g_prof_on = false;
  for (int v : {1, 2, 4}) {
    if (v == 4 && p->my > 1024) continue;
    p->ysolve = v;
    cudaError_t e = spatial<float>(p, p->tf, st);
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = spatial<float>(p, p->tf, st);
    cudaEventRecord(e1, st);
    cudaError_t se = cudaStreamSynchronize(st);
    if (e != cudaSuccess || se != cudaSuccess) {
      g_prof_on = prof;
      cudaEventDestroy(e0); cudaEventDestroy(e1); cudaStreamDestroy(st);
      return cuda_fail(e != cudaSuccess ? e : se, "autotune");
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; bestv = v; }
  }
  g_prof_on = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  p->ysolve = bestv;
  std::lock_guard<std::mutex> lk(mu);
  cache.push_back({key, bestv});
  return PINT_OK;
}

// MIXED sweep on the plan's double-float iterate (Uff); F_hat read in FP64
// The three time kernels of a MIXED sweep, each on its own (the tile-width tuner times them apart).
cudaError_t mixed_toeplitz(pint_plan p, cudaStream_t st) {
  ToepFFArgs ta{};
  float* yhi = reinterpret_cast<float*>(p->z);
  ta.U = p->Uff; ta.yhi = yhi; ta.ylo = yhi + (size_t)p->N * p->M; ta.what = p->what_ff; ta.tw = p->tw_ff;
  ta.N = p->N; ta.M = p->M; ta.C = p->Cz; ta.logC = ilog2c(p->Cz);
  return launch_toeplitz_ff(ta, st);
}

// The off-diagonal stencil weights are powers of two (m + 1 = 2^a per axis), so products with
// them are exact in FP32.
int stencil_pow2(pint_plan p) {
  auto p2 = [](double g) { return g == 0.0 || pow2((long)g); };
  return p2(p->gx) && p2(p->gy) && p2(p->gz) ? 1 : 0;
}

// Fc: Fhat is f, and F_hat's first kc levels are in Fc (BDF: F_hat = f beyond them; the fused
// right-hand side), else null
cudaError_t mixed_resid(pint_plan p, const double* Fhat, cudaStream_t st, const double* Fc = nullptr) {
  const int N = p->N, M = p->M;
  float* yhi = reinterpret_cast<float*>(p->z);
  ResidFwdArgs r{};
  r.U = p->Uff; r.F = Fhat; r.Fh = Fc; r.kc = Fc ? p->kc : 0;
  r.yhi = p->cq ? yhi : nullptr;
  r.ylo = p->cq ? yhi + (size_t)N * M : nullptr;
  r.S = reinterpret_cast<float2*>(p->S);
  r.s = p->tf.s; r.tw = reinterpret_cast<const float2*>(p->tf.tw_time);
  r.N = N; r.M = M; r.mx = p->mx; r.dim = p->dim; r.C = p->Cr; r.logC = ilog2c(p->Cr);
  const double ta = std::pow(p->tau, -p->alpha);
  // FD: c_0 includes the stencil centre; P1: the time terms act on M_h U and the stiffness
  // centre 2/h is applied separately (exact: h is a power of two)
  double c0 = p->fem ? 0.0 : 2.0 * p->gx + 2.0 * p->gy + 2.0 * p->gz;
  r.fem = p->fem ? 1 : 0;
  r.periodic = p->periodic ? 1 : 0;
  split_ff(1.0 / (6.0 * (p->mx + 1)), r.m_hi, r.m_lo);
  if (!p->cq) {
    r.k = p->k;
    c0 += p->omega[0] * ta;
    for (int j = 1; j <= p->k; ++j) split_ff(p->omega[j] * ta, r.c_hi[j], r.c_lo[j]);
  } else {
    r.k = 0;
  }
  split_ff(c0, r.c_hi[0], r.c_lo[0]);
  split_ff(p->gx, r.gx_hi, r.gx_lo);
  split_ff(p->gy, r.gy_hi, r.gy_lo);
  split_ff(p->gz, r.gz_hi, r.gz_lo);
  r.g_pow2 = stencil_pow2(p);
  r.maxlog = p->rml;
  r.my = p->my;
  r.react = p->react_on ? p->react : nullptr;
  return launch_resid_fwd(r, st);
}

cudaError_t mixed_update(pint_plan p, const double* v, cudaStream_t st) {
  InvUpdArgs u{};
  u.S = reinterpret_cast<const float2*>(p->S); u.U = p->Uff;
  u.inv_s = p->tf.inv_s; u.tw = reinterpret_cast<const float2*>(p->tf.tw_time);
  u.N = p->N; u.M = p->M; u.C = p->Ci; u.logC = ilog2c(p->Ci); u.norms = p->norms; u.v = v;
  u.maxlog = p->uml;
  return launch_inv_upd(u, st);
}

// MIXED sweep on the plan's double-float iterate (Uff); F_hat read in FP64
pint_status sweep_mixed(pint_plan p, const double* Fhat, cudaStream_t st, const double* Fc = nullptr) {
  cudaError_t e;
  if (p->cq && (e = mixed_toeplitz(p, st)) != cudaSuccess) return cuda_fail(e, "toeplitz kernel");
  PINT_CUDA(cudaMemsetAsync(p->norms, 0, 2 * sizeof(double), st));
  if ((e = mixed_resid(p, Fhat, st, Fc)) != cudaSuccess) return cuda_fail(e, "residual kernel");
  if ((e = spatial<float>(p, p->tf, st)) != cudaSuccess) return cuda_fail(e, "spatial kernel");
  if ((e = mixed_update(p, nullptr, st)) != cudaSuccess) return cuda_fail(e, "update kernel");
  return PINT_OK;
}

// Tile widths of the MIXED time kernels (residual, update, CQ history) by measurement: each kernel
// is launched alone on the plan's workspaces (zero right-hand side) at every admissible width,
// three timed launches after one warm-up, and the fastest width is kept. Results are cached per
// problem shape for the process.
pint_status tune_time_tiles(pint_plan p, int cmax_t, int cmax_z) {
  static std::mutex mu;
  struct Entry { long long key[4]; int cr, ci, cz; };
  static std::vector<Entry> cache;
  const long long key[4] = {(long long)p->N * 8192 + p->k, ((long long)p->mx * 4096 + p->my) * 4096 + p->mz,
                            (long long)p->dim * 16 + (p->cq ? 8 : 0) + (p->fem ? 4 : 0) + (p->periodic ? 2 : 0),
                            (long long)cmax_t * 64 + cmax_z};
  {
    std::lock_guard<std::mutex> lk(mu);
    for (const Entry& c : cache)
      if (std::equal(key, key + 4, c.key)) { p->Cr = c.cr; p->Ci = c.ci; p->Cz = c.cz; return PINT_OK; }
  }
  const size_t NM = (size_t)p->N * p->M;
  double* F = nullptr;
  {
    void* q = nullptr;
    const cudaError_t ea = lib_malloc(&q, NM * sizeof(double));
    if (ea != cudaSuccess) return fail(PINT_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(ea));
    F = (double*)q;
  }
  cudaStream_t st;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) { lib_free(F, NM * sizeof(double)); return cuda_fail(e, "tile tuning"); }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const bool prof = g_prof_on;
  g_prof_on = false;
  if (e == cudaSuccess) e = cudaMemsetAsync(F, 0, NM * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->Uff, 0, NM * sizeof(float2), st);
  if (e == cudaSuccess && p->cq) e = cudaMemsetAsync(p->z, 0, NM * sizeof(double), st);
  // kind 0: residual (Cr), 1: update (Ci), 2: CQ history (Cz)
  auto run = [&](int kind) -> cudaError_t {
    if (kind == 0) return mixed_resid(p, F, st);
    if (kind == 1) return mixed_update(p, nullptr, st);
    return mixed_toeplitz(p, st);
  };
  int* width[3] = {&p->Cr, &p->Ci, &p->Cz};
  for (int kind = 0; kind < 3 && e == cudaSuccess; ++kind) {
    if (kind == 2 && !p->cq) break;
    const int cmax = kind == 2 ? cmax_z : cmax_t;
    float best = 1e30f;
    int bestc = *width[kind];
    for (int c = 1; c <= cmax && e == cudaSuccess; c *= 2) {
      *width[kind] = c;
      e = run(kind);
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = run(kind);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < best) { best = ms; bestc = c; }
    }
    *width[kind] = bestc;
  }
  g_prof_on = prof;
  cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  lib_free(F, NM * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(e, "tile tuning");
  std::lock_guard<std::mutex> lk(mu);
  Entry en;
  std::copy(key, key + 4, en.key);
  en.cr = p->Cr; en.ci = p->Ci; en.cz = p->Cz;
  cache.push_back(en);
  return PINT_OK;
}

// Radix bound of the runtime-shape time FFTs (shapes without a compiled transform, e.g. N = 2048 or
// N = 100): the residual and the update kernel are each timed with radix <= 8 and radix <= 16
// passes on the plan's workspaces at their chosen widths, and each keeps its faster schedule (the
// forward and the inverse transform need not match: the half spectrum is stored in natural order).
// Cached per problem shape and widths for the process.
pint_status tune_radix(pint_plan p) {
  static std::mutex mu;
  struct Entry { long long key[4]; int rml, uml; };
  static std::vector<Entry> cache;
  const long long key[4] = {(long long)p->N * 8192 + p->k, ((long long)p->mx * 4096 + p->my) * 4096 + p->mz,
                            (long long)p->dim * 16 + (p->cq ? 8 : 0) + (p->fem ? 4 : 0) + (p->periodic ? 2 : 0),
                            (long long)p->Cr * 4096 + p->Ci};
  {
    std::lock_guard<std::mutex> lk(mu);
    for (const Entry& c : cache)
      if (std::equal(key, key + 4, c.key)) { p->rml = c.rml; p->uml = c.uml; return PINT_OK; }
  }
  const size_t NM = (size_t)p->N * p->M;
  double* F = nullptr;
  {
    void* q = nullptr;
    const cudaError_t ea = lib_malloc(&q, NM * sizeof(double));
    if (ea != cudaSuccess) return fail(PINT_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(ea));
    F = (double*)q;
  }
  cudaStream_t st;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) { lib_free(F, NM * sizeof(double)); return cuda_fail(e, "radix tuning"); }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const bool prof = g_prof_on;
  g_prof_on = false;
  if (e == cudaSuccess) e = cudaMemsetAsync(F, 0, NM * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->Uff, 0, NM * sizeof(float2), st);
  if (e == cudaSuccess && p->cq) e = cudaMemsetAsync(p->z, 0, NM * sizeof(double), st);
  int* ml[2] = {&p->rml, &p->uml};
  for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
    float best = 1e30f;
    int bestl = 4;
    for (int l = 3; l <= 4 && e == cudaSuccess; ++l) {
      *ml[kind] = l;
      auto run = [&]() { return kind == 0 ? mixed_resid(p, F, st) : mixed_update(p, nullptr, st); };
      e = run();
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = run();
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < best) { best = ms; bestl = l; }
    }
    *ml[kind] = bestl;
  }
  g_prof_on = prof;
  cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  lib_free(F, NM * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(e, "radix tuning");
  std::lock_guard<std::mutex> lk(mu);
  Entry en;
  std::copy(key, key + 4, en.key);
  en.rml = p->rml; en.uml = p->uml;
  cache.push_back(en);
  return PINT_OK;
}

// MIXED first sweep from U_0^n = v (Theorem 2.7): r_0 = F_hat - beta_n M v - A v in one pass over
// F_hat (no U read; for CQ no history product), the spatial solves, and U_1 = v + c written as
// the double-float iterate
pint_status sweep_mixed_v0(pint_plan p, const double* Fhat, const double* v, cudaStream_t st,
                           const double* Fc = nullptr) {
  const int N = p->N, M = p->M;
  PINT_CUDA(cudaMemsetAsync(p->norms, 0, 2 * sizeof(double), st));
  ResidFwdArgs r{};
  r.F = Fhat; r.v = v; r.beta_ff = p->beta_ff; r.Fh = Fc; r.kc = Fc ? p->kc : 0;
  r.S = reinterpret_cast<float2*>(p->S);
  r.s = p->tf.s; r.tw = reinterpret_cast<const float2*>(p->tf.tw_time);
  r.N = N; r.M = M; r.mx = p->mx; r.dim = p->dim; r.C = p->Cr; r.logC = ilog2c(p->Cr);
  r.fem = p->fem ? 1 : 0;
  r.periodic = p->periodic ? 1 : 0;
  split_ff(1.0 / (6.0 * (p->mx + 1)), r.m_hi, r.m_lo);
  split_ff(p->gx, r.gx_hi, r.gx_lo);
  split_ff(p->gy, r.gy_hi, r.gy_lo);
  split_ff(p->gz, r.gz_hi, r.gz_lo);
  r.g_pow2 = stencil_pow2(p);
  r.maxlog = p->rml;
  r.my = p->my;
  r.react = p->react_on ? p->react : nullptr;
  cudaError_t e = launch_resid_v0(r, st);
  if (e != cudaSuccess) return cuda_fail(e, "first-sweep residual kernel");
  e = spatial<float>(p, p->tf, st);
  if (e != cudaSuccess) return cuda_fail(e, "spatial kernel");
  e = mixed_update(p, v, st);
  if (e != cudaSuccess) return cuda_fail(e, "update kernel");
  return PINT_OK;
}

// FP64 / FP32 direct-form sweep: Uout = P^-1 (F + (P - K) Uin)
template <typename T>
pint_status sweep_direct(pint_plan p, const DevTables<T>& t, const T* F, const T* Uin, T* Uout,
                         cudaStream_t st) {
  const int N = p->N, M = p->M;
  if (p->cq) {
    ToepArgs ta{};
    if (sizeof(T) == 8) { ta.Ud = reinterpret_cast<const double*>(Uin); ta.ukind = 0; }
    else { ta.Uf = reinterpret_cast<const float*>(Uin); ta.ukind = 2; }
    ta.out = p->z; ta.what = p->what_up; ta.tw = p->tw_2n; ta.N = N; ta.M = M; ta.C = p->Cz;
    ta.logC = ilog2c(p->Cz); ta.half = 1;
    cudaError_t e = launch_toeplitz(ta, st);
    if (e != cudaSuccess) return cuda_fail(e, "toeplitz kernel");
  }
  PINT_CUDA(cudaMemsetAsync(p->norms, 0, 2 * sizeof(double), st));
  DirectFwdArgs<T> f{};
  f.F = F; f.U = Uin; f.z = p->cq ? p->z : nullptr; f.S = p->S; f.s = t.s; f.tw = t.tw_time;
  f.N = N; f.M = M; f.C = p->Ctd; f.logC = ilog2c(p->Ctd); f.k = p->cq ? 0 : p->k;
  f.fem = p->fem ? 1 : 0;
  f.h6 = (T)(1.0 / (6.0 * (p->mx + 1)));
  const double kt = p->kappa * std::pow(p->tau, -p->alpha);
  for (int j = 0; j <= p->k; ++j) f.kw[j] = (T)(kt * p->omega[j]);
  cudaError_t e = launch_direct_fwd(f, st);
  if (e != cudaSuccess) return cuda_fail(e, "direct fwd kernel");
  e = spatial<T>(p, t, st);
  if (e != cudaSuccess) return cuda_fail(e, "spatial kernel");
  DirectInvArgs<T> iv{};
  iv.S = p->S; iv.Uold = Uin; iv.Uout = Uout; iv.inv_s = t.inv_s; iv.tw = t.tw_time;
  iv.N = N; iv.M = M; iv.C = p->Ctd; iv.logC = ilog2c(p->Ctd); iv.norms = p->norms;
  e = launch_direct_inv(iv, st);
  if (e != cudaSuccess) return cuda_fail(e, "direct inv kernel");
  return PINT_OK;
}

pint_status read_norms(pint_plan p, cudaStream_t st, double* upd) {
  PINT_CUDA(cudaMemcpyAsync(p->h_norms, p->norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  PINT_CUDA(cudaMemcpyAsync(&p->h_ctl->err, &p->ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PINT_CUDA(cudaStreamSynchronize(st));
  if (p->h_ctl->err) {
    PINT_CUDA(cudaMemsetAsync(&p->ctl->err, 0, sizeof(int), st));
    return fail(PINT_ECUDA, "a device-side wait of the sweep gave up (bounded wait)");
  }
  const double c2 = p->h_norms[0], u2 = p->h_norms[1];
  *upd = u2 > 0.0 ? std::sqrt(c2 / u2) : std::sqrt(c2);
  return PINT_OK;
}

// sweep on FP64 user buffers
pint_status sweep_user(pint_plan p, const double* Fhat, const double* Uin, double* Uout, cudaStream_t st) {
  const size_t NM = (size_t)p->N * p->M;
  cudaError_t e;
  if (p->prec == PINT_FP64) return sweep_direct<double>(p, p->td, Fhat, Uin, Uout, st);
  if (p->prec == PINT_MIXED) {
    if ((e = launch_d2ff(Uin, p->Uff, NM, st)) != cudaSuccess) return cuda_fail(e, "convert");
    pint_status s = sweep_mixed(p, Fhat, st);
    if (s != PINT_OK) return s;
    if ((e = launch_ff2d(p->Uff, Uout, NM, st)) != cudaSuccess) return cuda_fail(e, "convert");
    return PINT_OK;
  }
  if ((e = launch_d2f(Fhat, p->Fhi, NM, st)) != cudaSuccess) return cuda_fail(e, "convert");
  if ((e = launch_d2f(Uin, p->Uhi, NM, st)) != cudaSuccess) return cuda_fail(e, "convert");
  pint_status s = sweep_direct<float>(p, p->tf, p->Fhi, p->Uhi, p->Uhi, st);
  if (s != PINT_OK) return s;
  if ((e = launch_f2d(p->Uhi, Uout, NM, st)) != cudaSuccess) return cuda_fail(e, "convert");
  return PINT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Whole solves as CUDA graphs: prologue (control init, conversions) -> while-node whose body is
// one sweep plus the device-side convergence check -> epilogue (conversion back, copy of the
// convergence state to pinned host memory). A solve is one graph launch; the host waits once.
// ---------------------------------------------------------------------------
namespace {

pint_status capture_begin(pint_plan p, cudaGraph_t g) {
  PINT_CUDA(cudaStreamBeginCaptureToGraph(p->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  return PINT_OK;
}
pint_status capture_end(pint_plan p, cudaGraph_t* g, pint_status body) {
  cudaGraph_t out = *g;
  cudaError_t e = cudaStreamEndCapture(p->cap, &out);
  if (body != PINT_OK) return body;
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  *g = out;
  return PINT_OK;
}

bool use_small(pint_plan p) { return p->small && !p->react_on; }

SmallArgs small_args(pint_plan p, const double* F, double* U, const double* v, double tol, int max_sweeps) {
  SmallArgs a{};
  a.F = F; a.U = U; a.v = v;
  a.tw_t = reinterpret_cast<const float2*>(p->tf.tw_time);
  a.s = p->tf.s; a.inv_s = p->tf.inv_s;
  a.sigma = reinterpret_cast<const float2*>(p->tf.sigma);
  a.lam = p->tf.lam_x;
  a.tw_x = reinterpret_cast<const float2*>(p->tf.tw_x);
  const double ta = std::pow(p->tau, -p->alpha);
  // as for the multi-kernel residual: c_0 carries the stencil centre 2/h^2
  split_ff(2.0 * p->gx + p->omega[0] * ta, a.c_hi[0], a.c_lo[0]);
  for (int j = 1; j <= p->k; ++j) split_ff(p->omega[j] * ta, a.c_hi[j], a.c_lo[j]);
  a.gx = (float)p->gx;
  a.k = p->k; a.N = p->N; a.M = p->M;
  a.Ct = p->small_Ct; a.logCt = ilog2c(p->small_Ct);
  a.L = 2 * (p->mx + 1);
  a.Cs = p->small_Cs; a.logCs = ilog2c(p->small_Cs);
  a.tol = tol; a.q_floor = p->q_floor; a.max_sweeps = max_sweeps;
  a.ctl = p->ctl;
  return a;
}

pint_status sweep_body(pint_plan p, const double* F, double* U, cudaStream_t st, const double* Fc = nullptr) {
  if (p->prec == PINT_MIXED) return sweep_mixed(p, F, st, Fc);
  if (p->prec == PINT_FP64) return sweep_direct<double>(p, p->td, F, U, U, st);
  return sweep_direct<float>(p, p->tf, p->Fhi, p->Uhi, p->Uhi, st);
}

}  // namespace

pint_status pint::add_solve_nodes(pint_plan p, cudaGraph_t g, const double* F, double* U, double tol,
                                  int max_sweeps, const double* v, cudaGraphNode_t dep, cudaGraphNode_t* last,
                                  const double* Fc) {
  const cudaGraphNode_t* deps = dep ? &dep : nullptr;
  const size_t ndeps = dep ? 1 : 0;
  const size_t NM = (size_t)p->N * p->M;
  const bool prof = g_prof_on;
  g_prof_on = false;  // per-kernel events are host-side records: keep them out of graphs
  if (use_small(p)) {
    // one kernel node (every sweep and the stopping rule) and the copy of its control block
    cudaGraph_t sub = nullptr;
    cudaGraphNode_t node;
    pint_status s = PINT_OK;
    if (cudaGraphCreate(&sub, 0) != cudaSuccess) {
      s = fail(PINT_ECUDA, "cudaGraphCreate");
    } else if ((s = capture_begin(p, sub)) == PINT_OK) {
      cudaError_t e = launch_small_solve(small_args(p, F, U, v, tol, max_sweeps), p->cap);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->h_ctl, p->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, p->cap);
      s = capture_end(p, &sub, e == cudaSuccess ? PINT_OK : cuda_fail(e, "small solve"));
      if (s == PINT_OK && cudaGraphAddChildGraphNode(&node, g, deps, ndeps, sub) != cudaSuccess)
        s = fail(PINT_ECUDA, "cudaGraphAddChildGraphNode");
      if (s == PINT_OK && last) *last = node;
    }
    if (sub) cudaGraphDestroy(sub);
    g_prof_on = prof;
    return s;
  }
  pint_status s = PINT_OK;
  cudaGraph_t pro = nullptr, epi = nullptr, body = nullptr;
  cudaGraphNode_t npro, nloop, nepi;
  do {
    // the while-node's condition (set by the convergence check of each sweep)
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { s = cuda_fail(e, "cudaGraphConditionalHandleCreate"); break; }
    // prologue (with v and MIXED: the first sweep from U_0^n = v and its convergence check)
    if (cudaGraphCreate(&pro, 0) != cudaSuccess) { s = fail(PINT_ECUDA, "cudaGraphCreate"); break; }
    if ((s = capture_begin(p, pro)) != PINT_OK) break;
    {
      pint_status b = PINT_OK;
      cudaError_t e1 = launch_ctl_init(p->ctl, tol, p->q_floor, max_sweeps, p->cap);
      if (e1 == cudaSuccess && v && p->prec != PINT_MIXED) e1 = launch_bcast_d(v, U, p->N, p->M, p->cap);
      if (e1 == cudaSuccess && p->prec == PINT_MIXED) {
        if (v) {
          b = sweep_mixed_v0(p, F, v, p->cap, Fc);
          if (b == PINT_OK) e1 = launch_converge(p->norms, p->ctl, h, p->cap);
        } else {
          e1 = launch_d2ff(U, p->Uff, NM, p->cap);
        }
      }
      if (e1 == cudaSuccess && p->prec == PINT_FP32) {
        e1 = launch_d2f(F, p->Fhi, NM, p->cap);
        if (e1 == cudaSuccess) e1 = launch_d2f(U, p->Uhi, NM, p->cap);
      }
      if (b == PINT_OK && e1 != cudaSuccess) b = cuda_fail(e1, "graph prologue");
      if ((s = capture_end(p, &pro, b)) != PINT_OK) break;
    }
    if (cudaGraphAddChildGraphNode(&npro, g, deps, ndeps, pro) != cudaSuccess) {
      s = fail(PINT_ECUDA, "cudaGraphAddChildGraphNode"); break;
    }
    // while-node with the sweep body
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&nloop, g, &npro, nullptr, 1, &cp);
    if (e != cudaSuccess) { s = cuda_fail(e, "cudaGraphAddNode(conditional)"); break; }
    body = cp.conditional.phGraph_out[0];
    if ((s = capture_begin(p, body)) != PINT_OK) break;
    {
      pint_status b = sweep_body(p, F, U, p->cap, Fc);
      if (b == PINT_OK) {
        cudaError_t e2 = launch_converge(p->norms, p->ctl, h, p->cap);
        if (e2 != cudaSuccess) b = cuda_fail(e2, "convergence kernel");
      }
      if ((s = capture_end(p, &body, b)) != PINT_OK) break;
    }
    // epilogue
    if (cudaGraphCreate(&epi, 0) != cudaSuccess) { s = fail(PINT_ECUDA, "cudaGraphCreate"); break; }
    if ((s = capture_begin(p, epi)) != PINT_OK) break;
    {
      cudaError_t e3 = cudaSuccess;
      if (p->prec == PINT_MIXED) e3 = launch_ff2d(p->Uff, U, NM, p->cap);
      else if (p->prec == PINT_FP32) e3 = launch_f2d(p->Uhi, U, NM, p->cap);
      if (e3 == cudaSuccess)
        e3 = cudaMemcpyAsync(p->h_ctl, p->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, p->cap);
      if ((s = capture_end(p, &epi, e3 == cudaSuccess ? PINT_OK : cuda_fail(e3, "graph epilogue"))) != PINT_OK)
        break;
    }
    if (cudaGraphAddChildGraphNode(&nepi, g, &nloop, 1, epi) != cudaSuccess) {
      s = fail(PINT_ECUDA, "cudaGraphAddChildGraphNode"); break;
    }
    if (last) *last = nepi;
  } while (0);
  if (pro) cudaGraphDestroy(pro);
  if (epi) cudaGraphDestroy(epi);
  g_prof_on = prof;
  return s;
}

pint_status pint::solve_enqueue(pint_plan p, const double* F, double* U, double tol, int max_sweeps,
                                cudaStream_t st, const double* v, const double* Fc) {
  SolveGraph* hit = nullptr;
  for (SolveGraph& c : p->sg)
    if (c.exec && c.F == F && c.Fc == Fc && c.U == U && c.v == v && c.tol == tol && c.max_sweeps == max_sweeps &&
        c.react == p->react_on)
      hit = &c;
  if (!hit) {
    // an empty slot, else the least recently used one
    hit = &p->sg[0];
    for (SolveGraph& c : p->sg) {
      if (!c.exec) { hit = &c; break; }
      if (c.last_use < hit->last_use) hit = &c;
    }
    SolveGraph& sg = *hit;
    if (sg.exec) {
      cudaGraphExecDestroy(sg.exec);
      sg.exec = nullptr;
    }
    cudaGraph_t g;
    PINT_CUDA(cudaGraphCreate(&g, 0));
    pint_status s = add_solve_nodes(p, g, F, U, tol, max_sweeps, v, nullptr, nullptr, Fc);
    if (s == PINT_OK) {
      cudaError_t e = cudaGraphInstantiate(&sg.exec, g, 0);
      if (e != cudaSuccess) s = cuda_fail(e, "cudaGraphInstantiate");
    }
    cudaGraphDestroy(g);
    if (s != PINT_OK) {
      sg.exec = nullptr;
      return s;
    }
    sg.F = F; sg.Fc = Fc; sg.U = U; sg.v = v; sg.tol = tol; sg.max_sweeps = max_sweeps; sg.react = p->react_on;
  }
  hit->last_use = ++p->sg_clock;
  PINT_CUDA(cudaGraphLaunch(hit->exec, st));
  return PINT_OK;
}

bool pint::solve_wait_gave_up(pint_plan p) { return p->h_ctl->err != 0; }

void pint::solve_result(pint_plan p, int* sweeps, double* upd, bool* converged) {
  if (sweeps) *sweeps = p->h_ctl->m;
  if (upd) *upd = p->h_ctl->upd;
  if (converged) *converged = p->h_ctl->done != 0;
}

void pint::plan_release(pint_plan p) { destroy_plan(p); }

size_t pint::plan_bytes_estimate(const pint_plan_desc* d) {
  const size_t N = d->N, M = (size_t)d->grid.mx * (d->grid.dim >= 2 ? d->grid.my : 1) *
                                 (d->grid.dim == 3 ? d->grid.mz : 1);
  const size_t NM = N * M, JM = (N / 2 + 1) * M;
  size_t b = 0;
  if (d->precision == PINT_MIXED) b += 8 * NM + 8 * JM + (d->alpha == 1.0 ? 8 * (size_t)d->k * M : 0);
  else if (d->precision == PINT_FP32) b += 8 * NM + 8 * JM;
  else b += 16 * JM;
  if (d->alpha != 1.0) b += 8 * NM;
  b += 64 * (N + d->grid.mx + d->grid.my) + 65536;  // tables, alignment slack
  if (d->xdst != 1 && dst_tc_line_ok(d->grid.mx) && d->grid.dim >= 2) b += dst_tc_table_bytes(d->grid.mx);
  if (d->xdst != 1 && d->grid.dim == 3 && (d->grid.my == 127 || d->grid.mz == 127)) b += dst_tc_table_bytes(127);
  return b;
}

extern "C" pint_status pint_wr_sweep(pint_plan p, const double* Fhat, const double* U_prev, double* U_next,
                                     double* upd_rel, void* stream) {
  if (!p || !Fhat || !U_prev || !U_next) return fail(PINT_EINVAL, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  pint_status s = sweep_user(p, Fhat, U_prev, U_next, st);
  if (s != PINT_OK) return s;
  if (upd_rel) return read_norms(p, st, upd_rel);
  return PINT_OK;
}

extern "C" pint_status pint_solve_async(pint_plan p, const double* Fhat, double* U, double tol, int max_sweeps,
                                        void* stream) {
  if (!p || !Fhat || !U) return fail(PINT_EINVAL, "NULL argument");
  if (!(tol > 0.0) || max_sweeps < 1) return fail(PINT_EINVAL, "tol must be > 0 and max_sweeps >= 1");
  if (g_prof_on) return fail(PINT_EINVAL, "pint_solve_async: not available while per-kernel profiling is on");
  return solve_enqueue(p, Fhat, U, tol, max_sweeps, (cudaStream_t)stream);
}

extern "C" pint_status pint_solve_v_async(pint_plan p, const double* Fhat, const double* v, double* U, double tol,
                                          int max_sweeps, void* stream) {
  if (!p || !Fhat || !v || !U) return fail(PINT_EINVAL, "NULL argument");
  if (!(tol > 0.0) || max_sweeps < 1) return fail(PINT_EINVAL, "tol must be > 0 and max_sweeps >= 1");
  if (g_prof_on) return fail(PINT_EINVAL, "pint_solve_v_async: not available while per-kernel profiling is on");
  return solve_enqueue(p, Fhat, U, tol, max_sweeps, (cudaStream_t)stream, v);
}

extern "C" int pint_plan_tuning(pint_plan p, int* out, int n) {
  if (!p || !out || n < 0) {
    set_last_error("NULL argument");
    return -1;
  }
  const bool mixed = p->prec == PINT_MIXED;
  const int v[10] = {p->Cr, p->Ci, p->Cz, p->ysolve,
                    mixed ? (compiled_time_fft_shape(p->N, p->Cr) ? 16 : 1 << p->rml) : 0,
                    mixed ? (compiled_update_shape(p->N, p->Ci) ? 16 : 1 << p->uml) : 0, p->small ? 1 : 0,
                    p->xdst, p->ydst, p->zsolve};
  const int k = n < 10 ? n : 10;
  for (int i = 0; i < k; ++i) out[i] = v[i];
  return 10;
}

extern "C" pint_status pint_solve_result(pint_plan p, int* sweeps_out, double* upd_rel_out) {
  if (!p) return fail(PINT_EINVAL, "NULL argument");
  int m = 0;
  double upd = 0.0;
  bool done = false;
  solve_result(p, &m, &upd, &done);
  if (sweeps_out) *sweeps_out = m;
  if (upd_rel_out) *upd_rel_out = upd;
  if (solve_wait_gave_up(p)) return fail(PINT_ECUDA, "a device-side wait of the solve gave up (bounded wait)");
  if (!done) return fail(PINT_ENOTCONV, "max_sweeps reached above tol");
  return PINT_OK;
}

namespace {
pint_status solve_sweeps(pint_plan p, const double* Fhat, const double* v, double* U, double tol, int max_sweeps,
                         int m0, double prev0, int* sweeps_out, double* upd_rel_out, cudaStream_t st,
                         const double* Fc = nullptr);

// pint_solve (v null: from the content of U) and pint_solve_v (from U_0^n = v); with Fc, Fhat is f
// and F_hat's first kc levels are in Fc (the fused right-hand side of pint_solve_fv)
pint_status solve_impl(pint_plan p, const double* Fhat, const double* v, double* U, double tol, int max_sweeps,
                       int* sweeps_out, double* upd_rel_out, cudaStream_t st, const double* Fc = nullptr) {
  if (!p || !Fhat || !U) return fail(PINT_EINVAL, "NULL argument");
  if (!(tol > 0.0) || max_sweeps < 1) return fail(PINT_EINVAL, "tol must be > 0 and max_sweeps >= 1");
  if (!g_prof_on) {
    // one graph launch runs every sweep; the host waits once for the result
    pint_status gs = solve_enqueue(p, Fhat, U, tol, max_sweeps, st, v, Fc);
    if (gs != PINT_OK) return gs;
    PINT_CUDA(cudaStreamSynchronize(st));
    int m = 0;
    double upd = 0.0;
    bool done = false;
    solve_result(p, &m, &upd, &done);
    if (sweeps_out) *sweeps_out = m;
    if (upd_rel_out) *upd_rel_out = upd;
    if (solve_wait_gave_up(p)) return fail(PINT_ECUDA, "a device-side wait of the solve gave up (bounded wait)");
    if (!done) return fail(PINT_ENOTCONV, "max_sweeps reached above tol");
    return PINT_OK;
  }
  cudaError_t e;
  if (use_small(p)) {
    // the one-CTA solve is one launch in either mode (its kernel appears in the profile)
    if ((e = launch_small_solve(small_args(p, Fhat, U, v, tol, max_sweeps), st)) != cudaSuccess)
      return cuda_fail(e, "small solve");
    PINT_CUDA(cudaMemcpyAsync(p->h_ctl, p->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, st));
    PINT_CUDA(cudaStreamSynchronize(st));
    if (sweeps_out) *sweeps_out = p->h_ctl->m;
    if (upd_rel_out) *upd_rel_out = p->h_ctl->upd;
    if (!p->h_ctl->done) return fail(PINT_ENOTCONV, "max_sweeps reached above tol");
    return PINT_OK;
  }
  return solve_sweeps(p, Fhat, v, U, tol, max_sweeps, 0, -1.0, sweeps_out, upd_rel_out, st, Fc);
}

// The sweeps of a solve launched one by one from the host, starting after m0 sweeps whose last
// relative update was prev0 (m0 = 0, prev0 < 0: a fresh solve; otherwise a resumed one, whose
// stopping decisions then match those of the uninterrupted solve).
pint_status solve_sweeps(pint_plan p, const double* Fhat, const double* v, double* U, double tol, int max_sweeps,
                         int m0, double prev0, int* sweeps_out, double* upd_rel_out, cudaStream_t st,
                         const double* Fc) {
  const size_t NM = (size_t)p->N * p->M;
  cudaError_t e;
  double prev = prev0, upd = prev0 > 0.0 ? prev0 : 0.0;
  int m = m0;
  bool done = false;
  pint_status s = PINT_OK;
  if (v && p->prec != PINT_MIXED && (e = launch_bcast_d(v, U, p->N, p->M, st)) != cudaSuccess)
    return cuda_fail(e, "initial guess kernel");
  if (p->prec == PINT_MIXED) {
    if (v) {
      // first sweep from U_0^n = v
      if ((s = sweep_mixed_v0(p, Fhat, v, st, Fc)) != PINT_OK) return s;
      m = 1;
      if ((s = read_norms(p, st, &upd)) != PINT_OK) return s;
      done = stop_decision(m, upd, prev, tol, p->q_floor);
      prev = upd;
    } else if ((e = launch_d2ff(U, p->Uff, NM, st)) != cudaSuccess) {
      return cuda_fail(e, "convert");
    }
  } else if (p->prec == PINT_FP32) {
    if ((e = launch_d2f(Fhat, p->Fhi, NM, st)) != cudaSuccess) return cuda_fail(e, "convert");
    if ((e = launch_d2f(U, p->Uhi, NM, st)) != cudaSuccess) return cuda_fail(e, "convert");
  }
  while (m < max_sweeps && !done) {
    if (p->prec == PINT_MIXED) s = sweep_mixed(p, Fhat, st, Fc);
    else if (p->prec == PINT_FP64) s = sweep_direct<double>(p, p->td, Fhat, U, U, st);
    else s = sweep_direct<float>(p, p->tf, p->Fhi, p->Uhi, p->Uhi, st);
    if (s != PINT_OK) return s;
    ++m;
    if ((s = read_norms(p, st, &upd)) != PINT_OK) return s;
    done = stop_decision(m, upd, prev, tol, p->q_floor);
    prev = upd;
  }
  if (p->prec == PINT_MIXED) {
    if ((e = launch_ff2d(p->Uff, U, NM, st)) != cudaSuccess) return cuda_fail(e, "convert");
  } else if (p->prec == PINT_FP32) {
    if ((e = launch_f2d(p->Uhi, U, NM, st)) != cudaSuccess) return cuda_fail(e, "convert");
  }
  if (sweeps_out) *sweeps_out = m;
  if (upd_rel_out) *upd_rel_out = upd;
  if (!done) return fail(PINT_ENOTCONV, "max_sweeps reached above tol");
  return PINT_OK;
}
}  // namespace

extern "C" pint_status pint_solve_resume(pint_plan p, const double* Fhat, double* U, int sweeps_done,
                                         double upd_last, double tol, int max_sweeps, int* sweeps_out,
                                         double* upd_rel_out, void* stream) {
  if (!p || !Fhat || !U) return fail(PINT_EINVAL, "NULL argument");
  if (!(tol > 0.0) || max_sweeps < 1 || sweeps_done < 0 || sweeps_done > max_sweeps || !(upd_last >= 0.0))
    return fail(PINT_EINVAL, "tol > 0, 0 <= sweeps_done <= max_sweeps and upd_last >= 0 are required");
  return solve_sweeps(p, Fhat, nullptr, U, tol, max_sweeps, sweeps_done, sweeps_done > 0 ? upd_last : -1.0,
                      sweeps_out, upd_rel_out, (cudaStream_t)stream);
}

extern "C" pint_status pint_solve(pint_plan p, const double* Fhat, double* U, double tol, int max_sweeps,
                                  int* sweeps_out, double* upd_rel_out, void* stream) {
  return solve_impl(p, Fhat, nullptr, U, tol, max_sweeps, sweeps_out, upd_rel_out, (cudaStream_t)stream);
}

extern "C" pint_status pint_solve_v(pint_plan p, const double* Fhat, const double* v, double* U, double tol,
                                    int max_sweeps, int* sweeps_out, double* upd_rel_out, void* stream) {
  if (!v) return fail(PINT_EINVAL, "NULL argument");
  return solve_impl(p, Fhat, v, U, tol, max_sweeps, sweeps_out, upd_rel_out, (cudaStream_t)stream);
}

bool pint::profiling_on() { return g_prof_on; }

bool pint::fused_rhs_ok(pint_plan p) {
  return p->prec == PINT_MIXED && p->fcorr && !p->react_on && !use_small(p);
}

pint_status pint::form_rhs_corr(pint_plan p, const double* v, const double* f, const double* fderiv, cudaStream_t st) {
  return form_rhs(p, v, f, fderiv, p->fcorr, st, nullptr, p->kc);
}

extern "C" pint_status pint_solve_fv(pint_plan p, const double* v, const double* f, const double* fderiv, double* U,
                                     double tol, int max_sweeps, int* sweeps_out, double* upd_rel_out,
                                     void* stream) {
  if (!p || !v || !f || !U) return fail(PINT_EINVAL, "NULL argument");
  if (p->k >= 2 && !fderiv) return fail(PINT_EINVAL, "fderiv is required for k >= 2");
  if (!(tol > 0.0) || max_sweeps < 1) return fail(PINT_EINVAL, "tol must be > 0 and max_sweeps >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  pint_status s;
  if (fused_rhs_ok(p)) {
    // fused: the residual kernels read F_hat's first kc levels from the plan's block, then f
    if ((s = form_rhs_corr(p, v, f, fderiv, st)) != PINT_OK) return s;
    return solve_impl(p, f, v, U, tol, max_sweeps, sweeps_out, upd_rel_out, st, p->fcorr);
  }
  if (!p->Fws && (s = dalloc(p, &p->Fws, (size_t)p->N * p->M)) != PINT_OK) return s;
  if ((s = form_rhs(p, v, f, fderiv, p->Fws, st, nullptr)) != PINT_OK) return s;
  return solve_impl(p, p->Fws, v, U, tol, max_sweeps, sweeps_out, upd_rel_out, st);
}

namespace {
// space-time unknowns from which one solve fills the GPU by itself (its time tiles give several
// waves of CTAs on every SM): such solves of a batch are chained rather than run side by side
constexpr size_t kBatchChainDof = (size_t)1 << 24;

// pint_batch_solve (v null: each solve from the content of its U) and pint_batch_solve_v
pint_status batch_impl(pint_plan* plans, int n, const double* const* Fhat, const double* const* v,
                       double* const* U, double tol, int max_sweeps, int* sweeps_out, double* upd_out,
                       cudaStream_t st) {
  if (n < 1 || !plans || !Fhat || !U) return fail(PINT_EINVAL, "bad batch arguments");
  if (!(tol > 0.0) || max_sweeps < 1) return fail(PINT_EINVAL, "tol must be > 0 and max_sweeps >= 1");
  std::vector<const void*> key;
  key.reserve(4 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || !Fhat[i] || !U[i] || (v && !v[i])) return fail(PINT_EINVAL, "NULL plan or array in batch");
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return fail(PINT_EINVAL, "a plan appears twice in one batch");
    key.push_back(plans[i]);
    key.push_back(Fhat[i]);
    key.push_back(U[i]);
    key.push_back(plans[i]->react_on ? plans[i]->react : nullptr);  // spatial solve captured
    key.push_back(v ? v[i] : nullptr);
  }
  std::lock_guard<std::mutex> lk(g_batch.mu);
  if (!g_batch.exec || g_batch.key != key || g_batch.tol != tol || g_batch.max_sweeps != max_sweeps) {
    if (g_batch.exec) {
      cudaGraphExecDestroy(g_batch.exec);
      g_batch.exec = nullptr;
    }
    cudaGraph_t g;
    PINT_CUDA(cudaGraphCreate(&g, 0));
    pint_status s = PINT_OK;
    // Problems large enough to fill the GPU on their own run one after another in a chain (running
    // them side by side only makes them contend: on the mixed 64-problem batch, 64 independent
    // branches took 959 ms against 907 ms for the same solves one at a time); the smaller ones run
    // as independent branches beside the chain, filling the GPU around it.
    cudaGraphNode_t chain = nullptr;
    for (int i = 0; i < n && s == PINT_OK; ++i) {
      const bool big = (size_t)plans[i]->N * plans[i]->M >= kBatchChainDof;
      cudaGraphNode_t tail = nullptr;
      s = add_solve_nodes(plans[i], g, Fhat[i], U[i], tol, max_sweeps, v ? v[i] : nullptr, big ? chain : nullptr,
                          &tail);
      if (big) chain = tail;
    }
    if (s == PINT_OK) {
      cudaError_t e = cudaGraphInstantiate(&g_batch.exec, g, 0);
      if (e != cudaSuccess) s = cuda_fail(e, "cudaGraphInstantiate");
    }
    cudaGraphDestroy(g);
    if (s != PINT_OK) {
      g_batch.exec = nullptr;
      return s;
    }
    g_batch.key = key;
    g_batch.tol = tol;
    g_batch.max_sweeps = max_sweeps;
  }
  cudaError_t e = cudaGraphLaunch(g_batch.exec, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "batch graph");
  bool all = true;
  for (int i = 0; i < n; ++i) {
    int m = 0;
    double upd = 0.0;
    bool done = false;
    solve_result(plans[i], &m, &upd, &done);
    if (sweeps_out) sweeps_out[i] = m;
    if (upd_out) upd_out[i] = upd;
    all = all && done;
    if (solve_wait_gave_up(plans[i]))
      return fail(PINT_ECUDA, "a device-side wait of a batch solve gave up (bounded wait)");
  }
  if (!all) return fail(PINT_ENOTCONV, "some problems reached max_sweeps above tol");
  return PINT_OK;
}
}  // namespace

extern "C" pint_status pint_batch_solve(pint_plan* plans, int n, const double* const* Fhat, double* const* U,
                                        double tol, int max_sweeps, int* sweeps_out, double* upd_out,
                                        void* stream) {
  return batch_impl(plans, n, Fhat, nullptr, U, tol, max_sweeps, sweeps_out, upd_out, (cudaStream_t)stream);
}

extern "C" pint_status pint_batch_solve_v(pint_plan* plans, int n, const double* const* Fhat,
                                          const double* const* v, double* const* U, double tol, int max_sweeps,
                                          int* sweeps_out, double* upd_out, void* stream) {
  if (!v) return fail(PINT_EINVAL, "bad batch arguments");
  return batch_impl(plans, n, Fhat, v, U, tol, max_sweeps, sweeps_out, upd_out, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// host-only queries and diagnostics
// ---------------------------------------------------------------------------
extern "C" pint_status pint_time_weights(int k, double alpha, int n, double* omega) {
  if (k < 1 || k > kMaxK || !(alpha > 0.0 && alpha <= 1.0) || n < 0 || (!omega && n > 0))
    return fail(PINT_EINVAL, "bad arguments");
  time_weights(k, alpha, n, omega);
  return PINT_OK;
}

extern "C" pint_status pint_correction_coefficients(int k, double* a, double* b) {
  if (k < 1 || k > kMaxK || !a || !b) return fail(PINT_EINVAL, "bad arguments");
  double bb[4][5];
  table1(k, a, bb);
  for (int l = 0; l < 4; ++l)
    for (int n = 0; n < 5; ++n) b[l * 5 + n] = bb[l][n];
  return PINT_OK;
}

extern "C" pint_status pint_circulant_eigenvalues(int k, double alpha, double kappa, int N,
                                                  pint_eig_variant eig, double* re, double* im) {
  if (k < 1 || k > kMaxK || !(alpha > 0.0 && alpha <= 1.0) || !(kappa > 0.0 && kappa < 1.0) ||
      !fft_len_ok(N) || N < 2 || N <= k || !re || !im)
    return fail(PINT_EINVAL, "bad arguments");
  std::vector<double> w(N);
  time_weights(k, alpha, N, w.data());
  std::vector<cd> g;
  eigenvalues(k, alpha, kappa, N, eig, w, g);
  for (int j = 0; j < N; ++j) {
    re[j] = g[j].real();
    im[j] = g[j].imag();
  }
  return PINT_OK;
}

extern "C" const char* pint_last_error(void) { return g_err.c_str(); }

extern "C" const char* pint_status_string(pint_status s) {
  switch (s) {
    case PINT_OK: return "PINT_OK";
    case PINT_EINVAL: return "PINT_EINVAL";
    case PINT_ENOMEM: return "PINT_ENOMEM";
    case PINT_ECUDA: return "PINT_ECUDA";
    case PINT_ENOTCONV: return "PINT_ENOTCONV";
    case PINT_ETIMEOUT: return "PINT_ETIMEOUT";
    case PINT_EAGAIN: return "PINT_EAGAIN";
    case PINT_EBUDGET: return "PINT_EBUDGET";
    case PINT_ENOTFOUND: return "PINT_ENOTFOUND";
  }
  return "unknown";
}

extern "C" const char* pint_version(void) { return "pint-gb300 0.1 (sm_103a)"; }

extern "C" pint_status pint_set_profiling(int enable) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = enable != 0;
  return PINT_OK;
}

extern "C" int pint_kernel_stats(int max, const char** names, int* launches, double* total_ms, int reset) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  std::vector<const char*> nm;
  std::vector<int> cnt;
  std::vector<double> tot;
  for (const ProfRec& r : g_prof_recs) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    size_t i = 0;
    for (; i < nm.size(); ++i)
      if (std::strcmp(nm[i], r.name) == 0) break;
    if (i == nm.size()) {
      nm.push_back(r.name);
      cnt.push_back(0);
      tot.push_back(0.0);
    }
    cnt[i] += 1;
    tot[i] += ms;
  }
  const int n = (int)nm.size();
  for (int i = 0; i < n && i < max; ++i) {
    if (names) names[i] = nm[i];
    if (launches) launches[i] = cnt[i];
    if (total_ms) total_ms[i] = tot[i];
  }
  if (reset) {
    for (const ProfRec& r : g_prof_recs) {
      g_prof_pool.push_back(r.a);
      g_prof_pool.push_back(r.b);
    }
    g_prof_recs.clear();
  }
  return n;
}

// ---------------------------------------------------------------------------
// Reaction term and the semilinear extension (Sec. 4.3, Algorithm 3)
// ---------------------------------------------------------------------------
namespace {

// reaction weight of a row: 1 (finite differences), h (P1 elements, nodal quadrature)
double react_weight(pint_plan p) { return p->fem ? 1.0 / (p->mx + 1) : 1.0; }

pint_status react_check(pint_plan p) {
  if (!p) return fail(PINT_EINVAL, "NULL plan");
  if (p->dim != 1 || p->periodic)
    return fail(PINT_EINVAL, "reaction terms are supported on 1D plans with Dirichlet boundaries");
  return PINT_OK;
}

pint_status react_alloc(pint_plan p) {
  if (p->react) return PINT_OK;
  const size_t JM = (size_t)(p->N / 2 + 1) * p->M;
  const size_t vb = p->prec == PINT_FP64 ? sizeof(double2) : sizeof(float2);
  pint_status s;
  unsigned char *ip, *cp;
  if ((s = dalloc(p, &ip, JM * vb)) != PINT_OK) return s;
  if ((s = dalloc(p, &cp, JM * vb)) != PINT_OK) return s;
  if ((s = dalloc(p, &p->react, (size_t)p->M)) != PINT_OK) return s;
  p->tri_ip = ip;
  p->tri_cp = cp;
  return PINT_OK;
}

// LU factors of (sigma_j M + A + diag(react)) for every frequency j
pint_status react_factor(pint_plan p, cudaStream_t st) {
  cudaError_t e;
  if (p->prec == PINT_FP64) {
    TriVarArgs<double> a{};
    a.ip = p->tri_ip; a.cp = p->tri_cp; a.sigma = p->td.sigma; a.r = p->react; a.n = p->mx; a.J = p->N / 2 + 1;
    row_coefficients(p, a.md, a.mo, a.kd, a.ko);
    e = launch_trivar_factor<double>(a, st);
  } else {
    TriVarArgs<float> a{};
    a.ip = p->tri_ip; a.cp = p->tri_cp; a.sigma = p->tf.sigma; a.r = p->react; a.n = p->mx; a.J = p->N / 2 + 1;
    row_coefficients(p, a.md, a.mo, a.kd, a.ko);
    e = launch_trivar_factor<float>(a, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "tridiagonal factor kernel");
  return PINT_OK;
}

pint_status nl_alloc_fd(pint_plan p) {
  if (p->nl_fd) return PINT_OK;
  return dalloc(p, &p->nl_fd, (size_t)(p->k - 1) * p->M);
}

pint_status poly_check(const pint_poly* g) {
  if (!g) return fail(PINT_EINVAL, "NULL nonlinearity");
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(g->c[i])) return fail(PINT_EINVAL, "non-finite nonlinearity coefficient");
  return PINT_OK;
}

NlPoly to_poly(const pint_poly* g) {
  NlPoly q;
  for (int i = 0; i < 4; ++i) q.c[i] = g->c[i];
  return q;
}

}  // namespace

extern "C" pint_status pint_set_reaction(pint_plan p, const double* c, void* stream) {
  pint_status s = react_check(p);
  if (s != PINT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (!c) {
    p->react_on = false;
    return PINT_OK;
  }
  if ((s = react_alloc(p)) != PINT_OK) return s;
  cudaError_t e = launch_scale(c, react_weight(p), p->M, p->react, st);
  if (e != cudaSuccess) return cuda_fail(e, "reaction kernel");
  if ((s = react_factor(p, st)) != PINT_OK) return s;
  p->react_on = true;
  return PINT_OK;
}

extern "C" pint_status pint_nl_form_rhs(pint_plan p, const pint_poly* g, const double* v, const double* f,
                                        const double* fderiv, double* Fhat, void* stream) {
  pint_status s = react_check(p);
  if (s != PINT_OK) return s;
  if ((s = poly_check(g)) != PINT_OK) return s;
  if (p->react_on) return fail(PINT_EINVAL, "a reaction term is installed (pint_set_reaction(plan, NULL) removes it)");
  const NlPoly q = to_poly(g);
  return form_rhs(p, v, f, fderiv, Fhat, (cudaStream_t)stream, &q);
}

// Outer stopping rule of Algorithm 3 after step l (upd = upd_l, prev = upd_{l-1}, prev2 = upd_{l-2}).
// The first update is the whole Newton step from the starting iterate, so the ratio upd_2 / upd_1
// measures how far that iterate was, not the contraction of the later steps (on Example 4 the
// step 2 -> 3 contraction is larger): it is never trusted alone. l = 1 or 2: stop only when the
// update itself is below tol / 100; l >= 3: q = the larger of the last two ratios, and the error
// estimate upd_l q / (1 - q) must be <= tol (upd_l <= tol if q >= 1).
static bool outer_stop_decision(int l, double upd, double prev, double prev2, double tol) {
  if (l <= 2) return upd <= 0.01 * tol;
  double q = prev > 0.0 ? upd / prev : 0.0;
  const double q2 = prev2 > 0.0 ? prev / prev2 : 0.0;
  if (q2 > q) q = q2;
  if (q < 1.0) return upd * q / (1.0 - q) <= tol;
  return upd <= tol;
}

extern "C" pint_status pint_nl_solve(pint_plan p, const pint_poly* g, const double* Fhat, double* U,
                                     double newton_tol, int max_steps, double tol, int max_sweeps,
                                     pint_nl_info* info, void* stream) {
  pint_status s = react_check(p);
  if (s != PINT_OK) return s;
  if ((s = poly_check(g)) != PINT_OK) return s;
  if (!Fhat || !U) return fail(PINT_EINVAL, "NULL argument");
  if (p->react_on) return fail(PINT_EINVAL, "a reaction term is installed (pint_set_reaction(plan, NULL) removes it)");
  if (!(newton_tol > 0.0) || !(tol > 0.0) || max_sweeps < 1 || max_steps < 1 || max_steps > PINT_NL_MAX_STEPS)
    return fail(PINT_EINVAL, "tolerances must be > 0, max_sweeps >= 1, 1 <= max_steps <= PINT_NL_MAX_STEPS");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t NM = (size_t)p->N * p->M;
  if ((s = react_alloc(p)) != PINT_OK) return s;
  if (!p->nl_F) {
    if ((s = dalloc(p, &p->nl_F, NM)) != PINT_OK) return s;
    if ((s = dalloc(p, &p->nl_U0, NM)) != PINT_OK) return s;
    if ((s = dalloc(p, &p->nl_norms, 2)) != PINT_OK) return s;
  }
  if (!p->nl_h) {
    p->nl_h = p->alloc ? (double*)p->alloc->host_alloc(2 * sizeof(double)) : nullptr;
    if (!p->alloc) {
      void* q = nullptr;
      p->nl_h = lib_malloc_host(&q, 2 * sizeof(double)) == cudaSuccess ? (double*)q : nullptr;
    }
    if (!p->nl_h) return fail(PINT_ENOMEM, "pinned host buffer");
  }
  const NlPoly q = to_poly(g);
  const double w = react_weight(p);
  if (info) std::memset(info, 0, sizeof(*info));
  p->react_on = true;
  double prev = 0.0, prev2 = 0.0;
  bool converged = false, inner_ok = true;
  int l = 0;
  while (l < max_steps && !converged) {
    ++l;
    // linearise at the time average of U_{l-1}: react = w g'(Ubar), its factors, and the
    // right-hand side F_hat - w g(U_{l-1}) + w D U_{l-1} of (K + I (x) w D) U_l = ...
    cudaError_t e = launch_nl_linearise(U, p->N, p->M, q, w, p->react, st);
    if (e == cudaSuccess) e = launch_nl_rhs(Fhat, U, p->react, q, w, p->N, p->M, p->nl_F, p->nl_U0, st);
    if (e != cudaSuccess) { p->react_on = false; return cuda_fail(e, "linearisation kernels"); }
    if ((s = react_factor(p, st)) != PINT_OK) { p->react_on = false; return s; }
    // the inner WR from U_{l-1} (W_0 = 0)
    int sweeps = 0;
    double upd_in = 0.0;
    s = pint_solve(p, p->nl_F, U, tol, max_sweeps, &sweeps, &upd_in, stream);
    if (s == PINT_ENOTCONV) inner_ok = false;
    else if (s != PINT_OK) { p->react_on = false; return s; }
    // ||U_l - U_{l-1}|| / ||U_l||
    e = cudaMemsetAsync(p->nl_norms, 0, 2 * sizeof(double), st);
    if (e == cudaSuccess) e = launch_nl_norms(U, p->nl_U0, NM, p->nl_norms, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->nl_h, p->nl_norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { p->react_on = false; return cuda_fail(e, "outer update norms"); }
    const double upd = p->nl_h[1] > 0.0 ? std::sqrt(p->nl_h[0] / p->nl_h[1]) : std::sqrt(p->nl_h[0]);
    if (info) {
      info->steps = l;
      info->sweeps[l - 1] = sweeps;
      info->upd[l - 1] = upd;
    }
    converged = outer_stop_decision(l, upd, prev, prev2, newton_tol);
    prev2 = prev;
    prev = upd;
  }
  p->react_on = false;
  if (!converged) return fail(PINT_ENOTCONV, "max_steps reached above newton_tol");
  if (!inner_ok) return fail(PINT_ENOTCONV, "an inner solve reached max_sweeps above tol");
  return PINT_OK;
}

extern "C" long long pint_device_bytes_held(void) { return pint::g_device_bytes.load(); }

extern "C" int pint_debug_fail_allocation(int n) { return pint::g_fail_countdown.exchange(n < 0 ? -1 : n); }
