// A kappa-circulant solve that allocates no device memory.
//
// Some callers cannot allocate device memory at call time: code that runs under a fixed
// memory budget decided up front, plugins hosted by a runtime that owns all allocations,
// or a real-time loop in which a cudaMalloc (which may synchronise the device) is not
// allowed. For them pint_kappa_solve_noalloc applies P_kappa^{-1} (Algorithm 1, steps 1-3:
// kappa^{n/N} scaling, DFT along time, the N shifted 1D systems, inverse DFT and unscaling)
// in FP64 with the same kernels as a plan, but the intermediate spectrum and the constant
// tables live in one file-scope static device array instead of plan-owned memory.
//
// The array is part of the library image: every GPU that loads the library holds it until the
// process exits. All calls share it, so calls whose GPU work overlaps (on different streams, or
// from different host threads) race on it; serialise them on one stream.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/pint.h"
#include "fft.cuh"
#include "pint_internal.h"

namespace pint {

// Capacity: the half spectrum (N/2+1) x mx complex doubles, plus tables for N <= 1024 and
// mx <= 1023.
constexpr size_t kNoAllocSpectrum = (size_t)1 << 18;        // complex doubles (4 MiB)
constexpr int kNoAllocMaxN = 1024;
constexpr int kNoAllocMaxMx = 1023;
constexpr size_t kNoAllocTables =
    sizeof(double2) * (kNoAllocMaxN + (kNoAllocMaxN / 2 + 1) + 2 * (kNoAllocMaxMx + 1)) +
    sizeof(double) * (2 * kNoAllocMaxN + kNoAllocMaxMx) + 4 * sizeof(double);
constexpr size_t kNoAllocBytes = sizeof(double2) * kNoAllocSpectrum + kNoAllocTables + 1024;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device ordinal, looked up on the first call made
// with that device current (cudaGetSymbolAddress; never a device pointer taken from host code).
// The address belongs to the context the library's module was loaded into: after a
// cudaDeviceReset the device gets a new primary context, the module is loaded again and the
// array may sit elsewhere. So each slot also records the ID of the context it was looked up in
// (cuCtxGetId, reached through the runtime's driver entry points, so no libcuda link), and a
// call made in another context looks the address up again.
struct NaSlot {
  unsigned long long ctx_id;
  void* ptr;
};
static std::mutex g_na_mu;
static NaSlot g_na[64] = {};

// ID of the calling thread's current context; false if there is none yet or the driver cannot
// report it (the caller then looks the address up on every call). Called under g_na_mu.
static bool current_ctx_id(unsigned long long* id) {
  using GetCur = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCur get_cur = nullptr;
  static GetId get_id = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<GetCur>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(p);
  }
  if (!get_cur || !get_id) return false;
  CUcontext ctx = nullptr;
  if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device ordinal of a device (or managed) allocation, -1 otherwise.
static int pointer_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the (non-sticky) error left by an unknown pointer
    return -1;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return -1;
  return at.device;
}

// Constant tables of the solve, computed on the device in FP64 (CUDA math functions):
// tw[m] = exp(-2 pi i m/N), s_i = kappa^{i/N}, inv_s_i = kappa^{-i/N}/N,
// sigma_j = delta_k(kappa^{1/N} e^{-2 pi i j/N}) / tau (Lemma 2.3, alpha = 1),
// twx[m] = exp(-2 pi i m/L), L = 2(mx+1), lam_p = (4/h^2) sin^2(p pi h/2).
__global__ void k_noalloc_tables(int k, double kappa, double tau, int N, int mx, double2* tw, double* s,
                                 double* inv_s, double2* sigma, double2* twx, double* lam) {
  const int L = 2 * (mx + 1);
  const int total = N + N + (N / 2 + 1) + L + mx;
  const double lk = log(kappa) / N;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int i = t;
    if (i < N) {
      double sn, cs;
      sincospi(2.0 * i / N, &sn, &cs);
      tw[i] = make_double2(cs, -sn);
      continue;
    }
    i -= N;
    if (i < N) {
      s[i] = exp(lk * i);
      inv_s[i] = exp(-lk * i) / N;
      continue;
    }
    i -= N;
    if (i < N / 2 + 1) {
      // 1 - z = (1 - r) + r (1 - e^{-i t}), 1 - e^{-i t} = 2 sin^2(t/2) + i sin t
      const double r = exp(lk), om = -expm1(lk);
      double sn, cs, sh, ch;
      sincospi(2.0 * i / N, &sn, &cs);
      sincospi((double)i / N, &sh, &ch);
      const double sr = om + r * 2.0 * sh * sh, si = r * sn;
      double pr = 1.0, pi = 0.0, dr = 0.0, di = 0.0;
      for (int l = 1; l <= k; ++l) {
        const double nr = pr * sr - pi * si, ni = pr * si + pi * sr;
        pr = nr;
        pi = ni;
        dr += pr / l;
        di += pi / l;
      }
      sigma[i] = make_double2(dr / tau, di / tau);
      continue;
    }
    i -= N / 2 + 1;
    if (i < L) {
      double sn, cs;
      sincospi(2.0 * i / L, &sn, &cs);
      twx[i] = make_double2(cs, -sn);
      continue;
    }
    i -= L;
    const double h = 1.0 / (mx + 1);
    double sn, cs;
    sincospi(0.5 * (i + 1) * h, &sn, &cs);
    lam[i] = 4.0 / (h * h) * sn * sn;
  }
}

static pint_status na_fail(pint_status st, const std::string& m) {
  set_last_error(m);
  return st;
}

}  // namespace pint

using namespace pint;

extern "C" pint_status pint_kappa_solve_noalloc(int k, double kappa, double tau, int N, int mx,
                                                const double* R, double* Q, void* stream) {
  if (!R || !Q) return na_fail(PINT_EINVAL, "NULL argument");
  if (k < 1 || k > kMaxK || !(kappa > 0.0 && kappa < 1.0) || !(tau > 0.0))
    return na_fail(PINT_EINVAL, "k must be in 1..6, kappa in (0,1), tau > 0");
  if (N < 8 || N > kNoAllocMaxN || (N & (N - 1)) || N <= k)
    return na_fail(PINT_EINVAL, "N must be a power of two in [8, 1024] and exceed k");
  if (mx < 3 || mx > kNoAllocMaxMx || ((mx + 1) & mx))
    return na_fail(PINT_EINVAL, "mx + 1 must be a power of two, 3 <= mx <= 1023");
  if ((size_t)(N / 2 + 1) * (size_t)mx > kNoAllocSpectrum)
    return na_fail(PINT_EINVAL, "(N/2+1)*mx exceeds the static scratch capacity of 262144 complex values");
  {
    // R and Q hold N * mx doubles each and may not overlap
    const size_t bytes = sizeof(double) * (size_t)N * (size_t)mx;
    const uintptr_t r0 = reinterpret_cast<uintptr_t>(R), q0 = reinterpret_cast<uintptr_t>(Q);
    if (r0 < q0 + bytes && q0 < r0 + bytes) return na_fail(PINT_EINVAL, "Q overlaps R");
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(PINT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return na_fail(PINT_EINVAL, "device ordinal out of range");
  // the scratch array used is the current device's: R and Q must live on that device too
  if (pointer_device(R) != dev || pointer_device(Q) != dev)
    return na_fail(PINT_EINVAL, "R and Q must be device arrays of the current device");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    unsigned long long id = 0;
    bool have_id = g_na[dev].ptr && current_ctx_id(&id);
    if (!have_id || g_na[dev].ctx_id != id) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return na_fail(PINT_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      have_id = current_ctx_id(&id);
      g_na[dev].ctx_id = have_id ? id : 0;
      g_na[dev].ptr = p;
    }
    base = reinterpret_cast<unsigned char*>(g_na[dev].ptr);
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int J = N / 2 + 1, L = 2 * (mx + 1);
  // carve the array (every piece 256-byte aligned)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off += (bytes + 255) & ~(size_t)255;
    return p;
  };
  double2* S = reinterpret_cast<double2*>(take(sizeof(double2) * (size_t)J * mx));
  double2* tw = reinterpret_cast<double2*>(take(sizeof(double2) * N));
  double* s = reinterpret_cast<double*>(take(sizeof(double) * N));
  double* inv_s = reinterpret_cast<double*>(take(sizeof(double) * N));
  double2* sigma = reinterpret_cast<double2*>(take(sizeof(double2) * J));
  double2* twx = reinterpret_cast<double2*>(take(sizeof(double2) * L));
  double* lam = reinterpret_cast<double*>(take(sizeof(double) * mx));
  double* norms = reinterpret_cast<double*>(take(2 * sizeof(double)));
  if (off > kNoAllocBytes) return na_fail(PINT_EINVAL, "static scratch too small for this size");

  // norms are accumulated with atomics: they must start at zero on every call
  e = cudaMemsetAsync(norms, 0, 2 * sizeof(double), st);
  if (e != cudaSuccess) return na_fail(PINT_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  k_noalloc_tables<<<8, 256, 0, st>>>(k, kappa, tau, N, mx, tw, s, inv_s, sigma, twx, lam);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(PINT_ECUDA, std::string("tables kernel: ") + cudaGetErrorString(e));

  // step 1: scale and DFT along time (direct-form kernel with no kappa corner term)
  int Ct = 32;
  while (Ct > 1 && (size_t)N * sizeof(double2) * Ct > 96 * 1024) Ct >>= 1;
  while (Ct < 32 && Ct * N < kThreads) Ct <<= 1;
  DirectFwdArgs<double> f{};
  f.F = R; f.U = R; f.z = nullptr; f.S = S; f.s = s; f.tw = tw;
  f.N = N; f.M = mx; f.C = Ct; f.logC = ilog2c(Ct); f.k = 0;
  e = launch_direct_fwd(f, st);
  if (e != cudaSuccess) return na_fail(PINT_ECUDA, std::string("time DFT kernel: ") + cudaGetErrorString(e));
  // step 2: (sigma_j + A_h) q_j = h_j by the sine transform along x
  int Cx = 16;
  while (Cx > 1 && (size_t)L * sizeof(double2) * Cx > 40 * 1024) Cx >>= 1;
  AxisArgs<double> ax{};
  ax.S = S; ax.n = mx; ax.lines = J; ax.mode = 0; ax.P = 1; ax.op = 1;
  ax.sigma = sigma; ax.lam_axis = lam; ax.lam_other = nullptr; ax.scale = 2.0 * (mx + 1);
  ax.lines_per_j = 1; ax.tw = twx; ax.C = Cx; ax.logC = ilog2c(Cx); ax.ld = Cx + 1;
  e = launch_axis(ax, st);
  if (e != cudaSuccess) return na_fail(PINT_ECUDA, std::string("spatial kernel: ") + cudaGetErrorString(e));
  // step 3: inverse DFT and unscaling into Q
  DirectInvArgs<double> iv{};
  iv.S = S; iv.Uold = R; iv.Uout = Q; iv.inv_s = inv_s; iv.tw = tw;
  iv.N = N; iv.M = mx; iv.C = Ct; iv.logC = ilog2c(Ct); iv.norms = norms;
  e = launch_direct_inv(iv, st);
  if (e != cudaSuccess) return na_fail(PINT_ECUDA, std::string("inverse DFT kernel: ") + cudaGetErrorString(e));
  return PINT_OK;
}
