// End-to-end solves through host buffers (pint_solve_host): the inputs v, f, d^l f(0) come from
// host memory, the solution goes back to host memory, and everything in between -- F_hat formation
// and the whole WR solve from U_0^n = v -- runs on the device as for pint_form_rhs +
// pint_solve_v_async.
//
// The plan keeps two sets of staging buffers (v, f, d^l f(0), U) and two copy streams, so that
// consecutive calls overlap their transfers with the neighbouring solves: the inputs of call i+1
// are copied in while call i solves, and the solution of call i-1 is copied out meanwhile.
// Ordering, per buffer set s (calls i, i+2, ... use the same set):
//   copy-in stream:  [wait: the solve of the previous user of s has read v_s, f_s] H2D -> in_done[s]
//   compute stream:  [wait in_done[s]; the copy-out of the previous user of s has read U_s]
//                    F_hat, solve -> comp_done[s]
//   copy-out stream: [wait comp_done[s]] D2H -> out_done[s]
// F_hat is one buffer: it is written and read on the compute stream only.
#include <cuda_runtime.h>

#include <string>

#include "../../include/pint.h"
#include "pint_internal.h"
#include "plan_internal.h"

namespace pint {

struct HostStage {
  double* v[2] = {nullptr, nullptr};
  double* f[2] = {nullptr, nullptr};
  double* fd[2] = {nullptr, nullptr};
  double* U[2] = {nullptr, nullptr};
  double* F = nullptr;
  size_t bytes[5] = {0, 0, 0, 0, 0};  // v, f, fd, U, F (per buffer)
  cudaStream_t sin = nullptr, sout = nullptr;
  cudaEvent_t in_done[2] = {nullptr, nullptr}, comp_done[2] = {nullptr, nullptr}, out_done[2] = {nullptr, nullptr};
  bool used[2] = {false, false};
  int next = 0;
};

void host_stage_free(pint_plan p) {
  HostStage* h = p->hstage;
  if (!h) return;
  if (h->sin) cudaStreamSynchronize(h->sin);
  if (h->sout) cudaStreamSynchronize(h->sout);
  for (int s = 0; s < 2; ++s) {
    lib_free(h->v[s], h->bytes[0]);
    lib_free(h->f[s], h->bytes[1]);
    lib_free(h->fd[s], h->bytes[2]);
    lib_free(h->U[s], h->bytes[3]);
    if (h->in_done[s]) cudaEventDestroy(h->in_done[s]);
    if (h->comp_done[s]) cudaEventDestroy(h->comp_done[s]);
    if (h->out_done[s]) cudaEventDestroy(h->out_done[s]);
  }
  lib_free(h->F, h->bytes[4]);
  if (h->sin) cudaStreamDestroy(h->sin);
  if (h->sout) cudaStreamDestroy(h->sout);
  delete h;
  p->hstage = nullptr;
}

static pint_status hs_fail(pint_status st, const std::string& m) {
  set_last_error(m);
  return st;
}

// the staging buffers, streams and events on first use; everything taken is given back on failure
static pint_status host_stage_get(pint_plan p, HostStage** out) {
  if (p->hstage) {
    *out = p->hstage;
    return PINT_OK;
  }
  HostStage* h = new HostStage();
  p->hstage = h;
  const size_t M = (size_t)p->M, NM = (size_t)p->N * M;
  h->bytes[0] = sizeof(double) * M;
  h->bytes[1] = sizeof(double) * NM;
  h->bytes[2] = sizeof(double) * M * (size_t)(p->k > 1 ? p->k - 1 : 1);
  h->bytes[3] = sizeof(double) * NM;
  h->bytes[4] = sizeof(double) * NM;
  auto take = [&](double** q, size_t b) {
    void* r = nullptr;
    const cudaError_t e = lib_malloc(&r, b);
    *q = (double*)r;
    return e == cudaSuccess;
  };
  bool ok = true;
  for (int s = 0; s < 2 && ok; ++s)
    ok = take(&h->v[s], h->bytes[0]) && take(&h->f[s], h->bytes[1]) && take(&h->fd[s], h->bytes[2]) &&
         take(&h->U[s], h->bytes[3]);
  ok = ok && take(&h->F, h->bytes[4]);
  if (!ok) {
    host_stage_free(p);
    return hs_fail(PINT_ENOMEM, "pint_solve_host: device staging buffers");
  }
  cudaError_t e = cudaStreamCreateWithFlags(&h->sin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->sout, cudaStreamNonBlocking);
  for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
    e = cudaEventCreateWithFlags(&h->in_done[s], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->comp_done[s], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->out_done[s], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    host_stage_free(p);
    (void)cudaGetLastError();
    return hs_fail(PINT_ECUDA, std::string("pint_solve_host: streams / events: ") + cudaGetErrorString(e));
  }
  *out = h;
  return PINT_OK;
}

}  // namespace pint

using namespace pint;

extern "C" pint_status pint_solve_host(pint_plan p, const double* v, const double* f, const double* fderiv,
                                       double* U_out, double tol, int max_sweeps, void* stream) {
  if (!p || !v || !f || !U_out || (p->k > 1 && !fderiv)) return hs_fail(PINT_EINVAL, "NULL argument");
  if (!(tol > 0.0) || max_sweeps < 1) return hs_fail(PINT_EINVAL, "tol must be > 0 and max_sweeps >= 1");
  HostStage* h = nullptr;
  pint_status st = host_stage_get(p, &h);
  if (st != PINT_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  const int s = h->next;
  auto cerr = [](cudaError_t e, const char* where) {
    (void)cudaGetLastError();
    return hs_fail(PINT_ECUDA, std::string("pint_solve_host: ") + where + ": " + cudaGetErrorString(e));
  };
  cudaError_t e = cudaSuccess;
  // 1. inputs into set s, once the solve of the previous user of s has read them
  if (h->used[s]) e = cudaStreamWaitEvent(h->sin, h->comp_done[s], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->v[s], v, h->bytes[0], cudaMemcpyHostToDevice, h->sin);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->f[s], f, h->bytes[1], cudaMemcpyHostToDevice, h->sin);
  if (e == cudaSuccess && p->k > 1)
    e = cudaMemcpyAsync(h->fd[s], fderiv, sizeof(double) * (size_t)p->M * (p->k - 1), cudaMemcpyHostToDevice,
                        h->sin);
  if (e == cudaSuccess) e = cudaEventRecord(h->in_done[s], h->sin);
  if (e != cudaSuccess) return cerr(e, "copy in");
  // 2. F_hat and the solve on the caller's stream, once the inputs are in and the previous copy-out
  //    of U_s is done
  e = cudaStreamWaitEvent(cs, h->in_done[s], 0);
  if (e == cudaSuccess && h->used[s]) e = cudaStreamWaitEvent(cs, h->out_done[s], 0);
  if (e != cudaSuccess) return cerr(e, "stream order");
  h->used[s] = true;
  h->next ^= 1;
  if (fused_rhs_ok(p)) {
    // F_hat not materialised: the residual kernels read f and the correction of the first levels
    // (graph-launched like pint_solve_v_async, hence not while per-kernel profiling is on)
    if (profiling_on()) return hs_fail(PINT_EINVAL, "pint_solve_host: not available while per-kernel profiling is on");
    st = form_rhs_corr(p, h->v[s], h->f[s], p->k > 1 ? h->fd[s] : nullptr, cs);
    if (st == PINT_OK) st = solve_enqueue(p, h->f[s], h->U[s], tol, max_sweeps, cs, h->v[s], p->fcorr);
  } else {
    st = pint_form_rhs(p, h->v[s], h->f[s], p->k > 1 ? h->fd[s] : nullptr, h->F, stream);
    if (st == PINT_OK) st = pint_solve_v_async(p, h->F, h->v[s], h->U[s], tol, max_sweeps, stream);
  }
  if (st != PINT_OK) return st;
  e = cudaEventRecord(h->comp_done[s], cs);
  // 3. the solution back to the host on the copy-out stream
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->sout, h->comp_done[s], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(U_out, h->U[s], h->bytes[3], cudaMemcpyDeviceToHost, h->sout);
  if (e == cudaSuccess) e = cudaEventRecord(h->out_done[s], h->sout);
  if (e != cudaSuccess) return cerr(e, "copy out");
  return PINT_OK;
}

extern "C" pint_status pint_solve_host_join(pint_plan p, void* stream) {
  if (!p) return hs_fail(PINT_EINVAL, "NULL argument");
  HostStage* h = p->hstage;
  if (!h) return PINT_OK;
  cudaStream_t cs = (cudaStream_t)stream;
  for (int s = 0; s < 2; ++s) {
    if (!h->used[s]) continue;
    const cudaError_t e = cudaStreamWaitEvent(cs, h->out_done[s], 0);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return hs_fail(PINT_ECUDA, std::string("pint_solve_host_join: ") + cudaGetErrorString(e));
    }
  }
  return PINT_OK;
}
