// Continuous-batching solve server: requests of any (N, grid, k, alpha, kappa) arrive at any
// time; a worker thread admits them while a device-memory budget and a slot count allow, runs
// each admitted request as one graph launch (F_hat formation and the whole WR solve from
// U_0 = v with its device-side convergence loop) on its own stream, and retires it when its completion
// event fires. Requests admitted while others run share the GPU: their kernels overlap.
// Iterates stay on the device from admission until the caller polls the result out.
//
// Device memory comes from one arena reserved at creation (the budget): plans and request
// arrays are sub-allocated from it (first fit, 256-byte granules, neighbours coalesced on
// release), so admission never calls cudaMalloc and never synchronises the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pint.h"
#include "pint_internal.h"
#include "plan_internal.h"

namespace pint {
namespace {

class Arena : public DevAllocator {
 public:
  // pinned: a host region of nslots blocks of kHostBlock bytes for plans' small read-back buffers
  static constexpr size_t kHostBlock = 256;
  Arena(char* base, size_t cap, char* pinned, int nslots) : base_(base), cap_(cap), pinned_(pinned) {
    free_[0] = cap;
    for (int i = nslots - 1; i >= 0; --i) host_free_.push_back(pinned_ + (size_t)i * kHostBlock);
  }
  void* host_alloc(size_t bytes) override {
    if (inject_alloc_failure()) return nullptr;
    std::lock_guard<std::mutex> lk(mu_);
    if (bytes > kHostBlock || host_free_.empty()) return nullptr;
    void* p = host_free_.back();
    host_free_.pop_back();
    return p;
  }
  void host_release(void* p) override {
    if (!p) return;
    std::lock_guard<std::mutex> lk(mu_);
    host_free_.push_back((char*)p);
  }
  void* alloc(size_t bytes) override {
    bytes = (bytes + 255) & ~(size_t)255;
    if (inject_alloc_failure()) return nullptr;  // the failure-path hook: as if the budget were full
    std::lock_guard<std::mutex> lk(mu_);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, sz = it->second;
        free_.erase(it);
        if (sz > bytes) free_[off + bytes] = sz - bytes;
        live_[off] = bytes;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return base_ + off;
      }
    }
    return nullptr;
  }
  void release(void* p) override {
    if (!p) return;
    std::lock_guard<std::mutex> lk(mu_);
    const size_t off = (size_t)((char*)p - base_);
    auto lv = live_.find(off);
    if (lv == live_.end()) return;
    size_t sz = lv->second;
    live_.erase(lv);
    used_ -= sz;
    size_t start = off;
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && nx->first == off + sz) {  // merge with the next free block
      sz += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {  // merge with the previous free block
      auto pv = std::prev(nx);
      if (pv->first + pv->second == start) {
        start = pv->first;
        sz += pv->second;
        free_.erase(pv);
      }
    }
    free_[start] = sz;
  }
  size_t used() {
    std::lock_guard<std::mutex> lk(mu_);
    return used_;
  }
  size_t peak() {
    std::lock_guard<std::mutex> lk(mu_);
    return peak_;
  }

 private:
  char* base_;
  size_t cap_;
  char* pinned_;
  std::vector<char*> host_free_;
  std::mutex mu_;
  std::map<size_t, size_t> free_;
  std::unordered_map<size_t, size_t> live_;
  size_t used_ = 0, peak_ = 0;
};

enum ReqState { QUEUED, RUNNING, DONE };

struct Request {
  uint64_t ticket;
  pint_request req;
  std::vector<double> v, f, fd;     // host inputs (copied at submit)
  const double *uv = nullptr, *uf = nullptr, *ufd = nullptr;  // caller-owned device inputs
  size_t need = 0;
  ReqState state = QUEUED;
  pint_status status = PINT_OK;
  std::string err;
  pint_plan plan = nullptr;
  double *dv = nullptr, *df = nullptr, *dfd = nullptr, *dF = nullptr, *dU = nullptr;
  std::vector<double> result;       // the solution, once moved to the host to free the budget
  bool held = false;                // finished, solution still on the device (dU), not yet polled
  bool spilling = false;            // the worker is moving the solution to the host
  int slot = -1;
  int sweeps = 0;
  double upd = 0.0;
  double t_submit = 0, t_start = 0, t_done = 0;
};

using clk = std::chrono::steady_clock;

}  // namespace
}  // namespace pint

using namespace pint;

struct pint_server_s {
  size_t budget = 0;
  int max_active = 0;
  char* base = nullptr;
  char* pinned = nullptr;
  Arena* arena = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<Request*> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::deque<Request*> held;        // finished requests whose solution waits on the device
  std::unordered_map<uint64_t, Request*> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  clk::time_point t0;
  int device = 0;
  // statistics
  double completed = 0, dof_done = 0, sweeps_done = 0, busy_s = 0;

  double now() const { return std::chrono::duration<double>(clk::now() - t0).count(); }
};

namespace {

size_t request_bytes(const pint_request& r) {
  const pint_plan_desc& d = r.desc;
  const size_t M = (size_t)d.grid.mx * (d.grid.dim == 2 ? d.grid.my : 1);
  const size_t NM = (size_t)d.N * M;
  // U on the device and F_hat unless the solve reads f directly (MIXED BDF, not the one-CTA solve,
  // which only takes problems of up to 4096 unknowns), plus copies of f, v and d^l f(0) when the
  // inputs come from the host
  const bool fused = d.precision == PINT_MIXED && d.alpha == 1.0 && NM > 4096;
  const size_t inputs = r.inputs_on_device ? 0 : 8 * NM + 8 * M * (size_t)(d.k + 1);
  return plan_bytes_estimate(&d) + (fused ? 1 : 2) * 8 * NM + inputs + 8 * 256;
}

// everything but the solution U
void release_request_inputs(pint_server_s* s, Request* r) {
  if (r->plan) {
    plan_release(r->plan);
    r->plan = nullptr;
  }
  double** arrays[] = {&r->dv, &r->df, &r->dfd, &r->dF};
  for (double** a : arrays) {
    if (*a) s->arena->release(*a);
    *a = nullptr;
  }
}

void release_request_memory(pint_server_s* s, Request* r) {
  release_request_inputs(s, r);
  if (r->dU) s->arena->release(r->dU);
  r->dU = nullptr;
}

size_t request_unknowns(const Request* r) {
  const pint_plan_desc& d = r->req.desc;
  return (size_t)d.N * d.grid.mx * (d.grid.dim == 2 ? d.grid.my : 1);
}

// Move the oldest finished-but-unpolled solution to host memory and return its device memory to the
// budget (when held results keep a queued request out). Returns false if none is held.
bool spill_oldest(pint_server_s* s) {
  Request* r = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->held.empty()) return false;
    r = s->held.front();
    s->held.pop_front();
    r->spilling = true;
  }
  r->result.resize(request_unknowns(r));
  const cudaError_t ce = cudaMemcpy(r->result.data(), r->dU, r->result.size() * sizeof(double),
                                    cudaMemcpyDeviceToHost);
  s->arena->release(r->dU);
  std::lock_guard<std::mutex> lk(s->mu);
  r->dU = nullptr;
  r->held = false;
  r->spilling = false;
  if (ce != cudaSuccess) {
    r->status = PINT_ECUDA;
    r->err = cudaGetErrorString(ce);
    r->result.clear();
  }
  s->cv_done.notify_all();
  return true;
}

// Set up one admitted request on its slot's stream: plan (from the arena), device arrays,
// uploads, F_hat, and the whole solve from U_0 = v as one graph launch, then the completion event.
void start_request(pint_server_s* s, Request* r) {
  cudaSetDevice(s->device);
  const pint_plan_desc& d = r->req.desc;
  const size_t M = (size_t)d.grid.mx * (d.grid.dim == 2 ? d.grid.my : 1);
  const size_t NM = (size_t)d.N * M;
  cudaStream_t st = s->streams[r->slot];
  pint_status status = plan_create_internal(&d, s->arena, &r->plan);
  auto take = [&](double** p, size_t n) {
    if (status != PINT_OK) return;
    *p = (double*)s->arena->alloc(std::max<size_t>(n, 1) * sizeof(double));
    if (!*p) status = PINT_ENOMEM;
  };
  const bool dev_in = r->req.inputs_on_device != 0;
  if (!dev_in) {
    take(&r->dv, M);
    take(&r->df, NM);
    if (d.k >= 2) take(&r->dfd, (size_t)(d.k - 1) * M);
  }
  // MIXED BDF: F_hat is not materialised (the residual reads f and F_hat's first k levels)
  const bool fused = status == PINT_OK && fused_rhs_ok(r->plan);
  if (!fused) take(&r->dF, NM);
  take(&r->dU, NM);
  cudaError_t e = cudaSuccess;
  const double* in_v = dev_in ? r->uv : r->dv;
  const double* in_f = dev_in ? r->uf : r->df;
  const double* in_fd = dev_in ? r->ufd : r->dfd;
  if (status == PINT_OK && !dev_in) {
    e = cudaMemcpyAsync(r->dv, r->v.data(), M * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->df, r->f.data(), NM * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && d.k >= 2)
      e = cudaMemcpyAsync(r->dfd, r->fd.data(), (size_t)(d.k - 1) * M * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) status = PINT_ECUDA;
  }
  // the whole solve from U_0^n = v (the first sweep reads v; U_0 is never written)
  if (fused) {
    if (status == PINT_OK) status = form_rhs_corr(r->plan, in_v, in_f, in_fd, st);
    if (status == PINT_OK)
      status = solve_enqueue(r->plan, in_f, r->dU, r->req.tol, r->req.max_sweeps, st, in_v, r->plan->fcorr);
  } else {
    if (status == PINT_OK) status = pint_form_rhs(r->plan, in_v, in_f, in_fd, r->dF, st);
    if (status == PINT_OK) status = solve_enqueue(r->plan, r->dF, r->dU, r->req.tol, r->req.max_sweeps, st, in_v);
  }
  if (status == PINT_OK) {
    e = cudaEventRecord(s->events[r->slot], st);
    if (e != cudaSuccess) status = PINT_ECUDA;
  }
  if (status == PINT_OK) {
    // the inputs are on the device now (pageable copies are staged before the call returns)
    std::vector<double>().swap(r->f);
    std::vector<double>().swap(r->fd);
  }
  if (status != PINT_OK) {
    r->status = status;
    r->err = pint_last_error();
    cudaStreamSynchronize(st);
    release_request_memory(s, r);
  }
}

void worker_loop(pint_server_s* s) {
  cudaSetDevice(s->device);
  std::vector<Request*> to_start;
  for (;;) {
    to_start.clear();
    bool progressed = false;
    bool spill = false;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      bool busy = false;
      for (Request* r : s->slots) busy = busy || r;
      if (s->stop) {
        // shutting down: queued requests are not admitted any more
        while (!s->queue.empty()) {
          Request* r = s->queue.front();
          s->queue.pop_front();
          r->status = PINT_ETIMEOUT;
          r->err = "server destroyed before the request was admitted";
          r->state = DONE;
          r->t_done = s->now();
        }
        s->cv_done.notify_all();
        if (!busy) break;
      }
      // admission: FIFO, while a slot is free and the budget allows
      while (!s->queue.empty()) {
        Request* r = s->queue.front();
        if (r->need > s->budget) {
          s->queue.pop_front();
          r->status = PINT_EBUDGET;
          r->err = "request larger than the server's device-memory budget";
          r->state = DONE;
          r->t_done = s->now();
          s->cv_done.notify_all();
          progressed = true;
          continue;
        }
        int slot = -1;
        for (int i = 0; i < s->max_active; ++i)
          if (!s->slots[i]) { slot = i; break; }
        if (slot < 0) break;
        // memory held by running and by finished-but-unpolled requests is what the arena holds;
        // unpolled solutions give way to queued work (moved to the host, oldest first)
        if (s->arena->used() + r->need > s->budget) {
          spill = !s->held.empty();
          break;
        }
        s->queue.pop_front();
        r->slot = slot;
        r->state = RUNNING;
        r->t_start = s->now();
        s->slots[slot] = r;
        to_start.push_back(r);
      }
    }
    if (spill && spill_oldest(s)) progressed = true;
    for (Request* r : to_start) {
      start_request(s, r);
      progressed = true;
      if (r->status != PINT_OK) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->slots[r->slot] = nullptr;
        bool others = false;
        for (Request* a : s->slots) others = others || a;
        if (r->status == PINT_ENOMEM && (others || !s->held.empty())) {
          // the arena is fragmented or the estimate was short: retry once others finish
          r->status = PINT_OK;
          r->state = QUEUED;
          r->slot = -1;
          s->queue.push_front(r);
          continue;
        }
        if (r->status == PINT_ENOMEM) r->status = PINT_EBUDGET;
        r->state = DONE;
        r->t_done = s->now();
        s->cv_done.notify_all();
      }
    }
    // retire finished requests
    for (int i = 0; i < s->max_active; ++i) {
      Request* r = nullptr;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        r = s->slots[i];
      }
      if (!r || r->status != PINT_OK) continue;
      const cudaError_t q = cudaEventQuery(s->events[i]);
      if (q == cudaErrorNotReady) continue;
      bool conv = false;
      if (q == cudaSuccess) {
        // the solution stays on the device until it is polled (or moved to the host when its
        // memory is needed for queued requests); everything else returns to the budget now
        solve_result(r->plan, &r->sweeps, &r->upd, &conv);
        r->status = solve_wait_gave_up(r->plan) ? PINT_ECUDA : (conv ? PINT_OK : PINT_ENOTCONV);
        release_request_inputs(s, r);
      } else {
        r->status = PINT_ECUDA;
        r->err = cudaGetErrorString(q);
        release_request_memory(s, r);
      }
      std::lock_guard<std::mutex> lk(s->mu);
      if (r->dU) {
        r->held = true;
        s->held.push_back(r);
      }
      r->t_done = s->now();
      r->state = DONE;
      s->slots[i] = nullptr;
      const pint_plan_desc& d = r->req.desc;
      s->completed += 1;
      s->dof_done += (double)d.N * d.grid.mx * (d.grid.dim == 2 ? d.grid.my : 1);
      s->sweeps_done += r->sweeps;
      s->cv_done.notify_all();
      progressed = true;
    }
    if (!progressed) {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
  }
}

pint_status srv_fail(pint_status st, const char* m) {
  set_last_error(m);
  return st;
}

}  // namespace

extern "C" pint_status pint_server_create(size_t hbm_budget_bytes, int max_active, pint_server* out) {
  if (!out || hbm_budget_bytes < ((size_t)1 << 20) || max_active < 1 || max_active > 256)
    return srv_fail(PINT_EINVAL, "budget must be >= 1 MiB and max_active in 1..256");
  pint_server_s* s = new pint_server_s();
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  cudaGetDevice(&s->device);
  void* base = nullptr;
  cudaError_t e = lib_malloc(&base, hbm_budget_bytes);
  if (e != cudaSuccess) {
    delete s;
    return srv_fail(PINT_ENOMEM, "cannot reserve the device-memory budget");
  }
  s->base = (char*)base;
  void* pinned = nullptr;
  if (lib_malloc_host(&pinned, (size_t)max_active * 4 * Arena::kHostBlock) != cudaSuccess) {
    lib_free(base, hbm_budget_bytes);
    delete s;
    return srv_fail(PINT_ENOMEM, "cannot allocate pinned host buffers");
  }
  s->pinned = (char*)pinned;
  s->arena = new Arena(s->base, hbm_budget_bytes, s->pinned, max_active * 4);
  s->streams.resize(max_active);
  s->events.resize(max_active);
  s->slots.assign(max_active, nullptr);
  for (int i = 0; i < max_active; ++i) {
    cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&s->events[i], cudaEventDisableTiming);
  }
  s->t0 = clk::now();
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return PINT_OK;
}

extern "C" pint_status pint_server_destroy(pint_server s) {
  if (!s) return PINT_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
  for (auto& kv : s->reqs) {
    release_request_memory(s, kv.second);
    delete kv.second;
  }
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
  delete s->arena;
  lib_free(s->base, s->budget);
  lib_free_host(s->pinned);
  delete s;
  return PINT_OK;
}

extern "C" pint_status pint_submit(pint_server s, const pint_request* req, const double* v, const double* f,
                                   const double* fderiv, uint64_t* ticket) {
  if (!s || !req || !v || !f || !ticket) return srv_fail(PINT_EINVAL, "NULL argument");
  const pint_plan_desc& d = req->desc;
  if (d.k < 1 || d.k > kMaxK || d.N < 8 || d.grid.mx < 1 || (d.grid.dim == 2 && d.grid.my < 1) ||
      (d.grid.dim != 1 && d.grid.dim != 2))
    return srv_fail(PINT_EINVAL, "invalid problem description");
  if (d.k >= 2 && !fderiv) return srv_fail(PINT_EINVAL, "fderiv is required for k >= 2");
  if (!(req->tol > 0.0) || req->max_sweeps < 1) return srv_fail(PINT_EINVAL, "tol must be > 0, max_sweeps >= 1");
  Request* r = new Request();
  r->req = *req;
  const size_t M = (size_t)d.grid.mx * (d.grid.dim == 2 ? d.grid.my : 1);
  const size_t NM = (size_t)d.N * M;
  if (req->inputs_on_device) {
    r->uv = v;
    r->uf = f;
    r->ufd = fderiv;
  } else {
    r->v.assign(v, v + M);
    r->f.assign(f, f + NM);
    if (d.k >= 2) r->fd.assign(fderiv, fderiv + (size_t)(d.k - 1) * M);
  }
  r->need = request_bytes(*req);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    r->t_submit = s->now();
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
  }
  s->cv_work.notify_all();
  return PINT_OK;
}

extern "C" pint_status pint_poll(pint_server s, uint64_t ticket, int timeout_us, double* U_out,
                                 pint_solve_info* info) {
  if (!s) return srv_fail(PINT_EINVAL, "NULL server");
  Request* r = nullptr;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return srv_fail(PINT_ENOTFOUND, "unknown ticket");
    r = it->second;
    if (r->state != DONE && timeout_us > 0)
      s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->state == DONE; });
    if (r->state != DONE) {
      if (info) {
        info->status = timeout_us > 0 ? PINT_ETIMEOUT : PINT_EAGAIN;
        info->sweeps = 0;
        info->upd_rel = 0.0;
        info->t_submit = r->t_submit;
        info->t_start = r->t_start;
        info->t_done = 0.0;
      }
      return timeout_us > 0 ? PINT_ETIMEOUT : PINT_EAGAIN;
    }
    // a solution being moved to the host by the worker: wait for the move (it is one copy)
    while (r->spilling) s->cv_done.wait_for(lk, std::chrono::milliseconds(10));
    s->reqs.erase(it);
    if (r->held) {
      s->held.erase(std::find(s->held.begin(), s->held.end(), r));
      r->held = false;
    }
  }
  pint_status st = r->status;
  if ((st == PINT_OK || st == PINT_ENOTCONV) && U_out) {
    if (r->dU) {
      const cudaError_t ce = cudaMemcpy(U_out, r->dU, request_unknowns(r) * sizeof(double), cudaMemcpyDeviceToHost);
      if (ce != cudaSuccess) {
        st = PINT_ECUDA;
        r->err = cudaGetErrorString(ce);
      }
    } else if (!r->result.empty()) {
      std::memcpy(U_out, r->result.data(), r->result.size() * sizeof(double));
    }
  }
  if (r->dU) s->arena->release(r->dU);
  r->dU = nullptr;
  if (info) {
    info->status = st;
    info->sweeps = r->sweeps;
    info->upd_rel = r->upd;
    info->t_submit = r->t_submit;
    info->t_start = r->t_start;
    info->t_done = r->t_done;
  }
  if (st != PINT_OK) set_last_error(r->err.empty() ? "solve did not converge" : r->err.c_str());
  delete r;
  return st;
}

extern "C" pint_status pint_server_stats(pint_server s, double* out) {
  if (!s || !out) return srv_fail(PINT_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  int active = 0;
  for (Request* r : s->slots) active += r ? 1 : 0;
  out[0] = s->completed;
  out[1] = active;
  out[2] = (double)s->queue.size();
  out[3] = (double)s->arena->used();
  out[4] = s->dof_done;
  out[5] = s->sweeps_done;
  out[6] = s->now();
  out[7] = (double)s->arena->peak();
  return PINT_OK;
}
