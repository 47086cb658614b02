// serve.cpp -- serving loop: continuous batching of control problems.
//
// A server owns `max_active` worker slots on one device.  Submitted requests
// (any kind, grid level, n_t, beta, nu, precision) wait in submission order;
// a free slot admits the oldest waiting request as soon as its device-memory
// estimate (pint_estimate_device_bytes) fits in what the requests on the GPU
// leave of the budget.  An admitted request gets its own handle and CUDA
// stream: its data and Krylov state stay resident on the device until it
// completes, and the kernels of all admitted requests run concurrently on
// the GPU.  A request that could not be created for lack of memory goes back
// to the head of the queue while other requests are running (and fails only
// when it cannot fit on an otherwise empty server).  Results, statuses and
// latencies (submission to completion) are kept until collected.
//
// With share_solves, each request's handle is a member of a group (same grid,
// domain, wind, nu, precision, inner-solver settings): its frequency solves
// run batched with those of the other members in the group's shared context
// (api.cu, batch.h), and admission counts the request's share of that
// context.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.h"
#include "pint.h"

namespace {

using clk = std::chrono::steady_clock;

struct Request {
  long long id = 0;
  pint_params p{};
  std::vector<double> vd, f, v0;
  size_t est = 0;
  size_t kkt_len = 0;
  long long retry_after = -1;  // admit again only after this many completions (+1)
  clk::time_point t_submit, t_done;
  bool done = false;
  pint_status status = PINT_OK;
  std::string msg;
  std::vector<double> x;
  pint_solve_info info{};
};

}  // namespace

struct pint_server_s {
  int dev = 0;
  size_t budget = 0;
  int max_active = 1;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::unordered_map<long long, Request*> all;
  long long next_id = 1;
  size_t in_use = 0, peak_bytes = 0;
  int active = 0, peak_active = 0;
  long long submitted = 0, completed = 0, failed = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  pint_batcher_s* batcher = nullptr;  // shared frequency solves (share_solves)

  void worker();
  bool run(Request* r, cudaStream_t st);
};

namespace {
thread_local std::string s_err;

size_t kkt_len_of(const pint_params& p) {
  const size_t N = (size_t)1 << p.level, ns = (2 * N + 1) * (2 * N + 1), nq = (N + 1) * (N + 1);
  return (size_t)p.n_t * (4 * ns + 2 * nq);
}
size_t ns_of(const pint_params& p) {
  const size_t N = (size_t)1 << p.level;
  return (2 * N + 1) * (2 * N + 1);
}
}  // namespace

// Solve one request on its own handle and stream; false if the handle could
// not be created for lack of device memory (the caller may retry later).
bool pint_server_s::run(Request* r, cudaStream_t st) {
  pint_handle h = nullptr;
  pint_status rc = batcher ? member_create(batcher, &r->p, st, &h) : pint_create(&r->p, st, &h);
  if (rc == PINT_ERR_OOM) return false;
  if (rc != PINT_OK) {
    r->status = rc;
    r->msg = pint_last_error(nullptr);
    return true;
  }
  rc = pint_set_data(h, r->vd.data(), r->f.empty() ? nullptr : r->f.data(), r->v0.empty() ? nullptr : r->v0.data());
  if (rc == PINT_OK) {
    r->x.assign(r->kkt_len, 0.0);
    rc = pint_solve_host(h, r->x.data(), &r->info);
  }
  if (rc != PINT_OK) r->msg = pint_last_error(h);
  r->status = rc;
  pint_destroy(h);
  r->vd.clear();
  r->vd.shrink_to_fit();
  r->f.clear();
  r->v0.clear();
  return true;
}

void pint_server_s::worker() {
  cudaSetDevice(dev);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait(lk, [&] {
        if (queue.empty()) return stop;
        const Request* h = queue.front();
        return h->est <= budget - in_use && h->retry_after < completed + failed;
      });
      if (queue.empty()) break;
      r = queue.front();
      queue.pop_front();
      in_use += r->est;
      peak_bytes = std::max(peak_bytes, in_use);
      ++active;
      peak_active = std::max(peak_active, active);
    }
    const bool finished = run(r, st);
    std::lock_guard<std::mutex> lk(mu);
    in_use -= r->est;
    --active;
    if (!finished) {
      if (active > 0) {
        r->retry_after = completed + failed;  // memory frees up when a running request completes
        queue.push_front(r);
        cv.notify_all();
        continue;
      }
      r->status = PINT_ERR_OOM;
      r->msg = "request does not fit in device memory";
    }
    r->done = true;
    r->t_done = clk::now();
    if (r->status == PINT_OK)
      ++completed;
    else
      ++failed;
    cv.notify_all();
  }
  cudaStreamDestroy(st);
}

extern "C" {

pint_status pint_server_create(const pint_server_params* sp, pint_server* out) {
  if (!sp || !out) return s_err = "null argument", PINT_ERR_ARG;
  if (sp->max_active < 1 || sp->max_active > 64) return s_err = "max_active must be in [1, 64]", PINT_ERR_ARG;
  pint_server s = new pint_server_s();
  cudaGetDevice(&s->dev);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    delete s;
    return s_err = "cudaMemGetInfo failed", PINT_ERR_CUDA;
  }
  s->budget = sp->device_budget ? std::min(sp->device_budget, free_b) : free_b / 10 * 9;
  s->max_active = sp->max_active;
  if (sp->share_solves) s->batcher = batcher_create();
  for (int i = 0; i < s->max_active; ++i) s->workers.emplace_back([s] { s->worker(); });
  *out = s;
  return PINT_OK;
}

pint_status pint_server_submit(pint_server s, const pint_params* p, const double* vd, const double* f,
                               const double* v0, long long* id) {
  if (!s || !p || !vd || !id) return s_err = "null argument", PINT_ERR_ARG;
  size_t est = pint_estimate_device_bytes(p);
  if (est == 0) return s_err = "invalid parameters", PINT_ERR_ARG;
  if (s->batcher) {
    // the member's own buffers plus its frequencies' share of the group's context
    size_t mb = 0, pf = 0;
    shared_estimates(p, &mb, &pf);
    est = mb + (size_t)(p->n_t / 2 + 1) * pf;
  }
  if (est > s->budget) return s_err = "request needs more device memory than the server's budget", PINT_ERR_OOM;
  Request* r = new Request();
  r->p = *p;
  r->est = est;
  r->kkt_len = kkt_len_of(*p);
  const size_t nv = (size_t)p->n_t * 2 * ns_of(*p);
  r->vd.assign(vd, vd + nv);
  if (f) r->f.assign(f, f + nv);
  if (v0) r->v0.assign(v0, v0 + 2 * ns_of(*p));
  r->t_submit = clk::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    delete r;
    return s_err = "server is shutting down", PINT_ERR_STATE;
  }
  r->id = s->next_id++;
  s->all[r->id] = r;
  s->queue.push_back(r);
  ++s->submitted;
  *id = r->id;
  s->cv.notify_all();
  return PINT_OK;
}

pint_status pint_server_wait(pint_server s, long long id, double* x_host, pint_solve_info* info, double* latency_ms) {
  if (!s) return s_err = "null server", PINT_ERR_ARG;
  Request* r = nullptr;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return s_err = "unknown or already collected request id", PINT_ERR_ARG;
    r = it->second;
    s->cv.wait(lk, [&] { return r->done; });
    s->all.erase(id);  // by key: the map may have rehashed while waiting
  }
  if (x_host && !r->x.empty()) std::copy(r->x.begin(), r->x.end(), x_host);
  if (info) *info = r->info;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  const pint_status st = r->status;
  s_err = r->msg;
  delete r;
  return st;
}

pint_status pint_server_get_stats(pint_server s, pint_server_stats* out) {
  if (!s || !out) return s_err = "null argument", PINT_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->active = s->active;
  out->queued = (long long)s->queue.size();
  out->budget_bytes = s->budget;
  out->bytes_in_use = s->in_use;
  out->bytes_peak = s->peak_bytes;
  out->active_peak = s->peak_active;
  pint_group_stats bs{};
  if (s->batcher) batcher_get_stats(s->batcher, &bs);
  out->shared_batches = bs.batches;
  out->shared_member_solves = bs.member_solves;
  out->shared_frequencies = bs.frequencies;
  out->shared_max_members = bs.max_members;
  return PINT_OK;
}

pint_status pint_server_destroy(pint_server s) {
  if (!s) return PINT_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  for (auto& t : s->workers) t.join();
  batcher_destroy(s->batcher);
  for (auto& kv : s->all) delete kv.second;
  delete s;
  return PINT_OK;
}

const char* pint_server_last_error(void) { return s_err.c_str(); }

}  // extern "C"
