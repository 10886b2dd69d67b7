// Serving: a request loop that runs Davidson solves of different cells,
// cut-offs and band counts as they arrive (continuous batching), admits them by
// a device-memory budget, keeps each solve's state on the device while it runs,
// and reports per-request latency.
//
// The paper's outlook (Sec. 4) observes that memory per card bounds the system
// size and that ensembles of many independent runs are the way to fill an
// exascale machine; Sec. 3.3 notes that over-subscribing one GPU with several
// small runs pays off.  Here every admitted request gets a slot: a worker thread
// with its own context and CUDA stream, so the kernels of concurrent solves
// overlap on the GPU.  A request is admitted, in arrival order, when a slot is
// idle and its estimated device footprint fits in what the budget has left;
// when a solve finishes its workspace goes back to the stream-ordered pool and
// the next request is admitted.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "common.h"

namespace qe {
int ctx_trim_public(qe_ctx* ctx);
size_t davidson_footprint(int npw, int nb, int max_dim, int nproj, const int grid[3], int nst);
int default_max_dim(int nb);
}  // namespace qe

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  qe_problem prob{};
  std::vector<double> vloc, beta, dmat, psi;   // owned copies of the inputs; psi is in/out
  std::vector<double> evals, resid;
  int precision = QE_FP64;
  double tol = 1e-8;
  int max_iter = 100;
  int npw = 0;
  size_t bytes = 0;
  Clock::time_point t_submit, t_done;
  int status = QE_PENDING;
  int iters = 0;
  bool running = false, done = false, canceled = false;
  std::string err;
};

struct Worker {
  std::thread th;
  qe_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
};

}  // namespace

struct qe_srv {
  int device = 0;
  size_t budget = 0, used = 0;
  int max_slots = 1, max_queue = 1;
  int flags = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> pending;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  uint64_t next_id = 1;
  bool stop = false;
  int running = 0;
  long long submitted = 0, completed = 0;
  std::vector<std::unique_ptr<Worker>> workers;
};

namespace {

// Test hook (QE_SERVE_FAKE_SOLVER): no GPU work; a "solve" sleeps max_iter
// milliseconds, copies psi through, returns evals = 0 and QE_OK, or QE_ENOCONV
// when tol > 1.  Exercises admission, queueing, cancellation and timeouts on
// machines without a GPU.
void fake_solve(Request& r) {
  std::this_thread::sleep_for(std::chrono::milliseconds(r.max_iter));
  std::fill(r.evals.begin(), r.evals.end(), 0.0);
  std::fill(r.resid.begin(), r.resid.end(), 0.0);
  r.iters = r.max_iter;
  r.status = r.tol > 1.0 ? QE_ENOCONV : QE_OK;
}

void worker_loop(qe_srv* s, Worker* w) {
  const bool fake = (s->flags & QE_SERVE_FAKE_SOLVER) != 0;
  if (!fake) cudaSetDevice(s->device);
  while (true) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] {
        return s->stop || (!s->pending.empty() && s->used + s->pending.front()->bytes <= s->budget);
      });
      if (s->stop) return;
      r = s->pending.front();
      s->pending.pop_front();
      s->used += r->bytes;
      s->running++;
      r->running = true;
    }
    if (fake) {
      fake_solve(*r);
    } else {
      r->prob.vloc_r = r->vloc.data();
      r->prob.beta = r->beta.empty() ? nullptr : r->beta.data();
      r->prob.dmat = r->dmat.empty() ? nullptr : r->dmat.data();
      r->prob.mem = QE_HOST;
      int it = 0;
      r->status = qe_davidson(w->ctx, &r->prob, r->precision, r->tol, r->max_iter, 0, r->psi.data(),
                              r->evals.data(), r->resid.data(), &it, w->st);
      r->iters = it;
      if (r->status != QE_OK) r->err = qe_last_error();
      // give the workspace back so that the budget accounting stays true
      qe::ctx_trim_public(w->ctx);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->t_done = Clock::now();
      r->running = false;
      r->done = true;
      if (r->canceled) r->status = QE_ECANCELED;
      s->used -= r->bytes;
      s->running--;
      s->completed++;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

int qe_serve_create(int device, size_t hbm_budget_bytes, int max_slots, int max_queue, int flags,
                    qe_srv** out) {
  qe::clear_error();
  if (!out || max_slots < 1 || max_queue < 1 || hbm_budget_bytes == 0) {
    qe::set_error("qe_serve_create: invalid argument");
    return QE_EINVAL;
  }
  *out = nullptr;
  auto s = std::make_unique<qe_srv>();
  s->device = device;
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  s->max_queue = max_queue;
  s->flags = flags;
  const bool fake = (flags & QE_SERVE_FAKE_SOLVER) != 0;
  for (int i = 0; i < max_slots; ++i) {
    auto w = std::make_unique<Worker>();
    if (!fake) {
      int rc = qe_ctx_create(device, &w->ctx);
      if (rc) {
        for (auto& x : s->workers) {
          if (x->ctx) qe_ctx_destroy(x->ctx);
          if (x->st) cudaStreamDestroy(x->st);
        }
        return rc;
      }
      if (cudaStreamCreateWithFlags(&w->st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        qe_ctx_destroy(w->ctx);
        for (auto& x : s->workers) {
          if (x->ctx) qe_ctx_destroy(x->ctx);
          if (x->st) cudaStreamDestroy(x->st);
        }
        qe::set_error("qe_serve_create: cudaStreamCreate failed");
        return QE_ECUDA;
      }
    }
    s->workers.push_back(std::move(w));
  }
  qe_srv* raw = s.release();
  for (auto& w : raw->workers) w->th = std::thread(worker_loop, raw, w.get());
  *out = raw;
  return QE_OK;
}

int qe_serve_submit(qe_srv* s, const qe_problem* prob, int precision, double tol, int max_iter,
                    const double* psi0, uint64_t* ticket) {
  qe::clear_error();
  if (!s || !prob || !psi0 || !ticket) { qe::set_error("qe_serve_submit: null argument"); return QE_EINVAL; }
  if (prob->mem != QE_HOST) { qe::set_error("qe_serve_submit: inputs must be host arrays"); return QE_EINVAL; }
  if (prob->nbnd < 1 || prob->nproj < 0 || !prob->vloc_r || (prob->nproj > 0 && (!prob->beta || !prob->dmat))) {
    qe::set_error("qe_serve_submit: invalid problem");
    return QE_EINVAL;
  }
  if (precision != QE_FP64 && precision != QE_MIXED) { qe::set_error("qe_serve_submit: bad precision"); return QE_EINVAL; }
  if (!(tol > 0.0) || max_iter < 0) { qe::set_error("qe_serve_submit: bad tol/max_iter"); return QE_EINVAL; }
  qe::PlanHost h;
  int rc = qe::build_plan_host(prob->lat, prob->k, prob->ecutwfc, prob->grid, h);
  if (rc) return rc;
  auto r = std::make_shared<Request>();
  r->prob = *prob;
  r->npw = h.npw;
  r->precision = precision;
  r->tol = tol;
  r->max_iter = max_iter;
  const int nb = prob->nbnd;
  if (nb > h.npw) { qe::set_error("qe_serve_submit: more bands than plane waves"); return QE_EINVAL; }
  r->bytes = qe::davidson_footprint(h.npw, nb, qe::default_max_dim(nb), prob->nproj, prob->grid, h.nst);
  if (r->bytes > s->budget) {
    qe::set_error("qe_serve_submit: request needs %zu bytes, budget is %zu", r->bytes, s->budget);
    return QE_EINVAL;
  }
  const size_t ng = (size_t)prob->grid[0] * prob->grid[1] * prob->grid[2];
  r->vloc.assign(prob->vloc_r, prob->vloc_r + ng);
  if (prob->nproj > 0) {
    r->beta.assign(prob->beta, prob->beta + (size_t)prob->nproj * h.npw * 2);
    r->dmat.assign(prob->dmat, prob->dmat + (size_t)prob->nproj * prob->nproj);
  }
  r->psi.assign(psi0, psi0 + (size_t)nb * h.npw * 2);
  r->evals.assign(nb, 0.0);
  r->resid.assign(nb, 0.0);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if ((int)s->pending.size() >= s->max_queue) {
      qe::set_error("qe_serve_submit: queue full (%d waiting)", (int)s->pending.size());
      return QE_EAGAIN;
    }
    r->id = s->next_id++;
    r->t_submit = Clock::now();
    s->pending.push_back(r);
    s->all[r->id] = r;
    s->submitted++;
    *ticket = r->id;
  }
  s->cv_work.notify_all();
  return QE_OK;
}

int qe_serve_poll(qe_srv* s, uint64_t ticket, int timeout_ms, double* psi_out, double* evals,
                  double* resid, int* iters, double* latency_s) {
  qe::clear_error();
  if (!s) { qe::set_error("qe_serve_poll: null server"); return QE_EINVAL; }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) { qe::set_error("qe_serve_poll: unknown ticket %llu", (unsigned long long)ticket); return QE_EINVAL; }
  std::shared_ptr<Request> r = it->second;
  if (!r->done && timeout_ms != 0) {
    auto pred = [&] { return r->done; };
    if (timeout_ms < 0) s->cv_done.wait(lk, pred);
    else s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred);
  }
  if (!r->done) return QE_PENDING;
  if (psi_out) std::memcpy(psi_out, r->psi.data(), r->psi.size() * sizeof(double));
  if (evals) std::memcpy(evals, r->evals.data(), r->evals.size() * sizeof(double));
  if (resid) std::memcpy(resid, r->resid.data(), r->resid.size() * sizeof(double));
  if (iters) *iters = r->iters;
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  s->all.erase(it);
  if (r->status != QE_OK) qe::set_error("%s", r->err.empty() ? "request did not complete" : r->err.c_str());
  return r->status;
}

int qe_serve_cancel(qe_srv* s, uint64_t ticket) {
  qe::clear_error();
  if (!s) { qe::set_error("qe_serve_cancel: null server"); return QE_EINVAL; }
  bool notify = false;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) { qe::set_error("qe_serve_cancel: unknown ticket"); return QE_EINVAL; }
    auto r = it->second;
    if (r->done) return QE_OK;
    r->canceled = true;
    if (!r->running) {
      for (auto p = s->pending.begin(); p != s->pending.end(); ++p)
        if ((*p)->id == ticket) { s->pending.erase(p); break; }
      r->done = true;
      r->status = QE_ECANCELED;
      r->t_done = Clock::now();
      notify = true;
    }
  }
  if (notify) { s->cv_done.notify_all(); s->cv_work.notify_all(); }
  return QE_OK;
}

int qe_serve_stats(qe_srv* s, long long* submitted, long long* completed, int* running,
                   int* queued, size_t* bytes_in_use) {
  if (!s) { qe::set_error("qe_serve_stats: null server"); return QE_EINVAL; }
  std::lock_guard<std::mutex> lk(s->mu);
  if (submitted) *submitted = s->submitted;
  if (completed) *completed = s->completed;
  if (running) *running = s->running;
  if (queued) *queued = (int)s->pending.size();
  if (bytes_in_use) *bytes_in_use = s->used;
  return QE_OK;
}

void qe_serve_destroy(qe_srv* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto& r : s->pending) {
      r->done = true;
      r->status = QE_ECANCELED;
    }
    s->pending.clear();
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  for (auto& w : s->workers)
    if (w->th.joinable()) w->th.join();
  for (auto& w : s->workers) {
    if (w->ctx) qe_ctx_destroy(w->ctx);
    if (w->st) cudaStreamDestroy(w->st);
  }
  delete s;
}

}  // extern "C"
