// Serving: a request loop that runs Davidson solves of different cells,
// cut-offs and band counts as they arrive (continuous batching), admits them by
// a device-memory budget, keeps each solve's state on the device while it runs,
// and reports per-request latency.
//
// The paper's outlook (Sec. 4) observes that memory per card bounds the system
// size and that ensembles of many independent runs are the way to fill an
// exascale machine; Sec. 3.3 notes that over-subscribing one GPU with several
// small runs pays off.  Here one engine thread owns a context and a stream and
// advances every admitted solve in lockstep rounds (dvtask.h): a round applies
// H to the new basis vectors of ALL running solves in one batched call (one
// persistent launch per FFT stage over every cell's bands), then takes one
// Rayleigh-Ritz step of each.  Between rounds, requests are admitted in arrival
// order while the number of running solves is below max_slots and the
// estimated device footprint fits in what the budget has left, so a new
// arrival joins at the next iteration boundary; a finished solve returns its
// results and its workspace.  A solve's arithmetic is the same whatever else
// runs (deterministic kernels, its own buffers): results are bit for bit those
// of the solve alone.
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
#include "dvtask.h"

namespace qe {
int ctx_begin(qe_ctx* ctx, cudaStream_t st);
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

// One running solve of the engine.
struct Active {
  std::shared_ptr<Request> r;
  qe::DvTask* task = nullptr;   // GPU solve
  int fake_left = 0;            // QE_SERVE_FAKE_SOLVER: rounds left
  bool failed = false;
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
  long long submitted = 0, completed = 0, rounds = 0;
  std::thread engine;
  qe_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  // side streams of the per-solve Rayleigh-Ritz steps and the fork/join events
  std::vector<void*> side, events;
};

// Side streams of the engine: the dense eigensolvers of that many running
// solves overlap within a round.
constexpr int kServeSideStreams = 8;

namespace {

// Test hook (QE_SERVE_FAKE_SOLVER): no GPU work; a "solve" takes max_iter
// rounds of 1 ms, copies psi through, returns evals = 0 and QE_OK, or
// QE_ENOCONV when tol > 1.  Exercises admission, queueing, cancellation and
// timeouts on machines without a GPU.
void fake_finish(Request& r) {
  std::fill(r.evals.begin(), r.evals.end(), 0.0);
  std::fill(r.resid.begin(), r.resid.end(), 0.0);
  r.iters = r.max_iter;
  r.status = r.tol > 1.0 ? QE_ENOCONV : QE_OK;
}

// Set up the device side of an admitted request; false (status set) on failure.
bool start_solve(qe_srv* s, Active& a) {
  Request& r = *a.r;
  if (s->flags & QE_SERVE_FAKE_SOLVER) {
    a.fake_left = r.max_iter;
    return true;
  }
  r.prob.vloc_r = r.vloc.data();
  r.prob.beta = r.beta.empty() ? nullptr : r.beta.data();
  r.prob.dmat = r.dmat.empty() ? nullptr : r.dmat.data();
  r.prob.mem = QE_HOST;
  const int rc = qe::dv_task_create(s->ctx, &r.prob, r.precision, r.tol, r.max_iter, 0, r.psi.data(),
                                    s->st, &a.task);
  if (rc) {
    r.status = rc;
    r.err = qe_last_error();
    return false;
  }
  return true;
}

// Results of a finished solve into the request; frees its device state.
void finish_solve(qe_srv* s, Active& a) {
  Request& r = *a.r;
  if (s->flags & QE_SERVE_FAKE_SOLVER) {
    fake_finish(r);
    return;
  }
  if (a.task) {
    int it = 0;
    r.status = qe::dv_task_result(s->ctx, a.task, r.psi.data(), r.evals.data(), r.resid.data(), &it,
                                  false, s->st);
    r.iters = it;
    if (r.status != QE_OK) r.err = qe_last_error();
    qe::dv_task_destroy(a.task, s->st);
    a.task = nullptr;
    cudaStreamSynchronize(s->st);
  }
}

void engine_loop(qe_srv* s) {
  const bool fake = (s->flags & QE_SERVE_FAKE_SOLVER) != 0;
  if (!fake) {
    cudaSetDevice(s->device);
    qe::ctx_begin(s->ctx, s->st);   // the context's buffers and plans follow the engine stream
  }
  std::vector<Active> act;
  while (true) {
    std::vector<std::shared_ptr<Request>> admit;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      auto can_admit = [&] {
        return !s->stop && !s->pending.empty() && (int)act.size() + (int)admit.size() < s->max_slots &&
               s->used + s->pending.front()->bytes <= s->budget;
      };
      if (act.empty()) s->cv_work.wait(lk, [&] { return s->stop || can_admit(); });
      if (s->stop && act.empty()) return;
      while (can_admit()) {
        auto r = s->pending.front();
        s->pending.pop_front();
        s->used += r->bytes;
        s->running++;
        r->running = true;
        admit.push_back(r);
      }
    }
    for (auto& r : admit) {
      Active a;
      a.r = r;
      a.failed = !start_solve(s, a);
      act.push_back(a);
    }
    // one lockstep round of every running solve
    if (fake) {
      bool any = false;
      for (auto& a : act) any = any || (!a.failed && a.fake_left > 0);
      if (any) std::this_thread::sleep_for(std::chrono::milliseconds(1));
      for (auto& a : act)
        if (a.fake_left > 0) --a.fake_left;
    } else {
      std::vector<qe::DvTask*> ts;
      for (auto& a : act)
        if (!a.failed && a.task && !qe::dv_task_done(a.task)) ts.push_back(a.task);
      if (!ts.empty())
        qe::dv_round(s->ctx, ts.data(), (int)ts.size(), s->st, s->side.data(), (int)s->side.size(),
                     s->events.data());
    }
    // completions
    std::vector<Active> keep;
    std::vector<Active> fin;
    for (auto& a : act) {
      const bool done = a.failed || (fake ? a.fake_left <= 0 : qe::dv_task_done(a.task));
      (done ? fin : keep).push_back(a);
    }
    act.swap(keep);
    for (auto& a : fin) {
      if (!a.failed) finish_solve(s, a);
      std::lock_guard<std::mutex> lk(s->mu);
      a.r->t_done = Clock::now();
      a.r->running = false;
      a.r->done = true;
      if (a.r->canceled) a.r->status = QE_ECANCELED;
      s->used -= a.r->bytes;
      s->running--;
      s->completed++;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->rounds++;
    }
    if (!fin.empty()) {
      // keep the plan cache and the shared workspaces from growing without
      // bound over a long stream of different cells
      if (!fake && act.empty()) qe::ctx_trim_public(s->ctx);
      s->cv_done.notify_all();
    }
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
  if (!(flags & QE_SERVE_FAKE_SOLVER)) {
    int rc = qe_ctx_create(device, &s->ctx);
    if (rc) return rc;
    bool ok = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; ok && i < kServeSideStreams; ++i) {
      cudaStream_t x = nullptr;
      ok = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) == cudaSuccess;
      if (ok) s->side.push_back(x);
    }
    for (int i = 0; ok && i <= kServeSideStreams; ++i) {
      cudaEvent_t e = nullptr;
      ok = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
      if (ok) s->events.push_back(e);
    }
    if (!ok) {
      cudaGetLastError();
      for (void* x : s->side) cudaStreamDestroy((cudaStream_t)x);
      for (void* e : s->events) cudaEventDestroy((cudaEvent_t)e);
      if (s->st) cudaStreamDestroy(s->st);
      qe_ctx_destroy(s->ctx);
      qe::set_error("qe_serve_create: stream or event creation failed");
      return QE_ECUDA;
    }
  }
  qe_srv* raw = s.release();
  raw->engine = std::thread(engine_loop, raw);
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
  if (s->engine.joinable()) s->engine.join();
  if (s->ctx) qe_ctx_destroy(s->ctx);
  for (void* x : s->side) cudaStreamDestroy((cudaStream_t)x);
  for (void* e : s->events) cudaEventDestroy((cudaEvent_t)e);
  if (s->st) cudaStreamDestroy(s->st);
  delete s;
}

}  // extern "C"
