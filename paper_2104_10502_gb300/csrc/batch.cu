// Batches of problems (k points of one cell, independent cells, different
// cut-offs, grids and band counts) in one set of launches, CUDA-graph replay
// of a fixed batch, and the FFT launch-shape autotuner.
//
// The paper's benchmarks parallelise over k points only (pools, Sec. 3.3) and
// note that over-subscribing a GPU with several small runs pays off; here the
// problems of a batch share each FFT stage: one persistent launch per stage
// pulls (problem, band, tile) items of every problem from a work counter, so
// small cells fill the GPU together instead of one after the other.
#include <algorithm>
#include <cstring>
#include <memory>
#include <type_traits>
#include <vector>

#include "ctx.h"

namespace qe {

#define BT_TRY(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)
#define BT_CU(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_error("%s: %s", #x, cudaGetErrorString(e_)); return QE_ECUDA; } } while (0)

void store_shape(const int grid[3], size_t elem_bytes, const FftShape& s);

static size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// Workspaces of a batched H|psi>.  An eager call uses the context's; a captured
// batch (qe_batch) owns its own, because the graph keeps their addresses.
struct BatchWork {
  cudaStream_t cur = nullptr;
  DevBuf ws, part, proj, projd, tc_work, tc_beta, tc_status, oz_work, oz_beta;
  BatchWork() {
    for (DevBuf* b : {&ws, &part, &proj, &projd, &tc_work, &tc_beta, &tc_status, &oz_work, &oz_beta})
      b->sp = &cur;
  }
  void release() {
    for (DevBuf* b : {&ws, &part, &proj, &projd, &tc_work, &tc_beta, &tc_status, &oz_work, &oz_beta})
      b->release();
  }
};

// Everything a batched H|psi> needs, laid out in one device buffer.
struct BatchLayout {
  std::vector<DevPlan*> plans;
  std::vector<OpView> ops;
  std::vector<size_t> vp_off, w_off;
  size_t jobs_off = 0, prefix_off = 0, counters_off = 0, total = 0;
  size_t smem_z = 0, smem_p = 0;
  size_t np_max_part = 0, np_max_proj = 0;   // nonlocal workspaces (largest problem)
  size_t tc_work = 0, tc_beta = 0;
  size_t oz_work = 0, oz_beta = 0;
  std::vector<char> pair;   // per problem: bands taken two per FFT (real in r, k = 0)
  bool all_sqz = true;      // every problem's z lines take the two-pass transform
};

// A problem's launch shape inside a batch: its tuned shape, except that when
// the batch's z stages run 256 threads (not every problem has two-pass z lines)
// the two-pass z lines take the 32-stick tiles that suit that thread count.
template <typename T>
static FftShape batch_shape(const DevPlan& P, bool all_sqz) {
  FftShape sh = tuned_shape(P, sizeof(T));
  if (!all_sqz && P.sqz && sh.spb == 0) sh.spb = default_spb<T>(P.grid[2]);
  return sh;
}

template <typename T>
static int batch_prepare(qe_ctx* ctx, BatchWork& W, int nprob, const qe_problem* probs,
                         const double* const* psi, double* const* hpsi, BatchLayout& L,
                         std::vector<char>& host_tables, cudaStream_t st,
                         const char* pair = nullptr) {
  W.cur = st;
  L = BatchLayout();
  size_t off = 0;
  for (int p = 0; p < nprob; ++p) {
    const qe_problem* pr = &probs[p];
    BT_TRY(check_problem(pr, "qe_hpsi_batch"));
    if (pr->mem != QE_DEVICE) {
      set_error("qe_hpsi_batch: problem %d: arrays must be device memory", p);
      return QE_EINVAL;
    }
    if (pr->nbnd > 0 && (!psi[p] || !hpsi[p])) {
      set_error("qe_hpsi_batch: problem %d: null psi/hpsi", p);
      return QE_EINVAL;
    }
    DevPlan* P = nullptr;
    BT_TRY(get_plan(ctx, pr->lat, pr->k, pr->ecutwfc, pr->grid, &P));
    OpView op;
    BT_TRY(resolve_operator(ctx, pr, *P, op, st));
    L.plans.push_back(P);
    L.all_sqz = L.all_sqz && P->sqz != 0;   // z stages: 128 threads suit the two-pass z lines
    L.ops.push_back(op);
    L.pair.push_back(pair && pair[p] && P->h.gamma ? 1 : 0);
    const size_t ngrid = (size_t)P->grid[0] * P->grid[1] * P->grid[2];
    L.vp_off.push_back(off);
    off += up256(ngrid * sizeof(T));
    L.w_off.push_back(off);
    off += up256(stick_bytes(*P, std::max(1, pr->nbnd), 2 * sizeof(T)));
    L.smem_p = std::max(L.smem_p, psm_bytes<T>(*P));
    if (op.nproj > 0) {
      L.np_max_part = std::max(L.np_max_part, gemm_inner_scratch(op.nproj, pr->nbnd, P->h.npw, sizeof(T)));
      L.np_max_proj = std::max(L.np_max_proj, (size_t)op.nproj * pr->nbnd * 2 * sizeof(double));
      L.tc_work = std::max(L.tc_work, nonlocal_tc_bytes(op.nproj, pr->nbnd, P->h.npw));
      L.tc_beta = std::max(L.tc_beta, nonlocal_tc_beta_bytes(op.nproj, P->h.npw));
      L.oz_work = std::max(L.oz_work, nonlocal_oz_bytes(op.nproj, pr->nbnd, P->h.npw));
      L.oz_beta = std::max(L.oz_beta, nonlocal_oz_beta_bytes(op.nproj, P->h.npw));
    }
  }
  for (int p = 0; p < nprob; ++p) {
    const int spb = make_job<T>(*L.plans[p], nullptr, nullptr, nullptr, nullptr, 0, 1,
                                batch_shape<T>(*L.plans[p], L.all_sqz)).spb;
    L.smem_z = std::max(L.smem_z, zsm_bytes<T>(L.plans[p]->grid[2], spb));
  }
  L.jobs_off = off;
  off += up256((size_t)nprob * sizeof(FftJob<T>));
  L.prefix_off = off;
  off += up256(2 * (size_t)(nprob + 1) * sizeof(int));
  L.counters_off = off;
  off += 256;
  L.total = off;
  BT_TRY(W.ws.ensure(L.total));
  if (L.np_max_part) {
    BT_TRY(W.part.ensure(L.np_max_part));
    BT_TRY(W.proj.ensure(L.np_max_proj));
    BT_TRY(W.projd.ensure(L.np_max_proj));
    if (std::is_same<T, float>::value) {
      BT_TRY(W.tc_work.ensure(L.tc_work));
      BT_TRY(W.tc_beta.ensure(L.tc_beta));
    } else if (fp64_gemm_on_tensor_cores()) {
      BT_TRY(W.oz_work.ensure(L.oz_work));
      BT_TRY(W.oz_beta.ensure(L.oz_beta));
    }
    if (!W.tc_status.p) {
      BT_TRY(W.tc_status.ensure(256));
      BT_CU(cudaMemsetAsync(W.tc_status.p, 0, 256, st));
    }
  }
  // job descriptors and the two prefix arrays (stick-block items, plane items)
  char* base = static_cast<char*>(W.ws.p);
  host_tables.assign(L.counters_off - L.jobs_off, 0);
  FftJob<T>* jobs = reinterpret_cast<FftJob<T>*>(host_tables.data());
  int* pre = reinterpret_cast<int*>(host_tables.data() + (L.prefix_off - L.jobs_off));
  pre[0] = 0;
  pre[nprob + 1] = 0;
  for (int p = 0; p < nprob; ++p) {
    const DevPlan& P = *L.plans[p];
    const FftShape sh = batch_shape<T>(P, L.all_sqz);
    jobs[p] = make_job<T>(P, psi[p], hpsi[p], reinterpret_cast<const T*>(base + L.vp_off[p]),
                          base + L.w_off[p], 0, probs[p].nbnd, sh, L.pair[p]);
    pre[p + 1] = pre[p] + jobs[p].nb * jobs[p].nsb;   // FFT bands (band pairs with pair)
    pre[nprob + 1 + p + 1] = pre[nprob + 1 + p] + jobs[p].nb * P.grid[2];
  }
  return QE_OK;
}

template <typename T>
static int batch_launch(BatchWork& W, int nprob, const qe_problem* probs, const double* const* psi,
                        double* const* hpsi, const BatchLayout& L, cudaStream_t st, Prof* pf) {
  char* base = static_cast<char*>(W.ws.p);
  for (int p = 0; p < nprob; ++p)
    BT_TRY(launch_vperm<T>(*L.plans[p], L.ops[p].vloc, reinterpret_cast<T*>(base + L.vp_off[p]), st, pf));
  BT_TRY(launch_local_kinetic_batch<T>(reinterpret_cast<const FftJob<T>*>(base + L.jobs_off),
                                       reinterpret_cast<const int*>(base + L.prefix_off), nprob,
                                       reinterpret_cast<int*>(base + L.counters_off), L.smem_z,
                                       L.smem_p, 256, L.all_sqz ? 128 : 256, st, pf));
  for (int p = 0; p < nprob; ++p) {
    const OpView& op = L.ops[p];
    const int nb = probs[p].nbnd, np = op.nproj, npw = L.plans[p]->h.npw;
    if (np <= 0 || nb <= 0) continue;
    const bool rp = L.pair[p] != 0;
    if (std::is_same<T, float>::value) {
      BT_TRY(nonlocal_tc(op.beta, op.dmat, psi[p], hpsi[p], np, nb, npw, W.tc_beta.p, true,
                         W.tc_work.p, W.tc_work.bytes, (int*)W.tc_status.p, st, pf, rp));
    } else if (oz_worth(np, nb, npw)) {
      BT_TRY(nonlocal_oz(op.beta, op.dmat, psi[p], hpsi[p], np, nb, npw, W.oz_beta.p, true,
                         W.oz_work.p, W.oz_work.bytes, (int*)W.tc_status.p, st, pf, rp));
    } else {
      BT_TRY(gemm_inner<GemmT<T>>(op.beta, npw, psi[p], npw, np, nb, npw, (double*)W.proj.p, nb,
                                  W.part.p, W.part.bytes, st, pf));
      BT_TRY(dmul(op.dmat, (const double*)W.proj.p, (double*)W.projd.p, np, nb, st, pf, rp));
      BT_TRY(gemm_outer<GemmT<T>>(op.beta, npw, (const double*)W.projd.p, nb, npw, nb, np, hpsi[p],
                                  npw, 1, st, pf));
    }
  }
  return QE_OK;
}

template <typename T>
static int hpsi_batch_t(qe_ctx* ctx, BatchWork& W, int nprob, const qe_problem* probs,
                        const double* const* psi, double* const* hpsi, cudaStream_t st,
                        const char* pair) {
  BatchLayout L;
  std::vector<char> tables;
  BT_TRY(batch_prepare<T>(ctx, W, nprob, probs, psi, hpsi, L, tables, st, pair));
  char* base = static_cast<char*>(W.ws.p);
  BT_CU(cudaMemcpyAsync(base + L.jobs_off, tables.data(), tables.size(), cudaMemcpyHostToDevice, st));
  BT_CU(cudaStreamSynchronize(st));   // the host tables are freed on return
  BT_TRY(batch_launch<T>(W, nprob, probs, psi, hpsi, L, st, &ctx->prof));
  if (W.tc_status.p) {
    int v = 0;
    BT_CU(cudaMemcpyAsync(&v, W.tc_status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    BT_CU(cudaStreamSynchronize(st));
    if (v) { set_error("a tensor-core GEMM wait timed out (code %d)", v); return QE_ETIMEOUT; }
  }
  return QE_OK;
}

BatchWork& ctx_batch_work(qe_ctx* ctx);

int hpsi_batch_core(qe_ctx* ctx, int nprob, const qe_problem* probs, int precision,
                    const double* const* psi, double* const* hpsi, cudaStream_t st,
                    const char* pair) {
  BatchWork& W = ctx_batch_work(ctx);
  if (precision == QE_FP64) return hpsi_batch_t<FftF64>(ctx, W, nprob, probs, psi, hpsi, st, pair);
  return hpsi_batch_t<float>(ctx, W, nprob, probs, psi, hpsi, st, pair);
}

// The context's batch workspace (created on first use, freed with the context).
BatchWork& ctx_batch_work(qe_ctx* ctx) {
  if (!ctx->batch) ctx->batch = std::make_shared<BatchWork>();
  return *std::static_pointer_cast<BatchWork>(ctx->batch);
}

void ctx_batch_release(qe_ctx* ctx) {
  if (ctx->batch) std::static_pointer_cast<BatchWork>(ctx->batch)->release();
}

}  // namespace qe

using namespace qe;

struct qe_batch {
  qe_ctx* ctx = nullptr;
  int precision = QE_FP64;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  BatchWork work;   // the graph's buffers: owned here so that nothing else moves them
};

extern "C" {

int qe_hpsi_batch(qe_ctx* ctx, int nprob, const qe_problem* probs, int precision,
                  const double* const* psi, double* const* hpsi, void* stream) {
  clear_error();
  if (!ctx || nprob < 0 || (nprob > 0 && (!probs || !psi || !hpsi))) {
    set_error("qe_hpsi_batch: invalid argument");
    return QE_EINVAL;
  }
  if (precision != QE_FP64 && precision != QE_MIXED) { set_error("qe_hpsi_batch: bad precision"); return QE_EINVAL; }
  if (nprob == 0) return QE_OK;
  BT_CU(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  BT_TRY(ctx_begin(ctx, st));
  return hpsi_batch_core(ctx, nprob, probs, precision, psi, hpsi, st);
}

int qe_batch_create(qe_ctx* ctx, int nprob, const qe_problem* probs, int precision,
                    const double* const* psi, double* const* hpsi, void* stream, qe_batch** out) {
  clear_error();
  if (!out || !ctx || nprob <= 0 || !probs || !psi || !hpsi) {
    set_error("qe_batch_create: invalid argument");
    return QE_EINVAL;
  }
  if (precision != QE_FP64 && precision != QE_MIXED) { set_error("qe_batch_create: bad precision"); return QE_EINVAL; }
  *out = nullptr;
  BT_CU(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  BT_TRY(ctx_begin(ctx, st));
  // one eager run sizes every workspace and uploads the tables; the graph then
  // records only device work on buffers that no longer move
  std::unique_ptr<qe_batch> b(new qe_batch());
  b->ctx = ctx;
  b->precision = precision;
  BatchWork& Wk = b->work;
  BatchLayout L;
  std::vector<char> tables;
  int rc = precision == QE_FP64
               ? batch_prepare<FftF64>(ctx, Wk, nprob, probs, psi, hpsi, L, tables, st)
               : batch_prepare<float>(ctx, Wk, nprob, probs, psi, hpsi, L, tables, st);
  if (rc) { Wk.release(); return rc; }
  char* base = static_cast<char*>(Wk.ws.p);
  BT_CU(cudaMemcpyAsync(base + L.jobs_off, tables.data(), tables.size(), cudaMemcpyHostToDevice, st));
  BT_CU(cudaStreamSynchronize(st));
  rc = precision == QE_FP64 ? batch_launch<FftF64>(Wk, nprob, probs, psi, hpsi, L, st, nullptr)
                            : batch_launch<float>(Wk, nprob, probs, psi, hpsi, L, st, nullptr);
  if (rc) { Wk.release(); return rc; }
  BT_CU(cudaStreamSynchronize(st));
  cudaStream_t cap = nullptr;
  BT_CU(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaStreamDestroy(cap);
    set_error("qe_batch_create: stream capture unavailable");
    return QE_ECUDA;
  }
  rc = precision == QE_FP64 ? batch_launch<FftF64>(Wk, nprob, probs, psi, hpsi, L, cap, nullptr)
                            : batch_launch<float>(Wk, nprob, probs, psi, hpsi, L, cap, nullptr);
  const cudaError_t ec = cudaStreamEndCapture(cap, &g);
  cudaStreamDestroy(cap);
  if (rc || ec != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    Wk.cur = st;
    Wk.release();
    if (!rc) set_error("qe_batch_create: capture failed: %s", cudaGetErrorString(ec));
    return rc ? rc : QE_ECUDA;
  }
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    Wk.cur = st;
    Wk.release();
    set_error("qe_batch_create: graph instantiation failed");
    return QE_ECUDA;
  }
  Wk.cur = st;
  b->graph = g;
  b->exec = ex;
  *out = b.release();
  return QE_OK;
}

int qe_batch_run(qe_batch* b, void* stream) {
  clear_error();
  if (!b) { set_error("qe_batch_run: null batch"); return QE_EINVAL; }
  BT_CU(cudaSetDevice(b->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (b->work.cur != st) {   // the graph's buffers are shared by its replays
    BT_CU(cudaStreamSynchronize(b->work.cur));
    b->work.cur = st;
  }
  BT_CU(cudaGraphLaunch(b->exec, st));
  b->ctx->prof.launches += 1;
  return QE_OK;
}

void qe_batch_destroy(qe_batch* b) {
  if (!b) return;
  cudaSetDevice(b->ctx->device);
  cudaStreamSynchronize(b->work.cur);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->work.release();
  cudaStreamSynchronize(b->work.cur);
  delete b;
}

int qe_autotune(qe_ctx* ctx, const qe_problem* prob, int precision, void* stream) {
  clear_error();
  if (!ctx) { set_error("qe_autotune: null context"); return QE_EINVAL; }
  BT_TRY(check_problem(prob, "qe_autotune"));
  if (precision != QE_FP64 && precision != QE_MIXED) { set_error("qe_autotune: bad precision"); return QE_EINVAL; }
  BT_CU(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  BT_TRY(ctx_begin(ctx, st));
  DevPlan* P = nullptr;
  BT_TRY(get_plan(ctx, prob->lat, prob->k, prob->ecutwfc, prob->grid, &P));
  OpView op;
  BT_TRY(resolve_operator(ctx, prob, *P, op, st));
  const size_t el = precision == QE_FP64 ? sizeof(double) : sizeof(float);
  const int nb = std::max(1, std::min(prob->nbnd > 0 ? prob->nbnd : 16, 16));
  const size_t nel = (size_t)nb * P->h.npw * 2;
  BT_TRY(ctx->h_psi.ensure(nel * sizeof(double)));
  BT_TRY(ctx->h_hpsi.ensure(nel * sizeof(double)));
  BT_CU(cudaMemsetAsync(ctx->h_psi.p, 0, nel * sizeof(double), st));
  const size_t ngrid = (size_t)P->grid[0] * P->grid[1] * P->grid[2];
  ctx->last_op = qe_ctx::LastOp{};   // the permuted potential is overwritten below
  BT_TRY(ctx->vp.ensure(ngrid * el));
  BT_TRY(ctx->sticks.ensure(stick_bytes(*P, nb, 2 * el)));
  cudaEvent_t e0, e1;
  BT_CU(cudaEventCreate(&e0));
  BT_CU(cudaEventCreate(&e1));
  auto run = [&](const FftShape& sh, float* ms) -> int {
    for (int rep = 0; rep < 4; ++rep) {
      if (rep == 1) cudaEventRecord(e0, st);
      const int rc = el == sizeof(double)
          ? launch_local_kinetic_shape<FftF64>(*P, (const double*)ctx->h_psi.p, (double*)ctx->h_hpsi.p,
                                               (const FftF64*)ctx->vp.p, ctx->sticks.p, 0, nb, sh, st, nullptr)
          : launch_local_kinetic_shape<float>(*P, (const double*)ctx->h_psi.p, (double*)ctx->h_hpsi.p,
                                              (const float*)ctx->vp.p, ctx->sticks.p, 0, nb, sh, st, nullptr);
      if (rc) return rc;
    }
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) { set_error("qe_autotune: timing failed"); return QE_ECUDA; }
    cudaEventElapsedTime(ms, e0, e1);
    return QE_OK;
  };
  FftShape best;
  float best_ms = 1e30f;
  const int spbs[] = {4, 8, 16, 32};
  const int zts[] = {128, 256, 512};
  for (int spb : spbs)
    for (int zt : zts) {
      FftShape sh;
      sh.spb = spb;
      sh.zthreads = zt;
      sh.pthreads = 256;
      if ((size_t)(P->grid[2] * spb + P->grid[2]) * 2 * el > 200 * 1024) continue;
      float ms = 0.f;
      const int rc = run(sh, &ms);
      if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
      if (ms < best_ms) { best_ms = ms; best = sh; }
    }
  const int pts[] = {128, 256, 512};
  FftShape zbest = best;
  for (int pt : pts) {
    FftShape sh = zbest;
    sh.pthreads = pt;
    float ms = 0.f;
    const int rc = run(sh, &ms);
    if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
    if (ms < best_ms) { best_ms = ms; best = sh; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  store_shape(P->grid, el, best);
  return QE_OK;
}

}  // extern "C"
