// C-ABI entry points: context, plan cache, builders and H|psi>.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <type_traits>
#include <vector>

#include "plan.h"
#include "ctx.h"

namespace qe {

int build_vloc(const double lat[9], const int grid[3], int natom, const double* tau_h, double amp,
               double sigma, double* v_dev, cudaStream_t st);
int build_beta(const double lat[9], const double k[3], double ecut, int natom, const double* tau_h,
               int nrad, const double* widths_h, double* beta_dev, int* npw_out, cudaStream_t st);

void Prof::begin(const char* name, cudaStream_t st, cudaEvent_t* ev) {
  ++launches;
  *ev = nullptr;
  if (!on) return;
  if (cudaEventCreate(ev) != cudaSuccess) { cudaGetLastError(); *ev = nullptr; return; }
  cudaEventRecord(*ev, st);
}

void Prof::end(const char* name, cudaStream_t st, cudaEvent_t ev) {
  if (!on || !ev) return;
  cudaEvent_t b;
  if (cudaEventCreate(&b) != cudaSuccess) { cudaGetLastError(); cudaEventDestroy(ev); return; }
  cudaEventRecord(b, st);
  std::lock_guard<std::mutex> lk(mu);
  recs.push_back({name, ev, b});
}

int Prof::fold() {
  int rc = QE_OK;
  std::lock_guard<std::mutex> lk(mu);
  for (auto& r : recs) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      rc = QE_ECUDA;
    }
    size_t i = 0;
    while (i < names.size() && names[i] != r.name) ++i;
    if (i == names.size()) { names.push_back(r.name); calls.push_back(0); ms.push_back(0.0); }
    calls[i] += 1;
    ms[i] += t;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  recs.clear();
  return rc;
}

void Prof::reset() {
  fold();
  names.clear();
  calls.clear();
  ms.clear();
  launches = 0;
}

int DevBuf::ensure(size_t nbytes) {
  if (nbytes <= bytes && p) return QE_OK;
  const cudaStream_t st = sp ? *sp : nullptr;
  release();
  if (nbytes == 0) return QE_OK;
  if (cudaMallocAsync(&p, nbytes, st) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMallocAsync of %zu bytes failed", nbytes);
    p = nullptr;
    return QE_ENOMEM;
  }
  bytes = nbytes;
  return QE_OK;
}

void DevBuf::release() {
  if (p) cudaFreeAsync(p, sp ? *sp : nullptr);
  p = nullptr;
  bytes = 0;
}

int ctx_trim_public(qe_ctx* ctx) {
  cudaSetDevice(ctx->device);
  return ctx_trim(ctx);
}

int ctx_begin(qe_ctx* ctx, cudaStream_t st) {
  if (ctx->has_cur && ctx->cur != st) {
    cudaError_t e = cudaStreamSynchronize(ctx->cur);
    if (e != cudaSuccess) {
      set_error("previous stream: %s", cudaGetErrorString(e));
      return QE_ECUDA;
    }
  }
  ctx->cur = st;
  ctx->has_cur = true;
  return QE_OK;
}

int ctx_trim(qe_ctx* ctx) {
  for (DevBuf* b : ctx->bufs()) b->release();
  for (auto& b : ctx->dvb_basis) b->release();
  for (auto& b : ctx->dvb_red) b->release();
  ctx->dvb_basis.clear();
  ctx->dvb_red.clear();
  ctx_batch_release(ctx);
  ctx->tc_beta_tag = 0;
  ctx->oz_beta_tag = 0;
  ctx->last_op = qe_ctx::LastOp{};
  for (auto& p : ctx->plans)
    if (p->block) cudaFreeAsync(p->block, ctx->cur);
  ctx->plans.clear();
  cudaError_t e = cudaStreamSynchronize(ctx->cur);
  if (e != cudaSuccess) {
    set_error("ctx_trim: %s", cudaGetErrorString(e));
    return QE_ECUDA;
  }
  return QE_OK;
}

static bool same_key(const DevPlan& P, const double lat[9], const double k[3], double ecut,
                     const int grid[3]) {
  return std::memcmp(P.lat, lat, sizeof(P.lat)) == 0 && std::memcmp(P.k, k, sizeof(P.k)) == 0 &&
         P.ecut == ecut && P.grid[0] == grid[0] && P.grid[1] == grid[1] && P.grid[2] == grid[2];
}

int get_plan(qe_ctx* ctx, const double lat[9], const double k[3], double ecut, const int grid[3],
             DevPlan** out) {
  for (auto& p : ctx->plans)
    if (same_key(*p, lat, k, ecut, grid)) { *out = p.get(); return QE_OK; }
  auto P = std::make_unique<DevPlan>();
  std::memcpy(P->lat, lat, sizeof(P->lat));
  std::memcpy(P->k, k, sizeof(P->k));
  P->ecut = ecut;
  std::memcpy(P->grid, grid, sizeof(P->grid));
  int rc = build_plan_host(lat, k, ecut, grid, P->h);
  if (rc) return rc;
  for (int c = 0; c < 3; ++c) make_radix(grid[c], P->rad[c]);
  const PlanHost& h = P->h;
  std::vector<int> perm[3];
  std::vector<double> tw[3];
  for (int c = 0; c < 3; ++c) { perm[c] = digit_reversal(P->rad[c]); tw[c] = twiddles(grid[c]); }
  // square planes with the register-resident transform keep x and y in its order
  P->sq = sq_plane_size(grid);
  if (P->sq) perm[0] = perm[1] = sq_order(P->sq);
  P->sqz = sq_line_size(grid[2]);
  if (P->sqz) perm[2] = sq_order(P->sqz);
  // one allocation: doubles first, then ints
  size_t nd = h.npw;
  for (int c = 0; c < 3; ++c) nd += tw[c].size();
  size_t ni = (h.nst + 1) + 3 * (size_t)h.npw + 2 * (size_t)h.nst + h.nax + h.mg.size();
  for (int c = 0; c < 3; ++c) ni += grid[c];
  const size_t bytes = nd * sizeof(double) + ni * sizeof(int);
  if (cudaMallocAsync(&P->block, bytes, ctx->cur) != cudaSuccess) {
    cudaGetLastError();
    set_error("plan: cudaMallocAsync of %zu bytes failed", bytes);
    return QE_ENOMEM;
  }
  std::vector<char> host(bytes);
  double* dp = reinterpret_cast<double*>(host.data());
  size_t od = 0;
  auto put_d = [&](const double* src, size_t n) { std::memcpy(dp + od, src, n * sizeof(double)); size_t o = od; od += n; return o; };
  const size_t o_kin = put_d(h.kin.data(), h.npw);
  size_t o_tw[3];
  for (int c = 0; c < 3; ++c) o_tw[c] = put_d(tw[c].data(), tw[c].size());
  int* ip = reinterpret_cast<int*>(host.data() + nd * sizeof(double));
  size_t oi = 0;
  auto put_i = [&](const int* src, size_t n) { std::memcpy(ip + oi, src, n * sizeof(int)); size_t o = oi; oi += n; return o; };
  const size_t o_ptr = put_i(h.st_ptr.data(), h.nst + 1);
  const size_t o_g = put_i(h.st_g.data(), h.npw);
  const size_t o_z = put_i(h.st_z.data(), h.npw);
  const size_t o_of = put_i(h.st_of.data(), h.npw);
  const size_t o_x = put_i(h.st_x.data(), h.nst);
  const size_t o_y = put_i(h.st_y.data(), h.nst);
  const size_t o_ax = put_i(h.ax.data(), h.nax);
  const size_t o_mg = put_i(h.mg.data(), h.mg.size());
  size_t o_perm[3];
  for (int c = 0; c < 3; ++c) o_perm[c] = put_i(perm[c].data(), perm[c].size());
  if (cudaMemcpyAsync(P->block, host.data(), bytes, cudaMemcpyHostToDevice, ctx->cur) != cudaSuccess ||
      cudaStreamSynchronize(ctx->cur) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeAsync(P->block, ctx->cur);
    set_error("plan: upload failed");
    return QE_ECUDA;
  }
  double* dd = reinterpret_cast<double*>(P->block);
  int* di = reinterpret_cast<int*>(reinterpret_cast<char*>(P->block) + nd * sizeof(double));
  P->kin = dd + o_kin;
  for (int c = 0; c < 3; ++c) { P->tw[c] = dd + o_tw[c]; P->perm[c] = di + o_perm[c]; }
  P->st_ptr = di + o_ptr;
  P->st_g = di + o_g;
  P->st_z = di + o_z;
  P->st_of = di + o_of;
  P->st_x = di + o_x;
  P->st_y = di + o_y;
  P->ax = di + o_ax;
  P->mg = h.gamma ? di + o_mg : nullptr;
  ctx->plans.push_back(std::move(P));
  *out = ctx->plans.back().get();
  return QE_OK;
}

int check_problem(const qe_problem* pr, const char* who) {
  if (!pr) { set_error("%s: null problem", who); return QE_EINVAL; }
  if (pr->mem != QE_HOST && pr->mem != QE_DEVICE) { set_error("%s: bad mem flag", who); return QE_EINVAL; }
  if (pr->nbnd < 0 || pr->nproj < 0) { set_error("%s: negative size", who); return QE_EINVAL; }
  for (int c = 0; c < 3; ++c)
    if (pr->grid[c] < 1) { set_error("%s: grid must be positive", who); return QE_EINVAL; }
  if (!pr->vloc_r) { set_error("%s: vloc_r is null", who); return QE_EINVAL; }
  if (pr->nproj > 0 && (!pr->beta || !pr->dmat)) { set_error("%s: beta/dmat null with nproj > 0", who); return QE_EINVAL; }
  return QE_OK;
}

#define QE_TRY(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)
#define QE_CU(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_error("%s: %s", #x, cudaGetErrorString(e_)); return QE_ECUDA; } } while (0)

// Device views of the problem's operator arrays (copied in when they are host arrays).
// psi of a host-memory call into dst in up to 8 band chunks on the copy stream,
// one event per chunk (after the buffers' stream-ordered allocation on st).
static int upload_psi_chunks(qe_ctx* ctx, const double* psi, double* dst, int nb, int npw,
                             cudaStream_t st) {
  if (!ctx->side) {
    QE_CU(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
    QE_CU(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    QE_CU(cudaEventCreateWithFlags(&ctx->ev_op, cudaEventDisableTiming));
  }
  const int chunk = (nb + 7) / 8, nch = (nb + chunk - 1) / chunk;
  while ((int)ctx->psi_ev.size() < nch) {
    cudaEvent_t e;
    QE_CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->psi_ev.push_back(e);
  }
  QE_CU(cudaEventRecord(ctx->ev_fork, st));
  QE_CU(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  const size_t band = (size_t)npw * 2;
  for (int c = 0; c < nch; ++c) {
    const int b0 = c * chunk, n = std::min(chunk, nb - b0);
    QE_CU(cudaMemcpyAsync(dst + (size_t)b0 * band, psi + (size_t)b0 * band, (size_t)n * band * sizeof(double),
                          cudaMemcpyHostToDevice, ctx->side));
    QE_CU(cudaEventRecord(ctx->psi_ev[c], ctx->side));
  }
  ctx->psi_ev_n = nch;
  ctx->psi_ev_bands = chunk;
  return QE_OK;
}

int resolve_operator(qe_ctx* ctx, const qe_problem* pr, const DevPlan& P, OpView& op,
                     cudaStream_t st, bool overlap) {
  const size_t ngrid = (size_t)P.grid[0] * P.grid[1] * P.grid[2];
  const size_t nbeta = (size_t)pr->nproj * P.h.npw * 2;
  const size_t nd = (size_t)pr->nproj * pr->nproj;
  op.nproj = pr->nproj;
  op.tag = ++ctx->op_tag;
  if (pr->mem == QE_DEVICE) {
    op.vloc = pr->vloc_r;
    op.beta = pr->beta;
    op.dmat = pr->dmat;
    return QE_OK;
  }
  QE_TRY(ctx->h_v.ensure(ngrid * sizeof(double)));
  QE_TRY(ctx->h_beta.ensure(nbeta * sizeof(double)));
  QE_TRY(ctx->h_d.ensure(nd * sizeof(double)));
  QE_CU(cudaMemcpyAsync(ctx->h_v.p, pr->vloc_r, ngrid * sizeof(double), cudaMemcpyHostToDevice, st));
  if (pr->nproj > 0 && overlap) {
    if (!ctx->side) {
      QE_CU(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
      QE_CU(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
      QE_CU(cudaEventCreateWithFlags(&ctx->ev_op, cudaEventDisableTiming));
    }
    // the buffers were (re)allocated in st's order: fork after that
    QE_CU(cudaEventRecord(ctx->ev_fork, st));
    QE_CU(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
    QE_CU(cudaMemcpyAsync(ctx->h_beta.p, pr->beta, nbeta * sizeof(double), cudaMemcpyHostToDevice,
                          ctx->side));
    QE_CU(cudaMemcpyAsync(ctx->h_d.p, pr->dmat, nd * sizeof(double), cudaMemcpyHostToDevice, ctx->side));
    QE_CU(cudaEventRecord(ctx->ev_op, ctx->side));
    op.ready = ctx->ev_op;
  } else if (pr->nproj > 0) {
    QE_CU(cudaMemcpyAsync(ctx->h_beta.p, pr->beta, nbeta * sizeof(double), cudaMemcpyHostToDevice, st));
    QE_CU(cudaMemcpyAsync(ctx->h_d.p, pr->dmat, nd * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  op.vloc = (const double*)ctx->h_v.p;
  op.beta = (const double*)ctx->h_beta.p;
  op.dmat = (const double*)ctx->h_d.p;
  return QE_OK;
}

template <typename T>
static int hpsi_device_nonlocal(qe_ctx* ctx, const DevPlan& P, const OpView& op, const double* psi,
                                double* hpsi, int nb, cudaStream_t st, bool pair);

// pair: the bands are real in r (k = 0 plan); two share each FFT and the
// projections are taken real.
template <typename T>
static int hpsi_device(qe_ctx* ctx, const DevPlan& P, const OpView& op, const double* psi,
                       double* hpsi, int nb, cudaStream_t st, bool pair, bool vp_ready = false) {
  const int npw = P.h.npw;
  pair = pair && P.h.gamma;
  const size_t ngrid = (size_t)P.grid[0] * P.grid[1] * P.grid[2];
  if (!vp_ready || !ctx->vp.p || ctx->vp.bytes < ngrid * sizeof(T)) {
    // the permuted potential no longer belongs to the last qe_hpsi operator
    ctx->last_op = qe_ctx::LastOp{};
    QE_TRY(ctx->vp.ensure(ngrid * sizeof(T)));
    QE_TRY(launch_vperm<T>(P, op.vloc, (T*)ctx->vp.p, st, &ctx->prof));
  }
  const size_t per_band = stick_bytes(P, 1, 2 * sizeof(T));
  const int per_fft = pair ? 2 : 1;   // bands per FFT
  int nfb = (int)std::max<size_t>(1, ctx->stick_budget / std::max<size_t>(per_band, 1));
  nfb = std::min(nfb, (nb + per_fft - 1) / per_fft);
  const int nbc = nfb * per_fft;
  QE_TRY(ctx->sticks.ensure(stick_bytes(P, nfb, 2 * sizeof(T))));
  int waited = 0;   // psi chunks of a host-memory call already joined
  for (int b0 = 0; b0 < nb; b0 += nbc) {
    const int n = std::min(nbc, nb - b0);
    if (ctx->psi_ev_n > 0) {
      const int need = std::min(ctx->psi_ev_n, (b0 + n + ctx->psi_ev_bands - 1) / ctx->psi_ev_bands);
      for (; waited < need; ++waited) QE_CU(cudaStreamWaitEvent(st, ctx->psi_ev[waited], 0));
    }
    QE_TRY(launch_local_kinetic<T>(P, psi, hpsi, (const T*)ctx->vp.p, ctx->sticks.p, b0, n, st,
                                   &ctx->prof, pair ? 1 : 0));
  }
  for (; waited < ctx->psi_ev_n; ++waited) QE_CU(cudaStreamWaitEvent(st, ctx->psi_ev[waited], 0));
  if (op.ready) QE_CU(cudaStreamWaitEvent(st, op.ready, 0));
  const bool use_oz = op.nproj > 0 && !std::is_same<T, float>::value && oz_worth(op.nproj, nb, npw);
  if (op.gen && op.nproj > 0 && !use_oz) {
    // generated projectors on the paths that read beta values: generate them here
    QE_TRY(ctx->gen_beta.ensure((size_t)op.nproj * npw * 2 * sizeof(double)));
    QE_TRY(gen_beta_values(*op.gen, (double*)ctx->gen_beta.p, st, &ctx->prof));
    OpView o2 = op;
    o2.gen = nullptr;
    o2.beta = (const double*)ctx->gen_beta.p;
    o2.tag = ++ctx->op_tag;
    return hpsi_device_nonlocal<T>(ctx, P, o2, psi, hpsi, nb, st, pair);
  }
  return hpsi_device_nonlocal<T>(ctx, P, op, psi, hpsi, nb, st, pair);
}

// The nonlocal term of hpsi_device.
template <typename T>
static int hpsi_device_nonlocal(qe_ctx* ctx, const DevPlan& P, const OpView& op, const double* psi,
                                double* hpsi, int nb, cudaStream_t st, bool pair) {
  const int npw = P.h.npw;
  if (op.nproj > 0 && std::is_same<T, float>::value) {
    // mixed precision: projector products on the tensor cores (TF32x3 split)
    const int np = op.nproj;
    QE_TRY(ctx->tc_work.ensure(nonlocal_tc_bytes(np, nb, npw)));
    if (!ctx->tc_status.p) {
      QE_TRY(ctx->tc_status.ensure(256));
      QE_CU(cudaMemsetAsync(ctx->tc_status.p, 0, 256, st));
    }
    const void* before = ctx->tc_beta.p;
    const size_t before_bytes = ctx->tc_beta.bytes;
    QE_TRY(ctx->tc_beta.ensure(nonlocal_tc_beta_bytes(np, npw)));
    if (ctx->tc_beta.p != before || ctx->tc_beta.bytes != before_bytes) ctx->tc_beta_tag = 0;
    const bool pack = ctx->tc_beta_tag == 0 || ctx->tc_beta_tag != op.tag;
    QE_TRY(nonlocal_tc(op.beta, op.dmat, psi, hpsi, np, nb, npw, ctx->tc_beta.p, pack,
                       ctx->tc_work.p, ctx->tc_work.bytes, (int*)ctx->tc_status.p, st, &ctx->prof,
                       pair));
    ctx->tc_beta_tag = op.tag;
  } else if (op.nproj > 0 && oz_worth(op.nproj, nb, npw)) {
    // FP64: FP64-accurate projector products on the BF16 tensor cores (Ozaki slices)
    const int np = op.nproj;
    QE_TRY(ctx->oz_work.ensure(nonlocal_oz_bytes(np, nb, npw)));
    if (!ctx->tc_status.p) {
      QE_TRY(ctx->tc_status.ensure(256));
      QE_CU(cudaMemsetAsync(ctx->tc_status.p, 0, 256, st));
    }
    const void* before = ctx->oz_beta.p;
    const size_t before_bytes = ctx->oz_beta.bytes;
    QE_TRY(ctx->oz_beta.ensure(nonlocal_oz_beta_bytes(np, npw)));
    if (ctx->oz_beta.p != before || ctx->oz_beta.bytes != before_bytes) ctx->oz_beta_tag = 0;
    // the kept column slices have one of two forms (complex or real-K)
    const int form = nonlocal_oz_real_outer(pair, np) ? 4 : 0;
    const bool slice = ctx->oz_beta_tag == 0 || ctx->oz_beta_tag != op.tag || ctx->oz_beta_form != form;
    if (op.gen && slice) {
      // projectors generated on the fly straight into the slices: no beta array
      QE_TRY(ctx->gen_scr.ensure(oz_gen_scratch_bytes(*op.gen)));
      QE_TRY(oz_gen_beta(*op.gen, ctx->oz_beta.p, ctx->gen_scr.p, st, &ctx->prof, form == 4));
    }
    QE_TRY(nonlocal_oz(op.beta, op.dmat, psi, hpsi, np, nb, npw, ctx->oz_beta.p, slice && !op.gen,
                       ctx->oz_work.p, ctx->oz_work.bytes, (int*)ctx->tc_status.p, st, &ctx->prof,
                       pair));
    ctx->oz_beta_tag = op.tag;
    ctx->oz_beta_form = form;
  } else if (op.nproj > 0) {
    const int np = op.nproj;
    QE_TRY(ctx->proj.ensure((size_t)np * nb * 2 * sizeof(double)));
    QE_TRY(ctx->projd.ensure((size_t)np * nb * 2 * sizeof(double)));
    const size_t sb = gemm_inner_scratch(np, nb, npw, sizeof(T));
    QE_TRY(ctx->part.ensure(sb));
    QE_TRY(gemm_inner<GemmT<T>>(op.beta, npw, psi, npw, np, nb, npw, (double*)ctx->proj.p, nb,
                                ctx->part.p, ctx->part.bytes, st, &ctx->prof));
    QE_TRY(dmul(op.dmat, (const double*)ctx->proj.p, (double*)ctx->projd.p, np, nb, st, &ctx->prof,
                pair));
    QE_TRY(gemm_outer<GemmT<T>>(op.beta, npw, (const double*)ctx->projd.p, nb, npw, nb, np, hpsi,
                                npw, 1, st, &ctx->prof));
  }
  return QE_OK;
}

int tc_check(qe_ctx* ctx, cudaStream_t st) {
  if (!ctx->tc_status.p) return QE_OK;
  int v = 0;
  QE_CU(cudaMemcpyAsync(&v, ctx->tc_status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  QE_CU(cudaStreamSynchronize(st));
  if (v != 0) {
    QE_CU(cudaMemsetAsync(ctx->tc_status.p, 0, sizeof(int), st));
    set_error("a tensor-core GEMM wait timed out (code %d); its products are invalid", v);
    return QE_ETIMEOUT;
  }
  return QE_OK;
}

int hpsi_core(qe_ctx* ctx, const DevPlan& P, const OpView& op, int precision, const double* psi,
              double* hpsi, int nb, cudaStream_t st, bool pair, bool fp64_pipe, bool vp_ready) {
  if (nb == 0) return QE_OK;
  if (precision == QE_FP64)
    return fp64_pipe ? hpsi_device<double>(ctx, P, op, psi, hpsi, nb, st, pair, vp_ready)
                     : hpsi_device<FftF64>(ctx, P, op, psi, hpsi, nb, st, pair, vp_ready);
  return hpsi_device<float>(ctx, P, op, psi, hpsi, nb, st, pair, vp_ready);
}

}  // namespace qe

using namespace qe;

extern "C" {

int qe_ctx_create(int device, qe_ctx** out) {
  clear_error();
  if (!out) { set_error("qe_ctx_create: null out"); return QE_EINVAL; }
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    set_error("qe_ctx_create: no CUDA device %d (%s)", device, cudaGetErrorString(e));
    return QE_ECUDA;
  }
  QE_CU(cudaSetDevice(device));
  qe_ctx* c = new qe_ctx();
  c->device = device;
  *out = c;
  return QE_OK;
}

void qe_ctx_destroy(qe_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->has_cur) cudaStreamSynchronize(ctx->cur);
  ctx->prof.reset();
  ctx_trim(ctx);
  if (ctx->side) {
    cudaStreamSynchronize(ctx->side);
    cudaStreamDestroy(ctx->side);
    cudaEventDestroy(ctx->ev_fork);
    cudaEventDestroy(ctx->ev_op);
  }
  for (cudaEvent_t e : ctx->psi_ev) cudaEventDestroy(e);
  for (void* x : ctx->round_side) {
    cudaStreamSynchronize((cudaStream_t)x);
    cudaStreamDestroy((cudaStream_t)x);
  }
  for (void* e : ctx->round_events) cudaEventDestroy((cudaEvent_t)e);
  delete ctx;
}

int qe_profile(qe_ctx* ctx, int enable) {
  clear_error();
  if (!ctx) { set_error("qe_profile: null context"); return QE_EINVAL; }
  QE_CU(cudaSetDevice(ctx->device));
  ctx->prof.reset();
  ctx->prof.on = enable != 0;
  return QE_OK;
}

int qe_test_grid_wait(qe_ctx* ctx, long long wait_ns) {
  clear_error();
  if (!ctx || wait_ns < 0) { set_error("qe_test_grid_wait: invalid argument"); return QE_EINVAL; }
  ctx->test_wait_ns = (unsigned long long)wait_ns;
  return QE_OK;
}

int qe_profile_read(qe_ctx* ctx, int index, char* name, int name_len, long long* calls,
                    double* ms, long long* launches) {
  clear_error();
  if (!ctx) { set_error("qe_profile_read: null context"); return QE_EINVAL; }
  QE_CU(cudaSetDevice(ctx->device));
  int rc = ctx->prof.fold();
  if (launches) *launches = ctx->prof.launches;
  if (index < 0) return rc;
  if (index >= (int)ctx->prof.names.size()) { set_error("qe_profile_read: no entry %d", index); return QE_EINVAL; }
  if (name && name_len > 0) {
    std::strncpy(name, ctx->prof.names[index].c_str(), name_len - 1);
    name[name_len - 1] = 0;
  }
  if (calls) *calls = ctx->prof.calls[index];
  if (ms) *ms = ctx->prof.ms[index];
  return rc;
}

int qe_vloc_gaussian(qe_ctx* ctx, const double lat[9], const int grid[3], int natom,
                     const double* tau, double amp, double sigma, double* vloc_out, int mem,
                     void* stream) {
  clear_error();
  if (!ctx || !lat || !grid || !vloc_out || (natom > 0 && !tau) || natom < 0 || !(sigma > 0)) {
    set_error("qe_vloc_gaussian: invalid argument");
    return QE_EINVAL;
  }
  if (mem != QE_HOST && mem != QE_DEVICE) { set_error("qe_vloc_gaussian: bad mem flag"); return QE_EINVAL; }
  QE_CU(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  QE_TRY(ctx_begin(ctx, st));
  const size_t ng = (size_t)grid[0] * grid[1] * grid[2];
  double* dst = vloc_out;
  if (mem == QE_HOST) {
    QE_TRY(ctx->h_v.ensure(ng * sizeof(double)));
    dst = (double*)ctx->h_v.p;
  }
  QE_TRY(build_vloc(lat, grid, natom, tau, amp, sigma, dst, st));
  if (mem == QE_HOST) {
    QE_CU(cudaMemcpyAsync(vloc_out, dst, ng * sizeof(double), cudaMemcpyDeviceToHost, st));
    QE_CU(cudaStreamSynchronize(st));
  }
  return QE_OK;
}

int qe_beta_gaussian(qe_ctx* ctx, const double lat[9], const double k[3], double ecut, int natom,
                     const double* tau, int nrad, const double* widths, double* beta_out, int mem,
                     void* stream) {
  clear_error();
  if (!ctx || !lat || !k || !beta_out || natom < 0 || nrad < 0 || (natom > 0 && !tau) ||
      (nrad > 0 && !widths)) {
    set_error("qe_beta_gaussian: invalid argument");
    return QE_EINVAL;
  }
  for (int n = 0; n < nrad; ++n)
    if (!(widths[n] > 0)) { set_error("qe_beta_gaussian: widths must be positive"); return QE_EINVAL; }
  if (mem != QE_HOST && mem != QE_DEVICE) { set_error("qe_beta_gaussian: bad mem flag"); return QE_EINVAL; }
  QE_CU(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  QE_TRY(ctx_begin(ctx, st));
  Sphere S;
  QE_TRY(build_sphere(lat, k, ecut, S));
  const size_t n = (size_t)4 * nrad * natom * S.npw * 2;
  double* dst = beta_out;
  if (mem == QE_HOST) {
    QE_TRY(ctx->h_beta.ensure(n * sizeof(double)));
    dst = (double*)ctx->h_beta.p;
  }
  int npw = 0;
  QE_TRY(build_beta(lat, k, ecut, natom, tau, nrad, widths, dst, &npw, st));
  if (mem == QE_HOST && n > 0) {
    QE_CU(cudaMemcpyAsync(beta_out, dst, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    QE_CU(cudaStreamSynchronize(st));
  }
  return QE_OK;
}

int qe_hpsi(qe_ctx* ctx, const qe_problem* prob, int precision, const double* psi, double* hpsi,
            void* stream) {
  clear_error();
  if (!ctx) { set_error("qe_hpsi: null context"); return QE_EINVAL; }
  QE_TRY(check_problem(prob, "qe_hpsi"));
  const bool pair = (precision & QE_GAMMA) != 0;
  const bool fp64_pipe = (precision & QE_FFT_FP64PIPE) != 0;
  const bool same_op = (precision & QE_SAME_OPERATOR) != 0;
  precision &= ~(QE_GAMMA | QE_FFT_FP64PIPE | QE_SAME_OPERATOR);
  if (precision != QE_FP64 && precision != QE_MIXED) { set_error("qe_hpsi: bad precision"); return QE_EINVAL; }
  if (prob->nbnd > 0 && (!psi || !hpsi)) { set_error("qe_hpsi: null psi/hpsi"); return QE_EINVAL; }
  QE_CU(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  QE_TRY(ctx_begin(ctx, st));
  DevPlan* P = nullptr;
  QE_TRY(get_plan(ctx, prob->lat, prob->k, prob->ecutwfc, prob->grid, &P));
  const int nb = prob->nbnd;
  const size_t nel = (size_t)nb * P->h.npw * 2;
  const double* dpsi = psi;
  double* dhpsi = hpsi;
  // the pending upload belongs to this call only, whatever path it leaves by
  struct PsiUploadReset {
    qe_ctx* c;
    ~PsiUploadReset() { c->psi_ev_n = 0; }
  } psi_upload_reset{ctx};
  ctx->psi_ev_n = 0;
  if (prob->mem == QE_HOST && nb > 0) {
    QE_TRY(ctx->h_psi.ensure(nel * sizeof(double)));
    QE_TRY(ctx->h_hpsi.ensure(nel * sizeof(double)));
    dpsi = (const double*)ctx->h_psi.p;
    dhpsi = (double*)ctx->h_hpsi.p;
    // psi in band chunks on the copy stream, ahead of beta: the FFTs of the
    // first chunks run while the rest arrives
    QE_TRY(upload_psi_chunks(ctx, psi, (double*)ctx->h_psi.p, nb, P->h.npw, st));
  }
  // host operator: V on st, beta and D on the side stream while the FFTs run
  OpView op;
  QE_TRY(resolve_operator(ctx, prob, *P, op, st, prob->mem == QE_HOST && nb > 0));
  // QE_SAME_OPERATOR: a device operator identical to the previous call's keeps
  // its prepared forms (the tag selects the kept slices or packs of beta)
  const int fft_type = precision == QE_MIXED ? 0 : (fp64_pipe ? 2 : 1);
  const qe_ctx::LastOp lo = ctx->last_op;
  bool vp_ready = false;
  if (prob->mem == QE_DEVICE && same_op && nb > 0 && lo.tag != 0 && lo.plan == P &&
      lo.vloc == op.vloc && lo.beta == op.beta && lo.dmat == op.dmat && lo.nproj == op.nproj &&
      lo.fft_type == fft_type) {
    op.tag = lo.tag;
    vp_ready = true;
  }
  const int rc_h = hpsi_core(ctx, *P, op, precision, dpsi, dhpsi, nb, st, pair, fp64_pipe, vp_ready);
  if (rc_h == QE_OK && prob->mem == QE_DEVICE && nb > 0)
    ctx->last_op = {P, op.vloc, op.beta, op.dmat, op.nproj, fft_type, op.tag};
  else
    ctx->last_op = qe_ctx::LastOp{};
  if (op.ready) QE_CU(cudaStreamWaitEvent(st, op.ready, 0));   // join the copy stream
  if (rc_h) return rc_h;
  if (prob->mem == QE_HOST) {
    if (nb > 0)
      QE_CU(cudaMemcpyAsync(hpsi, dhpsi, nel * sizeof(double), cudaMemcpyDeviceToHost, st));
    QE_CU(cudaStreamSynchronize(st));
    QE_TRY(tc_check(ctx, st));
  }
  return QE_OK;
}

}  // extern "C"
