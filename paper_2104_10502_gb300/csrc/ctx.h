// The context behind the opaque qe_ctx handle.
#pragma once

#include <memory>
#include <vector>

#include "plan.h"

struct qe_ctx {
  int device = 0;
  // The stream of the current call.  A context's buffers are shared by its
  // calls, so a call on a different stream first waits for the previous one.
  cudaStream_t cur = nullptr;
  bool has_cur = false;
  qe::Prof prof;
  std::vector<std::unique_ptr<qe::DevPlan>> plans;
  // H|psi> workspaces
  size_t stick_budget = (size_t)64 << 20;  // stick buffer per band chunk (kept L2-sized)
  qe::DevBuf sticks, vp, part, proj, projd;
  // device copies of host arrays
  qe::DevBuf h_v, h_beta, h_d, h_psi, h_hpsi;
  // Davidson workspaces
  qe::DevBuf dv_basis, dv_red;
  // charge density: per-group accumulators and the band weights; the
  // self-consistency step's work
  qe::DevBuf dens_acc, dens_w, scf_work;
  // generated projectors: Miller indices of a plan's sphere, phase tables,
  // radial table copy, exponent scratch, beta values for the non-sliced paths
  qe::DevBuf gen_mill, gen_tab, gen_rad, gen_scr, gen_beta;
  const void* gen_mill_plan = nullptr;
  // tensor-core path: packed operands and the kernel's status word (a bounded
  // wait that ran out writes a non-zero code; read at the next synchronising point)
  qe::DevBuf tc_work, tc_status, tc_beta;
  // FP64 path on the tensor cores: beta slices (tagged like tc_beta) and work
  qe::DevBuf oz_beta, oz_work;
  unsigned long long oz_beta_tag = 0;
  int oz_beta_form = 0;        // form of the kept column slices (0 complex, 4 real-K)
  // the packed beta in tc_beta belongs to the operator with this tag (0: none);
  // every API call that takes an operator gets a fresh tag
  unsigned long long tc_beta_tag = 0, op_tag = 0;
  // the operator of the last device-memory qe_hpsi (QE_SAME_OPERATOR reuses
  // its prepared forms: permuted potential, tensor-core slices or packs of beta)
  struct LastOp {
    const void* plan = nullptr;
    const double *vloc = nullptr, *beta = nullptr, *dmat = nullptr;
    int nproj = 0, fft_type = -1;
    unsigned long long tag = 0;
  } last_op;
  // copy stream for the operator of a host-memory qe_hpsi (beta and D go in
  // while the FFTs run) and its two events (created on first use)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_op = nullptr;
  // host-memory qe_hpsi: psi goes in on `side` in chunks of psi_ev_bands bands,
  // psi_ev[c] recorded after chunk c; the FFT of a band chunk waits only for
  // the copies it reads (psi_ev_n = 0: no pending upload)
  std::vector<cudaEvent_t> psi_ev;
  int psi_ev_n = 0, psi_ev_bands = 0;
  // batched H|psi> workspaces (created on first use; type private to batch.cu)
  std::shared_ptr<void> batch;
  // per-solve Davidson workspaces of a batched solve (basis, reduced matrices)
  std::vector<std::unique_ptr<qe::DevBuf>> dvb_basis, dvb_red;
  // side streams and fork/join events of lockstep Davidson rounds (created on
  // first use; cudaStream_t / cudaEvent_t values)
  std::vector<void*> round_side, round_events;
  // test hook (qe_test_grid_wait): when non-zero, the grid barriers of this
  // context's Davidson solves wait for an arrival that never comes, bounded by
  // this many nanoseconds, so that every one of them runs out
  unsigned long long test_wait_ns = 0;
  qe_ctx() {
    for (qe::DevBuf* b : bufs()) b->sp = &cur;
  }
  std::vector<qe::DevBuf*> bufs() {
    return {&sticks, &vp,       &part,     &proj,   &projd,   &h_v,     &h_beta,
            &h_d,    &h_psi,    &h_hpsi,   &dv_basis, &dv_red, &tc_work, &tc_status, &tc_beta,
            &oz_beta, &oz_work, &dens_acc, &dens_w, &scf_work, &gen_mill, &gen_tab, &gen_rad,
            &gen_scr, &gen_beta};
  }
};

namespace qe {

struct OpView {
  unsigned long long tag = 0;   // identifies the operator within one API call
  int nproj = 0;
  const double* vloc = nullptr;
  const double* beta = nullptr;
  const double* dmat = nullptr;
  // set when beta and D are still being copied on the context's side stream:
  // the projector products wait for it
  cudaEvent_t ready = nullptr;
  // projectors generated on the fly (qe_hpsi_gen): beta is not stored
  const GenProj* gen = nullptr;
};

// Start of an API call on stream st (see qe_ctx::cur).
int ctx_begin(qe_ctx* ctx, cudaStream_t st);
// Return every buffer and plan of the context to the pool (stream-ordered on
// the current stream, which is then synchronised).
int ctx_trim(qe_ctx* ctx);

int get_plan(qe_ctx* ctx, const double lat[9], const double k[3], double ecut, const int grid[3],
             DevPlan** out);
int check_problem(const qe_problem* pr, const char* who);
// overlap (host-memory problems): beta and D are copied on the context's side
// stream and op.ready is set; the caller must make st wait for it (hpsi_core
// does before the projector products) before the call returns.
int resolve_operator(qe_ctx* ctx, const qe_problem* pr, const DevPlan& P, OpView& op,
                     cudaStream_t st, bool overlap = false);
// H psi for nb bands already on the device.  pair (k = 0 plans): the bands are
// real in r, psi(-G) = conj psi(G); two share each FFT and the projections are
// taken real, so the result is H applied to that part of each band.  fp64_pipe
// (QE_FP64): the FFT in double on the FP64 pipe instead of in float-float pairs.
// vp_ready: the context's permuted potential already holds op.vloc for this
// plan and element type (QE_SAME_OPERATOR).
int hpsi_core(qe_ctx* ctx, const DevPlan& P, const OpView& op, int precision, const double* psi,
              double* hpsi, int nb, cudaStream_t st, bool pair = false, bool fp64_pipe = false,
              bool vp_ready = false);
// Status word of the tensor-core kernels since the last check (synchronises on
// `st`); QE_ETIMEOUT with a message if a bounded wait ran out, then resets it.
int tc_check(qe_ctx* ctx, cudaStream_t st);
// Batched H|psi> of device-resident problems on stream st (batch.cu); pair
// (per problem, may be null): as hpsi_core's.
int hpsi_batch_core(qe_ctx* ctx, int nprob, const qe_problem* probs, int precision,
                    const double* const* psi, double* const* hpsi, cudaStream_t st,
                    const char* pair = nullptr);
void ctx_batch_release(qe_ctx* ctx);

}  // namespace qe
