// Davidson solves advanced in lockstep rounds (davidson.cu), for drivers that
// admit new solves between rounds (the serving engine, serve.cpp).  Plain
// declarations only, so that host-only translation units can use them.
#pragma once

#include <cstddef>

#include "qegb.h"

namespace qe {

struct DvTask;

// A solve of prob: host arrays (prob->mem = QE_HOST) are copied to device
// buffers the task owns, device arrays are used in place (they must outlive
// the task); psi0 [nbnd][npw][2] lives where prob's arrays do.  precision:
// QE_FP64 or QE_MIXED with the qe_davidson flags; max_dim as qe_davidson's
// (0: default).  Ordered on `stream`; the task starts with its first H
// product pending.
int dv_task_create(qe_ctx* ctx, const qe_problem* prob, int precision, double tol, int max_iter,
                   int max_dim, const double* psi0, void* stream, DvTask** out);
// One round for every unfinished task: the pending H products of all of them
// in one batched call per precision on `stream`, then one Rayleigh-Ritz step
// each, task i on side[i % nside] (cudaStream_t values; ordered after the H
// products and joined back into `stream`), so that the latency-bound dense
// eigensolvers of different tasks overlap on the GPU.  A task's arithmetic is
// the same as in a solve of its own (bit for bit).  `events` holds nside + 1
// cudaEvent_t created with cudaEventDisableTiming.
int dv_round(qe_ctx* ctx, DvTask* const* tasks, int n, void* stream, void* const* side, int nside,
             void* const* events);
bool dv_task_done(const DvTask* t);
// Results of a finished task into host arrays, or device arrays with
// device_out (any may be NULL); returns its
// status (QE_OK, QE_ENOCONV or the error that ended it; the message is set).
int dv_task_result(qe_ctx* ctx, DvTask* t, double* psi, double* evals, double* resid, int* iters,
                   bool device_out, void* stream);
// Frees the task's device buffers (stream-ordered on `stream`).
void dv_task_destroy(DvTask* t, void* stream);

}  // namespace qe
