// Device-side bookkeeping of the CG state after an accurate residual, shared by
// the single-problem and batched iterations.
#pragma once

#include "internal.cuh"

namespace ds {

// Statuses kept in CgState::status.
enum CgStatus { CG_RUNNING = 0, CG_CONVERGED = 1, CG_MAX_ITER = 2, CG_BREAKDOWN = 3,
                CG_NONFINITE = 4, CG_STALLED = 5 };

// tot = ||b - A x||^2 just recomputed with the accurate operator (mixed plans) or
// the recursive residual of a float64 plan (exact up to rounding).  A residual
// that has not dropped 10x within stall_iters iterations marks the problem as
// stalled: an ill-posed system whose residual has reached its floor.
__device__ __forceinline__ void track_progress(CgState* st, double tot) {
  if (tot < 1e-2 * st->rr_progress) {
    st->rr_progress = tot;
    st->progress_iter = st->iter;
  }
}

__device__ __forceinline__ bool stalled(const CgState* st) {
  return st->stall_iters > 0 && st->iter - st->progress_iter >= st->stall_iters;
}

// Mixed plans, after the accurate residual refresh.
__device__ __forceinline__ void after_refresh(CgState* st, double tot) {
  // the float32 operator is not accurate enough for this problem when the true
  // residual sits far above the recursive one: iterate with the accurate one
  if (st->mixed && !st->accurate && tot > st->drift2 * st->rr) st->accurate = 1;
  if (tot < st->rr_best) {
    st->rr_best = tot;
    st->improved = 1;
  }
  st->rr = tot;
  st->rr_anchor = tot;
  st->rr_true = tot;
  st->n_reliable += 1;
  st->last_refresh = st->iter;
  st->need = 0;
  track_progress(st, tot);
  if (!isfinite(tot)) {
    st->status = CG_NONFINITE;
    st->done = 1;
  } else if (tot <= st->tol2) {
    st->status = CG_CONVERGED;
    st->done = 1;
  } else if (st->iter >= st->max_iter) {
    st->status = CG_MAX_ITER;
    st->done = 1;
  } else if (stalled(st)) {
    st->status = CG_STALLED;
    st->done = 1;
  }
}

}  // namespace ds
