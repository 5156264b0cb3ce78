// Stop rules of the relaxation (Eq. normres, Sec. III.C) for one iteration,
// run by a single thread: normalised residual r = <|R|> / eps (absolute when
// eps = 0) below tol: converged; it = max_iter, a residual rise while bad
// points were present, or no new minimum for `patience` iterations: stopped
// with the minimum-residual iterate; a non-finite R or eps: failed.  The
// iteration index is counted on the device (ctl->next_it), so one launch
// serves every iteration of a captured graph.
#pragma once
#include "kernels.cuh"

namespace dgp {

__device__ __forceinline__ void relax_control_step(SolveCtl* __restrict__ c, const double* __restrict__ stats,
                                                   const double* __restrict__ abs_src_sum,
                                                   double* __restrict__ hist, int max_iter, int patience,
                                                   double tol, double inv_m) {
  if (c->done) return;
  const int it = c->next_it;
  if (c->fault) {  // a wait of this iteration gave up: its statistics are incomplete
    c->status = CTL_FAULT;
    c->done = 1;
    return;
  }
  c->next_it = it + 1;
  if (it == 0) {
    const double eps = abs_src_sum[0] * inv_m;
    c->eps = eps;
    c->rnorm = eps > 0.0 ? eps : 1.0;
    c->rbest = INFINITY;
    c->rprev = INFINITY;
    c->prev_nbad = 0.0;
    c->best_it = -1;
    if (!isfinite(eps)) {
      c->status = CTL_NONFINITE;
      c->stop_it = 0;
      c->done = 1;
      return;
    }
  }
  const double r = stats[0] * inv_m / c->rnorm;
  const double nbad = stats[2];
  hist[it] = r;
  c->last_bad = nbad;
  c->stop_it = it;
  if (stats[3] > 0.0 || !isfinite(r)) {
    c->status = CTL_NONFINITE;
    c->done = 1;
    return;
  }
  if (r < c->rbest) {
    c->rbest = r;
    c->best_it = it;
  }
  if (r < tol) {
    c->status = CTL_CONVERGED;
    c->done = 1;
    return;
  }
  if (it == max_iter || (it > 0 && c->prev_nbad > 0.0 && r > c->rprev) || it - c->best_it >= patience) {
    c->status = CTL_STOPPED;
    c->done = 1;
    return;
  }
  c->rprev = r;
  c->prev_nbad = nbad;
}

// One CTA: the fixed-order FP64 sum of the fused relaxation's [nblocks][4]
// block partials into stats[0..3] (as launch_finalize), then the stop rules
// above applied to them by thread 0 (the finalize and controller launches of
// an iteration in one).  skip: as launch_finalize.
void launch_finalize_control(const double* partials, int nblocks, double* stats, SolveCtl* ctl,
                             const double* abs_src_sum, double* hist, int max_iter, int patience, double tol,
                             double inv_m, cudaStream_t s, const int* skip);

}  // namespace dgp
