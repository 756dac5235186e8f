// sl_control.cu - device-side control of implicit steps: the tests of Howard policy iteration,
// of the refinement / restart loop and of BiCGSTAB, applied on the device to the state in
// DevCtl, so that a CUDA graph with conditional nodes runs a step (or a march of steps)
// without a host round trip.  Each kernel is one thread: it reads the loop state, applies the
// same test as the host loop in sl_api.cu, and sets the conditional handle of the next node.
// Every while loop has its iteration counter compared with its cap here, so none can run on.
#include <cmath>

#include "../../include/sl_hjb.h"
#include "sl_launch.h"

namespace sl {

// Per-step values from the host (a single step graph is launched right after this kernel).
__global__ void k_ctl_step_prep(DevCtl *c, StepPrep p, double *d_tau) {
  for (int q = 0; q < p.ntau; ++q) d_tau[q] = p.tau[q];
  c->extrap = p.extrap;
  c->need_improve = p.need_improve;
  c->hier_valid = p.hier_valid;
  c->changes_since_build = p.changes_since_build;
  c->status = SL_OK;
  c->step = 1;
  c->nsteps = 1;
}
void launch_ctl_step_prep(DevCtl *c, const StepPrep &p, double *d_tau, cudaStream_t s) {
  note_launch();
  k_ctl_step_prep<<<1, 1, 0, s>>>(c, p, d_tau);
}

// Start of a march: the handle starts like a new one (no policy, no hierarchy).
__global__ void k_ctl_march_begin(DevCtl *c, int nsteps, int extrap_first, int need_improve_first,
                                  cudaGraphConditionalHandle march) {
  c->step = 1;
  c->nsteps = nsteps;
  c->status = SL_OK;
  c->extrap_first = extrap_first;
  c->need_improve_first = need_improve_first;
  c->hier_valid = 0;
  c->changes_since_build = 0;
  cudaGraphSetConditional(march, nsteps >= 1 ? 1u : 0u);
}
void launch_ctl_march_begin(DevCtl *c, int nsteps, int extrap_first, int need_improve_first,
                            cudaGraphConditionalHandle march, cudaStream_t s) {
  note_launch();
  k_ctl_march_begin<<<1, 1, 0, s>>>(c, nsteps, extrap_first, need_improve_first, march);
}

// Start of a step.  In a march (tau_table != nullptr) the step's time factors come from the
// table the host filled for every step, and only the march's first step may start without a
// policy or without extrapolation.
__global__ void k_ctl_step_begin(DevCtl *c, const double *tau_table, int ntau, double *d_tau,
                                 int extrap_opt, int howard_init, cudaGraphConditionalHandle improve0,
                                 cudaGraphConditionalHandle pre, cudaGraphConditionalHandle pi) {
  if (tau_table) {
    const int st = c->step;
    for (int q = 0; q < ntau; ++q) d_tau[q] = tau_table[size_t(st - 1) * ntau + q];
    c->extrap = st > 1 ? extrap_opt : c->extrap_first;
    c->need_improve = st > 1 ? 0 : c->need_improve_first;
  }
  c->pi_it = 0;
  c->c_steps += 1;
  c->skip_ok = 0;  // no improvement in this step yet
  cudaGraphSetConditional(improve0, c->need_improve ? 1u : 0u);
  // a step that keeps the previous policy improves it at its first iterate (howard_init 1)
  cudaGraphSetConditional(pre, (howard_init && !c->need_improve && c->status == SL_OK) ? 1u : 0u);
  cudaGraphSetConditional(pi, c->status == SL_OK ? 1u : 0u);
}
void launch_ctl_step_begin(DevCtl *c, const double *tau_table, int ntau, double *d_tau, int extrap_opt,
                           int howard_init, cudaGraphConditionalHandle improve0,
                           cudaGraphConditionalHandle pre, cudaGraphConditionalHandle pi, cudaStream_t s) {
  note_launch();
  k_ctl_step_begin<<<1, 1, 0, s>>>(c, tau_table, ntau, d_tau, extrap_opt, howard_init, improve0, pre, pi);
}

// After the improvement at a step's first iterate: its changes count toward the rebuild test;
// a NaN stops the step before its Howard loop.
__global__ void k_ctl_preimproved(DevCtl *c, const unsigned long long *changes, const int *flags,
                                  cudaGraphConditionalHandle pi) {
  c->c_pre += 1;
  if (*flags & 1) {
    c->status = SL_ENAN;
    cudaGraphSetConditional(pi, 0u);
    return;
  }
  const long long ch = (long long)*changes;
  c->changes_since_build += ch;
  c->c_changes += ch;
}
void launch_ctl_preimproved(DevCtl *c, const unsigned long long *changes, const int *flags,
                            cudaGraphConditionalHandle pi, cudaStream_t s) {
  note_launch();
  k_ctl_preimproved<<<1, 1, 0, s>>>(c, changes, flags, pi);
}

// After the first improvement of a march (the policy has changed wholesale).
__global__ void k_ctl_improved0(DevCtl *c) {
  c->hier_valid = 0;
  c->c_improve0 += 1;
}
void launch_ctl_improved0(DevCtl *c, cudaStream_t s) {
  note_launch();
  k_ctl_improved0<<<1, 1, 0, s>>>(c);
}

// X = 2 U - V on interior nodes when this step extrapolates (the k_extrapolate arithmetic).
__global__ void k_extrapolate_ctl(double *__restrict__ X, const double *__restrict__ U,
                                  const double *__restrict__ V, int n, const DevCtl *c) {
  if (!c->extrap) return;
  const size_t N = size_t(n) * n;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < N; i += size_t(gridDim.x) * blockDim.x) {
    const int i1 = int(i % n), i2 = int(i / n);
    if (i1 == 0 || i2 == 0 || i1 == n - 1 || i2 == n - 1) continue;
    X[i] = 2.0 * U[i] - V[i];
  }
}
void launch_extrapolate_ctl(double *X, const double *U, const double *V, int n, const DevCtl *c,
                            cudaStream_t s) {
  note_launch();
  k_extrapolate_ctl<<<kRedBlocks, 256, 0, s>>>(X, U, V, n, c);
}

// Howard iteration, before the solve: rebuild the hierarchy when it is not valid or when more
// than `thresh` rows changed control since it was built.
__global__ void k_ctl_pi_pre(DevCtl *c, long long thresh, cudaGraphConditionalHandle rebuild) {
  const bool rb = !c->hier_valid || c->changes_since_build > thresh;
  c->c_pibody += 1;
  if (rb) c->c_rebuild += 1;
  cudaGraphSetConditional(rebuild, rb ? 1u : 0u);
}
void launch_ctl_pi_pre(DevCtl *c, long long thresh, cudaGraphConditionalHandle rebuild, cudaStream_t s) {
  note_launch();
  k_ctl_pi_pre<<<1, 1, 0, s>>>(c, thresh, rebuild);
}

__global__ void k_ctl_built(DevCtl *c, NexplPtrs np) {
  c->hier_valid = 1;
  c->changes_since_build = 0;
  for (int l = 1; l < np.L && l < 16; ++l) c->nexpl[l] = *np.p[l];
}
void launch_ctl_built(DevCtl *c, const NexplPtrs &np, cudaStream_t s) {
  note_launch();
  k_ctl_built<<<1, 1, 0, s>>>(c, np);
}

// Start of a linear solve.
// Start of a linear solve: the first solve of a step's Howard iteration stops at loose_tol when
// that is set (sl_opts.howard_loose_tol), every other at tol.
__global__ void k_ctl_ls_begin(DevCtl *c, double tol, double loose_tol, cudaGraphConditionalHandle ir) {
  c->round = 0;
  c->total = 0;
  c->ls_loose = (loose_tol > 0.0 && c->pi_it == 0) ? 1 : 0;
  c->ls_tol = c->ls_loose ? loose_tol : tol;
  c->tolk = c->ls_tol;
  c->ls_done = 0;
  c->need_true = 1;
  c->rec_rounds = 0;
  cudaGraphSetConditional(ir, 1u);
}
void launch_ctl_ls_begin(DevCtl *c, double tol, double loose_tol, cudaGraphConditionalHandle ir, cudaStream_t s) {
  note_launch();
  k_ctl_ls_begin<<<1, 1, 0, s>>>(c, tol, loose_tol, ir);
}

// k_init_scalars with the threshold (tolk)^2 from the loop state, keeping the norms of the
// solve's right-hand side (computed once before its first round).
__global__ void k_init_scalars_ctl(BicgScalars *S, const DevCtl *c) {
  BicgScalars z = {};
  z.rho_old = 1.0;
  z.alpha = 1.0;
  z.omega = 1.0;
  const double tk = c->tolk;
  z.tolrel2 = tk * tk;
  z.bnorm2 = S->bnorm2;
  z.bmax = S->bmax;
  z.tol2 = z.tolrel2 * z.bnorm2;
  z.inject_bd = S->inject_bd;
  *S = z;
}
void launch_init_scalars_ctl(BicgScalars *S, const DevCtl *c, cudaStream_t s) {
  note_launch();
  k_init_scalars_ctl<<<1, 1, 0, s>>>(S, c);
}

// One refinement round, after the true residual: stop when ||r||_2 <= tol ||F||_2 and
// ||r||_inf <= tol ||F||_inf; tighten the recurrence's threshold tenfold when only the 2-norm
// test holds; in FP64 give up once kry_max Krylov iterations are spent.
__global__ void k_ctl_ir_decide(DevCtl *c, const BicgScalars *S, double tol, int fp64, int kry_max,
                                cudaGraphConditionalHandle enter) {
  c->c_true += 1;
  tol = c->ls_tol;  // this solve's tolerance (k_ctl_ls_begin)
  const double bn2 = S->bnorm2, bmax = S->bmax, rr = S->rr, rmax = S->rmax;
  unsigned go = 0;
  if (S->nonfinite || !isfinite(rr)) {
    c->status = SL_ENAN;
  } else {
    c->res_final = bn2 > 0 ? sqrt(rr / bn2) : sqrt(rr);
    const bool ok2 = rr <= tol * tol * bn2;
    const bool okinf = rmax <= tol * bmax;
    if (ok2 && okinf) {
      c->ls_done = 1;
    } else {
      if (ok2 && !okinf) c->tolk *= 0.1;
      if (fp64 && c->total >= kry_max) c->status = SL_ENOCONV_KRYLOV;
      else go = 1;
    }
  }
  if (go) c->c_enter += 1;
  cudaGraphSetConditional(enter, go);
}
void launch_ctl_ir_decide(DevCtl *c, const BicgScalars *S, double tol, int fp64, int kry_max,
                          cudaGraphConditionalHandle enter, cudaStream_t s) {
  note_launch();
  k_ctl_ir_decide<<<1, 1, 0, s>>>(c, S, tol, fp64, kry_max, enter);
}

__global__ void k_ctl_kry_begin(DevCtl *c, int fp64, int kry_max, cudaGraphConditionalHandle kry) {
  c->kry_it = 0;
  c->kry_res = KRY_RUNNING;
  c->kry_maxit = fp64 ? kry_max - c->total : kry_max;
  cudaGraphSetConditional(kry, c->kry_maxit >= 1 ? 1u : 0u);
  if (c->kry_maxit < 1) c->kry_res = KRY_CAP;
}
void launch_ctl_kry_begin(DevCtl *c, int fp64, int kry_max, cudaGraphConditionalHandle kry,
                          cudaStream_t s) {
  note_launch();
  k_ctl_kry_begin<<<1, 1, 0, s>>>(c, fp64, kry_max, kry);
}

// End of one BiCGSTAB iteration: the host loop's tests in its order (non-finite, converged,
// breakdown), then the iteration cap.
__global__ void k_ctl_kry_check(DevCtl *c, const BicgScalars *S, cudaGraphConditionalHandle kry) {
  c->kry_it += 1;
  c->total += 1;
  c->c_kry += 1;
  int res = KRY_RUNNING;
  if (S->nonfinite) res = KRY_NONFINITE;
  else if (S->rr <= S->tol2) res = KRY_CONVERGED;
  else if (S->breakdown) res = KRY_BREAKDOWN;
  else if (c->kry_it >= c->kry_maxit) res = KRY_CAP;
  c->kry_res = res;
  cudaGraphSetConditional(kry, res == KRY_RUNNING ? 1u : 0u);
}
void launch_ctl_kry_check(DevCtl *c, const BicgScalars *S, cudaGraphConditionalHandle kry, cudaStream_t s) {
  note_launch();
  k_ctl_kry_check<<<1, 1, 0, s>>>(c, S, kry);
}

// After BiCGSTAB: a non-finite value ends the solve; in FP64 so does the iteration cap (the
// refinement of mixed precision goes on to its next round, and a breakdown restarts from the
// true residual in either precision).
__global__ void k_ctl_kry_end(DevCtl *c, int fp64) {
  if (c->kry_res == KRY_NONFINITE) c->status = SL_ENAN;
  else if (fp64 && c->kry_res == KRY_CAP) c->status = SL_ENOCONV_KRYLOV;
}
void launch_ctl_kry_end(DevCtl *c, int fp64, cudaStream_t s) {
  note_launch();
  k_ctl_kry_end<<<1, 1, 0, s>>>(c, fp64);
}

__global__ void k_ctl_ir_end(DevCtl *c, int rounds, cudaGraphConditionalHandle ir) {
  c->round += 1;
  unsigned more = 0;
  if (c->status == SL_OK && !c->ls_done) {
    if (c->round >= rounds) c->status = SL_ENOCONV_KRYLOV;
    else more = 1;
  }
  cudaGraphSetConditional(ir, more);
}
void launch_ctl_ir_end(DevCtl *c, int rounds, cudaGraphConditionalHandle ir, cudaStream_t s) {
  note_launch();
  k_ctl_ir_end<<<1, 1, 0, s>>>(c, rounds, ir);
}

// Start of a refinement round: take a true residual (then k_ctl_ir_decide sets `enter`), or go
// straight to the inner solve on the previous inner solve's residual.
__global__ void k_ctl_ir_pre(DevCtl *c, cudaGraphConditionalHandle tr, cudaGraphConditionalHandle enter) {
  c->c_ir += 1;
  const bool t = c->need_true != 0;
  cudaGraphSetConditional(tr, t ? 1u : 0u);
  if (!t) {
    c->c_enter += 1;
    cudaGraphSetConditional(enter, 1u);
  }
}
void launch_ctl_ir_pre(DevCtl *c, cudaGraphConditionalHandle tr, cudaGraphConditionalHandle enter,
                       cudaStream_t s) {
  note_launch();
  k_ctl_ir_pre<<<1, 1, 0, s>>>(c, tr, enter);
}

// End of an inner solve of mixed precision: where the next round starts (ir_next_recursive; S
// still holds the norms of the last true residual); a breakdown or a failure always goes back
// to a true residual.
__global__ void k_ctl_ir_next(DevCtl *c, const BicgScalars *S, const BicgScalars *S32, int max_rec) {
  const bool ok = c->status == SL_OK && (c->kry_res == KRY_CONVERGED || c->kry_res == KRY_CAP);
  const bool rec = ok && ir_next_recursive(S32->rr, c->ls_tol, S->bnorm2, S->rr, c->rec_rounds, max_rec);
  c->need_true = rec ? 0 : 1;
  c->rec_rounds = rec ? c->rec_rounds + 1 : 0;
}
void launch_ctl_ir_next(DevCtl *c, const BicgScalars *S, const BicgScalars *S32, int max_rec,
                        cudaStream_t s) {
  note_launch();
  k_ctl_ir_next<<<1, 1, 0, s>>>(c, S, S32, max_rec);
}

// After the linear solve: improve only if it succeeded; a failure ends the Howard loop.
__global__ void k_ctl_after_ls(DevCtl *c, cudaGraphConditionalHandle ok, cudaGraphConditionalHandle pi) {
  const bool good = c->status == SL_OK;
  if (good) c->c_ok += 1;
  cudaGraphSetConditional(ok, good ? 1u : 0u);
  if (!good) cudaGraphSetConditional(pi, 0u);
}
void launch_ctl_after_ls(DevCtl *c, cudaGraphConditionalHandle ok, cudaGraphConditionalHandle pi,
                         cudaStream_t s) {
  note_launch();
  k_ctl_after_ls<<<1, 1, 0, s>>>(c, ok, pi);
}

// Howard stop test after an improvement: the policy is unchanged, or
// ||X^m - X^{m-1}||_inf <= pi_tol max(1, ||X^m||_inf); pi_max iterations at most.
__global__ void k_ctl_pi_post(DevCtl *c, const unsigned long long *changes, const int *flags,
                              const double *maxd, double pi_tol, int pi_max,
                              cudaGraphConditionalHandle pi) {
  unsigned more = 0;
  if (*flags & 1) {
    c->status = SL_ENAN;
  } else {
    const long long ch = (long long)*changes;
    c->skip_ok = 1;  // this improvement was at the iterate the next stop test measures from
    c->changes_since_build += ch;
    c->c_pi += 1;
    c->c_changes += ch;
    c->pi_it += 1;
    if (!isfinite(maxd[0])) {
      c->status = SL_ENAN;
    } else {
      const bool small = maxd[0] <= pi_tol * fmax(1.0, maxd[1]);
      // a loosely solved iterate never ends the iteration: the next solve is tight
      if (!(ch == 0 || small) || c->ls_loose) {
        if (c->pi_it >= pi_max) c->status = SL_ENOCONV_PI;
        else more = 1;
      }
    }
  }
  cudaGraphSetConditional(pi, more);
}
void launch_ctl_pi_post(DevCtl *c, const unsigned long long *changes, const int *flags,
                        const double *maxd, double pi_tol, int pi_max, cudaGraphConditionalHandle pi,
                        cudaStream_t s) {
  note_launch();
  k_ctl_pi_post<<<1, 1, 0, s>>>(c, changes, flags, maxd, pi_tol, pi_max, pi);
}

__global__ void k_ctl_march_end(DevCtl *c, cudaGraphConditionalHandle march) {
  c->step += 1;
  cudaGraphSetConditional(march, (c->status == SL_OK && c->step <= c->nsteps) ? 1u : 0u);
}
void launch_ctl_march_end(DevCtl *c, cudaGraphConditionalHandle march, cudaStream_t s) {
  note_launch();
  k_ctl_march_end<<<1, 1, 0, s>>>(c, march);
}

}  // namespace sl
