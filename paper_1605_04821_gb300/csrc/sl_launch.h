// sl_launch.h - host launchers of the sm_103a kernels (one declaration per kernel family).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sl_common.cuh"

namespace sl {

// Host-side count of kernel launches issued by the library (all handles, all threads), and
// the part issued by the calling host thread.
void note_launch(int n = 1);
long long launch_count();
long long thread_launch_count();

// Raises a kernel's dynamic shared-memory limit to the device's opt-in maximum, once per
// kernel and device (thread-safe).  The limit is process-wide state of the kernel: setting it
// to each launch's own size would race between host threads that launch the same kernel with
// different sizes.  prepare_*_kernels apply it to every kernel of a file that may need more
// than 48 KB; sl_hjb_create calls them, so no solve or graph capture changes the attribute.
cudaError_t allow_dynamic_smem(const void *func);
cudaError_t prepare_fine_kernels();
cudaError_t prepare_coarse_kernels();

enum FineOp { OP_APPLY = 0, OP_RESID = 1, OP_JACOBI = 2, OP_JACOBI0 = 3 };

struct ArgminArgs {
  FineTab tab;
  const int32_t *slin;     // [e*tmax + t] offset in the staged tile (dy*SW + dx)
  const int32_t *off;      // [e*tmax + t] packed (dy << 16) | (dx & 0xffff)
  const double *X;         // full grid, psi on the boundary
  const double *F;         // [nf][n*n] source basis values at t
  const float *F32;
  const double *phi;       // [K*nf]
  const float *phi32;
  const double *phimax;    // [nf] max_k |phi_km|
  int nf;
  double tie_rel;
  double cmax;             // max_k |c_k|
  float tie2_32;           // 2 fp32(tie_rel), cmax and phimax in FP32 for the screen's bound
  float cmax32;            // (converted on the host: no FP64 value enters the FP32 loop)
  float phimax32[4];
  const double *Wmax_class;  // [Q*Q]
  uint8_t *policy;         // in: current, out: improved
  unsigned long long *changes;
  int *flags;              // bit 0: non-finite control value
  int halo, SW, SH;        // staged tile: (32 + 2 halo) x (8 + 2 halo)
  int screen;
  // Skipping decisions that cannot change (k_argmin2).  gap[I]: a lower bound, in the units of
  // the control values, on how far every other control lies above the chosen one at the X of
  // the last improvement (Xprev), less the tie window; null: no skipping.  With dX = X - Xprev,
  // a control value moves by at most sum_t |w_t| |dX_t - dX_j| + |c_k| |dX_j|
  // <= Wabs osc(dX) + cmax max|dX| over a block's tile and halo, so a node whose gap exceeds
  // twice that keeps its control.  skip_flag != 0 only within a step after an improvement at
  // Xprev.
  float *gap;
  const double *Xprev;
  const int *skip_flag;
  double Wabs;             // max over table entries of sum_t |w_t|
};

// The packed taps {byte offset in the FP32 staged tile, fp32 weight bits} of the interior
// class of every control, [k*tmax + t], passed as a kernel parameter: rows of the interior
// class (all but a band of width B along the boundary) read them through the constant cache,
// every lane of a warp the same entry, instead of through L1.  The offset is in bytes so that
// the shared load can take it as a uniform register beside the thread's own address.  n = 0
// when they do not fit (K * tmax > kITapMax).
constexpr int kITapMax = 3584;  // 28 KB of kernel parameters
struct ArgminITaps {
  int n;
  int2 t[kITapMax];
};

void launch_coef(const double *G, int nf, int nq, const double *tau, const double *Psi, int npsi,
                 const double *tau_psi, int n, double *F, float *F32, double *Xext, double *Xb,
                 cudaStream_t s);
cudaError_t launch_argmin(const ArgminArgs &a, const ArgminITaps &it, cudaStream_t s);

// slin: staged-tile tap offsets (pitch SW), the same table as the argmin's.
// color (OP_JACOBI / OP_JACOBI0): -1 every row; 0 / 1 a half-sweep of the two-colour
// Gauss-Seidel smoother (rows with (i1 + i2) mod 2 == color updated, the others passed through).
template <typename T>
void launch_fine_op(int op, const FineTab &tab, const int32_t *slin, const uint8_t *policy, T dt,
                    T omega, const T *x, const T *b, T *y, int halo, int SW, cudaStream_t s, int color = -1);

// Jacobi scale omega / d_e of every fine table entry for step size dt (into od64 / od32).
void launch_fine_od(const FineTab &tab, double dt, double omega, double *od64, float *od32,
                    double *iod64, float *iod32, cudaStream_t s);

// r = U_prev - X + dt (L X + c X + f) for the current policy (interior), FP64.  With
// zero_inside = R > 0 the caller promises X = 0 on the interior and R >= the longest tap:
// rows farther than R from the boundary then skip their taps (r = U_prev + dt f).
// ub_out (if not null) receives U_prev + dt f on every interior row; a later residual at the
// same policy, U_prev, dt and source passes it back as ub_in and reads it in place of
// U_prev, F and phi: r = ub - X + dt (L X + c X).
void launch_hjb_resid(const FineTab &tab, const uint8_t *policy, const double *X,
                      const double *Uprev, const double *F, const double *phi, int nf, double dt,
                      double *r, int halo, int SW, cudaStream_t s, int zero_inside = 0,
                      double *ub_out = nullptr, const double *ub_in = nullptr);

template <typename T>
void launch_restrict(const T *rf, int nf, T *bc, int nc, cudaStream_t s);
template <typename T>
void launch_prolong_add(const T *xc, int nc, T *xf, int nf, cudaStream_t s);

// coarse levels
// chunk_scratch: 2 * ceil((n-2)^2 / 256) ints of device scratch.
void launch_classify(int level, const FineTab &tab, const uint8_t *policy, const int32_t *cls_prev,
                     int n_prev, int32_t *cls, int n, int32_t *erow, int *count, int *chunk_scratch,
                     cudaStream_t s);
template <typename T>
cudaError_t launch_rap_explicit(int level, const FineTab &tab, const int32_t *fine_off,
                                const uint8_t *policy, T dt, const CoarseLev<T> &prev,
                                const int32_t *prev_coff, const CoarseLev<T> &cur, int count,
                                T *ewin_out, cudaStream_t s);
template <typename T>
void launch_coarse_op(int op, const CoarseLev<T> &L, const int *nexpl_dev, T omega, const T *x,
                      const T *b, T *y, cudaStream_t s, int color = -1);

// Fused coarse-level passes of the Jacobi V-cycle (levels >= 1): down = (x = omega D^-1 b when
// xin is null, else x = xin) + residual + full-weighting restriction into bc; up = y = one
// Jacobi sweep from cur + P xc.
template <typename T>
void launch_coarse_down(const CoarseLev<T> &L, T omega, const T *b, const T *xin, T *xout, T *bc, int nc,
                        cudaStream_t s);
template <typename T>
void launch_coarse_up(const CoarseLev<T> &L, T omega, const T *b, const T *cur, const T *xc, int nc, T *y,
                      cudaStream_t s);

// Levels l0 .. L-1 of one V-cycle in a single thread block (x[l0] = M_l0^{-1} b[l0]).
template <typename T>
struct TailArgs {
  int l0, L, nu1, nu2;
  int rbgs;  // 1: two-colour Gauss-Seidel sweeps (relaxation omega); 0: damped Jacobi
  T omega;
  CoarseLev<T> lev[kMaxLevels];
  T *x[kMaxLevels], *t[kMaxLevels], *r[kMaxLevels], *b[kMaxLevels];
  const T *Ainv;
  const T *img;  // the levels' stencils packed in the shared-memory layout (launch_tail_pack), or null
};
template <typename T>
void launch_vcycle_tail(const TailArgs<T> &a, cudaStream_t s);
// Bytes of the packed tail stencils of a (0: they do not fit in one block's shared memory).
template <typename T>
size_t tail_image_bytes(const TailArgs<T> &a);
// Packs the tail levels' stencils into img (tail_image_bytes(a) bytes), in the layout the
// shared-memory tail copies; after every change of the hierarchy or of the tail's levels.
template <typename T>
void launch_tail_pack(const TailArgs<T> &a, T *img, cudaStream_t s);

template <typename T>
void launch_coarsest_setup(int level, const FineTab &tab, const uint8_t *policy, T dt,
                           const CoarseLev<T> &L, const int32_t *coff, double *work, T *Ainv,
                           cudaStream_t s);
// x = A^{-1} b, or x = A^{-T} b when trans != 0.
template <typename T>
void launch_coarsest_apply(const T *Ainv, int n, const T *b, T *x, cudaStream_t s, int trans = 0);

// ------------------------------------------------------------------ general fine level
// x-dependent diffusion shared by all controls (per-row taps) plus per-control drift taps
// from (control, boundary class) tables; see sl_general.cu.
struct GeneralArgs {
  int n, nd_stride;
  const int32_t *nd_off;   // [I*nd_stride + t] packed (dy << 16) | (dx & 0xffff) of row I's diffusion taps
  const double *nd_w;      // [I*nd_stride + t]
  const uint8_t *nd_nt;    // [I]
  const double *nd_W;      // [I] sum_p (A_p + B_p)/(2h) of the diffusion part
  const int32_t *dr_off;   // drift tables: [ed*tmax + t] packed offsets (weights in the FineTab)
};
struct GeneralOut {        // the assembled fine table (entry = interior row)
  int stride;
  int32_t *off, *lin;
  double *w64;
  float *w32;
  int2 *pk32;
  longlong2 *pk64;
  uint8_t *nt;
  double *W64, *ws64, *od64;
  float *W32, *ws32, *od32;
};
void launch_assemble_general(const GeneralArgs &g, const FineTab &dtab, const uint8_t *policy,
                             const double *c64, double dt, double omega, int SW, const GeneralOut &o,
                             cudaStream_t s);
void launch_argmin_general(const GeneralArgs &g, const FineTab &dtab, const double *c64, const double *X,
                           const double *F, const double *phi, int nf, double tie_rel, uint8_t *policy,
                           unsigned long long *changes, int *flags, cudaStream_t s);

// out[0..n] = exclusive prefix sums of in[0..n-1], out[n] = total (n >= 1);
// scratch: 2 * ceil(n / 1024) ints.
void launch_exclusive_scan(const int *in, int n, int32_t *out, int *scratch, cudaStream_t s);

// ------------------------------------------------------------------ adjoint (transposed solves)
// Explicit A^T of the fine level: row J (interior index of column j of A) lists the sources i
// with A[i, j] != 0, i != j, sorted by i; the diagonal is stored apart.
template <typename T>
struct CsrTView {
  int n, m;
  const int32_t *rowptr;  // [m*m + 1]
  const int32_t *col;     // [nnz] full-grid index of the source row i
  const T *v;             // [nnz] A[i, j]
  const T *d;             // [m*m] A[j, j]
};
// cnt: m*m ints, scan_scratch: 2 * ceil(m*m / 1024) ints; col/vtmp/v64/v32 sized for every
// tap; R0: the largest |dx|, |dy| of any tap (at most (2^25 - 1) / (n + 1) / 2).
void launch_csrT_build(const FineTab &tab, const int32_t *off, const uint8_t *policy, double dt, int R0,
                       int *cnt, int *scan_scratch, int32_t *rowptr, int32_t *col, double *vtmp,
                       double *v64, float *v32, double *d64, float *d32, cudaStream_t s);
template <typename T>
void launch_fineT_op(int op, const CsrTView<T> &A, T omega, const T *x, const T *b, T *y, cudaStream_t s);
// Dense windows of the rows of A_l^T (level l >= 1) from the forward level; cdense holds the
// class windows [k * win + e].
template <typename T>
void launch_denseT_build(const CoarseLev<T> &L, const T *cdense, T *WT, cudaStream_t s);
template <typename T>
void launch_denseT_op(int op, int n, int R, const T *WT, T omega, const T *x, const T *b, T *y,
                      cudaStream_t s);

// Derivative tables of the fine stencil for np parameters: entry (p, e) at p*E + e.
constexpr int kMaxParams = 8;
struct DTabView {
  int np, E, stride;
  const int32_t *lin;   // [(p*E + e)*stride + t] dy*n + dx
  const double *dw;     // [(p*E + e)*stride + t]
  const uint8_t *nt;    // [p*E + e]
  const double *dW;     // [p*E + e]
};
void launch_interior_copy(int n, const double *x, double *y, cudaStream_t s);
void launch_adj_dG(int n, int nf, int nq, const uint8_t *policy, const double *phi, const double *tau,
                   double dt, const double *mu, double *dG, cudaStream_t s);
// partials: kMaxParams * kRedBlocks doubles; out[p] += dt * mu^T (dL/dtheta_p U).
void launch_adj_dtheta(const FineTab &tab, const DTabView &d, const uint8_t *policy, const double *mu,
                       const double *U, double dt, double *partials, double *out, cudaStream_t s);

// vectors and reductions
template <typename T>
void launch_fill(T *x, size_t N, T v, cudaStream_t s);
template <typename Tin, typename Tout>
void launch_convert(const Tin *x, Tout *y, size_t N, cudaStream_t s, const int *flag = nullptr);
void launch_extrapolate(double *X, const double *U, const double *V, int n, cudaStream_t s);
void launch_add_f32_to_f64(double *x, const float *e, size_t N, cudaStream_t s);

enum Post { POST_RHO_INIT = 0, POST_ALPHA = 1, POST_SS = 2, POST_OMEGA = 3, POST_RHO = 4,
            POST_BNORM = 5, POST_RR = 6 };

template <typename T>
void launch_dot2(const T *a, const T *b, const T *c, const T *d, size_t N, int post,
                 BicgScalars *S, double *partials, unsigned *counter, cudaStream_t s);
template <typename T>
void launch_bicg_p(T *p, const T *r, const T *v, size_t N, int first, const BicgScalars *S,
                   cudaStream_t s);
template <typename T>
void launch_bicg_s(T *sv, const T *r, const T *v, size_t N, BicgScalars *S, double *partials,
                   unsigned *counter, cudaStream_t s);
template <typename T, typename TX>
void launch_bicg_xr(TX *x, const T *phat, const T *shat, const T *sv, const T *t, T *r,
                    const T *rhat, size_t N, BicgScalars *S, double *partials, unsigned *counter,
                    cudaStream_t s);
void launch_norms(const double *a, size_t N, int which, BicgScalars *S, double *partials,
                  unsigned *counter, cudaStream_t s);
void launch_init_scalars(BicgScalars *S, double tolrel2, cudaStream_t s);
void launch_init_scalars_keep_b(BicgScalars *S, double tolrel2, cudaStream_t s);
void launch_maxabs_diff(const double *a, const double *b, int n, double *out2,
                        unsigned *counter, double *partials, cudaStream_t s);


// ---- device-side control of implicit steps (sl_control.cu) ----------------------------------
// The loops of a step (Howard policy iteration, iterative refinement / restarts, BiCGSTAB) and
// of a march run on the device as conditional nodes of one CUDA graph.  These single-thread
// kernels read the loop state below, apply exactly the host loop's tests, and set the
// conditional handles; every loop's counter is capped, so each while node ends.
struct DevCtl {
  int extrap;            // this step's first solve starts from 2 U^{n-1} - U^{n-2}
  int need_improve;      // this step starts with an improvement on U^{n-1} (no policy yet)
  int extrap_first, need_improve_first;  // the same for the first step of a march
  int step, nsteps;      // march: current step (1-based) and its number of steps
  int status;            // sl_status of the step or march (the first failure)
  int pi_it;             // Howard iterations of the current step
  int hier_valid;        // the Galerkin hierarchy belongs to the current policy and step size
  int round, total;      // refinement round and Krylov iterations of the current solve
  int kry_it, kry_maxit, kry_res, ls_done;
  long long changes_since_build;
  double tolk;           // threshold handed to BiCGSTAB's recurrence
  double res_final;      // last relative 2-norm residual
  // counts, accumulated until the host clears them
  long long c_steps, c_improve0, c_pibody, c_pi, c_rebuild, c_ir, c_enter, c_kry, c_ok, c_changes;
  int nexpl[16];         // explicit rows of each level after the last rebuild in the graph
  int tma_err;           // a bounded wait of the TMA fine operator gave up (FineTab::tma_err)
  long long c_pre;       // improvements at a step's first iterate (sl_opts.howard_init 1)
  double ls_tol;         // stop tolerance of the current linear solve
  int ls_loose;          // the current solve is a step's first, at howard_loose_tol
  int skip_ok;           // the argmin may skip settled nodes (ArgminArgs::skip_flag)
  int need_true;         // the next refinement round starts from a true FP64 residual
  int rec_rounds;        // consecutive rounds on the inner solve's own residual
  long long c_true;      // true residuals taken by refinement rounds
};

// Mixed-precision refinement: the next round starts from the inner solve's own residual (the
// recursively updated FP32 r of BiCGSTAB, F - A X up to FP32 drift) when that residual's 2-norm
// is still above twice the stop threshold tol ||F||_2, no more than four orders of magnitude
// below the last true residual (rr_true = its squared 2-norm; the drift, about 1e-7 of that
// residual, then stays below 1e-3 of the one handed on), and fewer than max_rec rounds in a row
// have done so; otherwise it starts from a true FP64 residual, the only one the stop test reads.
// The host loop and the device-side control both decide with this function.
SL_HD bool ir_next_recursive(double inner_rr, double tol, double bn2, double rr_true, int rec_rounds,
                             int max_rec) {
  return rec_rounds < max_rec && inner_rr > 4.0 * (tol * tol * bn2) && inner_rr > 1e-8 * rr_true;
}

// Explicit-row counts of the coarse levels, gathered into DevCtl::nexpl (levels 1 .. L-1).
struct NexplPtrs {
  const int *p[16];
  int L;
};

// Kry results (DevCtl::kry_res)
enum { KRY_RUNNING = 0, KRY_CONVERGED = 1, KRY_BREAKDOWN = 2, KRY_NONFINITE = 3, KRY_CAP = 4 };

// Values the host hands to a single step graph (launched just before it).
struct StepPrep {
  double tau[8];         // tau_q(t_n), then tau'_q(t_n): the separable time factors
  int ntau, extrap, need_improve, hier_valid;
  long long changes_since_build;
};

void launch_ctl_step_prep(DevCtl *c, const StepPrep &p, double *d_tau, cudaStream_t s);
void launch_ctl_march_begin(DevCtl *c, int nsteps, int extrap_first, int need_improve_first,
                            cudaGraphConditionalHandle march, cudaStream_t s);
void launch_ctl_step_begin(DevCtl *c, const double *tau_table, int ntau, double *d_tau, int extrap_opt,
                           int howard_init, cudaGraphConditionalHandle improve0,
                           cudaGraphConditionalHandle pre, cudaGraphConditionalHandle pi, cudaStream_t s);
void launch_ctl_preimproved(DevCtl *c, const unsigned long long *changes, const int *flags,
                            cudaGraphConditionalHandle pi, cudaStream_t s);
void launch_ctl_improved0(DevCtl *c, cudaStream_t s);
void launch_extrapolate_ctl(double *X, const double *U, const double *V, int n, const DevCtl *c,
                            cudaStream_t s);
void launch_ctl_pi_pre(DevCtl *c, long long thresh, cudaGraphConditionalHandle rebuild, cudaStream_t s);
void launch_ctl_built(DevCtl *c, const NexplPtrs &np, cudaStream_t s);
void launch_ctl_ls_begin(DevCtl *c, double tol, double loose_tol, cudaGraphConditionalHandle ir, cudaStream_t s);
void launch_init_scalars_ctl(BicgScalars *S, const DevCtl *c, cudaStream_t s);
void launch_ctl_ir_decide(DevCtl *c, const BicgScalars *S, double tol, int fp64, int kry_max,
                          cudaGraphConditionalHandle enter, cudaStream_t s);
void launch_ctl_kry_begin(DevCtl *c, int fp64, int kry_max, cudaGraphConditionalHandle kry,
                          cudaStream_t s);
void launch_ctl_kry_check(DevCtl *c, const BicgScalars *S, cudaGraphConditionalHandle kry, cudaStream_t s);
void launch_ctl_kry_end(DevCtl *c, int fp64, cudaStream_t s);
void launch_ctl_ir_end(DevCtl *c, int rounds, cudaGraphConditionalHandle ir, cudaStream_t s);
void launch_ctl_ir_pre(DevCtl *c, cudaGraphConditionalHandle tr, cudaGraphConditionalHandle enter,
                       cudaStream_t s);
void launch_ctl_ir_next(DevCtl *c, const BicgScalars *S, const BicgScalars *S32, int max_rec,
                        cudaStream_t s);
void launch_ctl_after_ls(DevCtl *c, cudaGraphConditionalHandle ok, cudaGraphConditionalHandle pi,
                         cudaStream_t s);
void launch_ctl_pi_post(DevCtl *c, const unsigned long long *changes, const int *flags,
                        const double *maxd, double pi_tol, int pi_max, cudaGraphConditionalHandle pi,
                        cudaStream_t s);
void launch_ctl_march_end(DevCtl *c, cudaGraphConditionalHandle march, cudaStream_t s);

// Explicit Galerkin rows with their count read from device memory (*count_dev, at most cap):
// the launch shape does not depend on the classification, so a graph can rebuild the
// hierarchy without the host.  Same per-row arithmetic as launch_rap_explicit.
template <typename T>
cudaError_t launch_rap_explicit_dev(int level, const FineTab &tab, const int32_t *fine_off,
                                    const uint8_t *policy, T dt, const CoarseLev<T> &prev,
                                    const int32_t *prev_coff, const CoarseLev<T> &cur,
                                    const int *count_dev, int cap, T *ewin_out, cudaStream_t s);

}  // namespace sl
