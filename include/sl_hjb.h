/*
 * sl_hjb.h - C ABI of a GB300 (sm_103a) solver for the implicit truncated LISL Scheme 2
 * applied to two-dimensional Hamilton-Jacobi-Bellman equations
 *
 *     u_t - inf_{k} { tr(a^k D^2 u) + b^k . Du + c^k u + f^k(t, x) } = 0,  a^k = sigma^k sigma^k^T / 2,
 *
 * on a square grid with Dirichlet data psi and initial data g (Section 1, Eqs. 1.1-1.3).
 *
 * Each implicit Euler step (theta = 1 in Eq. 2.11) solves the nonlinear system
 * max_k (A^k X - F^k) = 0 (Eq. 1.10) by Howard policy iteration. Each iteration runs
 * two phases:
 *   - a per-node argmin over the discrete control set of the truncated wide-stencil operator
 *     (Section 2.1, Proposition 2.2, Eq. 2.9);
 *   - a BiCGSTAB solve at the fixed policy, right-preconditioned by a geometric multigrid
 *     V-cycle with Galerkin coarse operators (Section 3.3).
 *
 * Conventions shared by every entry point
 *   - Grid: nx == ny = n nodes per dimension, boundary included, uniform spacing
 *     h = (x_hi - x_lo) / (n - 1) = (y_hi - y_lo) / (n - 1).  Node (i1, i2) sits at
 *     (x_lo + h i1, y_lo + h i2).
 *   - Full-grid arrays are row-major [i2][i1] (x1 runs fastest), n*n entries.
 *   - Policy arrays cover the (n-2)^2 interior nodes, row-major, one uint8_t control index
 *     per node.
 *   - Every pointer named *_dev is device memory; the caller owns it, and the library never
 *     frees it.  The handle owns all workspace; sl_hjb_create allocates it and
 *     sl_hjb_destroy frees it.
 *   - Work is ordered on the given CUDA stream (a cudaStream_t passed as void*; NULL = legacy
 *     default stream).  Calls that return iteration counts or statistics synchronise that
 *     stream before returning.
 *   - Errors: every call returns an sl_status.  The first failure is recorded in the handle;
 *     sl_hjb_last_error returns a message.  No call traps or hangs the GPU: iteration loops
 *     are capped and report SL_ENOCONV_* when the cap is reached.
 */
#ifndef SL_HJB_H
#define SL_HJB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sl_hjb sl_hjb;

typedef enum {
  SL_OK = 0,
  SL_EINVAL = 1,          /* invalid argument or unsupported configuration */
  SL_ENOMEM = 2,          /* device allocation failed */
  SL_ECUDA = 3,           /* a CUDA runtime call failed */
  SL_ECFL = 4,            /* dt * c^k > 1 for some control (Proposition 2.4, theta = 1) */
  SL_ENOCONV_PI = 5,      /* Howard iteration reached pi_max */
  SL_ENOCONV_KRYLOV = 6,  /* BiCGSTAB / refinement reached its iteration cap */
  SL_EBREAKDOWN = 7,      /* BiCGSTAB breakdown (rho or omega vanished); handled inside the
                             solves by a restart, not returned by the step entry points */
  SL_ENAN = 8,            /* a NaN or Inf appeared in a residual or control value */
  SL_ETIMEOUT = 9         /* a bounded device-side wait gave up (the TMA tile copies of the
                             fine operator did not arrive) */
} sl_status;

/* Grid of Eq. 1.1 (Section 2.4: "N_x x N_x equispaced nodes"). */
typedef struct {
  int nx, ny;                     /* nodes per dimension, boundary included; nx == ny, 5 <= nx <= 46340
                                     (nx^2 < 2^31: grid indices are 32-bit) */
  double x_lo, x_hi, y_lo, y_hi;  /* square cells: x_hi - x_lo == y_hi - y_lo */
} sl_grid;

/* Discrete control set {k = 0..K-1} with x-independent coefficients (Eq. 1.4).
 * Column p of sigma^k (a 2 x P matrix) is (sigma[(k*2+0)*P + p], sigma[(k*2+1)*P + p]).
 * Scheme 2 (Section 1) uses the directions +-sqrt(h) sigma_p and h b. */
typedef struct {
  int K;                /* 1 .. 255 */
  int P;                /* 1 .. 4 */
  const double *sigma;  /* host, K*2*P, or NULL when sigma_field is given */
  const double *b;      /* host, K*2 drift, or NULL for b = 0 */
  const double *c;      /* host, K discount, or NULL for c = 0 */
  const double *sigma_field;  /* host, n*n*2*P, or NULL: an x-dependent diffusion shared by all
                                 controls (Section 2.4, Problem A), sigma_field[((i2*n + i1)*2 + d)*P + p]
                                 = component d of column p at node (i1, i2); sigma is then ignored.
                                 The controls differ through b and c; the policy improvement is FP64
                                 (argmin_screen ignored) and sl_hjb_adjoint gives no dJ/dtheta. */
} sl_controls;

/* Time factors tau(t) of the separable source and boundary data. */
enum { SL_TAU_ONE = 0, SL_TAU_EXP = 1 /* exp(rate t) */, SL_TAU_LINEAR = 2 /* t */ };

/* Coefficient callback.  Eqs. 1.1-1.3 let the source f^k(t, x) and the Dirichlet data psi(t, x)
 * be general functions of time and space; a callback fills their values on the device at each
 * implicit step's time t_n (theta = 1 evaluates them at t_n, Section 1).  The library calls it
 * on the host thread that runs the step, before any kernel of that step reads the values:
 *   - source callback: once for each m = 0 .. nf-1, to write F_m(t_n, .) into dev_out; the
 *     source of control k is then f^k(t_n, .) = sum_m phi[k*nf + m] F_m(t_n, .);
 *   - boundary callback: once (m = 0), to write psi(t_n, .) into dev_out on the boundary nodes
 *     (interior entries are ignored).
 * dev_out is library-owned device memory of n*n FP64 values in the full-grid layout; it is
 * valid for the duration of the call.  The callback must enqueue its writes on `stream` (a
 * cudaStream_t, the handle's stream for this call) or finish them before it returns; the
 * library reads dev_out in stream order afterwards.  `user` is sl_source.cb_user.  A callback
 * must not call back into the library with the same handle. */
typedef void (*sl_field_cb)(double t, const sl_grid *grid, int m, double *dev_out, void *user,
                            void *stream);

/* Source and boundary data.  Either the separable form
 *   f^k(t, x) = sum_m phi[k*nf + m] sum_q tau_q(t) G[((m*nq + q)*n + i2)*n + i1],
 *   psi(t, x) = sum_q tau'_q(t) Psi[(q*n + i2)*n + i1] (boundary entries),
 * whose tables G and Psi stay in the caller's device memory and must outlive the handle (the
 * fast path: the per-step tables are one kernel), or callbacks (sl_field_cb) for data of any
 * other form: with f_cb set, G_dev, nq, tau_kind and tau_rate are ignored; with psi_cb set,
 * npsi, Psi_dev, psi_kind and psi_rate are ignored.  phi and nf are used in both cases. */
typedef struct {
  int nf, nq;
  const double *phi;       /* host, K*nf */
  const double *G_dev;     /* device, nf*nq*n*n */
  const int *tau_kind;     /* host, nq */
  const double *tau_rate;  /* host, nq */
  int npsi;                /* 0: psi = 0 */
  const double *Psi_dev;   /* device, npsi*n*n, or NULL */
  const int *psi_kind;     /* host, npsi */
  const double *psi_rate;  /* host, npsi */
  sl_field_cb f_cb;        /* NULL: separable source from G_dev and tau */
  sl_field_cb psi_cb;      /* NULL: separable boundary data from Psi_dev (or psi = 0) */
  void *cb_user;           /* passed to both callbacks */
} sl_source;

typedef struct {
  int precision;        /* 0: FP64 throughout.  1: mixed - FP32 V-cycle, FP32 preconditioner
                           weights and FP32 inner BiCGSTAB inside FP64 iterative refinement;
                           FP64 outer residual and FP64 policy decision. */
  int levels;           /* multigrid levels including the finest; 0 = coarsen to 5 x 5 */
  int nu1, nu2;         /* damped-Jacobi pre- / post-smoothing sweeps */
  double omega;         /* Jacobi weight */
  double krylov_tol;    /* stop when ||F - A X||_2 <= krylov_tol ||F||_2 and
                           ||F - A X||_inf <= krylov_tol ||F||_inf (true FP64 residual).  With
                           c = 0, A^alpha has row sums >= 1, so one step's error is at most
                           krylov_tol ||F||_inf and n steps add at most n times that. */
  int kry_max;          /* BiCGSTAB iterations per solve (FP64) or per refinement (mixed) */
  double inner_tol;     /* mixed: relative tolerance of each inner FP32 solve */
  int ir_max;           /* mixed: refinement sweeps per solve */
  double pi_tol;        /* Howard stop: ||X^m - X^{m-1}||_inf <= pi_tol max(1, ||X^m||_inf) */
  int pi_max;           /* Howard iterations per step */
  double tie_rel;       /* argmin picks the lowest k with v_k <= v_min + tie_rel max(1, |v_min|) */
  int argmin_screen;    /* 1 (default): screen controls in FP32 with a rigorous rounding bound,
                           then decide in FP64 among the survivors (identical result, in either
                           precision); 0: all FP64 */
  double rebuild_frac;  /* rebuild the Galerkin hierarchy when more than rebuild_frac * N
                           rows changed control since the last build (0: on any change).
                           The fine level always applies the current policy; a coarse
                           hierarchy built for a policy that differs in a few rows is still
                           a close preconditioner, and the solve tolerance is unchanged.
                           Default 0.01: at 2049^2 fewer than 0.1 % of the rows change per
                           step, and rebuilding every step cost about 1.3 ms of a 19 ms step
                           for the same iteration count. */
  int use_graphs;       /* 2: each implicit step is one CUDA-graph launch: its Howard,
                           refinement / restart and BiCGSTAB loops are conditional graph nodes
                           whose tests run on the device (captured once per step size), so a step
                           reads the host only once at its end; used with the geometric V-cycle
                           and x-independent sigma outside sl_hjb_solve_record, otherwise as 1.
                           1: each BiCGSTAB iteration is one CUDA-graph launch (captured once per
                           precision and step size); 0: plain stream launches.  All three run the
                           same kernels in the same order and give the same result bit for bit. */
  int coarse_tail_rows; /* levels with at most this many rows run, from the first such level
                           down, in one thread block per V-cycle; 0: never; -1: default
                           (1024 rows in mixed precision, 0 in FP64, whose per-SM rate is low) */
  int extrapolate;      /* 1: when a step continues the previous one (same dt, t = t_prev + dt)
                           its first linear solve starts from 2 U^{n-1} - U^{n-2}; Howard's stop
                           test still measures against U^{n-1}.  0: start from U^{n-1}. */
  int precond;          /* BiCGSTAB preconditioner.  0: the geometric V-cycle (Section 3.3).
                           1: aggregation AMG with a K-cycle (the aggregation multigrid the paper
                           recommends in Section 3.4): two pairwise-matching passes per level
                           (aggregates of at most four unknowns, Galerkin P^T A P), damped Jacobi
                           (nu1, nu2, omega), GCR-accelerated coarse corrections, dense coarsest
                           solve.  The V-cycle entry points and sl_hjb_adjoint need precond 0. */
  int amg_k_levels;     /* precond 1: coarse levels 1..amg_k_levels take two GCR steps, deeper
                           levels one */
  int smoother;         /* smoother of the geometric V-cycle (nu1 / nu2 sweeps, relaxation weight
                           omega): 0 damped Jacobi; 1 two-colour (red-black) Gauss-Seidel, the
                           data-parallel form of the paper's Gauss-Seidel smoother (Section 3.3):
                           the nodes with i1 + i2 even, then the odd ones, each colour updated at
                           once from the current values of all nodes.  The wide stencils couple
                           nodes of one colour, which a colour's simultaneous update treats as
                           Jacobi does; for grid-aligned stencils of even reach all couplings are
                           within a colour (see the design notes), and omega = 1 can then diverge.
                           The aggregation K-cycle and the adjoint's transposed cycle use Jacobi. */
  int fine_tma;         /* staging of the FP32 fine-level operator's tiles (apply, residual, Jacobi
                           sweep; tap stride 12): 1 (default): the interior tiles' rows are copied
                           into shared memory by the TMA unit (cp.async.bulk completing on an
                           mbarrier), one tile per block; 2: a persistent kernel that keeps the
                           next tile's copies in flight while it computes the current one (two
                           buffers); 0: the threads stage every tile.  All three compute each row
                           the same way and give the same result bit for bit. */
  int coarse_fusion;    /* f >= 1: the V-cycle's levels l >= f (coarse levels only: f = 1 is the
                           first coarse level) above the single-block tail, with the Jacobi
                           smoother and nu1, nu2 >= 1, take two launches per level and cycle: the
                           last pre-smoothing sweep (or the first, from zero), the residual and
                           the full-weighting restriction in one kernel; the prolongation with
                           the first post-smoothing sweep in another; each tile of rows stages its
                           values once in shared memory.  0: one launch per operation on every
                           level.  All settings give the same result bit for bit.  Default 3: on
                           the first two coarse levels (the widest, where a tile's explicit rows
                           and its halo cost more than the launches saved) the one-pass kernels
                           are faster. */
  int howard_init;      /* initial policy of each implicit step's Howard iteration after the first
                           step (the first step improves on U^0): 0 (default): the previous step's
                           final policy; 1: that policy improved at the step's first iterate
                           (2 U^{n-1} - U^{n-2} when extrapolating, else U^{n-1}).  Howard's
                           iteration converges to the same discrete solution from either (the
                           stop rule is unchanged); 1 saves a linear solve in the steps whose
                           switching fronts the extrapolation predicts, at the cost of one policy
                           improvement in every step. */
  double howard_loose_tol; /* > 0: the first linear solve of each step's Howard iteration stops at
                           this relative residual instead of krylov_tol (it only has to place the
                           switching fronts for the next improvement); an iterate solved this
                           loosely never ends the iteration, so the step's last solve is always at
                           krylov_tol and its policy is the improvement of its result.  Default
                           1e-7; 0: every solve at krylov_tol.  At least krylov_tol. */
  int argmin_skip;      /* with the FP32 screen (argmin_screen 1): 1 (default): a policy
                           improvement after the first one of a step re-decides only the nodes
                           whose last decision could change.  Each decision's margin (how far,
                           in a rigorous bound, every other control lies above the chosen one) is
                           kept; a control value moves by at most (2 sum |w| + |c|) max|dX| when
                           X moves, so a node whose margin exceeds twice that bound for the X
                           change since the last improvement keeps its control, and a tile
                           whose nodes all keep theirs is not evaluated.  The policies are the
                           same as with 0 (every node re-decided). */
  int ir_recursive;     /* mixed precision: the most refinement rounds in a row that start from
                           the previous inner solve's own residual (its recursively updated FP32
                           r, which is F - A X up to FP32 drift) instead of a true FP64 residual,
                           taken while that residual's 2-norm exceeds twice the stop threshold
                           and lies within four orders of magnitude of the last true residual.
                           The stop test is only ever applied to a true FP64 residual.  Default
                           3; 0: every round starts from a true residual.  The backward solves
                           of sl_hjb_adjoint always start their rounds from a true residual. */
} sl_opts;

typedef struct {
  int steps;                  /* implicit steps taken */
  int pi_iters;               /* Howard iterations, summed over steps */
  int krylov_iters;           /* BiCGSTAB iterations (inner ones in mixed mode) */
  int ir_iters;               /* refinement sweeps (mixed mode) */
  int rebuilds;               /* Galerkin hierarchy builds */
  long long policy_changes;   /* rows whose control changed, summed over improvements */
  long long explicit_rows;    /* coarse rows stored explicitly in the last build */
  double res_final;           /* last relative residual ||F - A X||_2 / ||F||_2 */
  double t_argmin_ms, t_hier_ms, t_solve_ms;  /* host-timed phases (sync points; 0 for steps
                                                 that ran as one graph launch) */
  int graph_steps;            /* steps that ran as one graph launch (use_graphs 2) */
} sl_stats;

/* Fills o with the defaults: FP64, as many levels as possible, V(2,2), omega 0.8,
 * krylov_tol 1e-12, kry_max 200, inner_tol 1e-2, ir_max 30, pi_tol 1e-10, pi_max 100,
 * tie_rel 1e-12, argmin_screen 1, rebuild_frac 0.01, use_graphs 2, coarse_tail_rows -1,
 * extrapolate 1, precond 0, amg_k_levels 2, smoother 0, fine_tma 1, coarse_fusion 3, howard_init 0,
 * howard_loose_tol 1e-7, argmin_skip 1, ir_recursive 3. */
void sl_opts_default(sl_opts *o);

/* Creates a solver.  Builds the Scheme-2 stencil tables of every control on every
 * boundary-distance class in FP64 (Proposition 2.2: truncation factors mu, weights A, B;
 * bilinear taps) and allocates the workspace.  Validates the grid (square, n = 2^j + 1 when
 * levels > 1), K, P and the options.  Returns SL_EINVAL on bad input, SL_ENOMEM / SL_ECUDA on
 * device failure.  *h is NULL on failure. */
sl_status sl_hjb_create(sl_hjb **h, const sl_grid *grid, const sl_controls *ctrl,
                        const sl_source *src, const sl_opts *opts, void *stream);

/* One implicit step from t_n - dt to t_n (Eq. 2.11, theta = 1) with Howard iteration.
 * u_dev (n*n, FP64): in U^{n-1} (boundary ignored), out U^n with psi(t_n) on the boundary.
 * The policy of the previous step is the starting policy; the first step starts from an
 * improvement on U^{n-1}.  policy_out_dev ((n-2)^2 uint8) receives the final policy if not
 * NULL.  stats (host, may be NULL) is overwritten with this step's counts.  Returns
 * SL_ECFL if dt * c^k > 1, SL_ENOCONV_PI / SL_ENOCONV_KRYLOV / SL_ENAN on failure of an
 * iteration.  A BiCGSTAB breakdown is not an error of the step: the solve restarts from the
 * true residual, and only when the restarts run out does the step end with SL_ENOCONV_KRYLOV. */
sl_status sl_hjb_step(sl_hjb *h, double *u_dev, double t_n, double dt, uint8_t *policy_out_dev,
                      sl_stats *stats, void *stream);

/* n_steps uniform implicit steps from t0 to t0 + T; u_dev in: g, out: U(t0 + T).
 * stats accumulates over the steps. */
sl_status sl_hjb_solve(sl_hjb *h, double *u_dev, double t0, double T, int n_steps,
                       uint8_t *policy_out_dev, sl_stats *stats, void *stream);

/* ---- Discrete adjoint: gradients of J = sum_x w(x) U^N(x) through the implicit march ----
 *
 * Each step of Eq. 2.11 (theta = 1) at its converged policy alpha_n is the linear system
 * A_n U^n = U^{n-1} + dt f^{alpha_n}(t_n) + (boundary terms).  The paper solves these
 * systems forwards; the adjoint differentiates the same discrete march backwards at fixed
 * policies (valid wherever no policy switches under a small perturbation):
 *   A_N^T mu_N = w,  A_n^T mu_n = mu_{n+1}  (the unknowns are the interior nodes),
 *   dJ/dg                    = mu_1,
 *   dJ/dG[m][q](x)          = sum_n dt tau_q(t_n) phi[alpha_n(x), m] mu_n(x),
 *   dJ/dtheta                = sum_n dt mu_n^T (dL^{alpha_n}/dtheta U^n)
 * for a scalar parameter theta of the diffusion coefficients, with dL/dtheta the derivative
 * of the truncated Scheme-2 operator (Proposition 2.2, Eq. 2.9: endpoints, truncation
 * factors mu, weights A_p, B_p and the bilinear taps) on the piece of its piecewise-smooth
 * dependence on sigma that the current sigma lies in.  Each backward system is solved like a
 * forward one (BiCGSTAB preconditioned by a V-cycle built from the transposed Galerkin levels
 * A_l^T = R A_{l-1}^T P, or the mixed-precision refinement), to opts.krylov_tol. */

/* sl_hjb_solve that also records, for sl_hjb_adjoint, the policy of every step's last linear
 * solve (the policy that defines A_n; one byte per interior node and step) and U^n at every
 * multiple of ckpt_every and at the last step (full grid, FP64).  ckpt_every = 1 keeps every
 * U^n, so the backward pass solves nothing forward again; with ckpt_every = k > 1 the
 * backward pass re-solves the steps between two checkpoints at their recorded policies
 * (k - 1 extra fields of workspace).  The record lives in the handle until the next call;
 * ckpt_every >= 1, otherwise SL_EINVAL.  Synchronises the stream. */
sl_status sl_hjb_solve_record(sl_hjb *h, double *u_dev, double t0, double T, int n_steps,
                              int ckpt_every, sl_stats *stats, void *stream);

/* Backward pass over the last sl_hjb_solve_record.
 *   w_dev        device, n*n: weights of J (boundary entries do not enter).
 *   dJ_dg_dev    device, n*n out: dJ/dg (zero on the boundary, where g is not used).
 *   dJ_dG_dev    device, nf*nq*n*n out (layout of sl_source.G_dev), or NULL to skip.  With a
 *                source callback, nq counts as 1 with tau = 1: dJ_dG[m] is then the gradient
 *                with respect to a time-independent additive change of the table F_m.
 *   nparam       0 .. 8 scalar parameters theta_p of sigma.
 *   dsigma       host, nparam*K*2*P: d sigma / d theta_p, laid out like sl_controls.sigma.
 *   dJ_dtheta    host, nparam out.
 * Returns SL_EINVAL without a preceding record or with bad arguments, and the status of a
 * failing backward solve otherwise.  Leaves the handle's policy at the first step's;
 * synchronises the stream. */
sl_status sl_hjb_adjoint(sl_hjb *h, const double *w_dev, double *dJ_dg_dev, double *dJ_dG_dev,
                         int nparam, const double *dsigma, double *dJ_dtheta, sl_stats *stats,
                         void *stream);

/* Changes the launch configuration of a handle: use_graphs and coarse_tail_rows as in sl_opts
 * (the same steps, launched differently; the single-block tail adds its coarse-level sums in
 * another order, so moving levels into or out of it changes results at rounding level).
 * Captured graphs are dropped and captured again by the next step.  Synchronises the device.
 * SL_EINVAL for use_graphs outside 0..2. */
sl_status sl_hjb_set_launch(sl_hjb *h, int use_graphs, int coarse_tail_rows);

/* Copies the policy that defined step `step`'s system A_step in the last sl_hjb_solve_record
 * (1 <= step <= n_steps; the policy of the step's last linear solve, the one the adjoint
 * differentiates at) to policy_dev ((n-2)^2 uint8, device).  Marching again with these
 * policies fixed (sl_hjb_set_policy + sl_hjb_linear_solve per step) evaluates the smooth piece
 * of the march whose derivative sl_hjb_adjoint returns.  SL_EINVAL without a record or for a
 * step out of range.  Stream-ordered. */
sl_status sl_hjb_recorded_policy(sl_hjb *h, int step, uint8_t *policy_dev, void *stream);

const char *sl_hjb_last_error(const sl_hjb *h);
void sl_hjb_destroy(sl_hjb *h);

/* ---- Aggregation AMG on a given matrix (the preconditioner of precond = 1, standalone) ----
 * Builds the aggregation hierarchy of an n x n matrix given in CSR form (host arrays:
 * rowptr[n+1], col[nnz] sorted ascending within each row, no repeated column, a diagonal entry
 * in every row; val[nnz] FP64) with opts->nu1, nu2, omega and amg_k_levels, exactly as the
 * solver does for its step matrices.  SL_EINVAL for a malformed matrix or when the coarsening
 * stops above 256 unknowns. */
typedef struct sl_amg sl_amg;
sl_status sl_amg_create(sl_amg **a, int n, const int *rowptr, const int *col, const double *val,
                        const sl_opts *opts);
int sl_amg_num_levels(const sl_amg *a);
/* Level `level` (0 = the given matrix): unknowns *n, entries *nnz, and, for non-NULL host
 * arrays, agg[n] = the level-(level+1) unknown of each unknown (levels below the coarsest), and
 * the level's matrix (rowptr[n+1], col[nnz], val[nnz]).  Synchronises. */
sl_status sl_amg_level(const sl_amg *a, int level, int *n, long long *nnz, int *agg, int *rowptr,
                       int *col, double *val);
/* x = one K-cycle applied to b (device vectors of n entries, FP64 for precision 0, FP32 for
 * precision 1).  Stream-ordered; no host synchronisation. */
sl_status sl_amg_apply(sl_amg *a, int precision, const void *b_dev, void *x_dev, void *stream);
const char *sl_amg_last_error(const sl_amg *a);
void sl_amg_destroy(sl_amg *a);

/* Forgets the march state of the handle: the current policy (the next step starts from an
 * improvement on its U^{n-1}, as the first step of a new handle does), the previous step used
 * for extrapolation and the Galerkin hierarchy.  A solve after a reset gives the same result
 * as the same solve on a new handle. */
sl_status sl_hjb_reset(sl_hjb *h);

/* ---- Batched solves: many independent instances on one GPU ----
 *
 * The paper solves one problem at a time; a batch runs many independent instances (each its
 * own grid, control set and source, as for sl_hjb_create) concurrently on one device.  The
 * library assigns instances to n_workers host threads by the longest-processing-time-first
 * rule on the estimated cost nx*ny*n_steps*(K + 32); each worker owns one CUDA stream and
 * solves its instances in decreasing cost, so kernels of different instances overlap on the
 * device.  Every instance runs exactly the launch sequence of sl_hjb_solve on a new handle,
 * so its result equals that solve bit for bit. */
typedef struct {
  sl_grid grid;
  sl_controls ctrl;    /* host arrays are copied by sl_batch_create */
  sl_source src;       /* G_dev / Psi_dev must outlive the batch */
  double *u_dev;       /* device, nx*ny: in g, out U(t0 + T); owned by the caller */
  double t0, T;
  int n_steps;
} sl_instance;

typedef struct sl_batch sl_batch;

/* Creates one handle per instance (all with opts) and the workers' streams.  Returns
 * SL_EINVAL for bad arguments or the status of the first failing sl_hjb_create (then *b is
 * NULL). */
sl_status sl_batch_create(sl_batch **b, int n_inst, const sl_instance *inst, const sl_opts *opts,
                          int n_workers);

/* Solves every instance from its u_dev (reset first, see sl_hjb_reset) and returns when all
 * are done.  status_out / stats_out (host, n_inst entries, may be NULL) receive each
 * instance's status and statistics; a failing instance does not stop the others.  Returns
 * SL_OK or the status of the lowest-numbered failing instance. */
sl_status sl_batch_run(sl_batch *b, sl_status *status_out, sl_stats *stats_out);

/* Worker (0 .. n_workers-1) that runs instance i, or -1. */
int sl_batch_worker_of(const sl_batch *b, int i);

/* LPT plan used by the batch (pure host function): bin_of[i] = bin of item i for n_bins bins,
 * items taken in decreasing cost (ties by index) and each placed in the least-loaded bin
 * (ties by the lowest bin).  Returns SL_OK or SL_EINVAL. */
int sl_batch_plan(int n_items, const double *cost, int n_bins, int *bin_of);

/* One grid size's launch configuration, as chosen by sl_batch_autotune. */
typedef struct {
  int n;                  /* nodes per dimension of the instances it applies to */
  int instances;          /* instances of the batch with that size */
  int coarse_tail_rows;   /* chosen single-block V-cycle tail (sl_opts.coarse_tail_rows; 0 = none) */
  double probe_seconds;   /* wall time of the fastest probe run of the whole batch */
} sl_tune_choice;

/* Autotuner of the batch's launch configuration; the paper has no counterpart.  Once many small
 * grids run concurrently, a batch is limited by kernel launches more than by arithmetic, and the
 * single-block V-cycle tail trades grid-wide launches on the coarse levels for the work of one
 * thread block.  For each grid size of the batch, in decreasing order of its share of the work,
 * every tail size that moves the tail to another level (levels of at most max_tail_rows rows,
 * and none) is timed by a probe run of the whole batch -- every instance, probe_steps implicit
 * steps after one untimed step that captures the graphs, from its current state -- with the
 * other sizes at their current choice, and the fastest is kept (coordinate descent, one pass).
 * The instances' state vectors are restored afterwards, so sl_batch_run starts from the same
 * data, and each handle keeps its chosen configuration (sl_hjb_set_launch).  The choices go to
 * out (capacity max_out; *n_out receives their number).  The tail only changes the order of the
 * coarse levels' sums: every instance still equals, bit for bit, a single solve with the same
 * configuration.  Allocates one state copy per instance for the duration of the call. */
sl_status sl_batch_autotune(sl_batch *b, int probe_steps, int max_tail_rows, sl_tune_choice *out,
                            int max_out, int *n_out);

const char *sl_batch_last_error(const sl_batch *b);
void sl_batch_destroy(sl_batch *b);

/* ---- Stage entry points: single phases of a step, for parity checks and diagnostics ---- */

/* Policy improvement (row-wise linear search of Eq. 1.10) on x_ext_dev (n*n FP64,
 * psi on the boundary) at time t: v_k(j) = (L^k X)_j + c^k X_j + f^k(t, x_j); the new policy
 * becomes the handle's policy and is copied to policy_out_dev if not NULL.  *changes
 * (host, may be NULL) receives the number of rows whose control changed. */
sl_status sl_hjb_improve(sl_hjb *h, const double *x_ext_dev, double t, uint8_t *policy_out_dev,
                         long long *changes, void *stream);

/* Replaces the handle's policy ((n-2)^2 uint8, device). */
sl_status sl_hjb_set_policy(sl_hjb *h, const uint8_t *policy_dev, void *stream);

/* Builds the Galerkin hierarchy A_{l+1} = R A_l P (bilinear P, full-weighting R) for the
 * current policy and step size dt, in the precision of opts.precision (FP64, or FP32
 * copies in mixed mode). */
sl_status sl_hjb_build_hierarchy(sl_hjb *h, double dt, void *stream);

/* y = A_level x on level `level` (0 = finest) with the current policy / hierarchy.
 * x_dev, y_dev: n_l*n_l full-grid vectors of that level, FP64 (precision 0) or FP32
 * (precision 1); x has zero boundary entries, y's boundary entries are left untouched.
 * Stream-ordered and asynchronous (no host synchronisation), so it can be captured in a
 * CUDA graph. */
sl_status sl_hjb_apply(sl_hjb *h, int level, int precision, const void *x_dev, void *y_dev,
                       void *stream);

/* One V(nu1, nu2) cycle from x = 0 for A_0 x = b (the preconditioner application).
 * b_dev, x_dev: n*n full-grid vectors, FP64 (precision 0) or FP32 (precision 1).  The
 * boundary entries of x_dev must be zero on entry (they are read as the Dirichlet zero of
 * the correction) and are left unchanged; every interior entry is written. */
sl_status sl_hjb_vcycle(sl_hjb *h, int precision, const void *b_dev, void *x_dev, void *stream);

/* sl_hjb_vcycle without any device allocation.  The paper has no counterpart: this entry
 * point is for callers that cannot call cudaMalloc while they run.  Examples are a host
 * application whose own pool allocator has reserved the device memory, so that a library's
 * cudaMalloc would fail or split that pool, and a latency-bound loop in which the device-wide
 * synchronisation that cudaMalloc and cudaFree may cause is not acceptable.  Same arguments
 * and same result as sl_hjb_vcycle (to rounding: the coarse levels run one launch per level
 * operation instead of the single-block tail), but the V-cycle's work vectors live in one
 * 2 MiB file-scope device array of the library instead of the handle's buffers, so they must
 * fit there: fine grids up to 257 x 257 nodes in either precision (513 x 513 would need
 * about 3.5 MB in FP32).  Larger grids get SL_EINVAL with a message giving the bytes needed;
 * nothing is allocated and nothing runs.  Every GPU that loads the library holds the array
 * until the process exits.
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); that first call should come before any
 * stream capture.  Every call shares the one array, keeps nothing from the previous call
 * (it clears the part it uses first), and calls that overlap on the GPU (other streams,
 * threads or handles) race with one another.  Stream-ordered; returns without
 * synchronising. */
sl_status sl_hjb_vcycle_noalloc(sl_hjb *h, int precision, const void *b_dev, void *x_dev,
                                void *stream);

/* Solves A^alpha X = F^alpha of the step at time t with step dt for the current policy,
 * starting from x_ext_dev (n*n FP64, overwritten with the solution and psi(t) on the
 * boundary); u_prev_dev is U^{n-1}.  Uses BiCGSTAB (precision 0) or refinement (1). */
sl_status sl_hjb_linear_solve(sl_hjb *h, const double *u_prev_dev, double *x_ext_dev, double t,
                              double dt, sl_stats *stats, void *stream);

/* Sizes of level `level` of the current hierarchy: nodes per dimension, stored explicit
 * rows, and the number of non-zeros (class rows counted with their table's non-zeros,
 * explicit rows with the non-zero entries of their windows; -1 on the matrix-free level 0).
 * Reads the tables back from the device: synchronises with the device (diagnostic use). */
sl_status sl_hjb_level_info(const sl_hjb *h, int level, int *n, long long *explicit_rows,
                            long long *nnz);

/* Storage statistics of one level of the Galerkin hierarchy (Section 3.3's R A P operators),
 * for diagnostics: the fine level is matrix-free; a coarse row is either a class row (stencil
 * from a per-control table) or an explicit row (a dense (2 reach + 1)^2 window). */
typedef struct {
  int n;                       /* nodes per dimension */
  int reach;                   /* stencil reach in nodes (level 0: the fine operator's halo) */
  long long explicit_rows;     /* rows stored as dense windows (0 on level 0) */
  long long class_nnz;         /* non-zeros of the class rows (-1 on level 0) */
  long long explicit_nnz;      /* non-zero entries of the explicit windows
                                  (both count coefficients of interior columns only: rows next
                                  to the boundary also hold weights of boundary nodes, which
                                  multiply the Dirichlet zero of the correction) */
  long long explicit_entries;  /* stored window entries: explicit_rows * (2 reach + 1)^2 */
} sl_level_stats;

/* Fills *out for level `level`.  SL_EINVAL for a null handle or output or a level outside
 * [0, sl_hjb_num_levels).  Synchronises with the device (the tables are read back). */
sl_status sl_hjb_level_stats(const sl_hjb *h, int level, sl_level_stats *out);

/* Number of levels in use. */
int sl_hjb_num_levels(const sl_hjb *h);

/* Test hook for the breakdown path of BiCGSTAB.  Marks the `iterations`-th BiCGSTAB iteration
 * from now (counted over every later solve of the handle, separately for the FP64 iteration
 * and the FP32 inner iteration of mixed precision) as a breakdown, as if rho had vanished; the
 * solve then restarts from the true residual as after a real breakdown.  iterations == 0
 * cancels a pending mark.  If the marked iteration meets the stop test, the solve ends as
 * converged and the mark is spent.  SL_EINVAL for a null handle or a negative count.
 * Synchronises with the device; call it between steps. */
sl_status sl_hjb_inject_breakdown(sl_hjb *h, int iterations);

/* Number of CUDA kernel launches the library has issued since it was loaded, over all
 * handles (host-side counter; used to report how many of the library's kernels ran in a
 * timed region). */
long long sl_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SL_HJB_H */
