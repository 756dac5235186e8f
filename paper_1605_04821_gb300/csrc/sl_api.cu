// sl_api.cu - C ABI and host orchestration: Howard policy iteration around a
// multigrid-preconditioned BiCGSTAB (FP64) or FP64 iterative refinement of an FP32
// BiCGSTAB with an FP32 V-cycle (mixed).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/sl_hjb.h"
#include "sl_amg.h"
#include "sl_geometry.h"
#include "sl_launch.h"

using namespace sl;

namespace {

struct CoarseBuf {
  int n = 0, m = 0, R = 0, win = 0, cap = 0, nexpl = 0, ctmax = 0;
  int *d_nexpl = nullptr;  // explicit-row count on the device (read by the explicit kernels)
  int32_t *cls = nullptr, *erow = nullptr, *clin = nullptr, *coff = nullptr, *cnt = nullptr;
  int2 *cpk32 = nullptr;
  longlong2 *cpk64 = nullptr;
  double *ewin64 = nullptr, *cw64 = nullptr, *cdiag64 = nullptr;
  float *ewin32 = nullptr, *cw32 = nullptr, *cdiag32 = nullptr;
  double *cdense64 = nullptr, *WT64 = nullptr;  // class windows [k*win + e]; rows of A_l^T
  float *cdense32 = nullptr, *WT32 = nullptr;
  std::vector<int> cnt_host;       // taps per class
  std::vector<int32_t> coff_host;  // class taps' packed offsets (dy << 16) | (dx & 0xffff)
};

template <typename T> T *pick(double *a, float *b);
template <> double *pick<double>(double *a, float *) { return a; }
template <> float *pick<float>(double *, float *b) { return b; }

struct VBuf {  // V-cycle vectors of one level
  double *x64 = nullptr, *t64 = nullptr, *r64 = nullptr, *b64 = nullptr;
  float *x32 = nullptr, *t32 = nullptr, *r32 = nullptr, *b32 = nullptr;
};

struct IterGraph {  // one captured BiCGSTAB iteration
  cudaGraphExec_t exec = nullptr;
  double dt = -1.0;
  long long kernels = 0;
  long long gen = -1;  // AMG hierarchy generation it was captured with
};

// One captured implicit step (use_graphs 2): the Howard, refinement and BiCGSTAB loops are
// conditional nodes of the graph, so a step is one graph launch.  The counts are the kernels
// captured directly in each loop body (the host adds them up from the device's loop counts).
struct DevStepGraph {
  cudaGraphExec_t exec = nullptr;
  double dt = -1.0;
  long long k_step = 0, k_imp0 = 0, k_pre = 0, k_pi = 0, k_rebuild = 0, k_ir = 0, k_enter = 0, k_kry = 0,
            k_ok = 0, k_true = 0;
};

struct KBuf {  // BiCGSTAB vectors on the finest level
  double *r64 = nullptr, *rh64 = nullptr, *p64 = nullptr, *v64 = nullptr, *s64 = nullptr,
         *t64 = nullptr, *ph64 = nullptr, *sh64 = nullptr;
  float *r32 = nullptr, *rh32 = nullptr, *p32 = nullptr, *v32 = nullptr, *s32 = nullptr,
        *t32 = nullptr, *ph32 = nullptr, *sh32 = nullptr, *e32 = nullptr;
};

}  // namespace

struct sl_hjb {
  int n = 0, m = 0, K = 0, P = 0, nf = 0, nq = 0, npsi = 0;
  double h = 0;
  sl_opts o{};
  std::vector<double> phi, phimax, tau_rate, psi_rate, cvec, sigma;
  std::vector<int> tau_kind, psi_kind;
  const double *G = nullptr, *Psi = nullptr;
  // coefficient callbacks: they fill Gcb (nf tables, read with nq = 1 and tau = 1) and Psicb
  // (read as one boundary table with tau = 1) at each step's time
  sl_field_cb f_cb = nullptr, psi_cb = nullptr;
  void *cb_user = nullptr;
  sl_grid grid{};
  double *Gcb = nullptr, *Psicb = nullptr;
  FineTabHost ft;
  FineTab tab{};
  // device tables
  int32_t *d_lin = nullptr, *d_slin = nullptr, *d_off = nullptr;
  int2 *d_pk32 = nullptr;
  longlong2 *d_pk64 = nullptr;
  double *d_w64 = nullptr, *d_W64 = nullptr, *d_ws64 = nullptr, *d_c64 = nullptr, *d_Wmaxc = nullptr;
  float *d_w32 = nullptr, *d_W32 = nullptr, *d_ws32 = nullptr, *d_c32 = nullptr;
  uint8_t *d_nt = nullptr;
  double *d_phi = nullptr, *d_phimax = nullptr, *d_tau = nullptr, *d_tpsi = nullptr;
  double *d_od64 = nullptr;
  float *d_od32 = nullptr;
  int4 *d_ipk32 = nullptr;          // interior taps, tap-major (FineTab::ipk32)
  longlong2 *d_ipk64 = nullptr;
  double *d_iWc64 = nullptr, *d_iod64 = nullptr;
  float *d_iWc32 = nullptr, *d_iod32 = nullptr;
  // general fine level (x-dependent diffusion): drift tables, per-row diffusion taps, and the
  // per-row table assembled for the current policy (h->tab then describes the latter)
  bool general = false;
  FineTab dtab{};
  GeneralArgs gen{};
  GeneralOut gout{};
  NodeTabHost nd;
  float *d_phi32 = nullptr;
  int halo = 0, SW = 0, SH = 0;
  // step state (full-grid FP64 vectors)
  double *X = nullptr, *Xb = nullptr, *Uprev = nullptr, *F = nullptr, *R = nullptr, *Xpi = nullptr,
         *Fvec = nullptr, *Uprev2 = nullptr;
  double *Ub = nullptr;  // U^{n-1} + dt f at the policy of the current solve (its ||F|| pass)
  bool have_prev2 = false;   // Uprev2 holds U^{n-2} of the step just taken (for extrapolation)
  double prev_t = 0.0, prev_dt = 0.0;
  float *F32 = nullptr;
  uint8_t *policy = nullptr;
  bool have_policy = false;
  // hierarchy
  int L = 1;
  CoarseBuf cl[kMaxLevels];
  VBuf vb[kMaxLevels];
  KBuf kb;
  double *cwork = nullptr, *Ainv64 = nullptr;
  float *Ainv32 = nullptr;
  bool hier_valid = false, class_valid = false;
  double hier_dt = -1.0, class_dt = -1.0;
  long long changes_since_build = 0;
  // reductions
  BicgScalars *S = nullptr, *S32 = nullptr, *hS = nullptr;
  double *partials = nullptr, *d_maxd = nullptr, *h_maxd = nullptr;
  unsigned *counter = nullptr;
  unsigned long long *d_changes = nullptr, *h_changes = nullptr;
  int *d_flags = nullptr, *h_flags = nullptr, *d_count = nullptr, *h_count = nullptr;
  IterGraph graph[2];           // [precision]
  IterGraph graphT[2];          // [precision], transposed operators (adjoint solves)
  bool transposed = false;      // level operators act as A_l^T (backward solves)
  int *chunk_scratch = nullptr; // classification counts / offsets
  int tail_l0 = 0;              // first level run by the single-block V-cycle tail (0: none)
  unsigned char *tail_img = nullptr;  // the tail levels' stencils packed for the shared-memory tail
  size_t tail_img_bytes = 0;          // its size (0: the tail runs from global memory)
  size_t tail_img_cap = 0;            // bytes allocated
  double ls_tol = 0.0;                // > 0: the tolerance of the next linear_solve (else krylov_tol)
  cudaStream_t cap_stream = nullptr;
  // adjoint: fine A^T (CSR), gradient tables and the recorded forward march
  int32_t *t_rowptr = nullptr, *t_col = nullptr;
  int *t_cnt = nullptr, *t_scan = nullptr;
  double *t_v64 = nullptr, *t_d64 = nullptr, *t_vtmp = nullptr;
  float *t_v32 = nullptr, *t_d32 = nullptr;
  double *mu = nullptr, *lam = nullptr;        // full grid, zero boundary
  double *d_dtheta = nullptr, *d_dpart = nullptr;
  int32_t *dt_lin = nullptr;
  double *dt_dw = nullptr, *dt_dW = nullptr;
  uint8_t *dt_nt = nullptr;
  size_t dt_cap[4] = {0, 0, 0, 0};            // capacities of dt_lin, dt_dw, dt_nt, dt_dW
  uint8_t *rec_pol = nullptr;                  // [step][m*m] policy of each step's last solve
  double *rec_U = nullptr;                     // checkpoints U^{c k} and U^N, full grid
  double *rec_seg = nullptr;                   // recomputed U^s inside one segment
  size_t rec_pol_cap = 0, rec_U_cap = 0, rec_seg_cap = 0;
  uint8_t *rec_slot = nullptr;                 // where step_impl stores the solve policy
  int rec_N = 0, rec_k = 0;
  double rec_t0 = 0.0, rec_dt = 0.0;
  bool rec_valid = false;
  // device-driven steps (use_graphs 2): loop state on the device and its pinned host mirror,
  // the streams that capture nested conditional bodies, and the captured step
  DevCtl *ctl = nullptr, *h_ctl = nullptr;
  cudaStream_t cap_pool[8] = {};
  DevStepGraph sgraph;
  bool dev_off = false;                        // a capture failed: host-driven steps from then on
  AmgEngine amg;                               // precond 1
  ArgminITaps *itaps = nullptr;                // interior-class taps for the argmin's parameter
  float *d_gap = nullptr;                      // per interior node: margin of its last decision
  double Wabs = 0.0;                           // max over table entries of sum |w|
  long long amg_gen = 0;                       // bumped by every AMG setup (its sizes change)
  std::vector<void *> allocs;
  std::string err;
  sl_status sticky = SL_OK;
};

namespace {

sl_status fail(sl_hjb *h, sl_status st, const std::string &msg) {
  if (h) {
    if (h->sticky == SL_OK) h->sticky = st;
    h->err = msg;
  }
  return st;
}

#define CK(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(h, SL_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
  } while (0)

template <typename T>
sl_status dalloc(sl_hjb *h, T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
  if (e != cudaSuccess) return fail(h, SL_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  h->allocs.push_back(*p);
  e = cudaMemset(*p, 0, count * sizeof(T));
  if (e != cudaSuccess) return fail(h, SL_ECUDA, std::string("cudaMemset: ") + cudaGetErrorString(e));
  return SL_OK;
}

#define AL(ptr, count)                             \
  do {                                             \
    sl_status s_ = dalloc(h, &(ptr), (count));     \
    if (s_ != SL_OK) return s_;                    \
  } while (0)

template <typename T>
sl_status upload(sl_hjb *h, T **p, const std::vector<T> &v) {
  AL(*p, v.size());
  if (!v.empty()) CK(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SL_OK;
}

#define UP(ptr, vec)                               \
  do {                                             \
    sl_status s_ = upload(h, &(ptr), (vec));       \
    if (s_ != SL_OK) return s_;                    \
  } while (0)

double tau_eval(int kind, double rate, double t) {
  if (kind == SL_TAU_ONE) return 1.0;
  if (kind == SL_TAU_EXP) return std::exp(rate * t);
  return t;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

size_t NN(const sl_hjb *h, int l) { return size_t(h->cl[l].n) * h->cl[l].n; }

// First level run by the single-block V-cycle tail (0: none), from opts.coarse_tail_rows.
void set_tail(sl_hjb *h) {
  h->tail_l0 = 0;
  const int tail_rows = h->o.coarse_tail_rows >= 0 ? h->o.coarse_tail_rows : (h->o.precision == 0 ? 0 : 1024);
  for (int l = 1; l < h->L - 1 && tail_rows > 0; ++l)
    if (h->cl[l].m * h->cl[l].m <= tail_rows) {
      h->tail_l0 = l;
      break;
    }
}

// Drops every captured graph (they hold launch shapes and the V-cycle's structure).
void drop_graphs(sl_hjb *h) {
  for (auto &g : h->graph)
    if (g.exec) { cudaGraphExecDestroy(g.exec); g = IterGraph{}; }
  for (auto &g : h->graphT)
    if (g.exec) { cudaGraphExecDestroy(g.exec); g = IterGraph{}; }
  if (h->sgraph.exec) cudaGraphExecDestroy(h->sgraph.exec);
  h->sgraph = DevStepGraph{};
}

// ---------------------------------------------------------------------- per-step tables
sl_status coef(sl_hjb *h, double t, double *Xext, cudaStream_t s) {
  const size_t NNc = size_t(h->n) * h->n;
  if (h->f_cb)
    for (int mm = 0; mm < h->nf; ++mm) h->f_cb(t, &h->grid, mm, h->Gcb + mm * NNc, h->cb_user, s);
  if (h->psi_cb) h->psi_cb(t, &h->grid, 0, h->Psicb, h->cb_user, s);
  if (h->f_cb || h->psi_cb) CK(cudaGetLastError());
  std::vector<double> tv(std::max(1, h->nq) + std::max(1, h->npsi), 0.0);
  for (int q = 0; q < h->nq; ++q) tv[q] = tau_eval(h->tau_kind[q], h->tau_rate[q], t);
  for (int q = 0; q < h->npsi; ++q) tv[h->nq + q] = tau_eval(h->psi_kind[q], h->psi_rate[q], t);
  CK(cudaMemcpyAsync(h->d_tau, tv.data(), tv.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  // the copy source is a host temporary: make sure it has been consumed
  CK(cudaStreamSynchronize(s));
  launch_coef(h->G, h->nf, h->nq, h->d_tau, h->Psi, h->npsi, h->d_tau + h->nq, h->n, h->F, h->F32,
              Xext, h->Xb, s);
  CK(cudaGetLastError());
  return SL_OK;
}

// ---------------------------------------------------------------------- argmin
// Arguments of the policy improvement on Xext (psi on the boundary) for the handle's tables.
ArgminArgs argmin_args(sl_hjb *h, const double *Xext, bool skip = false) {
  ArgminArgs a{};
  a.tab = h->tab;
  a.slin = h->d_slin;
  a.off = h->d_off;
  a.X = Xext;
  a.F = h->F;
  a.F32 = h->F32;
  a.phi = h->d_phi;
  a.phi32 = h->d_phi32;
  a.phimax = h->d_phimax;
  a.nf = h->nf;
  a.tie_rel = h->o.tie_rel;
  a.cmax = 0.0;
  for (double c : h->cvec) a.cmax = std::max(a.cmax, std::fabs(c));
  a.tie2_32 = float(a.tie_rel) * 2.0f;
  a.cmax32 = float(a.cmax);
  for (int mm = 0; mm < 4; ++mm) a.phimax32[mm] = mm < h->nf ? float(h->phimax[mm]) : 0.f;
  a.Wmax_class = h->d_Wmaxc;
  a.policy = h->policy;
  a.changes = h->d_changes;
  a.flags = h->d_flags;
  a.halo = h->halo;
  a.SW = h->SW;
  a.SH = h->SH;
  a.screen = h->o.argmin_screen;
  // decisions that cannot change are skipped inside a step (the paired screen only: it is the
  // kernel that records the margins)
  const bool paired = a.screen && h->tab.tmax == 12 && h->itaps && h->itaps->n > 0;
  a.gap = paired ? h->d_gap : nullptr;
  a.skip_flag = (paired && skip && h->o.argmin_skip == 1) ? &h->ctl->skip_ok : nullptr;
  a.Xprev = h->Xpi;
  a.Wabs = h->Wabs;
  return a;
}

sl_status improve(sl_hjb *h, const double *Xext, long long *changes, cudaStream_t s, bool skip = false) {
  if (h->general) {
    CK(cudaMemsetAsync(h->d_changes, 0, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(h->d_flags, 0, sizeof(int), s));
    launch_argmin_general(h->gen, h->dtab, h->dtab.c64, Xext, h->F, h->d_phi, h->nf, h->o.tie_rel,
                          h->policy, h->d_changes, h->d_flags, s);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->h_changes, h->d_changes, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->h_flags, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (*h->h_flags & 1) return fail(h, SL_ENAN, "non-finite control value in the policy improvement");
    if (changes) *changes = (long long)*h->h_changes;
    h->have_policy = true;
    return SL_OK;
  }
  const ArgminArgs a = argmin_args(h, Xext, skip);
  CK(cudaMemsetAsync(h->d_changes, 0, sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(h->d_flags, 0, sizeof(int), s));
  CK(launch_argmin(a, *h->itaps, s));
  CK(cudaMemcpyAsync(h->h_changes, h->d_changes, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->h_flags, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (*h->h_flags & 1) return fail(h, SL_ENAN, "non-finite control value in the policy improvement");
  if (changes) *changes = (long long)*h->h_changes;
  h->have_policy = true;
  return SL_OK;
}

// ---------------------------------------------------------------------- hierarchy
template <typename T>
CoarseLev<T> lev_view(sl_hjb *h, int l) {
  CoarseBuf &c = h->cl[l];
  CoarseLev<T> L{};
  L.n = c.n;
  L.m = c.m;
  L.R = c.R;
  L.win = c.win;
  L.cls = c.cls;
  L.clin = c.clin;
  L.coff = c.coff;
  L.cpk32 = c.cpk32;
  L.cpk64 = c.cpk64;
  L.cw = pick<T>(c.cw64, c.cw32);
  L.cnt = c.cnt;
  L.cdiag = pick<T>(c.cdiag64, c.cdiag32);
  L.ctmax = c.ctmax;
  L.nk = h->K;
  L.ewin = pick<T>(c.ewin64, c.ewin32);
  L.erow = c.erow;
  L.cap = c.cap;
  return L;
}

// Translation-invariant class stencils S_k^l (host, FP64), rebuilt when dt changes.
sl_status build_class_tables(sl_hjb *h, double dt) {
  const bool interior_exists = !h->general && (h->n - 1 >= 2 * h->ft.B);
  std::vector<std::vector<double>> prev(h->K);
  int Rprev = h->ft.R0;
  if (interior_exists)
    for (int k = 0; k < h->K; ++k) prev[k] = fine_interior_window(h->ft, k, dt);
  for (int l = 1; l < h->L; ++l) {
    CoarseBuf &c = h->cl[l];
    std::vector<std::vector<double>> cur(h->K);
    std::vector<int32_t> lin, off;
    std::vector<double> w, diag(h->K, 1.0);
    std::vector<int> cnt(h->K, 0);
    int ctmax = 1;
    std::vector<std::vector<std::pair<int, double>>> taps(h->K);
    const int Wd = 2 * c.R + 1;
    for (int k = 0; k < h->K; ++k) {
      if (!interior_exists) break;
      cur[k] = rap_class_window(prev[k], Rprev, c.R);
      for (int e = 0; e < Wd * Wd; ++e) {
        const double v = cur[k][e];
        if (v == 0.0) continue;
        taps[k].push_back({e, v});
        if (e == c.R * Wd + c.R) diag[k] = v;
      }
      ctmax = std::max(ctmax, int(taps[k].size()));
    }
    lin.assign(size_t(h->K) * ctmax, 0);
    off.assign(size_t(h->K) * ctmax, 0);
    w.assign(size_t(h->K) * ctmax, 0.0);
    for (int k = 0; k < h->K; ++k) {
      cnt[k] = int(taps[k].size());
      for (size_t t = 0; t < taps[k].size(); ++t) {
        const int e = taps[k][t].first;
        const int dy = e / Wd - c.R, dx = e % Wd - c.R;
        lin[size_t(k) * ctmax + t] = dy * c.n + dx;
        off[size_t(k) * ctmax + t] = (dy << 16) | (dx & 0xffff);
        w[size_t(k) * ctmax + t] = taps[k][t].second;
      }
    }
    if (c.ctmax < ctmax) {
      // (re)allocate: sizes only grow
      AL(c.clin, size_t(h->K) * ctmax);
      AL(c.coff, size_t(h->K) * ctmax);
      AL(c.cw64, size_t(h->K) * ctmax);
      AL(c.cw32, size_t(h->K) * ctmax);
      AL(c.cpk32, size_t(h->K) * ctmax);
      AL(c.cpk64, size_t(h->K) * ctmax);
    }
    {
      const int SWl = coarse_pitch(c.R);
      std::vector<int2> p32(size_t(h->K) * ctmax, make_int2(0, 0));
      std::vector<longlong2> p64(size_t(h->K) * ctmax);
      for (size_t i = 0; i < p64.size(); ++i) { p64[i].x = 0; p64[i].y = 0; }
      for (int k = 0; k < h->K; ++k)
        for (size_t t = 0; t < taps[k].size(); ++t) {
          const int e = taps[k][t].first;
          const int dy = e / Wd - c.R, dx = e % Wd - c.R;
          const size_t ix = size_t(k) * ctmax + t;
          const float w32 = float(taps[k][t].second);
          int wb;
          std::memcpy(&wb, &w32, sizeof(int));
          p32[ix] = make_int2(dy * SWl + dx, wb);
          long long wb64;
          std::memcpy(&wb64, &taps[k][t].second, sizeof(long long));
          p64[ix].x = dy * SWl + dx;
          p64[ix].y = wb64;
        }
      CK(cudaMemcpy(c.cpk32, p32.data(), p32.size() * sizeof(int2), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(c.cpk64, p64.data(), p64.size() * sizeof(longlong2), cudaMemcpyHostToDevice));
    }
    if (!c.cnt) {
      AL(c.cnt, size_t(h->K));
      AL(c.cdiag64, size_t(h->K));
      AL(c.cdiag32, size_t(h->K));
      AL(c.cdense64, size_t(h->K) * c.win);
      AL(c.cdense32, size_t(h->K) * c.win);
    }
    {
      // dense class windows (read by the transposed coarse rows of the adjoint)
      std::vector<double> dn(size_t(h->K) * c.win, 0.0);
      for (int k = 0; k < h->K && interior_exists; ++k)
        std::copy(cur[k].begin(), cur[k].end(), dn.begin() + size_t(k) * c.win);
      std::vector<float> dn32(dn.begin(), dn.end());
      CK(cudaMemcpy(c.cdense64, dn.data(), dn.size() * sizeof(double), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(c.cdense32, dn32.data(), dn32.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    c.ctmax = ctmax;
    std::vector<float> w32(w.begin(), w.end()), d32(diag.begin(), diag.end());
    CK(cudaMemcpy(c.clin, lin.data(), lin.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c.coff, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c.cw64, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c.cw32, w32.data(), w32.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c.cnt, cnt.data(), cnt.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c.cdiag64, diag.data(), diag.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c.cdiag32, d32.data(), d32.size() * sizeof(float), cudaMemcpyHostToDevice));
    c.cnt_host = cnt;
    c.coff_host = off;
    prev.swap(cur);
    Rprev = c.R;
  }
  h->class_valid = true;
  h->class_dt = dt;
  return SL_OK;
}

void tail_pack(sl_hjb *h, cudaStream_t s);

template <typename T>
sl_status build_hierarchy_T(sl_hjb *h, double dt, cudaStream_t s) {
  for (int l = 1; l < h->L; ++l) {
    CoarseBuf &c = h->cl[l];
    CoarseBuf &p = h->cl[l - 1];
    launch_classify(l, h->tab, h->policy, p.cls, p.n, c.cls, c.n, c.erow, c.d_nexpl, h->chunk_scratch, s);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->h_count, c.d_nexpl, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    c.nexpl = *h->h_count;
    CoarseLev<T> prevv = lev_view<T>(h, l - 1), curv = lev_view<T>(h, l);
    CK(launch_rap_explicit<T>(l, h->tab, h->d_off, h->policy, T(dt), prevv, p.coff, curv, c.nexpl,
                              pick<T>(c.ewin64, c.ewin32), s));
  }
  const int lc = h->L - 1;
  CoarseLev<T> cv = lev_view<T>(h, lc);
  launch_coarsest_setup<T>(lc, h->tab, h->policy, T(dt), cv, lc == 0 ? h->d_off : h->cl[lc].coff,
                           h->cwork, pick<T>(h->Ainv64, h->Ainv32), s);
  tail_pack(h, s);
  CK(cudaGetLastError());
  return SL_OK;
}

// Host-built class stencils and the fine Jacobi scales for step size dt (when dt changes).
sl_status ensure_class_tables(sl_hjb *h, double dt, cudaStream_t s) {
  if (h->class_valid && h->class_dt == dt) return SL_OK;
  sl_status st = build_class_tables(h, dt);
  if (st != SL_OK) return st;
  if (!h->general) launch_fine_od(h->tab, dt, h->o.omega, h->d_od64, h->d_od32, h->d_iod64, h->d_iod32, s);
  CK(cudaGetLastError());
  return SL_OK;
}

sl_status build_hierarchy(sl_hjb *h, double dt, cudaStream_t s) {
  if (h->general) {  // the fine rows of the current policy and step size
    launch_assemble_general(h->gen, h->dtab, h->policy, h->dtab.c64, dt, h->o.omega, h->SW, h->gout, s);
    CK(cudaGetLastError());
  }
  if (h->o.precond == 1) {  // aggregation AMG on the assembled step matrix
    cudaError_t e = amg_level0_from_tables(h->amg, h->tab, h->d_off, h->policy, dt, s);
    if (e == cudaSuccess) e = amg_setup(h->amg, s);
    if (e != cudaSuccess)
      return fail(h, e == cudaErrorInvalidValue && !h->amg.err_msg.empty() ? SL_EINVAL : SL_ECUDA,
                  h->amg.err_msg.empty() ? std::string("AMG setup: ") + cudaGetErrorString(e) : h->amg.err_msg);
    h->hier_valid = true;
    h->hier_dt = dt;
    h->changes_since_build = 0;
    // level sizes and buffers may have changed: captured iterations must be captured again
    ++h->amg_gen;
    return SL_OK;
  }
  sl_status st = ensure_class_tables(h, dt, s);
  if (st != SL_OK) return st;
  st = (h->o.precision == 0) ? build_hierarchy_T<double>(h, dt, s)
                                       : build_hierarchy_T<float>(h, dt, s);
  if (st != SL_OK) return st;
  h->hier_valid = true;
  h->hier_dt = dt;
  h->changes_since_build = 0;
  return SL_OK;
}

// ---------------------------------------------------------------------- V-cycle
template <typename T>
CsrTView<T> csrT_view(sl_hjb *h) {
  CsrTView<T> A{};
  A.n = h->n;
  A.m = h->m;
  A.rowptr = h->t_rowptr;
  A.col = h->t_col;
  A.v = pick<T>(h->t_v64, h->t_v32);
  A.d = pick<T>(h->t_d64, h->t_d32);
  return A;
}

template <typename T>
void level_op(sl_hjb *h, int l, int op, double dt, const T *x, const T *b, T *y, cudaStream_t s,
              int color = -1) {
  if (h->transposed) {
    if (l == 0)
      launch_fineT_op<T>(op, csrT_view<T>(h), T(h->o.omega), x, b, y, s);
    else
      launch_denseT_op<T>(op, h->cl[l].n, h->cl[l].R, pick<T>(h->cl[l].WT64, h->cl[l].WT32),
                          T(h->o.omega), x, b, y, s);
    return;
  }
  if (l == 0)
    launch_fine_op<T>(op, h->tab, h->d_slin, h->policy, T(dt), T(h->o.omega), x, b, y, h->halo, h->SW, s,
                      color);
  else
    launch_coarse_op<T>(op, lev_view<T>(h, l), h->cl[l].d_nexpl, T(h->o.omega), x, b, y, s, color);
}

// `sweeps` sweeps of the level-l smoother on A_l x = b, ping-ponging between cur and other
// (from_zero: the first sweep starts at x = 0 and writes cur).  Damped Jacobi, or with
// smoother 1 the two-colour Gauss-Seidel sweep (Section 3.3's Gauss-Seidel in data-parallel
// form): rows with i1 + i2 even, then odd, each half updated from the current values.  The
// transposed solves of the adjoint smooth with Jacobi.
template <typename T>
void smooth(sl_hjb *h, int l, double dt, const T *b, T *&cur, T *&other, int sweeps, bool from_zero,
            cudaStream_t s) {
  const bool gs = h->o.smoother == 1 && !h->transposed;
  for (int it = 0; it < sweeps; ++it) {
    if (gs) {
      for (int c = 0; c < 2; ++c) {
        if (from_zero && it == 0 && c == 0) {
          level_op<T>(h, l, OP_JACOBI0, dt, nullptr, b, cur, s, 0);
        } else {
          level_op<T>(h, l, OP_JACOBI, dt, cur, b, other, s, c);
          std::swap(cur, other);
        }
      }
    } else if (from_zero && it == 0) {
      level_op<T>(h, l, OP_JACOBI0, dt, nullptr, b, cur, s);
    } else {
      level_op<T>(h, l, OP_JACOBI, dt, cur, b, other, s);
      std::swap(cur, other);
    }
  }
}

// Number of times smooth() exchanges its two buffers over one V-cycle level: every sweep (or
// half-sweep) that reads one buffer and writes the other.  A cycle that starts its
// pre-smoothing in the work buffer when this is odd ends its post-smoothing in x, with no copy.
inline int smooth_swaps(const sl_hjb *h) {
  const int per = (h->o.smoother == 1 && !h->transposed) ? 2 : 1;
  const int pre = h->o.nu1 > 0 ? per * h->o.nu1 - 1 : 0;
  return pre + per * h->o.nu2;
}

template <typename T>
void vbufs(VBuf &v, T **x, T **t, T **r, T **b);
template <>
void vbufs<double>(VBuf &v, double **x, double **t, double **r, double **b) {
  *x = v.x64; *t = v.t64; *r = v.r64; *b = v.b64;
}
template <>
void vbufs<float>(VBuf &v, float **x, float **t, float **r, float **b) {
  *x = v.x32; *t = v.t32; *r = v.r32; *b = v.b32;
}

// The arguments of the single-block V-cycle tail from level l0 = h->tail_l0 down.
template <typename T>
TailArgs<T> tail_args(sl_hjb *h) {
  TailArgs<T> a{};
  const int l = h->tail_l0;
  a.l0 = l;
  a.L = h->L;
  a.nu1 = h->o.nu1;
  a.nu2 = h->o.nu2;
  a.rbgs = h->o.smoother == 1 ? 1 : 0;
  a.omega = T(h->o.omega);
  for (int q = l; q < h->L; ++q) {
    a.lev[q] = lev_view<T>(h, q);
    vbufs<T>(h->vb[q], &a.x[q], &a.t[q], &a.r[q], &a.b[q]);
  }
  a.Ainv = pick<T>(h->Ainv64, h->Ainv32);
  a.img = h->tail_img_bytes ? reinterpret_cast<const T *>(h->tail_img) : nullptr;
  return a;
}

// Packs the tail levels' stencils of the current hierarchy for the shared-memory tail; every
// path that builds the hierarchy calls this at its end.
void tail_pack(sl_hjb *h, cudaStream_t s) {
  // before the first hierarchy the class tables do not exist yet: nothing to pack
  if (h->tail_l0 <= 0 || h->tail_img_bytes == 0 || !h->class_valid) return;
  if (h->o.precision == 0) launch_tail_pack<double>(tail_args<double>(h), reinterpret_cast<double *>(h->tail_img), s);
  else launch_tail_pack<float>(tail_args<float>(h), reinterpret_cast<float *>(h->tail_img), s);
}

// Room for the packed tail stencils (sizes only grow); none when the tail's levels do not fit in
// one block's shared memory.
sl_status alloc_tail_image(sl_hjb *h) {
  h->tail_img_bytes = 0;
  if (h->tail_l0 <= 0) return SL_OK;
  const size_t need = h->o.precision == 0 ? tail_image_bytes<double>(tail_args<double>(h))
                                          : tail_image_bytes<float>(tail_args<float>(h));
  if (need == 0) return SL_OK;
  if (need > h->tail_img_cap) {
    AL(h->tail_img, need);
    h->tail_img_cap = need;
  }
  h->tail_img_bytes = need;
  return SL_OK;
}

// x = M_l^{-1} b: V(nu1, nu2) from a zero initial guess, exact solve on the coarsest level.
template <typename T>
sl_status vcycle(sl_hjb *h, int l, double dt, const T *b, T *x, cudaStream_t s) {
  const size_t N = NN(h, l);
  if (l > 0 && l == h->tail_l0 && l < h->L - 1 && !h->transposed) {
    // coarse end of the cycle in one thread block; b and x are this level's own buffers
    const TailArgs<T> a = tail_args<T>(h);
    if (b != a.b[l] || x != a.x[l]) return fail(h, SL_EINVAL, "V-cycle tail called on foreign buffers");
    launch_vcycle_tail<T>(a, s);
    CK(cudaGetLastError());
    return SL_OK;
  }
  if (l == h->L - 1) {
    launch_coarsest_apply<T>(pick<T>(h->Ainv64, h->Ainv32), h->cl[l].n, b, x, s, h->transposed ? 1 : 0);
    return SL_OK;
  }
  T *bx, *bt, *br, *bb;
  vbufs<T>(h->vb[l], &bx, &bt, &br, &bb);
  // the buffer the pre-smoothing starts in is chosen so that the last sweep writes x; bt's
  // boundary entries are zero (no operator writes a boundary entry), as x's must be
  T *cur = x, *other = bt;
  if (smooth_swaps(h) & 1) std::swap(cur, other);
  T *cx, *ct, *cr, *cb;
  vbufs<T>(h->vb[l + 1], &cx, &ct, &cr, &cb);
  const int nc = h->cl[l + 1].n;
  // coarse levels with the Jacobi smoother: two fused passes (sl_opts.coarse_fusion)
  const bool fused = l > 0 && h->o.coarse_fusion > 0 && l >= h->o.coarse_fusion && h->o.smoother == 0 &&
                     !h->transposed && h->o.nu1 >= 1 && h->o.nu2 >= 1;
  if (fused) {
    const CoarseLev<T> L = lev_view<T>(h, l);
    if (h->o.nu1 == 1) {
      launch_coarse_down<T>(L, T(h->o.omega), b, nullptr, cur, cb, nc, s);
    } else {
      smooth<T>(h, l, dt, b, cur, other, h->o.nu1, true, s);
      launch_coarse_down<T>(L, T(h->o.omega), b, cur, nullptr, cb, nc, s);
    }
    sl_status st = vcycle<T>(h, l + 1, dt, cb, cx, s);
    if (st != SL_OK) return st;
    launch_coarse_up<T>(L, T(h->o.omega), b, cur, cx, nc, other, s);
    std::swap(cur, other);
    smooth<T>(h, l, dt, b, cur, other, h->o.nu2 - 1, false, s);
    if (cur != x) CK(cudaMemcpyAsync(x, cur, N * sizeof(T), cudaMemcpyDeviceToDevice, s));
    CK(cudaGetLastError());
    return SL_OK;
  }
  if (h->o.nu1 == 0) launch_fill<T>(cur, N, T(0), s);
  else smooth<T>(h, l, dt, b, cur, other, h->o.nu1, true, s);
  level_op<T>(h, l, OP_RESID, dt, cur, b, br, s);
  launch_restrict<T>(br, h->cl[l].n, cb, nc, s);
  sl_status st = vcycle<T>(h, l + 1, dt, cb, cx, s);
  if (st != SL_OK) return st;
  launch_prolong_add<T>(cx, nc, cur, h->cl[l].n, s);
  smooth<T>(h, l, dt, b, cur, other, h->o.nu2, false, s);
  if (cur != x) CK(cudaMemcpyAsync(x, cur, N * sizeof(T), cudaMemcpyDeviceToDevice, s));
  CK(cudaGetLastError());
  return SL_OK;
}

// x = M^{-1} b on the finest level: the V-cycle, or the aggregation K-cycle (precond 1) on the
// interior unknowns gathered from b and scattered back into x.
template <typename T>
sl_status precond(sl_hjb *h, double dt, const T *b, T *x, cudaStream_t s) {
  if (h->o.precond == 1) {
    AmgLevel &L0 = h->amg.lev[0];
    T *cb = pick<T>(L0.vec64[AV_B], L0.vec32[AV_B]), *cx = pick<T>(L0.vec64[AV_X], L0.vec32[AV_X]);
    amg_full_to_compact<T>(h->n, b, cb, s);
    amg_cycle<T>(h->amg, cb, cx, s);
    amg_compact_to_full<T>(h->n, cx, x, s);
    CK(cudaGetLastError());
    return SL_OK;
  }
  return vcycle<T>(h, 0, dt, b, x, s);
}

// ---------------------------------------------------------------------- BiCGSTAB
// Right-preconditioned BiCGSTAB for A e = r0 with x += e accumulated in place (x may be FP64
// while the Krylov vectors are FP32: TX / T).  On entry r holds the initial residual and S
// carries ||b||^2 and the stop threshold (tol ||b||)^2.  Returns SL_OK on convergence,
// SL_ENOCONV_KRYLOV at the cap, SL_EBREAKDOWN, or SL_ENAN; only SL_ENAN is recorded as an error.
// The work of one BiCGSTAB iteration (no host synchronisation inside).
template <typename T, typename TX>
sl_status issue_iteration(sl_hjb *h, double dt, TX *x, T *r, T *rh, T *p, T *v, T *sv, T *t, T *ph,
                          T *sh, BicgScalars *S, cudaStream_t s) {
  const size_t N = NN(h, 0);
  launch_bicg_p<T>(p, r, v, N, 0, S, s);
  sl_status st = precond<T>(h, dt, p, ph, s);
  if (st != SL_OK) return st;
  level_op<T>(h, 0, OP_APPLY, dt, ph, nullptr, v, s);
  launch_dot2<T>(rh, v, nullptr, nullptr, N, POST_ALPHA, S, h->partials, h->counter, s);
  launch_bicg_s<T>(sv, r, v, N, S, h->partials, h->counter, s);
  st = precond<T>(h, dt, sv, sh, s);
  if (st != SL_OK) return st;
  level_op<T>(h, 0, OP_APPLY, dt, sh, nullptr, t, s);
  launch_dot2<T>(t, sv, t, t, N, POST_OMEGA, S, h->partials, h->counter, s);
  launch_bicg_xr<T, TX>(x, ph, sh, sv, t, r, rh, N, S, h->partials, h->counter, s);
  CK(cudaGetLastError());
  return SL_OK;
}

// Captures one iteration into a CUDA graph (once per precision and step size: pointers,
// launch shapes and dt are fixed; counts and scalars live in device memory).
template <typename T, typename TX>
sl_status ensure_graph(sl_hjb *h, int prec, double dt, TX *x, T *r, T *rh, T *p, T *v, T *sv, T *t,
                       T *ph, T *sh, BicgScalars *S) {
  IterGraph &g = h->transposed ? h->graphT[prec] : h->graph[prec];
  // the V-cycle's buffers and launch shapes are fixed at create; the AMG ones are not
  if (g.exec && g.dt == dt && (h->o.precond == 0 || g.gen == h->amg_gen)) return SL_OK;
  if (g.exec) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
  }
  if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  const long long before = thread_launch_count();  // other threads may launch meanwhile
  CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  sl_status st = issue_iteration<T, TX>(h, dt, x, r, rh, p, v, sv, t, ph, sh, S, h->cap_stream);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
  if (st != SL_OK) return st;
  CK(e);
  g.kernels = thread_launch_count() - before;
  note_launch(int(-g.kernels));  // captured, not executed
  e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  CK(e);
  g.dt = dt;
  g.gen = h->amg_gen;
  return SL_OK;
}

// Right-preconditioned BiCGSTAB for A e = r0 with x += e accumulated in place (x may be FP64
// while the Krylov vectors are FP32: TX / T).  On entry r holds the initial residual and S
// carries ||b||^2 and the stop threshold (tol ||b||)^2.  Returns SL_OK on convergence,
// SL_ENOCONV_KRYLOV at the cap, SL_EBREAKDOWN, or SL_ENAN; only SL_ENAN is recorded as an error.
// Each iteration is one CUDA-graph launch followed by a read of the residual norm.
template <typename T, typename TX>
sl_status bicgstab(sl_hjb *h, double dt, TX *x, T *r, T *rh, T *p, T *v, T *sv, T *t, T *ph, T *sh,
                   BicgScalars *S, int maxit, int *iters, cudaStream_t s) {
  const size_t N = NN(h, 0);
  const int prec = sizeof(T) == 8 ? 0 : 1;
  if (h->o.use_graphs) {
    sl_status st = ensure_graph<T, TX>(h, prec, dt, x, r, rh, p, v, sv, t, ph, sh, S);
    if (st != SL_OK) return st;
  }
  CK(cudaMemcpyAsync(rh, r, N * sizeof(T), cudaMemcpyDeviceToDevice, s));
  launch_dot2<T>(r, r, r, r, N, POST_RHO_INIT, S, h->partials, h->counter, s);
  *iters = 0;
  for (int it = 1; it <= maxit; ++it) {
    if (h->o.use_graphs) {
      IterGraph &g = h->transposed ? h->graphT[prec] : h->graph[prec];
      CK(cudaGraphLaunch(g.exec, s));
      note_launch(int(g.kernels));
    } else {
      sl_status st = issue_iteration<T, TX>(h, dt, x, r, rh, p, v, sv, t, ph, sh, S, s);
      if (st != SL_OK) return st;
    }
    CK(cudaMemcpyAsync(h->hS, S, sizeof(BicgScalars), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *iters = it;
    const BicgScalars &hs = *h->hS;
    if (hs.nonfinite) return fail(h, SL_ENAN, "non-finite value in BiCGSTAB");
    if (hs.rr <= hs.tol2) return SL_OK;
    if (hs.breakdown) return SL_EBREAKDOWN;
  }
  return SL_ENOCONV_KRYLOV;
}

// True FP64 residual of the step system at h->X into `r`, with ||r||_2^2, ||r||_inf and the
// matching norms of F.
struct ResNorms {
  double rr, rmax, bn2, bmax;
};

sl_status true_residual(sl_hjb *h, double dt, double tolk, double *r, ResNorms *nr, cudaStream_t s) {
  const size_t N = NN(h, 0);
  if (h->transposed)  // backward solve A^T mu = lambda
    launch_fineT_op<double>(OP_RESID, csrT_view<double>(h), h->o.omega, h->mu, h->lam, r, s);
  else
    launch_hjb_resid(h->tab, h->policy, h->X, h->Uprev, h->F, h->d_phi, h->nf, dt, r, h->halo, h->SW, s,
                     0, nullptr, h->Ub);
  // ||F|| (or ||lambda||) was taken once by linear_solve before its first round, which also
  // left U^{n-1} + dt f of this policy in h->Ub
  launch_init_scalars_keep_b(h->S, tolk * tolk, s);
  launch_norms(r, N, 1, h->S, h->partials, h->counter, s);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h->hS, h->S, sizeof(BicgScalars), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  nr->bn2 = h->hS->bnorm2;
  nr->bmax = h->hS->bmax;
  nr->rr = h->hS->rr;
  nr->rmax = h->hS->rmax;
  if (h->hS->nonfinite || !std::isfinite(nr->rr)) return fail(h, SL_ENAN, "non-finite residual");
  return SL_OK;
}

// Solves A^alpha X = F^alpha at the current policy from the iterate h->X (psi on the boundary).
// Stop test on the true FP64 residual r = F - A X:
//   ||r||_2 <= krylov_tol ||F||_2  and  ||r||_inf <= krylov_tol ||F||_inf.
// A^alpha is an M-matrix with row sums >= 1 - dt c (Section 3.4), so for c = 0 the max-norm
// test bounds the error of the step: ||X - X*||_inf <= ||r||_inf.  When the Krylov recurrence
// meets the 2-norm test but the true max-norm test fails, the inner threshold is tightened
// tenfold and BiCGSTAB restarts from the true residual.  In mixed precision each round is an
// FP32 inner solve of A e = r followed by X += e in FP64; r is the true residual, or, while
// ir_next_recursive() allows it, the previous inner solve's own residual r - A e, so that the
// true residual (and the stop test on it) is formed only once the solve may have converged.
//
// With h->transposed set, the same loop solves the backward system A^T mu = lambda of the
// adjoint (h->mu from its initial value, right-hand side h->lam).
sl_status linear_solve(sl_hjb *h, double dt, sl_stats *st, cudaStream_t s) {
  const size_t N = NN(h, 0);
  // ||F||: the residual at X = (0 inside, psi on the boundary) is F itself
  if (!h->transposed)  // Xb vanishes inside: rows beyond the stencil reach need no taps
    launch_hjb_resid(h->tab, h->policy, h->Xb, h->Uprev, h->F, h->d_phi, h->nf, dt, h->Fvec, h->halo,
                     h->SW, s, std::max(1, h->cl[0].R), h->Ub);
  CK(cudaGetLastError());
  // the right-hand side's norms, once per solve (every round keeps them in S)
  launch_init_scalars(h->S, 0.0, s);
  launch_norms(h->transposed ? h->lam : h->Fvec, N, 0, h->S, h->partials, h->counter, s);
  double *X = h->transposed ? h->mu : h->X;
  KBuf &k = h->kb;
  const double tol = h->ls_tol > 0.0 ? h->ls_tol : h->o.krylov_tol;
  double tolk = tol;   // threshold handed to BiCGSTAB's recurrence
  int total = 0;
  const bool fp64 = h->o.precision == 0;
  const int rounds = fp64 ? 12 : h->o.ir_max + 1;
  bool need_true = true;  // mixed: this round starts from a true residual (ir_next_recursive)
  int rec_rounds = 0;
  // The backward solves of the adjoint (A^T mu = lambda) took 40 % more Krylov iterations with
  // rounds on the inner residual (1,797 against 1,285 over a 64-step backward pass at 1025^2):
  // their rounds always start from the true residual.
  const int max_rec = h->transposed ? 0 : h->o.ir_recursive;
  double bn2 = 0.0;       // ||F||_2^2 of the solve
  double rr_true = 0.0;   // ||r||_2^2 of the last true residual
  for (int round = 0; round < rounds; ++round) {
    sl_status r = SL_OK;
    if (need_true) {
      ResNorms nr{};
      double *r64 = fp64 ? k.r64 : h->R;
      r = true_residual(h, dt, tolk, r64, &nr, s);
      if (r != SL_OK) return r;
      bn2 = nr.bn2;
      rr_true = nr.rr;
      const double rel2 = nr.bn2 > 0 ? std::sqrt(nr.rr / nr.bn2) : std::sqrt(nr.rr);
      if (st) st->res_final = rel2;
      const bool ok2 = nr.rr <= tol * tol * nr.bn2;
      const bool okinf = nr.rmax <= tol * nr.bmax;
      if (ok2 && okinf) return SL_OK;
      if (ok2 && !okinf) tolk *= 0.1;
      if (fp64 && total >= h->o.kry_max) break;
    }
    int it = 0;
    if (fp64) {
      // BiCGSTAB on the true residual; S holds ||F||_2 and the threshold (tolk ||F||_2)^2
      r = bicgstab<double, double>(h, dt, X, k.r64, k.rh64, k.p64, k.v64, k.s64, k.t64, k.ph64,
                                   k.sh64, h->S, h->o.kry_max - total, &it, s);
    } else {
      // refinement: FP32 inner solve of A e = fp32(r) from e = 0, then X += e in FP64; r is the
      // true residual, or the previous inner solve's own residual r - A e (left in k.r32)
      if (st) st->ir_iters += 1;
      if (need_true) launch_convert<double, float>(h->R, k.r32, N, s);
      launch_fill<float>(k.e32, N, 0.0f, s);
      launch_init_scalars(h->S32, h->o.inner_tol * h->o.inner_tol, s);
      launch_dot2<float>(k.r32, k.r32, nullptr, nullptr, N, POST_BNORM, h->S32, h->partials, h->counter, s);
      r = bicgstab<float, float>(h, dt, k.e32, k.r32, k.rh32, k.p32, k.v32, k.s32, k.t32, k.ph32,
                                 k.sh32, h->S32, h->o.kry_max, &it, s);
      launch_add_f32_to_f64(X, k.e32, N, s);
      CK(cudaGetLastError());
      // bicgstab() left the inner solve's last scalars (S32) in h->hS
      const bool rec = (r == SL_OK || r == SL_ENOCONV_KRYLOV) &&
                       ir_next_recursive(h->hS->rr, tol, bn2, rr_true, rec_rounds, max_rec);
      need_true = !rec;
      rec_rounds = rec ? rec_rounds + 1 : 0;
    }
    total += it;
    if (st) st->krylov_iters += it;
    if (r == SL_ENAN) return r;
    if (r != SL_OK && r != SL_ENOCONV_KRYLOV && r != SL_EBREAKDOWN) return r;
    if (fp64 && r == SL_ENOCONV_KRYLOV) break;
  }
  return fail(h, SL_ENOCONV_KRYLOV, fp64 ? "BiCGSTAB reached its iteration cap"
                                         : "iterative refinement reached ir_max");
}

// ---------------------------------------------------------------------- one step
sl_status step_impl(sl_hjb *h, double *u, double t, double dt, uint8_t *pol_out, sl_stats *st,
                    cudaStream_t s) {
  if (!(dt > 0)) return fail(h, SL_EINVAL, "dt must be positive");
  for (double c : h->cvec)
    if (dt * c > 1.0) return fail(h, SL_ECFL, "dt * c > 1 violates the positivity condition");
  const size_t N = NN(h, 0);
  double t0 = now_ms();
  // consecutive equal steps continue the march: U^{n-2} is the previous step's U^{n-1}
  const bool extrap = h->o.extrapolate && h->have_prev2 && h->prev_dt == dt &&
                      std::fabs(h->prev_t + dt - t) <= 1e-12 * std::max(1.0, std::fabs(t));
  if (h->o.extrapolate) {
    // keep U^{n-1} for the next step's extrapolation (Uprev still holds the previous U^{n-1})
    std::swap(h->Uprev, h->Uprev2);
  }
  CK(cudaMemcpyAsync(h->Uprev, u, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->X, u, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  sl_status r = coef(h, t, h->X, s);
  if (r != SL_OK) return r;
  CK(cudaMemsetAsync(&h->ctl->skip_ok, 0, sizeof(int), s));  // no improvement in this step yet
  const bool first_improve = !h->have_policy;
  if (first_improve) {
    long long ch = 0;
    r = improve(h, h->X, &ch, s);
    if (r != SL_OK) return r;
    h->hier_valid = false;
  }
  // Howard's stop test measures against X^0 = U^{n-1}
  CK(cudaMemcpyAsync(h->Xpi, h->X, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (extrap) {
    // first linear solve starts from 2 U^{n-1} - U^{n-2} (interior; psi(t_n) stays on the boundary)
    launch_extrapolate(h->X, h->Uprev, h->Uprev2, h->n, s);
    CK(cudaGetLastError());
  }
  if (!first_improve && h->o.howard_init == 1) {
    // the previous step's policy, improved at this step's first iterate
    long long ch = 0;
    r = improve(h, h->X, &ch, s);
    if (r != SL_OK) return r;
    h->changes_since_build += ch;
    if (st) st->policy_changes += ch;
  }
  h->have_prev2 = h->o.extrapolate != 0;
  h->prev_t = t;
  h->prev_dt = dt;
  if (st) st->steps += 1;
  for (int it = 1; it <= h->o.pi_max; ++it) {
    // a general fine level re-assembles its rows on every policy change
    const long long thresh = h->general ? 0 : (long long)(h->o.rebuild_frac * double(h->m) * h->m);
    if (!h->hier_valid || h->hier_dt != dt || h->changes_since_build > thresh) {
      double tb = now_ms();
      r = build_hierarchy(h, dt, s);
      if (r != SL_OK) return r;
      CK(cudaStreamSynchronize(s));
      if (st) {
        st->rebuilds += 1;
        st->t_hier_ms += now_ms() - tb;
        long long ex = 0;
        for (int l = 1; l < h->L; ++l) ex += h->cl[l].nexpl;
        st->explicit_rows = ex;
      }
    }
    double ts = now_ms();
    // the first solve of the iteration at howard_loose_tol when that is set
    const bool loose = h->o.howard_loose_tol > 0.0 && it == 1;
    h->ls_tol = loose ? h->o.howard_loose_tol : 0.0;
    r = linear_solve(h, dt, st, s);
    h->ls_tol = 0.0;
    if (st) st->t_solve_ms += now_ms() - ts;
    if (r != SL_OK) return r;
    if (h->rec_slot)  // the policy that defines A_n for the adjoint
      CK(cudaMemcpyAsync(h->rec_slot, h->policy, size_t(h->m) * h->m, cudaMemcpyDeviceToDevice, s));
    double ta = now_ms();
    long long ch = 0;
    // the stop test's max |X - X^{m-1}| first: the argmin's skip test reads it
    launch_maxabs_diff(h->X, h->Xpi, h->n, h->d_maxd, h->counter, h->partials, s);
    r = improve(h, h->X, &ch, s, true);
    if (r != SL_OK) return r;
    CK(cudaMemsetAsync(&h->ctl->skip_ok, 1, sizeof(int), s));  // this improvement was at X = X^m
    h->changes_since_build += ch;
    CK(cudaMemcpyAsync(h->h_maxd, h->d_maxd, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (st) {
      st->t_argmin_ms += now_ms() - ta;
      st->pi_iters += 1;
      st->policy_changes += ch;
    }
    if (!std::isfinite(h->h_maxd[0])) return fail(h, SL_ENAN, "non-finite iterate");
    const bool small = h->h_maxd[0] <= h->o.pi_tol * std::max(1.0, h->h_maxd[1]);
    if ((ch == 0 || small) && !loose) {  // a loosely solved iterate is solved again, tightly
      CK(cudaMemcpyAsync(u, h->X, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
      if (pol_out)
        CK(cudaMemcpyAsync(pol_out, h->policy, size_t(h->m) * h->m, cudaMemcpyDeviceToDevice, s));
      (void)t0;
      if (h->tab.tma) {  // a bounded wait of the TMA fine operator that gave up
        CK(cudaMemcpyAsync(&h->h_ctl->tma_err, &h->ctl->tma_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (h->h_ctl->tma_err) {
          CK(cudaMemsetAsync(&h->ctl->tma_err, 0, sizeof(int), s));
          return fail(h, SL_ETIMEOUT, "a bounded wait for the TMA tile copies of the fine operator gave up");
        }
      }
      return SL_OK;
    }
    CK(cudaMemcpyAsync(h->Xpi, h->X, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  CK(cudaMemcpyAsync(u, h->X, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return fail(h, SL_ENOCONV_PI, "Howard iteration reached pi_max");
}

// ---------------------------------------------------------------------- device-driven steps
// use_graphs 2: a step is captured once per step size as one CUDA graph whose Howard,
// refinement and BiCGSTAB loops are conditional nodes.  The graph runs the kernels of
// step_impl / linear_solve / bicgstab in the same order on the same buffers; the single-thread
// control kernels of sl_control.cu take the host loop's decisions on the device, so a step
// costs one graph launch and one read of the loop state.

cudaError_t cap_stream_at(sl_hjb *h, int depth, cudaStream_t *out) {
  if (depth < 0 || depth >= 8) return cudaErrorInvalidValue;
  if (!h->cap_pool[depth]) {
    cudaError_t e = cudaStreamCreateWithFlags(&h->cap_pool[depth], cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  *out = h->cap_pool[depth];
  return cudaSuccess;
}

// A conditional handle of the graph that stream s is capturing into.
cudaError_t new_cond_handle(cudaStream_t s, cudaGraphConditionalHandle *hd) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive || !g) return cudaErrorStreamCaptureInvalidated;
  return cudaGraphConditionalHandleCreate(hd, g, 0, 0);
}

// Captures body(stream, depth, &nested) into a new graph body; nested collects the kernels of
// deeper conditionals so that each body's own kernel count stays separate.
using BodyFn = std::function<sl_status(cudaStream_t, int, long long *)>;

// Adds a conditional node (while / if on handle hd) after the work captured so far on s,
// captures the body on the capture stream of the next depth, and orders the next work on s
// after the node.  *direct: kernels captured in the body itself; *total: with deeper bodies.
sl_status add_cond(sl_hjb *h, cudaStream_t s, int depth, cudaGraphConditionalHandle hd,
                   cudaGraphConditionalNodeType type, long long *direct, long long *total,
                   const BodyFn &body) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  const cudaGraphEdgeData *ed = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &ed, &nd));
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = hd;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  CK(cudaGraphAddNode(&node, g, deps, ed, nd, &p));
  cudaStream_t sb = nullptr;
  CK(cap_stream_at(h, depth + 1, &sb));
  CK(cudaStreamBeginCaptureToGraph(sb, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                   cudaStreamCaptureModeThreadLocal));
  const long long before = thread_launch_count();
  long long nested = 0;
  const sl_status st = body(sb, depth + 1, &nested);
  cudaGraph_t og = nullptr;
  const cudaError_t e = cudaStreamEndCapture(sb, &og);
  if (st != SL_OK) return st;
  CK(e);
  *total = thread_launch_count() - before;
  *direct = *total - nested;
  CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return SL_OK;
}

// Ends any capture left open on the handle's capture streams (after a failed capture).
void abandon_captures(sl_hjb *h) {
  for (int d = 7; d >= 0; --d) {
    cudaStream_t cs = h->cap_pool[d];
    if (!cs) continue;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(cs, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(cs, &g);
      if (g) cudaGraphDestroy(g);
    }
  }
  cudaGetLastError();
}

// Galerkin hierarchy for the current policy with every launch shape fixed: the explicit-row
// counts stay on the device (build_hierarchy_T reads them back to size its launches).
template <typename T>
sl_status cap_hierarchy_T(sl_hjb *h, double dt, cudaStream_t s) {
  for (int l = 1; l < h->L; ++l) {
    CoarseBuf &c = h->cl[l];
    CoarseBuf &p = h->cl[l - 1];
    launch_classify(l, h->tab, h->policy, p.cls, p.n, c.cls, c.n, c.erow, c.d_nexpl, h->chunk_scratch, s);
    CoarseLev<T> prevv = lev_view<T>(h, l - 1), curv = lev_view<T>(h, l);
    CK(launch_rap_explicit_dev<T>(l, h->tab, h->d_off, h->policy, T(dt), prevv, p.coff, curv, c.d_nexpl,
                                  c.cap, pick<T>(c.ewin64, c.ewin32), s));
  }
  const int lc = h->L - 1;
  CoarseLev<T> cv = lev_view<T>(h, lc);
  launch_coarsest_setup<T>(lc, h->tab, h->policy, T(dt), cv, lc == 0 ? h->d_off : h->cl[lc].coff,
                           h->cwork, pick<T>(h->Ainv64, h->Ainv32), s);
  tail_pack(h, s);
  CK(cudaGetLastError());
  return SL_OK;
}

// BiCGSTAB on the Krylov vectors of precision T (x accumulated in TX), the iterations a while
// node: the prologue of bicgstab(), then issue_iteration() and the device stop test.
template <typename T, typename TX>
sl_status cap_bicgstab(sl_hjb *h, double dt, TX *x, T *r, T *rh, T *p, T *v, T *sv, T *t, T *ph,
                       T *sh, BicgScalars *S, cudaStream_t s, int depth, long long *nested,
                       DevStepGraph &G) {
  const size_t N = NN(h, 0);
  const int fp64 = sizeof(T) == 8 ? 1 : 0;
  cudaGraphConditionalHandle hk;
  CK(new_cond_handle(s, &hk));
  CK(cudaMemcpyAsync(rh, r, N * sizeof(T), cudaMemcpyDeviceToDevice, s));
  launch_dot2<T>(r, r, r, r, N, POST_RHO_INIT, S, h->partials, h->counter, s);
  launch_ctl_kry_begin(h->ctl, fp64, h->o.kry_max, hk, s);
  long long tot = 0;
  const sl_status st = add_cond(h, s, depth, hk, cudaGraphCondTypeWhile, &G.k_kry, &tot,
                                [&](cudaStream_t sb, int, long long *) -> sl_status {
                                  sl_status r2 = issue_iteration<T, TX>(h, dt, x, r, rh, p, v, sv, t, ph, sh, S, sb);
                                  if (r2 != SL_OK) return r2;
                                  launch_ctl_kry_check(h->ctl, S, hk, sb);
                                  CK(cudaGetLastError());
                                  return SL_OK;
                                });
  *nested += tot;
  return st;
}

// linear_solve() with its refinement / restart rounds a while node; in a round, the true
// residual with the stop test is an if node (skipped when the round starts from the previous
// inner solve's residual) and the Krylov part another.
sl_status cap_linear_solve(sl_hjb *h, double dt, cudaStream_t s, int depth, long long *nested,
                           DevStepGraph &G) {
  const size_t N = NN(h, 0);
  const bool fp64 = h->o.precision == 0;
  KBuf &k = h->kb;
  launch_hjb_resid(h->tab, h->policy, h->Xb, h->Uprev, h->F, h->d_phi, h->nf, dt, h->Fvec, h->halo,
                   h->SW, s, std::max(1, h->cl[0].R), h->Ub);
  // the right-hand side's norms, once per solve (every round keeps them in S)
  launch_init_scalars(h->S, 0.0, s);
  launch_norms(h->Fvec, N, 0, h->S, h->partials, h->counter, s);
  cudaGraphConditionalHandle hir;
  CK(new_cond_handle(s, &hir));
  launch_ctl_ls_begin(h->ctl, h->o.krylov_tol, h->o.howard_loose_tol, hir, s);
  const int rounds = fp64 ? 12 : h->o.ir_max + 1;
  long long tot = 0;
  const sl_status st = add_cond(
      h, s, depth, hir, cudaGraphCondTypeWhile, &G.k_ir, &tot,
      [&](cudaStream_t sb, int d, long long *nest) -> sl_status {
        double *r64 = fp64 ? k.r64 : h->R;
        cudaGraphConditionalHandle htr, hen;
        CK(new_cond_handle(sb, &htr));
        CK(new_cond_handle(sb, &hen));
        // a true residual and the stop test (if node), or the previous inner solve's residual
        launch_ctl_ir_pre(h->ctl, htr, hen, sb);
        long long t1 = 0;
        const sl_status s1 = add_cond(
            h, sb, d, htr, cudaGraphCondTypeIf, &G.k_true, &t1,
            [&](cudaStream_t sc, int, long long *) -> sl_status {
              launch_hjb_resid(h->tab, h->policy, h->X, h->Uprev, h->F, h->d_phi, h->nf, dt, r64, h->halo,
                               h->SW, sc, 0, nullptr, h->Ub);
              launch_init_scalars_ctl(h->S, h->ctl, sc);
              launch_norms(r64, N, 1, h->S, h->partials, h->counter, sc);
              launch_ctl_ir_decide(h->ctl, h->S, h->o.krylov_tol, fp64 ? 1 : 0, h->o.kry_max, hen, sc);
              CK(cudaGetLastError());
              return SL_OK;
            });
        *nest += t1;
        if (s1 != SL_OK) return s1;
        long long t2 = 0;
        const sl_status s2 = add_cond(
            h, sb, d, hen, cudaGraphCondTypeIf, &G.k_enter, &t2,
            [&](cudaStream_t sc, int d2, long long *nest2) -> sl_status {
              sl_status s3;
              if (fp64) {
                s3 = cap_bicgstab<double, double>(h, dt, h->X, k.r64, k.rh64, k.p64, k.v64, k.s64, k.t64,
                                                  k.ph64, k.sh64, h->S, sc, d2, nest2, G);
              } else {
                launch_convert<double, float>(h->R, k.r32, N, sc, &h->ctl->need_true);
                launch_fill<float>(k.e32, N, 0.0f, sc);
                launch_init_scalars(h->S32, h->o.inner_tol * h->o.inner_tol, sc);
                launch_dot2<float>(k.r32, k.r32, nullptr, nullptr, N, POST_BNORM, h->S32, h->partials,
                                   h->counter, sc);
                s3 = cap_bicgstab<float, float>(h, dt, k.e32, k.r32, k.rh32, k.p32, k.v32, k.s32, k.t32,
                                                k.ph32, k.sh32, h->S32, sc, d2, nest2, G);
                if (s3 == SL_OK) launch_add_f32_to_f64(h->X, k.e32, N, sc);
              }
              if (s3 != SL_OK) return s3;
              launch_ctl_kry_end(h->ctl, fp64 ? 1 : 0, sc);
              if (!fp64) launch_ctl_ir_next(h->ctl, h->S, h->S32, h->o.ir_recursive, sc);
              CK(cudaGetLastError());
              return SL_OK;
            });
        *nest += t2;
        if (s2 != SL_OK) return s2;
        launch_ctl_ir_end(h->ctl, rounds, hir, sb);
        CK(cudaGetLastError());
        return SL_OK;
      });
  *nested += tot;
  return st;
}

// The argmin with its change counter and flags cleared first (improve() without the host read).
sl_status cap_improve(sl_hjb *h, cudaStream_t s, bool skip = false) {
  CK(cudaMemsetAsync(h->d_changes, 0, sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(h->d_flags, 0, sizeof(int), s));
  CK(launch_argmin(argmin_args(h, h->X, skip), *h->itaps, s));
  return SL_OK;
}

// One Howard iteration: rebuild (if node), linear solve, then improvement and stop test (if
// node, taken when the solve succeeded).
sl_status cap_pi_body(sl_hjb *h, double dt, cudaStream_t s, int depth, long long *nested,
                      DevStepGraph &G, cudaGraphConditionalHandle hpi) {
  const size_t N = NN(h, 0);
  cudaGraphConditionalHandle hrb, hok;
  CK(new_cond_handle(s, &hrb));
  CK(new_cond_handle(s, &hok));
  const long long thresh = (long long)(h->o.rebuild_frac * double(h->m) * h->m);
  launch_ctl_pi_pre(h->ctl, thresh, hrb, s);
  long long t = 0;
  sl_status st = add_cond(h, s, depth, hrb, cudaGraphCondTypeIf, &G.k_rebuild, &t,
                          [&](cudaStream_t sb, int, long long *) -> sl_status {
                            const sl_status r = h->o.precision == 0 ? cap_hierarchy_T<double>(h, dt, sb)
                                                                    : cap_hierarchy_T<float>(h, dt, sb);
                            if (r != SL_OK) return r;
                            NexplPtrs np{};
                            np.L = h->L;
                            for (int l = 1; l < h->L && l < 16; ++l) np.p[l] = h->cl[l].d_nexpl;
                            launch_ctl_built(h->ctl, np, sb);
                            return SL_OK;
                          });
  *nested += t;
  if (st != SL_OK) return st;
  st = cap_linear_solve(h, dt, s, depth, nested, G);
  if (st != SL_OK) return st;
  launch_ctl_after_ls(h->ctl, hok, hpi, s);
  st = add_cond(h, s, depth, hok, cudaGraphCondTypeIf, &G.k_ok, &t,
                [&](cudaStream_t sb, int, long long *) -> sl_status {
                  // the stop test's max |X - X^{m-1}| first: the argmin's skip test reads it
                  launch_maxabs_diff(h->X, h->Xpi, h->n, h->d_maxd, h->counter, h->partials, sb);
                  const sl_status r = cap_improve(h, sb, true);
                  if (r != SL_OK) return r;
                  launch_ctl_pi_post(h->ctl, h->d_changes, h->d_flags, h->d_maxd, h->o.pi_tol,
                                     h->o.pi_max, hpi, sb);
                  CK(cudaMemcpyAsync(h->Xpi, h->X, N * sizeof(double), cudaMemcpyDeviceToDevice, sb));
                  CK(cudaGetLastError());
                  return SL_OK;
                });
  *nested += t;
  return st;
}

// The work of one step after U^{n-1} is in Uprev (and U^{n-2} in Uprev2): tables, the first
// improvement of a march (if node), extrapolation, and the Howard loop (while node).
// tau_table: per-step time factors of a march (nullptr: d_tau is set before each launch).
sl_status cap_step_body(sl_hjb *h, double dt, cudaStream_t s, int depth, long long *nested,
                        DevStepGraph &G, const double *tau_table) {
  const size_t N = NN(h, 0);
  cudaGraphConditionalHandle him, hpre, hpi;
  CK(new_cond_handle(s, &him));
  CK(new_cond_handle(s, &hpre));
  CK(new_cond_handle(s, &hpi));
  launch_ctl_step_begin(h->ctl, tau_table, h->nq + h->npsi, h->d_tau, h->o.extrapolate, h->o.howard_init, him,
                        hpre, hpi, s);
  CK(cudaMemcpyAsync(h->X, h->Uprev, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  launch_coef(h->G, h->nf, h->nq, h->d_tau, h->Psi, h->npsi, h->d_tau + h->nq, h->n, h->F, h->F32,
              h->X, h->Xb, s);
  long long t = 0;
  sl_status st = add_cond(h, s, depth, him, cudaGraphCondTypeIf, &G.k_imp0, &t,
                          [&](cudaStream_t sb, int, long long *) -> sl_status {
                            const sl_status r = cap_improve(h, sb);
                            if (r != SL_OK) return r;
                            launch_ctl_improved0(h->ctl, sb);
                            return SL_OK;
                          });
  *nested += t;
  if (st != SL_OK) return st;
  CK(cudaMemcpyAsync(h->Xpi, h->X, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  launch_extrapolate_ctl(h->X, h->Uprev, h->Uprev2, h->n, h->ctl, s);
  st = add_cond(h, s, depth, hpre, cudaGraphCondTypeIf, &G.k_pre, &t,
                [&](cudaStream_t sb, int, long long *) -> sl_status {
                  const sl_status r = cap_improve(h, sb);
                  if (r != SL_OK) return r;
                  launch_ctl_preimproved(h->ctl, h->d_changes, h->d_flags, hpi, sb);
                  return SL_OK;
                });
  *nested += t;
  if (st != SL_OK) return st;
  st = add_cond(h, s, depth, hpi, cudaGraphCondTypeWhile, &G.k_pi, &t,
                [&](cudaStream_t sb, int d, long long *nest) -> sl_status {
                  return cap_pi_body(h, dt, sb, d, nest, G, hpi);
                });
  *nested += t;
  CK(cudaGetLastError());
  return st;
}

// Steps run on the device when nothing in the middle of a step needs the host: the geometric
// V-cycle, the class-table fine level, no recording for the adjoint.
bool dev_step_ok(const sl_hjb *h) {
  return h->o.use_graphs == 2 && !h->dev_off && !h->general && h->o.precond == 0 && !h->rec_slot &&
         !h->transposed && h->nq + h->npsi <= 8;
}

// Kernels one step graph launch ran, from the device's loop counts.
long long dev_kernels(const DevStepGraph &G, const DevCtl &c) {
  return G.k_step * c.c_steps + G.k_imp0 * c.c_improve0 + G.k_pre * c.c_pre + G.k_pi * c.c_pibody +
         G.k_rebuild * c.c_rebuild +
         G.k_ir * c.c_ir + G.k_true * c.c_true + G.k_enter * c.c_enter + G.k_kry * c.c_kry +
         G.k_ok * c.c_ok;
}

// Captures the step graph for step size dt (after the host-side tables for dt).
sl_status ensure_step_graph(sl_hjb *h, double dt, cudaStream_t s) {
  DevStepGraph &G = h->sgraph;
  if (G.exec && G.dt == dt) return SL_OK;
  if (G.exec) cudaGraphExecDestroy(G.exec);
  G = DevStepGraph{};
  sl_status st = ensure_class_tables(h, dt, s);
  if (st != SL_OK) return st;
  CK(cudaStreamSynchronize(s));
  cudaStream_t cs = nullptr;
  CK(cap_stream_at(h, 0, &cs));
  const long long before = thread_launch_count();
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  long long nested = 0;
  st = cap_step_body(h, dt, cs, 0, &nested, G, nullptr);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  const long long captured = thread_launch_count() - before;
  note_launch(int(-captured));  // captured, not executed
  G.k_step = captured - nested;
  if (st == SL_OK && e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (st != SL_OK || e != cudaSuccess) {
    abandon_captures(h);
    if (G.exec) cudaGraphExecDestroy(G.exec);
    G = DevStepGraph{};
    return st != SL_OK ? st : fail(h, SL_ECUDA, std::string("step graph: ") + cudaGetErrorString(e));
  }
  G.dt = dt;
  return SL_OK;
}

sl_status step_impl(sl_hjb *h, double *u, double t, double dt, uint8_t *pol_out, sl_stats *st,
                    cudaStream_t s);

// One implicit step as one graph launch (the same kernels and results as step_impl).
sl_status step_device(sl_hjb *h, double *u, double t, double dt, uint8_t *pol_out, sl_stats *st,
                      cudaStream_t s) {
  if (!(dt > 0)) return fail(h, SL_EINVAL, "dt must be positive");
  for (double c : h->cvec)
    if (dt * c > 1.0) return fail(h, SL_ECFL, "dt * c > 1 violates the positivity condition");
  if (ensure_step_graph(h, dt, s) != SL_OK) {
    h->dev_off = true;
    std::fprintf(stderr, "sl_hjb: step graph unavailable (%s); steps are host-driven\n", h->err.c_str());
    return step_impl(h, u, t, dt, pol_out, st, s);
  }
  const size_t N = NN(h, 0);
  const bool extrap = h->o.extrapolate && h->have_prev2 && h->prev_dt == dt &&
                      std::fabs(h->prev_t + dt - t) <= 1e-12 * std::max(1.0, std::fabs(t));
  if (h->o.extrapolate) CK(cudaMemcpyAsync(h->Uprev2, h->Uprev, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->Uprev, u, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (h->f_cb)
    for (int mm = 0; mm < h->nf; ++mm) h->f_cb(t, &h->grid, mm, h->Gcb + mm * N, h->cb_user, s);
  if (h->psi_cb) h->psi_cb(t, &h->grid, 0, h->Psicb, h->cb_user, s);
  StepPrep p{};
  p.ntau = h->nq + h->npsi;
  for (int q = 0; q < h->nq; ++q) p.tau[q] = tau_eval(h->tau_kind[q], h->tau_rate[q], t);
  for (int q = 0; q < h->npsi; ++q) p.tau[h->nq + q] = tau_eval(h->psi_kind[q], h->psi_rate[q], t);
  p.extrap = extrap ? 1 : 0;
  p.need_improve = h->have_policy ? 0 : 1;
  p.hier_valid = (h->hier_valid && h->hier_dt == dt) ? 1 : 0;
  p.changes_since_build = h->changes_since_build;
  CK(cudaMemsetAsync(h->ctl, 0, sizeof(DevCtl), s));
  launch_ctl_step_prep(h->ctl, p, h->d_tau, s);
  CK(cudaGraphLaunch(h->sgraph.exec, s));
  CK(cudaMemcpyAsync(u, h->X, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (pol_out) CK(cudaMemcpyAsync(pol_out, h->policy, size_t(h->m) * h->m, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const DevCtl &c = *h->h_ctl;
  note_launch(int(dev_kernels(h->sgraph, c)));
  h->have_policy = true;
  h->have_prev2 = h->o.extrapolate != 0;
  h->prev_t = t;
  h->prev_dt = dt;
  h->hier_valid = c.hier_valid != 0;
  if (c.c_rebuild) h->hier_dt = dt;
  h->changes_since_build = c.changes_since_build;
  if (c.c_rebuild)
    for (int l = 1; l < h->L && l < 16; ++l) h->cl[l].nexpl = c.nexpl[l];
  if (st) {
    st->steps += 1;
    st->graph_steps += 1;
    st->pi_iters += int(c.c_pi);
    st->krylov_iters += int(c.c_kry);
    if (h->o.precision != 0) st->ir_iters += int(c.c_enter);
    st->rebuilds += int(c.c_rebuild);
    st->policy_changes += c.c_changes;
    st->res_final = c.res_final;
    if (c.c_rebuild) {
      long long ex = 0;
      for (int l = 1; l < h->L; ++l) ex += h->cl[l].nexpl;
      st->explicit_rows = ex;
    }
  }
  if (c.tma_err) return fail(h, SL_ETIMEOUT, "a bounded wait for the TMA tile copies of the fine operator gave up");
  switch (c.status) {
    case SL_OK: return SL_OK;
    case SL_ENAN: return fail(h, SL_ENAN, "non-finite value in the step (control value, residual or iterate)");
    case SL_ENOCONV_PI: return fail(h, SL_ENOCONV_PI, "Howard iteration reached pi_max");
    case SL_ENOCONV_KRYLOV:
      return fail(h, SL_ENOCONV_KRYLOV, h->o.precision == 0 ? "BiCGSTAB reached its iteration cap"
                                                             : "iterative refinement reached ir_max");
    default: return fail(h, sl_status(c.status), "step failed on the device");
  }
}

// The step of the public entry points.
sl_status step_any(sl_hjb *h, double *u, double t, double dt, uint8_t *pol_out, sl_stats *st,
                   cudaStream_t s) {
  return dev_step_ok(h) ? step_device(h, u, t, dt, pol_out, st, s) : step_impl(h, u, t, dt, pol_out, st, s);
}

// ---------------------------------------------------------------------- adjoint
// Grows a device buffer (contents are not kept).
template <typename T>
sl_status dgrow(sl_hjb *h, T **p, size_t *cap, size_t count) {
  if (*p && *cap >= count) return SL_OK;
  if (*p) {
    CK(cudaDeviceSynchronize());
    h->allocs.erase(std::find(h->allocs.begin(), h->allocs.end(), static_cast<void *>(*p)));
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
  }
  sl_status st = dalloc(h, p, count);
  if (st != SL_OK) return st;
  *cap = count;
  return SL_OK;
}

sl_status ensure_adjoint_buffers(sl_hjb *h) {
  if (h->t_rowptr) return SL_OK;
  // the fine table in use: the class tables, or the per-row tables of a general level (whose
  // rows hold diffusion and drift taps and reach farther than the drift tables alone)
  if (double(h->cl[0].R) * (h->n + 1) >= double(1 << 24))  // packed sort keys of the fine A^T
    return fail(h, SL_EINVAL, "stencil reach too large for the transposed fine operator");
  const size_t M = size_t(h->m) * h->m, N = size_t(h->n) * h->n;
  const size_t nnz = M * size_t(h->tab.tmax);  // every tap of every row at most once
  AL(h->t_rowptr, M + 1);
  AL(h->t_cnt, M);
  AL(h->t_scan, 2 * ((M + 1023) / 1024) + 2);
  AL(h->t_col, nnz);
  AL(h->t_v64, nnz);
  AL(h->t_vtmp, nnz);
  AL(h->t_v32, nnz);
  AL(h->t_d64, M);
  AL(h->t_d32, M);
  AL(h->mu, N);
  AL(h->lam, N);
  AL(h->d_dtheta, kMaxParams);
  AL(h->d_dpart, size_t(kMaxParams) * kRedBlocks);
  for (int l = 1; l < h->L; ++l) {
    CoarseBuf &c = h->cl[l];
    const size_t cnt = size_t(c.win) * c.m * c.m;
    if (h->o.precision == 0) AL(c.WT64, cnt);
    else AL(c.WT32, cnt);
  }
  return SL_OK;
}

// Transposed operators of the current policy and step size (after build_hierarchy).
sl_status build_transposed(sl_hjb *h, double dt, cudaStream_t s) {
  launch_csrT_build(h->tab, h->d_off, h->policy, dt, h->cl[0].R, h->t_cnt, h->t_scan, h->t_rowptr,
                    h->t_col, h->t_vtmp, h->t_v64, h->t_v32, h->t_d64, h->t_d32, s);
  for (int l = 1; l < h->L; ++l) {
    CoarseBuf &c = h->cl[l];
    if (h->o.precision == 0) launch_denseT_build<double>(lev_view<double>(h, l), c.cdense64, c.WT64, s);
    else launch_denseT_build<float>(lev_view<float>(h, l), c.cdense32, c.WT32, s);
  }
  CK(cudaGetLastError());
  return SL_OK;
}

size_t rec_checkpoints(int N, int k) { return size_t(N / k) + 1 + (N % k ? 1 : 0); }

// U^s of the recorded march, if stored (nullptr inside a segment).
double *rec_stored(sl_hjb *h, int s) {
  const size_t NNf = size_t(h->n) * h->n;
  if (s % h->rec_k == 0) return h->rec_U + size_t(s / h->rec_k) * NNf;
  if (s == h->rec_N) return h->rec_U + (rec_checkpoints(h->rec_N, h->rec_k) - 1) * NNf;
  return nullptr;
}

// Re-solves steps base+1 .. top-1 of segment c at their recorded policies into rec_seg.
sl_status recompute_segment(sl_hjb *h, int c, sl_stats *st, cudaStream_t s) {
  const size_t NNf = size_t(h->n) * h->n, M = size_t(h->m) * h->m;
  const int base = c * h->rec_k, top = std::min(base + h->rec_k, h->rec_N);
  const double dt = h->rec_dt;
  for (int j = base + 1; j < top; ++j) {
    const double *prev = (j - 1 == base) ? rec_stored(h, base) : h->rec_seg + size_t(j - 2 - base) * NNf;
    CK(cudaMemcpyAsync(h->Uprev, prev, NNf * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(h->X, prev, NNf * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(h->policy, h->rec_pol + size_t(j - 1) * M, M, cudaMemcpyDeviceToDevice, s));
    sl_status r = coef(h, h->rec_t0 + j * dt, h->X, s);
    if (r != SL_OK) return r;
    r = build_hierarchy(h, dt, s);
    if (r != SL_OK) return r;
    r = linear_solve(h, dt, st, s);
    if (r != SL_OK) return r;
    CK(cudaMemcpyAsync(h->rec_seg + size_t(j - 1 - base) * NNf, h->X, NNf * sizeof(double),
                       cudaMemcpyDeviceToDevice, s));
  }
  return SL_OK;
}

sl_status upload_dtables(sl_hjb *h, int np, const double *dsigma, DTabView *dv) {
  const int E = h->K * h->ft.Q * h->ft.Q;
  const size_t per = size_t(h->K) * 2 * h->P;
  std::vector<FineDTabHost> tabs;
  int stride = 1;
  for (int p = 0; p < np; ++p) {
    tabs.push_back(build_fine_dtables(h->ft, h->h, h->P, h->sigma.data(), dsigma + p * per));
    stride = std::max(stride, tabs.back().stride);
  }
  std::vector<int32_t> lin(size_t(np) * E * stride, 0);
  std::vector<double> dw(lin.size(), 0.0), dW(size_t(np) * E, 0.0);
  std::vector<uint8_t> nt(size_t(np) * E, 0);
  for (int p = 0; p < np; ++p)
    for (int e = 0; e < E; ++e) {
      const FineDTabHost &d = tabs[p];
      const size_t pe = size_t(p) * E + e;
      nt[pe] = d.nt[e];
      dW[pe] = d.dW[e];
      for (int t = 0; t < d.nt[e]; ++t) {
        const size_t src = size_t(e) * d.stride + t;
        lin[pe * stride + t] = d.dy[src] * h->n + d.dx[src];
        dw[pe * stride + t] = d.dw[src];
      }
    }
  sl_status r = dgrow(h, &h->dt_lin, &h->dt_cap[0], lin.size());
  if (r == SL_OK) r = dgrow(h, &h->dt_dw, &h->dt_cap[1], dw.size());
  if (r == SL_OK) r = dgrow(h, &h->dt_nt, &h->dt_cap[2], nt.size());
  if (r == SL_OK) r = dgrow(h, &h->dt_dW, &h->dt_cap[3], dW.size());
  if (r != SL_OK) return r;
  CK(cudaMemcpy(h->dt_lin, lin.data(), lin.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->dt_dw, dw.data(), dw.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->dt_nt, nt.data(), nt.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->dt_dW, dW.data(), dW.size() * sizeof(double), cudaMemcpyHostToDevice));
  dv->np = np;
  dv->E = E;
  dv->stride = stride;
  dv->lin = h->dt_lin;
  dv->dw = h->dt_dw;
  dv->nt = h->dt_nt;
  dv->dW = h->dt_dW;
  return SL_OK;
}

}  // namespace

// ---------------------------------------------------------------------- no-allocation V-cycle
// Scratch of sl_hjb_vcycle_noalloc: a file-scope device array, so that the entry point needs no
// cudaMalloc.  Every GPU that loads the library holds it until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(2) << 20;  // 2 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Host code cannot use g_noalloc_scratch as a device address (on the host it names a shadow
// variable); its device address is looked up once per device, with that device current.
constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[kMaxDevices] = {};

sl_status noalloc_scratch(sl_hjb *h, void **out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(h, SL_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return SL_OK;
}

// The V-cycle of vcycle() with every work vector taken from caller-provided storage
// (t, r: smoother ping-pong and residual per level; cb, cx: coarse right-hand side and
// correction per level >= 1).
template <typename T>
sl_status vcycle_into(sl_hjb *h, int l, double dt, const T *b, T *x, T *const *t, T *const *r,
                      T *const *cb, T *const *cx, cudaStream_t s) {
  const size_t N = NN(h, l);
  if (l == h->L - 1) {
    launch_coarsest_apply<T>(pick<T>(h->Ainv64, h->Ainv32), h->cl[l].n, b, x, s);
    return SL_OK;
  }
  T *cur = x, *other = t[l];
  if (smooth_swaps(h) & 1) std::swap(cur, other);
  if (h->o.nu1 == 0) launch_fill<T>(cur, N, T(0), s);
  else smooth<T>(h, l, dt, b, cur, other, h->o.nu1, true, s);
  level_op<T>(h, l, OP_RESID, dt, cur, b, r[l], s);
  launch_restrict<T>(r[l], h->cl[l].n, cb[l + 1], h->cl[l + 1].n, s);
  sl_status st = vcycle_into<T>(h, l + 1, dt, cb[l + 1], cx[l + 1], t, r, cb, cx, s);
  if (st != SL_OK) return st;
  launch_prolong_add<T>(cx[l + 1], h->cl[l + 1].n, cur, h->cl[l].n, s);
  smooth<T>(h, l, dt, b, cur, other, h->o.nu2, false, s);
  if (cur != x) CK(cudaMemcpyAsync(x, cur, N * sizeof(T), cudaMemcpyDeviceToDevice, s));
  CK(cudaGetLastError());
  return SL_OK;
}

// Lays the work vectors out in the static scratch (each vector 256-byte aligned), clears the
// part that is used (boundary entries must read as zero and the array keeps the previous
// call's contents), and runs the cycle.
template <typename T>
sl_status vcycle_noalloc_T(sl_hjb *h, const T *b, T *x, cudaStream_t s) {
  T *t[kMaxLevels] = {}, *r[kMaxLevels] = {}, *cb[kMaxLevels] = {}, *cx[kMaxLevels] = {};
  size_t need = 0;
  auto take = [&](size_t count) {
    const size_t off = need;
    need += (count * sizeof(T) + 255) / 256 * 256;
    return off;
  };
  size_t ot[kMaxLevels], orr[kMaxLevels], ob[kMaxLevels], ox[kMaxLevels];
  for (int l = 0; l < h->L; ++l) {
    const size_t Nl = NN(h, l);
    ot[l] = take(Nl);
    orr[l] = take(Nl);
    if (l > 0) {
      ob[l] = take(Nl);
      ox[l] = take(Nl);
    }
  }
  if (need > kNoAllocScratchBytes)
    return fail(h, SL_EINVAL, "sl_hjb_vcycle_noalloc: the V-cycle of this grid needs " +
                                  std::to_string(need) + " bytes of scratch, more than the " +
                                  std::to_string(kNoAllocScratchBytes) + " bytes available");
  void *base = nullptr;
  sl_status st = noalloc_scratch(h, &base);
  if (st != SL_OK) return st;
  unsigned char *p = static_cast<unsigned char *>(base);
  for (int l = 0; l < h->L; ++l) {
    t[l] = reinterpret_cast<T *>(p + ot[l]);
    r[l] = reinterpret_cast<T *>(p + orr[l]);
    if (l > 0) {
      cb[l] = reinterpret_cast<T *>(p + ob[l]);
      cx[l] = reinterpret_cast<T *>(p + ox[l]);
    }
  }
  CK(cudaMemsetAsync(base, 0, need, s));
  return vcycle_into<T>(h, 0, h->hier_dt, b, x, t, r, cb, cx, s);
}

// ====================================================================== C ABI
extern "C" {

void sl_opts_default(sl_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = 0;
  o->levels = 0;
  o->nu1 = 2;
  o->nu2 = 2;
  o->omega = 0.8;
  o->krylov_tol = 1e-12;
  o->kry_max = 200;
  o->inner_tol = 1e-2;
  o->ir_max = 30;
  o->pi_tol = 1e-10;
  o->pi_max = 100;
  o->tie_rel = 1e-12;
  o->argmin_screen = 1;
  o->rebuild_frac = 0.01;
  o->use_graphs = 2;
  o->coarse_tail_rows = -1;
  o->extrapolate = 1;
  o->precond = 0;
  o->amg_k_levels = 2;
  o->fine_tma = 1;
  o->smoother = 0;
  o->coarse_fusion = 3;
  o->howard_init = 0;
  o->howard_loose_tol = 1e-7;
  o->argmin_skip = 1;
  o->ir_recursive = 3;
}

const char *sl_hjb_last_error(const sl_hjb *h) { return h ? h->err.c_str() : "null handle"; }

void sl_hjb_destroy(sl_hjb *h) {
  if (!h) return;
  cudaDeviceSynchronize();
  for (auto &g : h->graph)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto &g : h->graphT)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->sgraph.exec) cudaGraphExecDestroy(h->sgraph.exec);
  for (cudaStream_t cs : h->cap_pool)
    if (cs) cudaStreamDestroy(cs);
  if (h->h_ctl) cudaFreeHost(h->h_ctl);
  amg_free(h->amg);
  for (void *p : h->allocs) cudaFree(p);
  if (h->hS) cudaFreeHost(h->hS);
  if (h->h_maxd) cudaFreeHost(h->h_maxd);
  if (h->h_changes) cudaFreeHost(h->h_changes);
  if (h->h_flags) cudaFreeHost(h->h_flags);
  if (h->h_count) cudaFreeHost(h->h_count);
  delete h->itaps;
  delete h;
}

static sl_status create_impl(sl_hjb *h, const sl_grid *g, const sl_controls *c, const sl_source *src,
                             const sl_opts *opts) {
  if (!g || !c || !src) return fail(h, SL_EINVAL, "null argument");
  if (g->nx != g->ny || g->nx < 5) return fail(h, SL_EINVAL, "grid must be square with nx >= 5");
  if (g->nx > 46340) return fail(h, SL_EINVAL, "nx must be at most 46340 (grid indices are 32-bit)");
  const double hx = (g->x_hi - g->x_lo) / (g->nx - 1), hy = (g->y_hi - g->y_lo) / (g->ny - 1);
  if (!(hx > 0) || std::fabs(hx - hy) > 1e-12 * hx) return fail(h, SL_EINVAL, "cells must be square");
  if (c->K < 1 || c->K > 255) return fail(h, SL_EINVAL, "K must be in 1..255");
  if (c->P < 1 || c->P > 4 || (!c->sigma && !c->sigma_field))
    return fail(h, SL_EINVAL, "P must be in 1..4 with sigma or sigma_field given");
  const bool fcb = src->f_cb != nullptr, pcb = src->psi_cb != nullptr;
  if (src->nf < 1 || src->nf > 4 || !src->phi ||
      (!fcb && (src->nq < 1 || !src->G_dev || !src->tau_kind || !src->tau_rate)))
    return fail(h, SL_EINVAL, "source: need 1 <= nf <= 4, phi, and nq >= 1, G, tau or a source callback");
  if (!pcb && (src->npsi < 0 || (src->npsi > 0 && (!src->Psi_dev || !src->psi_kind || !src->psi_rate))))
    return fail(h, SL_EINVAL, "boundary data incomplete");
  if (opts) h->o = *opts; else sl_opts_default(&h->o);
  if (h->o.precision != 0 && h->o.precision != 1) return fail(h, SL_EINVAL, "precision must be 0 or 1");
  if (h->o.nu1 < 0 || h->o.nu2 < 0 || h->o.kry_max < 1 || h->o.pi_max < 1 || !(h->o.omega > 0))
    return fail(h, SL_EINVAL, "bad iteration options");
  if (h->o.precond != 0 && h->o.precond != 1) return fail(h, SL_EINVAL, "precond must be 0 or 1");
  if (h->o.smoother != 0 && h->o.smoother != 1) return fail(h, SL_EINVAL, "smoother must be 0 or 1");
  if (h->o.coarse_fusion < 0) return fail(h, SL_EINVAL, "coarse_fusion must be >= 0");
  if (h->o.howard_init != 0 && h->o.howard_init != 1) return fail(h, SL_EINVAL, "howard_init must be 0 or 1");
  if (h->o.argmin_skip != 0 && h->o.argmin_skip != 1) return fail(h, SL_EINVAL, "argmin_skip must be 0 or 1");
  if (h->o.ir_recursive < 0) return fail(h, SL_EINVAL, "ir_recursive must be >= 0");
  if (!(h->o.howard_loose_tol >= 0.0) || (h->o.howard_loose_tol > 0.0 && h->o.howard_loose_tol < h->o.krylov_tol))
    return fail(h, SL_EINVAL, "howard_loose_tol must be 0 or at least krylov_tol");
  if (h->o.precond == 1 && (h->o.nu1 < 1 || h->o.amg_k_levels < 0))
    return fail(h, SL_EINVAL, "the aggregation K-cycle needs nu1 >= 1 and amg_k_levels >= 0");
  h->amg.nu1 = h->o.nu1;
  h->amg.nu2 = h->o.nu2;
  h->amg.omega = h->o.omega;
  h->amg.k_levels = h->o.amg_k_levels;
  h->n = g->nx;
  h->m = g->nx - 2;
  h->h = hx;
  h->K = c->K;
  h->P = c->P;
  h->nf = src->nf;
  h->nq = fcb ? 1 : src->nq;
  h->npsi = pcb ? 1 : src->npsi;
  h->G = src->G_dev;
  h->Psi = src->Psi_dev;
  h->f_cb = src->f_cb;
  h->psi_cb = src->psi_cb;
  h->cb_user = src->cb_user;
  h->grid = *g;
  h->phi.assign(src->phi, src->phi + size_t(c->K) * src->nf);
  if (fcb) {
    h->tau_kind.assign(1, SL_TAU_ONE);
    h->tau_rate.assign(1, 0.0);
  } else {
    h->tau_kind.assign(src->tau_kind, src->tau_kind + src->nq);
    h->tau_rate.assign(src->tau_rate, src->tau_rate + src->nq);
  }
  if (pcb) {
    h->psi_kind.assign(1, SL_TAU_ONE);
    h->psi_rate.assign(1, 0.0);
  } else if (src->npsi > 0) {
    h->psi_kind.assign(src->psi_kind, src->psi_kind + src->npsi);
    h->psi_rate.assign(src->psi_rate, src->psi_rate + src->npsi);
  }
  h->cvec.assign(c->K, 0.0);
  if (c->c) h->cvec.assign(c->c, c->c + c->K);
  if (c->sigma) h->sigma.assign(c->sigma, c->sigma + size_t(c->K) * 2 * c->P);
  h->general = c->sigma_field != nullptr;
  h->phimax.assign(h->nf, 0.0);
  for (int k = 0; k < h->K; ++k)
    for (int mm = 0; mm < h->nf; ++mm)
      h->phimax[mm] = std::max(h->phimax[mm], std::fabs(h->phi[size_t(k) * h->nf + mm]));
  // levels
  int maxL = 1;
  {
    int nn = h->n;
    while (nn > 5 && (nn - 1) % 2 == 0) { nn = (nn + 1) / 2; ++maxL; }
  }
  h->L = h->o.levels > 0 ? h->o.levels : maxL;
  if (h->L > maxL || h->L > kMaxLevels) return fail(h, SL_EINVAL, "too many levels for this grid (need n = 2^j + 1)");
  {
    int nn = h->n;
    for (int l = 0; l < h->L; ++l) {
      h->cl[l].n = nn;
      h->cl[l].m = nn - 2;
      nn = (nn + 1) / 2;
    }
    const int mc = h->cl[h->L - 1].m;
    if (mc * mc > kCoarsestMax) return fail(h, SL_EINVAL, "coarsest level too large for the dense solve: use more levels");
  }
  // kernels that may take more than 48 KB of dynamic shared memory (once per device)
  CK(prepare_fine_kernels());
  CK(prepare_coarse_kernels());
  // stencil tables
  try {
    if (h->general) {
      // drift taps per (control, boundary class), diffusion taps per row
      h->ft = build_fine_tables(h->n, h->h, h->K, 0, nullptr, c->b, c->c);
      h->nd = build_node_tables(h->n, h->h, h->P, c->sigma_field);
    } else {
      h->ft = build_fine_tables(h->n, h->h, h->K, h->P, c->sigma, c->b, c->c);
    }
  } catch (const std::exception &e) {
    return fail(h, SL_EINVAL, e.what());
  }
  const FineTabHost &ft = h->ft;
  const int R0 = h->general ? std::max(ft.R0, h->nd.R0) : ft.R0;
  h->halo = std::max(1, R0);
  // Row pitch of the staged fine tiles: at least 3 columns beyond the 32 + 2 halo staged ones,
  // and congruent to n mod 4, so that each tile row and its global row have the same offset
  // within 16 bytes: a row can then be copied by the TMA unit (cp.async.bulk) from its
  // 16-byte-aligned start, the extra columns taking the rounding at either end.
  h->SW = 32 + 2 * h->halo + 3;
  while ((h->SW - h->n) % 4 != 0) ++h->SW;
  h->SH = 8 + 2 * h->halo;
  if (size_t(h->SW) * (32 + 2 * h->halo) * sizeof(double) > 200 * 1024)
    return fail(h, SL_EINVAL, "stencil too wide for the shared-memory tiles");
  const size_t ET = ft.dx.size();
  std::vector<int32_t> lin(ET), slin(ET), off(ET);
  std::vector<int2> pk32(ET);
  std::vector<longlong2> pk64(ET);
  for (size_t i = 0; i < ET; ++i) {
    lin[i] = ft.dy[i] * h->n + ft.dx[i];
    slin[i] = ft.dy[i] * h->SW + ft.dx[i];
    off[i] = (ft.dy[i] << 16) | (ft.dx[i] & 0xffff);
    const float w32 = float(ft.w[i]);
    int wbits;
    std::memcpy(&wbits, &w32, sizeof(int));
    pk32[i] = make_int2(slin[i], wbits);
    long long wb64;
    std::memcpy(&wb64, &ft.w[i], sizeof(long long));
    pk64[i].x = slin[i];
    pk64[i].y = wb64;
  }
  std::vector<float> w32(ft.w.begin(), ft.w.end()), W32(ft.W.begin(), ft.W.end()),
      ws32(ft.ws.begin(), ft.ws.end()), c32(ft.c.begin(), ft.c.end()),
      phi32(h->phi.begin(), h->phi.end());
  // interior-class taps of every control for the argmin (the class path only)
  h->itaps = new (std::nothrow) ArgminITaps();
  if (!h->itaps) return fail(h, SL_ENOMEM, "host allocation failed");
  h->itaps->n = 0;
  if (!h->general && h->n - 1 >= 2 * ft.B && size_t(h->K) * ft.tmax <= size_t(kITapMax)) {
    for (int k = 0; k < h->K; ++k) {
      const int e = ft.entry(k, ft.B, ft.B);
      for (int t = 0; t < ft.tmax; ++t) {
        const int2 p = pk32[size_t(e) * ft.tmax + t];
        h->itaps->t[k * ft.tmax + t] = make_int2(p.x * int(sizeof(float)), p.y);  // byte offset
      }
    }
    h->itaps->n = h->K * ft.tmax;
  }
  // the argmin's skip test: a control value moves by at most sum_t |w_t| |dX_t - dX_j|
  // + |c_k| |dX_j| when X moves by dX
  h->Wabs = 0.0;
  for (int e = 0; e < int(ft.nt.size()); ++e) {
    double sw = 0.0;
    for (int t = 0; t < ft.nt[e]; ++t) sw += std::fabs(ft.w[size_t(e) * ft.tmax + t]);
    h->Wabs = std::max(h->Wabs, sw);
  }
  h->Wabs *= 1.0 + 1e-12;
  if (h->o.argmin_screen && !h->general) AL(h->d_gap, size_t(h->m) * h->m);
  UP(h->d_lin, lin);
  UP(h->d_slin, slin);
  UP(h->d_off, off);
  UP(h->d_pk32, pk32);
  UP(h->d_pk64, pk64);
  UP(h->d_w64, ft.w);
  UP(h->d_w32, w32);
  UP(h->d_nt, ft.nt);
  UP(h->d_W64, ft.W);
  UP(h->d_W32, W32);
  UP(h->d_ws64, ft.ws);
  UP(h->d_ws32, ws32);
  UP(h->d_c64, ft.c);
  UP(h->d_c32, c32);
  UP(h->d_Wmaxc, ft.Wmax_class);
  UP(h->d_phi, h->phi);
  UP(h->d_phi32, phi32);
  UP(h->d_phimax, h->phimax);
  AL(h->d_tau, size_t(h->nq + h->npsi + 2));
  FineTab &t = h->tab;
  t.n = h->n; t.m = h->m; t.B = ft.B; t.Q = ft.Q; t.tmax = ft.tmax; t.K = h->K;
  t.lin = h->d_lin; t.w64 = h->d_w64; t.w32 = h->d_w32; t.nt = h->d_nt; t.W64 = h->d_W64;
  t.W32 = h->d_W32; t.ws64 = h->d_ws64; t.ws32 = h->d_ws32; t.c64 = h->d_c64; t.c32 = h->d_c32;
  t.pk32 = h->d_pk32; t.pk64 = h->d_pk64;
  t.ipk32 = nullptr; t.ipk64 = nullptr; t.iWc64 = nullptr; t.iWc32 = nullptr;
  t.iod64 = nullptr; t.iod32 = nullptr;
  if (!h->general && h->n - 1 >= 2 * ft.B && ft.tmax % 2 == 0) {
    // the interior entries again, tap-major with the controls adjacent
    const int K = h->K, tm = ft.tmax;
    std::vector<int4> ipk32(size_t(tm / 2) * K);
    std::vector<longlong2> ipk64(size_t(tm) * K);
    std::vector<double> iWc64(K);
    std::vector<float> iWc32(K);
    for (int k = 0; k < K; ++k) {
      const int e = ft.entry(k, ft.B, ft.B);
      for (int tt = 0; tt < tm; ++tt) {
        const int2 p = pk32[size_t(e) * tm + tt];
        int4 &q = ipk32[size_t(tt / 2) * K + k];
        if (tt % 2 == 0) { q.x = p.x; q.y = p.y; } else { q.z = p.x; q.w = p.y; }
        ipk64[size_t(tt) * K + k] = pk64[size_t(e) * tm + tt];
      }
      iWc64[k] = ft.W[e] - ft.c[k];
      const float Wf = W32[e], cf = c32[k];
      iWc32[k] = Wf - cf;
    }
    UP(h->d_ipk32, ipk32);
    UP(h->d_ipk64, ipk64);
    UP(h->d_iWc64, iWc64);
    UP(h->d_iWc32, iWc32);
    AL(h->d_iod64, size_t(K));
    AL(h->d_iod32, size_t(K));
    t.ipk32 = h->d_ipk32; t.ipk64 = h->d_ipk64; t.iWc64 = h->d_iWc64; t.iWc32 = h->d_iWc32;
    t.iod64 = h->d_iod64; t.iod32 = h->d_iod32;
  }
  AL(h->d_od64, size_t(h->K) * ft.Q * ft.Q);
  AL(h->d_od32, size_t(h->K) * ft.Q * ft.Q);
  t.od64 = h->d_od64; t.od32 = h->d_od32;
  t.general = 0;
  t.tma = 0;
  t.tma_err = nullptr;
  if (h->general) {
    // the tables above hold the drift part; the fine level reads per-row entries
    h->dtab = t;
    const NodeTabHost &nd = h->nd;
    const size_t M = size_t(h->m) * h->m;
    std::vector<int32_t> ndoff(nd.dx.size());
    for (size_t i = 0; i < ndoff.size(); ++i) ndoff[i] = (nd.dy[i] << 16) | (nd.dx[i] & 0xffff);
    GeneralArgs &g = h->gen;
    g.n = h->n;
    g.nd_stride = nd.stride;
    int32_t *p_off = nullptr;
    double *p_w = nullptr, *p_W = nullptr;
    uint8_t *p_nt = nullptr;
    UP(p_off, ndoff);
    UP(p_w, nd.w);
    UP(p_nt, nd.nt);
    UP(p_W, nd.W);
    g.nd_off = p_off; g.nd_w = p_w; g.nd_nt = p_nt; g.nd_W = p_W;
    g.dr_off = h->d_off;
    GeneralOut &o = h->gout;
    o.stride = nd.stride + ft.tmax;
    const size_t ES = M * o.stride;
    AL(o.off, ES); AL(o.lin, ES); AL(o.w64, ES); AL(o.w32, ES); AL(o.pk32, ES); AL(o.pk64, ES);
    AL(o.nt, M); AL(o.W64, M); AL(o.W32, M); AL(o.ws64, M); AL(o.ws32, M); AL(o.od64, M); AL(o.od32, M);
    t.general = 1;
    t.tmax = o.stride;
    t.lin = o.lin; t.w64 = o.w64; t.w32 = o.w32; t.nt = o.nt; t.W64 = o.W64; t.W32 = o.W32;
    t.ws64 = o.ws64; t.ws32 = o.ws32; t.od64 = o.od64; t.od32 = o.od32; t.pk32 = o.pk32; t.pk64 = o.pk64;
    h->d_off = o.off;  // Galerkin, coarsest and transposed builds read the assembled rows
  }
  // vectors
  const size_t N = size_t(h->n) * h->n;
  AL(h->X, N);
  AL(h->Xb, N);
  AL(h->Uprev, N);
  AL(h->Uprev2, N);
  AL(h->R, N);
  AL(h->Xpi, N);
  AL(h->Fvec, N);
  AL(h->Ub, N);
  AL(h->F, N * h->nf);
  AL(h->F32, N * h->nf);
  if (h->f_cb) {
    AL(h->Gcb, N * h->nf);
    h->G = h->Gcb;
  }
  if (h->psi_cb) {
    AL(h->Psicb, N);
    h->Psi = h->Psicb;
  }
  AL(h->policy, size_t(h->m) * h->m);
  const bool p64 = h->o.precision == 0;
  KBuf &k = h->kb;
  if (p64) {
    AL(k.r64, N); AL(k.rh64, N); AL(k.p64, N); AL(k.v64, N); AL(k.s64, N); AL(k.t64, N);
    AL(k.ph64, N); AL(k.sh64, N);
  } else {
    AL(k.r32, N); AL(k.rh32, N); AL(k.p32, N); AL(k.v32, N); AL(k.s32, N); AL(k.t32, N);
    AL(k.ph32, N); AL(k.sh32, N); AL(k.e32, N);
  }
  // multigrid levels
  h->cl[0].R = R0;
  for (int l = 0; l < h->L; ++l) {
    CoarseBuf &cb = h->cl[l];
    const size_t Nl = size_t(cb.n) * cb.n;
    VBuf &v = h->vb[l];
    if (p64) { AL(v.x64, Nl); AL(v.t64, Nl); AL(v.r64, Nl); AL(v.b64, Nl); }
    else { AL(v.x32, Nl); AL(v.t32, Nl); AL(v.r32, Nl); AL(v.b32, Nl); }
    if (l == 0) continue;
    cb.R = (h->cl[l - 1].R + 2) / 2;
    cb.win = (2 * cb.R + 1) * (2 * cb.R + 1);
    cb.cap = cb.m * cb.m;
    AL(cb.cls, size_t(cb.m) * cb.m);
    AL(cb.d_nexpl, 1);
    AL(cb.erow, size_t(cb.cap));
    if (p64) AL(cb.ewin64, size_t(cb.win) * cb.cap);
    else AL(cb.ewin32, size_t(cb.win) * cb.cap);
  }
  if (h->L > 1) {
    const size_t m1 = size_t(h->cl[1].m);
    AL(h->chunk_scratch, 2 * ((m1 * m1 + 255) / 256) + 2);
  }
  set_tail(h);
  {
    const sl_status ts = alloc_tail_image(h);
    if (ts != SL_OK) return ts;
  }
  const int mc = h->cl[h->L - 1].m;
  AL(h->cwork, size_t(2) * mc * mc * mc * mc);
  if (p64) AL(h->Ainv64, size_t(mc) * mc * mc * mc);
  else AL(h->Ainv32, size_t(mc) * mc * mc * mc);
  // reductions
  AL(h->S, 1);
  AL(h->S32, 1);
  AL(h->partials, size_t(2) * kRedBlocks + 2 * 65536);
  AL(h->counter, 1);
  AL(h->d_maxd, 2);
  AL(h->d_changes, 1);
  AL(h->d_flags, 1);
  AL(h->d_count, 1);
  AL(h->ctl, 1);
  h->tab.tma = h->general ? 0 : std::max(0, std::min(2, h->o.fine_tma));
  h->tab.tma_err = &h->ctl->tma_err;
  CK(cudaMallocHost(reinterpret_cast<void **>(&h->h_ctl), sizeof(DevCtl)));
  std::memset(h->h_ctl, 0, sizeof(DevCtl));
  CK(cudaMallocHost(reinterpret_cast<void **>(&h->hS), sizeof(BicgScalars)));
  CK(cudaMallocHost(reinterpret_cast<void **>(&h->h_maxd), 2 * sizeof(double)));
  CK(cudaMallocHost(reinterpret_cast<void **>(&h->h_changes), sizeof(unsigned long long)));
  CK(cudaMallocHost(reinterpret_cast<void **>(&h->h_flags), sizeof(int)));
  CK(cudaMallocHost(reinterpret_cast<void **>(&h->h_count), sizeof(int)));
  CK(cudaDeviceSynchronize());
  return SL_OK;
}

sl_status sl_hjb_create(sl_hjb **out, const sl_grid *g, const sl_controls *c, const sl_source *src,
                        const sl_opts *opts, void *stream) {
  (void)stream;
  if (!out) return SL_EINVAL;
  *out = nullptr;
  sl_hjb *h = new (std::nothrow) sl_hjb();
  if (!h) return SL_ENOMEM;
  sl_status st = create_impl(h, g, c, src, opts);
  if (st != SL_OK) {
    std::fprintf(stderr, "sl_hjb_create: %s\n", h->err.c_str());
    sl_hjb_destroy(h);
    return st;
  }
  *out = h;
  return SL_OK;
}

sl_status sl_hjb_step(sl_hjb *h, double *u, double t_n, double dt, uint8_t *pol_out, sl_stats *st,
                      void *stream) {
  if (!h || !u) return SL_EINVAL;
  if (st) std::memset(st, 0, sizeof(*st));
  return step_any(h, u, t_n, dt, pol_out, st, static_cast<cudaStream_t>(stream));
}

sl_status sl_hjb_solve(sl_hjb *h, double *u, double t0, double T, int n_steps, uint8_t *pol_out,
                       sl_stats *st, void *stream) {
  if (!h || !u || n_steps < 1 || !(T > 0)) return SL_EINVAL;
  if (st) std::memset(st, 0, sizeof(*st));
  const double dt = T / n_steps;
  for (int i = 1; i <= n_steps; ++i) {
    sl_status r = step_any(h, u, t0 + i * dt, dt, pol_out, st, static_cast<cudaStream_t>(stream));
    if (r != SL_OK) return r;
  }
  return SL_OK;
}

sl_status sl_hjb_reset(sl_hjb *h) {
  if (!h) return SL_EINVAL;
  h->have_policy = false;
  h->have_prev2 = false;
  h->hier_valid = false;
  h->changes_since_build = 0;
  return SL_OK;
}

sl_status sl_hjb_improve(sl_hjb *h, const double *x_ext, double t, uint8_t *pol_out,
                         long long *changes, void *stream) {
  if (!h || !x_ext) return SL_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  sl_status r = coef(h, t, h->X, s);
  if (r != SL_OK) return r;
  long long ch = 0;
  r = improve(h, x_ext, &ch, s);
  if (r != SL_OK) return r;
  h->changes_since_build += ch;
  h->hier_valid = h->hier_valid && ch == 0;
  if (changes) *changes = ch;
  if (pol_out) CK(cudaMemcpyAsync(pol_out, h->policy, size_t(h->m) * h->m, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  return SL_OK;
}

sl_status sl_hjb_set_policy(sl_hjb *h, const uint8_t *pol, void *stream) {
  if (!h || !pol) return SL_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaMemcpyAsync(h->policy, pol, size_t(h->m) * h->m, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  h->have_policy = true;
  h->hier_valid = false;
  return SL_OK;
}

sl_status sl_hjb_build_hierarchy(sl_hjb *h, double dt, void *stream) {
  if (!h || !(dt > 0)) return SL_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  sl_status r = build_hierarchy(h, dt, s);
  if (r != SL_OK) return r;
  CK(cudaStreamSynchronize(s));
  return SL_OK;
}

sl_status sl_hjb_apply(sl_hjb *h, int level, int precision, const void *x, void *y, void *stream) {
  if (!h || !x || !y || level < 0 || level >= h->L) return SL_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (level > 0 && (!h->hier_valid || precision != h->o.precision || h->o.precond != 0))
    return fail(h, SL_EINVAL, "coarse levels need a built V-cycle hierarchy in the handle's precision");
  const double dt = h->hier_valid ? h->hier_dt : (h->class_valid ? h->class_dt : -1.0);
  if (level == 0 && !(dt > 0)) return fail(h, SL_EINVAL, "build the hierarchy first (it fixes dt)");
  if (precision == 0)
    level_op<double>(h, level, OP_APPLY, dt, static_cast<const double *>(x), nullptr,
                     static_cast<double *>(y), s);
  else
    level_op<float>(h, level, OP_APPLY, dt, static_cast<const float *>(x), nullptr,
                    static_cast<float *>(y), s);
  CK(cudaGetLastError());
  return SL_OK;
}

sl_status sl_hjb_vcycle(sl_hjb *h, int precision, const void *b, void *x, void *stream) {
  if (!h || !b || !x) return SL_EINVAL;
  if (h->o.precond != 0) return fail(h, SL_EINVAL, "the V-cycle needs precond 0");
  if (!h->hier_valid || precision != h->o.precision)
    return fail(h, SL_EINVAL, "V-cycle needs a built hierarchy in the handle's precision");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  sl_status r = precision == 0
                    ? vcycle<double>(h, 0, h->hier_dt, static_cast<const double *>(b), static_cast<double *>(x), s)
                    : vcycle<float>(h, 0, h->hier_dt, static_cast<const float *>(b), static_cast<float *>(x), s);
  if (r != SL_OK) return r;
  CK(cudaStreamSynchronize(s));
  return SL_OK;
}

sl_status sl_hjb_vcycle_noalloc(sl_hjb *h, int precision, const void *b, void *x, void *stream) {
  if (!h || !b || !x) return SL_EINVAL;
  if (h->o.precond != 0) return fail(h, SL_EINVAL, "the V-cycle needs precond 0");
  if (!h->hier_valid || precision != h->o.precision)
    return fail(h, SL_EINVAL, "V-cycle needs a built hierarchy in the handle's precision");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return precision == 0
             ? vcycle_noalloc_T<double>(h, static_cast<const double *>(b), static_cast<double *>(x), s)
             : vcycle_noalloc_T<float>(h, static_cast<const float *>(b), static_cast<float *>(x), s);
}

sl_status sl_hjb_linear_solve(sl_hjb *h, const double *u_prev, double *x_ext, double t, double dt,
                              sl_stats *st, void *stream) {
  if (!h || !u_prev || !x_ext || !(dt > 0)) return SL_EINVAL;
  if (!h->have_policy) return fail(h, SL_EINVAL, "no policy set");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (st) std::memset(st, 0, sizeof(*st));
  const size_t N = NN(h, 0);
  CK(cudaMemcpyAsync(h->Uprev, u_prev, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->X, x_ext, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  sl_status r = coef(h, t, h->X, s);
  if (r != SL_OK) return r;
  if (!h->hier_valid || h->hier_dt != dt) {
    r = build_hierarchy(h, dt, s);
    if (r != SL_OK) return r;
  }
  r = linear_solve(h, dt, st, s);
  CK(cudaMemcpyAsync(x_ext, h->X, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  return r;
}

sl_status sl_hjb_solve_record(sl_hjb *h, double *u, double t0, double T, int n_steps, int ckpt_every,
                              sl_stats *st, void *stream) {
  if (!h || !u || n_steps < 1 || !(T > 0) || ckpt_every < 1) return SL_EINVAL;
  if (st) std::memset(st, 0, sizeof(*st));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->rec_valid = false;
  const size_t M = size_t(h->m) * h->m, NNf = size_t(h->n) * h->n;
  const int k = std::min(ckpt_every, n_steps);
  const double dt = T / n_steps;
  sl_status r = dgrow(h, &h->rec_pol, &h->rec_pol_cap, size_t(n_steps) * M);
  if (r == SL_OK) r = dgrow(h, &h->rec_U, &h->rec_U_cap, rec_checkpoints(n_steps, k) * NNf);
  if (r == SL_OK && k > 1) r = dgrow(h, &h->rec_seg, &h->rec_seg_cap, size_t(k - 1) * NNf);
  if (r != SL_OK) return r;
  h->rec_N = n_steps;
  h->rec_k = k;
  CK(cudaMemcpyAsync(h->rec_U, u, NNf * sizeof(double), cudaMemcpyDeviceToDevice, s));
  for (int i = 1; i <= n_steps; ++i) {
    h->rec_slot = h->rec_pol + size_t(i - 1) * M;
    r = step_impl(h, u, t0 + i * dt, dt, nullptr, st, s);
    h->rec_slot = nullptr;
    if (r != SL_OK) return r;
    double *dst = rec_stored(h, i);
    if (dst) CK(cudaMemcpyAsync(dst, u, NNf * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  h->rec_t0 = t0;
  h->rec_dt = dt;
  h->rec_valid = true;
  CK(cudaStreamSynchronize(s));
  return SL_OK;
}

sl_status sl_hjb_adjoint(sl_hjb *h, const double *w, double *dJ_dg, double *dJ_dG, int nparam,
                         const double *dsigma, double *dJ_dtheta, sl_stats *st, void *stream) {
  if (!h || !w || !dJ_dg || nparam < 0 || nparam > kMaxParams) return SL_EINVAL;
  if (nparam > 0 && (!dsigma || !dJ_dtheta)) return SL_EINVAL;
  if (!h->rec_valid) return fail(h, SL_EINVAL, "sl_hjb_adjoint needs a preceding sl_hjb_solve_record");
  if (nparam > 0 && h->general)
    return fail(h, SL_EINVAL, "dJ/dtheta needs an x-independent sigma (sl_controls.sigma)");
  if (h->o.precond != 0) return fail(h, SL_EINVAL, "the adjoint's transposed V-cycle needs precond 0");
  if (st) std::memset(st, 0, sizeof(*st));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  sl_status r = ensure_adjoint_buffers(h);
  if (r != SL_OK) return r;
  DTabView dv{};
  if (nparam > 0) {
    r = upload_dtables(h, nparam, dsigma, &dv);
    if (r != SL_OK) return r;
  }
  const size_t M = size_t(h->m) * h->m, NNf = size_t(h->n) * h->n;
  const double dt = h->rec_dt;
  CK(cudaMemsetAsync(h->d_dtheta, 0, kMaxParams * sizeof(double), s));
  if (dJ_dG) CK(cudaMemsetAsync(dJ_dG, 0, size_t(h->nf) * h->nq * NNf * sizeof(double), s));
  launch_interior_copy(h->n, w, h->lam, s);  // lambda_N = dJ/dU^N on the unknowns
  int seg = -1;
  for (int sn = h->rec_N; sn >= 1; --sn) {
    const double t = h->rec_t0 + sn * dt;
    const double *U = rec_stored(h, sn);
    if (!U) {
      const int c = sn / h->rec_k;
      if (c != seg) {
        r = recompute_segment(h, c, st, s);
        if (r != SL_OK) return r;
        seg = c;
      }
      U = h->rec_seg + size_t(sn - 1 - c * h->rec_k) * NNf;
    }
    CK(cudaMemcpyAsync(h->policy, h->rec_pol + size_t(sn - 1) * M, M, cudaMemcpyDeviceToDevice, s));
    h->have_policy = true;
    r = coef(h, t, h->X, s);  // tau_q(t_n) for the source gradient
    if (r != SL_OK) return r;
    r = build_hierarchy(h, dt, s);
    if (r == SL_OK) r = build_transposed(h, dt, s);
    if (r != SL_OK) return r;
    // A_n^T mu_n = lambda_n, started from lambda_n (A_n = I + O(dt))
    CK(cudaMemcpyAsync(h->mu, h->lam, NNf * sizeof(double), cudaMemcpyDeviceToDevice, s));
    h->transposed = true;
    r = linear_solve(h, dt, st, s);
    h->transposed = false;
    if (r != SL_OK) return r;
    if (st) st->steps += 1;
    if (dJ_dG) launch_adj_dG(h->n, h->nf, h->nq, h->policy, h->d_phi, h->d_tau, dt, h->mu, dJ_dG, s);
    if (nparam > 0) launch_adj_dtheta(h->tab, dv, h->policy, h->mu, U, dt, h->d_dpart, h->d_dtheta, s);
    // lambda_{n-1} = mu_n (U^{n-1} enters step n as -I)
    CK(cudaMemcpyAsync(h->lam, h->mu, NNf * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(dJ_dg, h->lam, NNf * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (nparam > 0)
    CK(cudaMemcpyAsync(dJ_dtheta, h->d_dtheta, nparam * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // the handle's policy and hierarchy now belong to step 1; the next march starts afresh
  h->hier_valid = false;
  h->have_prev2 = false;
  return SL_OK;
}

sl_status sl_hjb_set_launch(sl_hjb *h, int use_graphs, int coarse_tail_rows) {
  if (!h || use_graphs < 0 || use_graphs > 2) return SL_EINVAL;
  CK(cudaDeviceSynchronize());
  h->o.use_graphs = use_graphs;
  h->o.coarse_tail_rows = coarse_tail_rows;
  set_tail(h);
  sl_status st = alloc_tail_image(h);
  if (st != SL_OK) return st;
  tail_pack(h, nullptr);  // the current hierarchy's stencils for the new tail levels
  CK(cudaDeviceSynchronize());
  drop_graphs(h);
  return SL_OK;
}

sl_status sl_hjb_recorded_policy(sl_hjb *h, int step, uint8_t *policy_dev, void *stream) {
  if (!h || !policy_dev) return SL_EINVAL;
  if (!h->rec_valid || step < 1 || step > h->rec_N)
    return fail(h, SL_EINVAL, "sl_hjb_recorded_policy: no recorded march, or step out of range");
  const size_t M = size_t(h->m) * h->m;
  CK(cudaMemcpyAsync(policy_dev, h->rec_pol + size_t(step - 1) * M, M, cudaMemcpyDeviceToDevice,
                     static_cast<cudaStream_t>(stream)));
  return SL_OK;
}

sl_status sl_hjb_level_stats(const sl_hjb *h, int level, sl_level_stats *out) {
  if (!h || !out || level < 0 || level >= h->L) return SL_EINVAL;
  const CoarseBuf &c = h->cl[level];
  *out = sl_level_stats{};
  out->n = c.n;
  if (level == 0) {
    out->reach = h->halo;
    out->class_nnz = -1;
    return SL_OK;
  }
  out->reach = c.R;
  if (cudaDeviceSynchronize() != cudaSuccess) return SL_ECUDA;
  int nexpl = 0;
  if (cudaMemcpy(&nexpl, c.d_nexpl, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SL_ECUDA;
  std::vector<int32_t> cls(size_t(c.m) * c.m);
  if (cudaMemcpy(cls.data(), c.cls, cls.size() * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return SL_ECUDA;
  // only coefficients of interior columns count: a row next to the boundary may also carry
  // weights of boundary nodes, which multiply the Dirichlet zero of the correction
  auto interior = [&](int i1, int i2) { return i1 >= 1 && i1 <= c.m && i2 >= 1 && i2 <= c.m; };
  for (size_t I = 0; I < cls.size(); ++I) {
    const int k = cls[I];
    if (k < 0 || size_t(k) >= c.cnt_host.size()) continue;
    const int I1 = 1 + int(I % c.m), I2 = 1 + int(I / c.m);
    for (int t = 0; t < c.cnt_host[k]; ++t) {
      const int o = c.coff_host[size_t(k) * c.ctmax + t];
      const int dx = int(int16_t(o & 0xffff)), dy = o >> 16;
      out->class_nnz += interior(I1 + dx, I2 + dy);
    }
  }
  out->explicit_rows = nexpl;
  out->explicit_entries = (long long)nexpl * c.win;
  if (nexpl > 0) {
    const bool fp64 = h->o.precision == 0;
    std::vector<int32_t> erow(nexpl);
    if (cudaMemcpy(erow.data(), c.erow, nexpl * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return SL_ECUDA;
    std::vector<double> w64;
    std::vector<float> w32;
    const int Wd = 2 * c.R + 1;
    for (int e = 0; e < c.win; ++e) {  // one window entry of every explicit row at a time
      const int dy = e / Wd - c.R, dx = e % Wd - c.R;
      cudaError_t err;
      if (fp64) {
        w64.resize(nexpl);
        err = cudaMemcpy(w64.data(), c.ewin64 + size_t(e) * c.cap, nexpl * sizeof(double),
                         cudaMemcpyDeviceToHost);
      } else {
        w32.resize(nexpl);
        err = cudaMemcpy(w32.data(), c.ewin32 + size_t(e) * c.cap, nexpl * sizeof(float),
                         cudaMemcpyDeviceToHost);
      }
      if (err != cudaSuccess) return SL_ECUDA;
      for (int q = 0; q < nexpl; ++q) {
        const bool nz = fp64 ? w64[q] != 0.0 : w32[q] != 0.0f;
        out->explicit_nnz += nz && interior(erow[q] % c.n + dx, erow[q] / c.n + dy);
      }
    }
  }
  return SL_OK;
}

sl_status sl_hjb_level_info(const sl_hjb *h, int level, int *n, long long *explicit_rows, long long *nnz) {
  sl_level_stats st;
  const sl_status r = sl_hjb_level_stats(h, level, &st);
  if (r != SL_OK) return r;
  if (n) *n = st.n;
  if (explicit_rows) *explicit_rows = st.explicit_rows;
  if (nnz) *nnz = level == 0 ? -1 : st.class_nnz + st.explicit_nnz;
  return SL_OK;
}

int sl_hjb_num_levels(const sl_hjb *h) { return h ? h->L : 0; }

sl_status sl_hjb_inject_breakdown(sl_hjb *h, int iterations) {
  if (!h || iterations < 0) return SL_EINVAL;
  CK(cudaDeviceSynchronize());
  BicgScalars *both[2] = {h->S, h->S32};
  for (BicgScalars *S : both)
    CK(cudaMemcpy(&S->inject_bd, &iterations, sizeof(int), cudaMemcpyHostToDevice));
  return SL_OK;
}

long long sl_launch_count(void) { return launch_count(); }

}  // extern "C"
