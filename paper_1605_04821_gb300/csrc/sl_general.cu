// sl_general.cu - fine level with an x-dependent diffusion coefficient (Section 2.4,
// Problem A: sigma = sqrt(2) (sin(x1 + x2), cos(x1 + x2)), the same for every control) and a
// per-control drift.
//
// Row j of L^k is the sum of a diffusion part that depends on the node only (Scheme 2 with
// sigma(x_j), truncated at the boundary: Proposition 2.2, Eq. 2.9) and a drift part that
// depends on the control and on the distance to the boundary (A = B = 1/mu, Eq. 2.2).
// The node parts come from a per-row table built once on the host, the drift parts from the
// (control, boundary class) tables of the regular path.  After each policy improvement every
// row's entry of the fine table is assembled for its control, so that the operator, residual,
// Galerkin and transposed kernels of the regular path read it unchanged (fine_row_entry).
#include "sl_launch.h"

namespace sl {

constexpr int kGenThreads = 256;

// Entry I of the fine table for the row's current control: node taps, then drift taps.
__global__ void __launch_bounds__(kGenThreads) k_assemble_general(GeneralArgs g, FineTab dtab,
                                                                   const uint8_t *__restrict__ policy,
                                                                   const double *__restrict__ c64,
                                                                   double dt, double omega, int SW,
                                                                   GeneralOut o) {
  const int n = g.n, m = n - 2;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= m * m) return;
  const int i1 = 1 + I % m, i2 = 1 + I / m;
  const int k = policy[I];
  const int ed = (k * dtab.Q + class_q(i2, n, dtab.B)) * dtab.Q + class_q(i1, n, dtab.B);
  const int nn = g.nd_nt[I], ndr = dtab.nt[ed];
  const size_t base = size_t(I) * o.stride;
  double ws = 0.0;
  int t = 0;
  auto put = [&](int packed, double w) {
    const int dx = int(int16_t(packed & 0xffff)), dy = packed >> 16;
    const size_t ix = base + t;
    o.off[ix] = packed;
    o.lin[ix] = dy * n + dx;
    o.w64[ix] = w;
    o.w32[ix] = float(w);
    const int so = dy * SW + dx;
    const float w32 = float(w);
    o.pk32[ix] = make_int2(so, __float_as_int(w32));
    longlong2 p;
    p.x = so;
    p.y = __double_as_longlong(w);
    o.pk64[ix] = p;
    if ((dx | dy) == 0) ws += w;
    ++t;
  };
  for (int a = 0; a < nn; ++a) put(g.nd_off[size_t(I) * g.nd_stride + a], g.nd_w[size_t(I) * g.nd_stride + a]);
  for (int a = 0; a < ndr; ++a) put(g.dr_off[size_t(ed) * dtab.tmax + a], dtab.w64[size_t(ed) * dtab.tmax + a]);
  for (; t < o.stride; ++t) {  // zero the padding (kernels may loop over the full stride)
    const size_t ix = base + t;
    o.off[ix] = 0;
    o.lin[ix] = 0;
    o.w64[ix] = 0.0;
    o.w32[ix] = 0.f;
    o.pk32[ix] = make_int2(0, 0);
    longlong2 p;
    p.x = 0;
    p.y = 0;
    o.pk64[ix] = p;
  }
  const double W = g.nd_W[I] + dtab.W64[ed];
  o.nt[I] = uint8_t(nn + ndr);
  o.W64[I] = W;
  o.W32[I] = float(W);
  o.ws64[I] = ws;
  o.ws32[I] = float(ws);
  const double d = 1.0 + dt * (W - c64[k] - ws);
  o.od64[I] = omega / d;
  o.od32[I] = float(omega / d);
}

void launch_assemble_general(const GeneralArgs &g, const FineTab &dtab, const uint8_t *policy,
                             const double *c64, double dt, double omega, int SW, const GeneralOut &o,
                             cudaStream_t s) {
  const int M = (g.n - 2) * (g.n - 2);
  note_launch();
  k_assemble_general<<<(M + kGenThreads - 1) / kGenThreads, kGenThreads, 0, s>>>(g, dtab, policy, c64, dt,
                                                                                 omega, SW, o);
}

// Policy improvement on a general fine level, in FP64 (Eq. 1.10, linear search):
// v_k(j) = (L_sigma X)_j + (L_b^k X)_j + c_k X_j + sum_m phi_km F_m(j), where the diffusion
// part is the same for every control and is evaluated once per row.  alpha_j = lowest k with
// v_k <= v_min + tie_rel max(1, |v_min|).
__global__ void __launch_bounds__(kGenThreads) k_argmin_general(GeneralArgs g, FineTab dtab,
                                                                 const double *__restrict__ c64,
                                                                 const double *__restrict__ X,
                                                                 const double *__restrict__ F,
                                                                 const double *__restrict__ phi, int nf,
                                                                 double tie_rel, uint8_t *__restrict__ policy,
                                                                 unsigned long long *__restrict__ changes,
                                                                 int *__restrict__ flags) {
  const int n = g.n, m = n - 2;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned changed = 0;
  if (I < m * m) {
    const int i1 = 1 + I % m, i2 = 1 + I / m;
    const int j = i2 * n + i1;
    const double xj = X[j];
    double vd = 0.0;
    for (int a = 0; a < g.nd_nt[I]; ++a) {
      const int o = g.nd_off[size_t(I) * g.nd_stride + a];
      const int dx = int(int16_t(o & 0xffff)), dy = o >> 16;
      vd = fma(g.nd_w[size_t(I) * g.nd_stride + a], X[j + dy * n + dx] - xj, vd);
    }
    const size_t N = size_t(n) * n;
    const int q1 = class_q(i1, n, dtab.B), q2 = class_q(i2, n, dtab.B);
    auto value = [&](int k) {
      const int ed = (k * dtab.Q + q2) * dtab.Q + q1;
      double v = vd;
      for (int a = 0; a < dtab.nt[ed]; ++a) {
        const int o = g.dr_off[size_t(ed) * dtab.tmax + a];
        const int dx = int(int16_t(o & 0xffff)), dy = o >> 16;
        v = fma(dtab.w64[size_t(ed) * dtab.tmax + a], X[j + dy * n + dx] - xj, v);
      }
      double f = 0.0;
      for (int mm = 0; mm < nf; ++mm) f = fma(phi[k * nf + mm], F[mm * N + j], f);
      return v + fma(c64[k], xj, f);
    };
    double vmin = INFINITY;
    bool bad = false;
    for (int k = 0; k < dtab.K; ++k) {
      const double v = value(k);
      if (!(v == v)) bad = true;
      else vmin = fmin(vmin, v);
    }
    int best = -1;
    if (!bad && vmin < INFINITY) {
      const double thr = vmin + tie_rel * fmax(1.0, fabs(vmin));
      for (int k = 0; k < dtab.K && best < 0; ++k)
        if (value(k) <= thr) best = k;
    }
    if (best < 0) {
      atomicOr(flags, 1);
    } else if (policy[I] != uint8_t(best)) {
      policy[I] = uint8_t(best);
      changed = 1;
    }
  }
  const unsigned c = __reduce_add_sync(0xffffffffu, changed);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(changes, (unsigned long long)c);
}

void launch_argmin_general(const GeneralArgs &g, const FineTab &dtab, const double *c64, const double *X,
                           const double *F, const double *phi, int nf, double tie_rel, uint8_t *policy,
                           unsigned long long *changes, int *flags, cudaStream_t s) {
  const int M = (g.n - 2) * (g.n - 2);
  note_launch();
  k_argmin_general<<<(M + kGenThreads - 1) / kGenThreads, kGenThreads, 0, s>>>(g, dtab, c64, X, F, phi, nf,
                                                                               tie_rel, policy, changes, flags);
}

}  // namespace sl
