// sl_fine.cu - fine-level kernels: source tables, policy improvement, matrix-free operator,
// FP64 HJB residual and grid transfers.
#include <cfloat>
#include <cmath>

#include "sl_launch.h"

namespace sl {

// ----------------------------------------------------------------------------- source tables
// F_m(t, x) = sum_q tau_q(t) G[m][q](x) on the full grid, and psi(t) on the boundary nodes of
// the iterate X and of Xb (the vector that is psi on the boundary and 0 inside).
__global__ void k_coef(const double *__restrict__ G, int nf, int nq, const double *__restrict__ tau,
                       const double *__restrict__ Psi, int npsi, const double *__restrict__ tpsi,
                       int n, double *__restrict__ F, float *__restrict__ F32,
                       double *__restrict__ Xext, double *__restrict__ Xb) {
  const size_t N = size_t(n) * n;
  for (size_t j = blockIdx.x * size_t(blockDim.x) + threadIdx.x; j < N;
       j += size_t(gridDim.x) * blockDim.x) {
    for (int m = 0; m < nf; ++m) {
      double acc = 0.0;
      for (int q = 0; q < nq; ++q) acc += tau[q] * G[(size_t(m) * nq + q) * N + j];
      F[size_t(m) * N + j] = acc;
      F32[size_t(m) * N + j] = float(acc);
    }
    const int i1 = int(j % n), i2 = int(j / n);
    if (i1 == 0 || i2 == 0 || i1 == n - 1 || i2 == n - 1) {
      double ps = 0.0;
      for (int q = 0; q < npsi; ++q) ps += tpsi[q] * Psi[size_t(q) * N + j];
      Xext[j] = ps;
      Xb[j] = ps;
    }
  }
}

void launch_coef(const double *G, int nf, int nq, const double *tau, const double *Psi, int npsi,
                 const double *tau_psi, int n, double *F, float *F32, double *Xext, double *Xb,
                 cudaStream_t s) {
  note_launch();
  k_coef<<<kRedBlocks, 256, 0, s>>>(G, nf, nq, tau, Psi, npsi, tau_psi, n, F, F32, Xext, Xb);
}

// ----------------------------------------------------------------------------- argmin
// Policy improvement (Eq. nonlinear_sys, linear search over the control set):
//   v_k(j) = sum_t w_t (X_{j+o_t} - X_j) + c_k X_j + sum_m phi_km F_m(j)
// alpha_j = lowest k with v_k <= v_min + tie_rel max(1, |v_min|), decided in FP64.
//
// Pass 1 screens all controls from a shared-memory tile of X (tile 32 x 8 nodes plus a halo
// of the longest tap).  With screen = 0 it is FP64; with screen = 1 it is FP32 on
// X - X_ref (X_ref the tile's centre value) and every screened value carries the rigorous
// rounding bound E described below, so the FP64 minimiser and all its FP64 near-ties lie in
// the candidate list.  Pass 2 re-evaluates the candidates in FP64 only when more than one
// survives; with one survivor it is the FP64 answer.
//
// Rounding bound of the FP32 screen (unit roundoff u = 2^-24), D = max |X - X_ref| over the
// staged tile, W = sum_t w_t, n_t taps:
//   |d_t - (X_nb - X_j)| <= 4 u D for the staged differences,
//   |sum w32 d - sum w (X_nb - X_j)| <= u D W (6 + 2 n_t)       (FMA chain, weights rounded),
//   |f32_k - f_k| <= (nf + 3) u sum_m |phi_km| |F_m|,  |c32 x32 - c x| <= 3 u |c| |X_j|,
//   final additions <= 2 u |v|.
// Two values that are both within their bounds differ by at most the sum of the bounds; the
// candidate window uses twice that sum plus the FP64 tie window.

constexpr int kTX = 32, kTY = 8;

template <typename T>
__device__ __forceinline__ T eval_smem(const FineTab &tab, const int32_t *__restrict__ slin,
                                       int e, const T *__restrict__ xs, int sidx) {
  const int nt = tab.nt[e];
  const T *w = tab_w<T>(tab);
  const T x0 = xs[sidx];
  T acc = T(0);
  for (int t = 0; t < nt; ++t) {
    const int ix = e * tab.tmax + t;
    acc = fma(__ldg(w + ix), xs[sidx + __ldg(slin + ix)] - x0, acc);
  }
  return acc;
}

__device__ __forceinline__ double eval_global64(const FineTab &tab, int e, const double *__restrict__ X,
                                                int j) {
  const int nt = tab.nt[e];
  const double x0 = X[j];
  double acc = 0.0;
  for (int t = 0; t < nt; ++t) {
    const int ix = e * tab.tmax + t;
    acc = fma(__ldg(tab.w64 + ix), __ldg(X + j + __ldg(tab.lin + ix)) - x0, acc);
  }
  return acc;
}

template <int SCREEN>
__global__ void __launch_bounds__(kTX *kTY) k_argmin(ArgminArgs a) {
  using TS = typename std::conditional<SCREEN, float, double>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TS *xs = reinterpret_cast<TS *>(smem_raw);
  __shared__ float red_max[kTX * kTY / 32];
  __shared__ unsigned red_cnt[kTX * kTY / 32];

  const FineTab &tab = a.tab;
  const int n = tab.n, m = tab.m;
  const int tid = threadIdx.y * kTX + threadIdx.x;
  const int o1 = 1 + blockIdx.x * kTX - a.halo;  // grid coordinate of staged column 0
  const int o2 = 1 + blockIdx.y * kTY - a.halo;
  // reference value of the tile (its centre node, clamped into the grid)
  double xref = 0.0;
  if (SCREEN) {
    const int c1 = min(1 + int(blockIdx.x) * kTX + kTX / 2, n - 1);
    const int c2 = min(1 + int(blockIdx.y) * kTY + kTY / 2, n - 1);
    xref = a.X[size_t(c2) * n + c1];
  }
  float dmax = 0.f;
  const int S = a.SW * a.SH;
  for (int s = tid; s < S; s += kTX * kTY) {
    const int g1 = o1 + s % a.SW, g2 = o2 + s / a.SW;
    TS v = TS(0);
    if (g1 >= 0 && g1 < n && g2 >= 0 && g2 < n) {
      const double xv = a.X[size_t(g2) * n + g1];
      if (SCREEN) {
        const double d = xv - xref;
        v = TS(d);
        dmax = fmaxf(dmax, float(fabs(d)) * (1.0f + 1.2e-7f));
      } else {
        v = TS(xv);
      }
    }
    xs[s] = v;
  }
  if (SCREEN) {
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((tid & 31) == 0) red_max[tid >> 5] = dmax;
  }
  __syncthreads();
  float D = 0.f;
  if (SCREEN) {
    for (int w = 0; w < kTX * kTY / 32; ++w) D = fmaxf(D, red_max[w]);
  }

  const int i1 = 1 + blockIdx.x * kTX + threadIdx.x;
  const int i2 = 1 + blockIdx.y * kTY + threadIdx.y;
  unsigned changed = 0;
  if (i1 <= m && i2 <= m) {
    const int j = i2 * n + i1;
    const int q1 = class_q(i1, n, tab.B), q2 = class_q(i2, n, tab.B);
    const int sidx = (threadIdx.y + a.halo) * a.SW + threadIdx.x + a.halo;
    const size_t N = size_t(n) * n;
    const int nf = a.nf;
    double Fv[4];
    float Fv32[4];
    double Fabs = 0.0;
    for (int mm = 0; mm < nf && mm < 4; ++mm) {
      Fv[mm] = a.F[mm * N + j];
      Fv32[mm] = a.F32[mm * N + j];
      Fabs += a.phimax[mm] * fabs(Fv[mm]);
    }
    const double Xj = a.X[j];
    // per-node part of the FP32 screen bound
    const double u = 5.9604644775390625e-8;
    const double E0 = SCREEN ? 1.001 * u * ((6.0 + 2.0 * tab.tmax) * a.Wmax_class[q2 * tab.Q + q1] * double(D)
                                             + (nf + 3.0) * Fabs + 3.0 * a.cmax * fabs(Xj))
                             : 0.0;
    // pass 1.  The candidate window is 2 (2 E0 + 4 u |v|) + 2 tie_rel max(1, |v|): twice what
    // two bounded values can differ by, so it stays rigorous when the comparison itself is
    // evaluated in the screening precision (its rounding is below the slack).
    const TS c1 = SCREEN ? TS(8.0 * u + 2.0 * a.tie_rel) : TS(2.0 * a.tie_rel * (1.0 + 1e-9));
    const TS M0 = SCREEN ? TS(4.0 * E0 * 1.0001 + 2.0 * a.tie_rel) : TS(0);
    TS vmin = TS(INFINITY);
    unsigned long long cand = 0ull;
    int ncand = 0;
    bool overflow = false;
    for (int k = 0; k < tab.K; ++k) {
      const int e = (k * tab.Q + q2) * tab.Q + q1;
      TS v = eval_smem<TS>(tab, a.slin, e, xs, sidx);
      TS fk;
      if (SCREEN) {
        float f = 0.f;
        for (int mm = 0; mm < nf && mm < 4; ++mm) f = fmaf(__ldg(a.phi32 + k * nf + mm), Fv32[mm], f);
        fk = fmaf(tab.c32[k], float(Xj), f);
      } else {
        double f = 0.0;
        for (int mm = 0; mm < nf && mm < 4; ++mm) f = fma(__ldg(a.phi + k * nf + mm), Fv[mm], f);
        fk = fma(tab.c64[k], Xj, f);
      }
      v = v + fk;
      if (!(v == v)) continue;  // NaN never enters the candidate list
      const TS av = v < vmin ? (v < TS(0) ? -v : v) : (vmin < TS(0) ? -vmin : vmin);
      const TS av1 = av > TS(1) ? av : TS(1);
      const TS margin = SCREEN ? M0 + c1 * av1 : c1 * av1;
      if (v < vmin) {
        if (v < vmin - margin) {
          cand = (unsigned long long)k;
          ncand = 1;
          overflow = false;
        } else {
          if (ncand < kMaxCand) cand |= (unsigned long long)k << (8 * ncand++);
          else overflow = true;
        }
        vmin = v;
      } else if (v <= vmin + margin) {
        if (ncand < kMaxCand) cand |= (unsigned long long)k << (8 * ncand++);
        else overflow = true;
      }
    }
    int best = -1;
    if (ncand == 1 && !overflow) {
      best = int(cand & 0xffull);
    } else if (ncand > 1 || overflow) {
      // pass 2: exact FP64 decision among the candidates (all controls on overflow)
      const int cnt = overflow ? tab.K : ncand;
      double vm = INFINITY;
      for (int c = 0; c < cnt; ++c) {
        const int k = overflow ? c : int((cand >> (8 * c)) & 0xffull);
        const int e = (k * tab.Q + q2) * tab.Q + q1;
        double f = 0.0;
        for (int mm = 0; mm < nf && mm < 4; ++mm) f = fma(__ldg(a.phi + k * nf + mm), Fv[mm], f);
        const double v = eval_global64(tab, e, a.X, j) + fma(tab.c64[k], Xj, f);
        vm = fmin(vm, v);
      }
      const double thr = vm + a.tie_rel * fmax(1.0, fabs(vm));
      for (int c = 0; c < cnt && best < 0; ++c) {
        const int k = overflow ? c : int((cand >> (8 * c)) & 0xffull);
        const int e = (k * tab.Q + q2) * tab.Q + q1;
        double f = 0.0;
        for (int mm = 0; mm < nf && mm < 4; ++mm) f = fma(__ldg(a.phi + k * nf + mm), Fv[mm], f);
        const double v = eval_global64(tab, e, a.X, j) + fma(tab.c64[k], Xj, f);
        if (v <= thr) best = k;
      }
    }
    const int pidx = (i2 - 1) * m + (i1 - 1);
    if (best < 0) {
      atomicOr(a.flags, 1);
    } else {
      const uint8_t old = a.policy[pidx];
      if (old != uint8_t(best)) {
        changed = 1;
        a.policy[pidx] = uint8_t(best);
      }
    }
  }
  // count changed rows
  unsigned c = __reduce_add_sync(0xffffffffu, changed);
  if ((tid & 31) == 0) red_cnt[tid >> 5] = c;
  __syncthreads();
  if (tid == 0) {
    unsigned tot = 0;
    for (int w = 0; w < kTX * kTY / 32; ++w) tot += red_cnt[w];
    if (tot) atomicAdd(a.changes, (unsigned long long)tot);
  }
}

cudaError_t launch_argmin(const ArgminArgs &a, cudaStream_t s) {
  dim3 blk(kTX, kTY), grd((a.tab.m + kTX - 1) / kTX, (a.tab.m + kTY - 1) / kTY);
  const size_t bytes = size_t(a.SW) * a.SH * (a.screen ? sizeof(float) : sizeof(double));
  cudaError_t err;
  if (a.screen) {
    err = cudaFuncSetAttribute(k_argmin<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (err != cudaSuccess) return err;
    note_launch();
    k_argmin<1><<<grd, blk, bytes, s>>>(a);
  } else {
    err = cudaFuncSetAttribute(k_argmin<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (err != cudaSuccess) return err;
    note_launch();
    k_argmin<0><<<grd, blk, bytes, s>>>(a);
  }
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------- fine operator
// (A x)_j = (1 + dt (W - c_k)) x_j - dt sum_t w_t x_{j+o_t}  (Eq. FullScheme, theta = 1; x has
// zero boundary entries, so boundary taps drop out as they belong to the right-hand side).
// Diagonal entry d_j = 1 + dt (W - c_k - w_self).
template <typename T, int OP>
__global__ void __launch_bounds__(256) k_fine_op(FineTab tab, const uint8_t *__restrict__ policy, T dt,
                                                 T omega, const T *__restrict__ x,
                                                 const T *__restrict__ b, T *__restrict__ y) {
  const int i1 = 1 + blockIdx.x * 32 + threadIdx.x;
  const int i2 = 1 + blockIdx.y * 8 + threadIdx.y;
  const int n = tab.n, m = tab.m;
  if (i1 > m || i2 > m) return;
  const int j = i2 * n + i1;
  const int k = policy[(i2 - 1) * m + (i1 - 1)];
  const int e = (k * tab.Q + class_q(i2, n, tab.B)) * tab.Q + class_q(i1, n, tab.B);
  const T W = tab_W<T>(tab)[e], c = tab_c<T>(tab)[k];
  const T d = T(1) + dt * (W - c - tab_ws<T>(tab)[e]);
  if (OP == OP_JACOBI0) {
    y[j] = omega * b[j] / d;
    return;
  }
  const int nt = tab.nt[e];
  const T *w = tab_w<T>(tab);
  T acc = T(0);
  for (int t = 0; t < nt; ++t) {
    const int ix = e * tab.tmax + t;
    acc = fma(__ldg(w + ix), __ldg(x + j + __ldg(tab.lin + ix)), acc);
  }
  const T xj = x[j];
  const T ax = (T(1) + dt * (W - c)) * xj - dt * acc;
  if (OP == OP_APPLY) y[j] = ax;
  else if (OP == OP_RESID) y[j] = b[j] - ax;
  else y[j] = xj + omega * (b[j] - ax) / d;
}

template <typename T>
void launch_fine_op(int op, const FineTab &tab, const uint8_t *policy, T dt, T omega, const T *x,
                    const T *b, T *y, cudaStream_t s) {
  dim3 blk(32, 8), grd((tab.m + 31) / 32, (tab.m + 7) / 8);
  switch (op) {
    case OP_APPLY: note_launch(); k_fine_op<T, OP_APPLY><<<grd, blk, 0, s>>>(tab, policy, dt, omega, x, b, y); break;
    case OP_RESID: note_launch(); k_fine_op<T, OP_RESID><<<grd, blk, 0, s>>>(tab, policy, dt, omega, x, b, y); break;
    case OP_JACOBI: note_launch(); k_fine_op<T, OP_JACOBI><<<grd, blk, 0, s>>>(tab, policy, dt, omega, x, b, y); break;
    default: note_launch(); k_fine_op<T, OP_JACOBI0><<<grd, blk, 0, s>>>(tab, policy, dt, omega, x, b, y); break;
  }
}
template void launch_fine_op<double>(int, const FineTab &, const uint8_t *, double, double,
                                     const double *, const double *, double *, cudaStream_t);
template void launch_fine_op<float>(int, const FineTab &, const uint8_t *, float, float,
                                    const float *, const float *, float *, cudaStream_t);

// ----------------------------------------------------------------------------- HJB residual
// r_j = F_j - (A X)_j = U^{n-1}_j - X_j + dt (sum_t w_t (X_{j+o_t} - X_j) + c_k X_j + f_k(j)),
// X carrying psi on the boundary (the boundary columns of Remark 2.2 are included here).
__global__ void __launch_bounds__(256) k_hjb_resid(FineTab tab, const uint8_t *__restrict__ policy,
                                                   const double *__restrict__ X,
                                                   const double *__restrict__ U,
                                                   const double *__restrict__ F,
                                                   const double *__restrict__ phi, int nf, double dt,
                                                   double *__restrict__ r) {
  const int i1 = 1 + blockIdx.x * 32 + threadIdx.x;
  const int i2 = 1 + blockIdx.y * 8 + threadIdx.y;
  const int n = tab.n, m = tab.m;
  if (i1 > m || i2 > m) return;
  const int j = i2 * n + i1;
  const int k = policy[(i2 - 1) * m + (i1 - 1)];
  const int e = (k * tab.Q + class_q(i2, n, tab.B)) * tab.Q + class_q(i1, n, tab.B);
  const size_t N = size_t(n) * n;
  double f = 0.0;
  for (int mm = 0; mm < nf; ++mm) f = fma(__ldg(phi + k * nf + mm), F[mm * N + j], f);
  const double Xj = X[j];
  const double v = eval_global64(tab, e, X, j) + (f + tab.c64[k] * Xj);
  r[j] = (U[j] - Xj) + dt * v;
}

void launch_hjb_resid(const FineTab &tab, const uint8_t *policy, const double *X,
                      const double *Uprev, const double *F, const double *phi, int nf, double dt,
                      double *r, cudaStream_t s) {
  dim3 blk(32, 8), grd((tab.m + 31) / 32, (tab.m + 7) / 8);
  note_launch();
  k_hjb_resid<<<grd, blk, 0, s>>>(tab, policy, X, Uprev, F, phi, nf, dt, r);
}

// ----------------------------------------------------------------------------- transfers
// Full weighting: b_c(I) = sum_{a in {-1,0,1}^2} w_a1 w_a2 r_f(2I + a), w = (1/4, 1/2, 1/4).
template <typename T>
__global__ void k_restrict(const T *__restrict__ rf, int nf, T *__restrict__ bc, int nc) {
  const int I1 = 1 + blockIdx.x * 32 + threadIdx.x;
  const int I2 = 1 + blockIdx.y * 8 + threadIdx.y;
  if (I1 > nc - 2 || I2 > nc - 2) return;
  const T *r0 = rf + size_t(2 * I2) * nf + 2 * I1;
  const T rowm = T(0.25) * r0[-nf - 1] + T(0.5) * r0[-nf] + T(0.25) * r0[-nf + 1];
  const T row0 = T(0.25) * r0[-1] + T(0.5) * r0[0] + T(0.25) * r0[1];
  const T rowp = T(0.25) * r0[nf - 1] + T(0.5) * r0[nf] + T(0.25) * r0[nf + 1];
  bc[size_t(I2) * nc + I1] = T(0.25) * rowm + T(0.5) * row0 + T(0.25) * rowp;
}

// Bilinear prolongation and correction: x_f(i) += sum_J P_{iJ} x_c(J).
template <typename T>
__global__ void k_prolong_add(const T *__restrict__ xc, int nc, T *__restrict__ xf, int nf) {
  const int i1 = 1 + blockIdx.x * 32 + threadIdx.x;
  const int i2 = 1 + blockIdx.y * 8 + threadIdx.y;
  if (i1 > nf - 2 || i2 > nf - 2) return;
  const int J1 = i1 >> 1, J2 = i2 >> 1;
  const bool odd1 = i1 & 1, odd2 = i2 & 1;
  T v;
  const T *c0 = xc + size_t(J2) * nc + J1;
  if (!odd1 && !odd2) v = c0[0];
  else if (odd1 && !odd2) v = T(0.5) * (c0[0] + c0[1]);
  else if (!odd1 && odd2) v = T(0.5) * (c0[0] + c0[nc]);
  else v = T(0.25) * ((c0[0] + c0[1]) + (c0[nc] + c0[nc + 1]));
  xf[size_t(i2) * nf + i1] += v;
}

template <typename T>
void launch_restrict(const T *rf, int nf, T *bc, int nc, cudaStream_t s) {
  dim3 blk(32, 8), grd((nc - 2 + 31) / 32, (nc - 2 + 7) / 8);
  note_launch();
  k_restrict<T><<<grd, blk, 0, s>>>(rf, nf, bc, nc);
}
template <typename T>
void launch_prolong_add(const T *xc, int nc, T *xf, int nf, cudaStream_t s) {
  dim3 blk(32, 8), grd((nf - 2 + 31) / 32, (nf - 2 + 7) / 8);
  note_launch();
  k_prolong_add<T><<<grd, blk, 0, s>>>(xc, nc, xf, nf);
}
template void launch_restrict<double>(const double *, int, double *, int, cudaStream_t);
template void launch_restrict<float>(const float *, int, float *, int, cudaStream_t);
template void launch_prolong_add<double>(const double *, int, double *, int, cudaStream_t);
template void launch_prolong_add<float>(const float *, int, float *, int, cudaStream_t);

}  // namespace sl
