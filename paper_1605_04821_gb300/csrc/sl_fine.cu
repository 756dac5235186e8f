// sl_fine.cu - fine-level kernels: source tables, policy improvement, matrix-free operator,
// FP64 HJB residual and grid transfers.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdint>
#include <type_traits>

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
  const size_t st = size_t(gridDim.x) * blockDim.x;
  for (size_t j0 = blockIdx.x * size_t(blockDim.x) + threadIdx.x; j0 < N; j0 += 4 * st) {
    // four nodes per pass, the loads of each (m, q) issued for all four before the sums
    for (int m = 0; m < nf; ++m) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int q = 0; q < nq; ++q) {
        double g[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) g[u] = j0 + u * st < N ? G[(size_t(m) * nq + q) * N + j0 + u * st] : 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] += tau[q] * g[u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const size_t j = j0 + u * st;
        if (j < N) {
          F[size_t(m) * N + j] = acc[u];
          F32[size_t(m) * N + j] = float(acc[u]);
        }
      }
    }
  }
  // the 4 (n - 1) boundary nodes, walked side by side: bottom, right, top, left
  for (size_t b = blockIdx.x * size_t(blockDim.x) + threadIdx.x; b < size_t(4) * (n - 1); b += st) {
    const int side = int(b / (n - 1)), p = int(b % (n - 1));
    const int i1 = side == 0 ? p : side == 1 ? n - 1 : side == 2 ? n - 1 - p : 0;
    const int i2 = side == 0 ? 0 : side == 1 ? p : side == 2 ? n - 1 : n - 1 - p;
    const size_t j = size_t(i2) * n + i1;
    double ps = 0.0;
    for (int q = 0; q < npsi; ++q) ps += tpsi[q] * Psi[size_t(q) * N + j];
    Xext[j] = ps;
    Xb[j] = ps;
  }
}

void launch_coef(const double *G, int nf, int nq, const double *tau, const double *Psi, int npsi,
                 const double *tau_psi, int n, double *F, float *F32, double *Xext, double *Xb,
                 cudaStream_t s) {
  note_launch();
  k_coef<<<kRedBlocks, 256, 0, s>>>(G, nf, nq, tau, Psi, npsi, tau_psi, n, F, F32, Xext, Xb);
}

// ----------------------------------------------------------------------------- argmin
// Policy improvement (Eq. 1.10, linear search over the control set):
//   v_k(j) = sum_t w_t (X_{j+o_t} - X_j) + c_k X_j + sum_m phi_km F_m(j)
// alpha_j = lowest k with v_k <= v_min + tie_rel max(1, |v_min|), decided in FP64.
//
// Pass 1 screens all controls from a shared-memory tile of X (tile 32 x 8 nodes plus a halo of
// the longest tap).  With screen = 0 it is FP64.  With screen = 1 it is FP32 on the centred
// tile x'_s = fp32(X_s - c), c = X at the tile's centre node (the subtraction in FP64), and
// each screened value carries a rigorous bound E_k on its distance from the exact value;
// pass 2 decides in FP64 among the controls that the bounds cannot exclude, and with a single
// survivor that survivor is the FP64 answer.
//
// Bound of the FP32 screen (unit roundoff u = 2^-24, n_t taps, d_t = X_{j+o_t} - X_j,
// D = max |X_s - c| over the staged nodes inside the grid):
//   |x'_s - (X_s - c)| <= u |X_s - c|, so the difference dd_t = fp32(x'_nb - x'_j) satisfies
//   |dd_t - d_t| <= u |d_t| + 2 u (1 + u) D;
//   |sum_t w32_t dd_t - sum_t w_t d_t| <= (n_t + 4) u S + 2 u (1 + u) D W,  S = sum_t w_t |d_t|;
//   |f32_k - f_k| <= (nf + 3) u sum_m |phi_km| |F_m|;  |c32 x32 - c x| <= 3 u |c| |X_j|;
//   the two final additions <= 2 u |v~_k|.
// E_k doubles the sum of these terms (S taken from its FP32 evaluation), which also absorbs
// the rounding of the FP32 comparisons below.  With lb_k = v~_k - E_k and ub_k = v~_k + E_k the
// exact minimiser and its FP64 near-ties always satisfy lb_k <= min_l ub_l + tie window, and a
// control is dropped from the list only when another control's upper bound lies below its
// lower bound by more than the tie window.

constexpr int kTX = 32, kTY = 8;

// Bytes of the staged argmin tile, rounded up to 16 so that the per-control constants of the
// screen start aligned behind it.
__host__ __device__ inline size_t argmin_tile_bytes(int SW, int SH, bool screen) {
  return (size_t(SW) * SH * (screen ? sizeof(float) : sizeof(double)) + 15) / 16 * 16;
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

__device__ __forceinline__ double eval_smem64(const FineTab &tab, const int32_t *__restrict__ slin, int e,
                                              const double *__restrict__ xs, int sidx) {
  const int nt = tab.nt[e];
  const double x0 = xs[sidx];
  double acc = 0.0;
  for (int t = 0; t < nt; ++t) {
    const int ix = e * tab.tmax + t;
    acc = fma(__ldg(tab.w64 + ix), xs[sidx + __ldg(slin + ix)] - x0, acc);
  }
  return acc;
}

// FP32 screen of one control: returns sum_t w (dd_t) and S = sum_t w |dd_t| on the centred
// tile xs.  Taps are packed {tile offset, weight}; with TMAX > 0 the loop runs over the padded
// width, fully unrolled.
template <int TMAX>
__device__ __forceinline__ float eval_smem32(const FineTab &tab, int e, const float *__restrict__ xs,
                                             int sidx, float x0, float &S) {
  float acc = 0.f, sa = 0.f;
  if (TMAX > 0) {
#pragma unroll
    for (int t = 0; t < TMAX; ++t) {
      int o;
      float w;
      PackedTap<float>::get(tab, e * TMAX + t, o, w);
      const float dd = xs[sidx + o] - x0;
      acc = fmaf(w, dd, acc);
      sa = fmaf(w, fabsf(dd), sa);
    }
  } else {
    const int nt = tab.nt[e];
    for (int t = 0; t < nt; ++t) {
      int o;
      float w;
      PackedTap<float>::get(tab, e * tab.tmax + t, o, w);
      const float dd = xs[sidx + o] - x0;
      acc = fmaf(w, dd, acc);
      sa = fmaf(w, fabsf(dd), sa);
    }
  }
  S = sa;
  return acc;
}

// The same screen for an interior-class row, with the taps from the kernel parameter.
template <int TMAX>
__device__ __forceinline__ float eval_itap32(const ArgminITaps &it, int k, const float *__restrict__ xs,
                                             int sidx, float x0, float &S) {
  float acc = 0.f, sa = 0.f;
  const char *xb = reinterpret_cast<const char *>(xs + sidx);
#pragma unroll
  for (int t = 0; t < TMAX; ++t) {
    const int2 p = it.t[k * TMAX + t];
    const float dd = *reinterpret_cast<const float *>(xb + p.x) - x0;
    const float w = __int_as_float(p.y);
    acc = fmaf(w, dd, acc);
    sa = fmaf(w, fabsf(dd), sa);
  }
  S = sa;
  return acc;
}

__device__ __forceinline__ void cand_push(unsigned long long &cand, int &ncand, bool &overflow, int k) {
  if (ncand < kMaxCand) cand |= (unsigned long long)k << (8 * ncand++);
  else overflow = true;
}

template <int SCREEN, int TMAX>
__global__ void __launch_bounds__(kTX *kTY) k_argmin(const __grid_constant__ ArgminArgs a,
                                                     const __grid_constant__ ArgminITaps it) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned red_cnt[kTX * kTY / 32];
  __shared__ float red_max[kTX * kTY / 32];
  double *xs64 = reinterpret_cast<double *>(smem_raw);
  float *xs32 = reinterpret_cast<float *>(smem_raw);
  // screen: the per-control constants every lane reads in the same order, staged once per
  // block beside the tile (one broadcast shared load each instead of global loads and
  // address arithmetic per control): phi_k (zero-padded to four source functions) and
  // {c_k, W and tap count of the control's interior entry, 0}
  float4 *ctl_phi = reinterpret_cast<float4 *>(smem_raw + argmin_tile_bytes(a.SW, a.SH, true));
  float4 *ctl_cw = ctl_phi + a.tab.K;

  const FineTab &tab = a.tab;
  const int n = tab.n, m = tab.m;
  const int tid = threadIdx.y * kTX + threadIdx.x;
  const int o1 = 1 + blockIdx.x * kTX - a.halo;  // grid coordinate of staged column 0
  const int o2 = 1 + blockIdx.y * kTY - a.halo;
  // centre of the FP32 tile: X at the tile's middle node (inside the grid)
  double xc = 0.0;
  if (SCREEN) {
    const int c1 = min(1 + blockIdx.x * kTX + kTX / 2, n - 2), c2 = min(1 + blockIdx.y * kTY + kTY / 2, n - 2);
    xc = a.X[size_t(c2) * n + c1];
  }
  float dmax = 0.f;
  if (SCREEN) {
    // taps never leave the grid: the values staged outside it are unused (and not in D)
    stage_window<4, float>(xs32, a.SW, a.SH, threadIdx.x, threadIdx.y, [&](int r, int cc) {
      const int g2 = o2 + r, g1 = o1 + cc;
      const bool in = g1 >= 0 && g1 < n && g2 >= 0 && g2 < n;
      const float xd = float((in ? a.X[size_t(g2) * n + g1] : 0.0) - xc);
      if (in) dmax = fmaxf(dmax, fabsf(xd));
      return xd;
    }, 32 + 2 * a.halo);
  } else {
    stage_window<4, double>(xs64, a.SW, a.SH, threadIdx.x, threadIdx.y, [&](int r, int cc) {
      const int g2 = o2 + r, g1 = o1 + cc;
      return (g1 >= 0 && g1 < n && g2 >= 0 && g2 < n) ? a.X[size_t(g2) * n + g1] : 0.0;
    }, 32 + 2 * a.halo);
  }
  if (SCREEN) {
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((tid & 31) == 0) red_max[tid >> 5] = dmax;
    const bool inner_exists = n - 1 >= 2 * tab.B;
    for (int k = tid; k < tab.K; k += kTX * kTY) {
      float p[4];
#pragma unroll
      for (int mm = 0; mm < 4; ++mm) p[mm] = mm < a.nf ? __ldg(a.phi32 + k * a.nf + mm) : 0.f;
      ctl_phi[k] = make_float4(p[0], p[1], p[2], p[3]);
      const int ei = (k * tab.Q + tab.B) * tab.Q + tab.B;
      ctl_cw[k] = make_float4(tab.c32[k], inner_exists ? tab.W32[ei] : 0.f,
                              inner_exists ? float(tab.nt[ei]) : 0.f, 0.f);
    }
  }
  __syncthreads();
  float Dmax = 0.f;
  if (SCREEN)
    for (int w = 0; w < kTX * kTY / 32; ++w) Dmax = fmaxf(Dmax, red_max[w]);

  const int i1 = 1 + blockIdx.x * kTX + threadIdx.x;
  const int i2 = 1 + blockIdx.y * kTY + threadIdx.y;
  unsigned changed = 0;
  if (i1 <= m && i2 <= m) {
    const int j = i2 * n + i1;
    const int q1 = class_q(i1, n, tab.B), q2 = class_q(i2, n, tab.B);
    const int sidx = (threadIdx.y + a.halo) * a.SW + threadIdx.x + a.halo;
    const size_t N = size_t(n) * n;
    const int nf = a.nf;  // 1..4 (checked at create)
    // The node's FP64 values (X_j, F_m(j)) are loaded by the FP64 comparisons that use them
    // and are not held across the FP32 screen: with them live there, the compiler recomputed
    // their FP32 copies inside the control loop, about two FP64 -> FP32 conversions per
    // control and node, which filled GB300's narrow FP64 pipe (87 % busy).
    auto load_fv = [&](double (&Fv)[4]) {
#pragma unroll
      for (int mm = 0; mm < 4; ++mm) Fv[mm] = mm < nf ? a.F[mm * N + j] : 0.0;
    };
    unsigned long long cand = 0ull;
    int ncand = 0;
    bool overflow = false;
    if (SCREEN) {
      const float u = 5.9604645e-8f;
      float Fv32[4];
      float Fabs = 0.f;
#pragma unroll
      for (int mm = 0; mm < 4; ++mm) {
        Fv32[mm] = mm < nf ? a.F32[mm * N + j] : 0.f;
        if (mm < nf) Fabs = fmaf(a.phimax32[mm], fabsf(Fv32[mm]), Fabs);
      }
      const float xj32 = float(a.X[j]);
      // node-constant part of E_k: f-term, c-term and the centring term 2 u (1 + u) D
      // (Dmax * 1.001 covers D: the staged |x'| are within a factor 1 + u of |X - c|)
      const float Ef = u * ((nf + 3.0f) * Fabs * 1.001f + 3.0f * a.cmax32 * fabsf(xj32) * 1.001f);
      const float eta = 2.0f * u * Dmax * 1.001f + 1e-30f;
      const float x0 = xs32[sidx];
      const bool itap = TMAX > 0 && it.n > 0 && q1 == tab.B && q2 == tab.B;
      const float tw_rel = a.tie2_32;
      float Umin = INFINITY, Lmin = INFINITY;
      for (int k = 0; k < tab.K; ++k) {
        const int e = (k * tab.Q + q2) * tab.Q + q1;
        float S;
        const float acc = itap ? eval_itap32<TMAX>(it, k, xs32, sidx, x0, S)
                               : eval_smem32<TMAX>(tab, e, xs32, sidx, x0, S);
        const float4 ph = ctl_phi[k], cw = ctl_cw[k];
        // f_k = sum_m phi_km F_m, in the order m = 0, 1, ... (padding terms add +0)
        float f = fmaf(ph.x, Fv32[0], 0.f);
        f = fmaf(ph.y, Fv32[1], f);
        f = fmaf(ph.z, Fv32[2], f);
        if (nf > 3) f = fmaf(ph.w, Fv32[3], f);
        const float v = acc + fmaf(cw.x, xj32, f);
        if (!(v == v)) continue;  // NaN never enters the candidate list
        // tap count and W of the entry: the interior ones from shared memory; the count
        // becomes a float by the exponent trick (exact below 2^23), not a conversion
        const float ntf = itap ? cw.z : __int_as_float(0x4B000000 | int(tab.nt[e])) - 8388608.0f;
        const float We = itap ? cw.y : __ldg(tab.W32 + e);
        const float E = 2.0f * (u * ((ntf + 4.0f) * S * 1.001f + 2.0f * fabsf(v)) + Ef +
                                eta * We) + 4.0f * u * fabsf(v);
        const float lb = v - E, ub = v + E;
        const float tw = tw_rel * fmaxf(1.0f, fabsf(v)) + 4.0f * u * fabsf(v);
        Umin = fminf(Umin, ub);
        if (ub + tw < Lmin) {          // every listed control is excluded by this one
          cand = (unsigned long long)k;
          ncand = 1;
          overflow = false;
          Lmin = lb;
        } else if (lb <= Umin + tw) {
          cand_push(cand, ncand, overflow, k);
          Lmin = fminf(Lmin, lb);
        }
      }
    } else {
      double Fv[4];
      load_fv(Fv);
      const double Xj = a.X[j];
      double vmin = INFINITY;
      for (int k = 0; k < tab.K; ++k) {
        const int e = (k * tab.Q + q2) * tab.Q + q1;
        double f = 0.0;
        #pragma unroll
        for (int mm = 0; mm < 4; ++mm)
          if (mm < nf) f = fma(__ldg(a.phi + k * nf + mm), Fv[mm], f);
        const double v = eval_smem64(tab, a.slin, e, xs64, sidx) + fma(tab.c64[k], Xj, f);
        if (!(v == v)) continue;
        const double margin = 2.0 * a.tie_rel * fmax(1.0, fabs(v < vmin ? v : vmin)) * (1.0 + 1e-9);
        if (v < vmin) {
          if (v < vmin - margin) {
            cand = (unsigned long long)k;
            ncand = 1;
            overflow = false;
          } else {
            cand_push(cand, ncand, overflow, k);
          }
          vmin = v;
        } else if (v <= vmin + margin) {
          cand_push(cand, ncand, overflow, k);
        }
      }
    }
    int best = -1;
    if (ncand == 1 && !overflow) {
      best = int(cand & 0xffull);
    } else if (ncand > 1 || overflow) {
      // pass 2: exact FP64 decision among the candidates (all controls on overflow)
      const int cnt = overflow ? tab.K : ncand;
      double Fv[4];
      load_fv(Fv);
      const double Xj = a.X[j];
      double vm = INFINITY;
      double vals[kMaxCand];
      for (int c = 0; c < cnt; ++c) {
        const int k = overflow ? c : int((cand >> (8 * c)) & 0xffull);
        const int e = (k * tab.Q + q2) * tab.Q + q1;
        double f = 0.0;
        #pragma unroll
        for (int mm = 0; mm < 4; ++mm)
          if (mm < nf) f = fma(__ldg(a.phi + k * nf + mm), Fv[mm], f);
        const double v = eval_global64(tab, e, a.X, j) + fma(tab.c64[k], Xj, f);
        if (c < kMaxCand) vals[c] = v;
        vm = fmin(vm, v);
      }
      const double thr = vm + a.tie_rel * fmax(1.0, fabs(vm));
      for (int c = 0; c < cnt && best < 0; ++c) {
        const int k = overflow ? c : int((cand >> (8 * c)) & 0xffull);
        double v;
        if (c < kMaxCand) {
          v = vals[c];
        } else {
          const int e = (k * tab.Q + q2) * tab.Q + q1;
          double f = 0.0;
          #pragma unroll
        for (int mm = 0; mm < 4; ++mm)
          if (mm < nf) f = fma(__ldg(a.phi + k * nf + mm), Fv[mm], f);
          v = eval_global64(tab, e, a.X, j) + fma(tab.c64[k], Xj, f);
        }
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

// ----------------------------------------------------------------------------- argmin, two nodes
// The FP32 screen of k_argmin<1, TMAX> with two nodes per thread: rows ty and ty + 8 of a 32 x 16
// tile.  The nodes of the interior class share each tap's {offset, weight} (a uniform load) and
// keep their accumulators as FP32 pairs (__ffma2_rn / __fadd2_rn: per lane the rounding of a
// scalar FMA / add), so a tap costs two shared loads and four paired operations for both nodes.
// The screen's bound is the one of k_argmin, evaluated as
//   E_k = A_k S + 8 u |v| + (2 E_f + 2 eta W_k),   A_k = 2 u (n_t + 4) 1.001  (per control),
// the same sum of positive terms; its own rounding (a few u relative) is far inside the factor 2
// and the 1.001 margins of the derivation, so the screen stays rigorous and the FP64 decision
// among the survivors gives the same policy.  Nodes outside the interior class, and threads
// whose two nodes are not both interior, run k_argmin's per-node screen.
constexpr int kTY2 = 16;  // node rows per block

struct NodeScreen {
  int j, q1, q2, sidx;
  bool valid, itap;
  float Fv32[4], xj32, Ef, x0;
  unsigned long long cand;
  int ncand;
  bool overflow;
  float l1, l2, umin;  // smallest and second smallest lower bound, smallest upper bound
  int i1;              // the control of l1
};

// The two smallest lower bounds of a node's screen and the control of the smallest.
__device__ __forceinline__ void track_lb(NodeScreen &ns, float lb, int k) {
  if (lb < ns.l1) {
    ns.l2 = ns.l1;
    ns.l1 = lb;
    ns.i1 = k;
  } else {
    ns.l2 = fminf(ns.l2, lb);
  }
}

// k_argmin's screen of one node over every control (any table entry).
template <int TMAX>
__device__ __forceinline__ void screen_one(const ArgminArgs &a, const ArgminITaps &it, const float *xs32,
                                           const float4 *ctl_phi, const float4 *ctl_cw, float eta,
                                           NodeScreen &ns) {
  const FineTab &tab = a.tab;
  const float u = 5.9604645e-8f;
  const int nf = a.nf;
  float Umin = INFINITY, Lmin = INFINITY;
  for (int k = 0; k < tab.K; ++k) {
    const int e = (k * tab.Q + ns.q2) * tab.Q + ns.q1;
    float S;
    const float acc = ns.itap ? eval_itap32<TMAX>(it, k, xs32, ns.sidx, ns.x0, S)
                              : eval_smem32<TMAX>(tab, e, xs32, ns.sidx, ns.x0, S);
    const float4 ph = ctl_phi[k], cw = ctl_cw[k];
    float f = fmaf(ph.x, ns.Fv32[0], 0.f);
    f = fmaf(ph.y, ns.Fv32[1], f);
    f = fmaf(ph.z, ns.Fv32[2], f);
    if (nf > 3) f = fmaf(ph.w, ns.Fv32[3], f);
    const float v = acc + fmaf(cw.x, ns.xj32, f);
    if (!(v == v)) continue;
    const float ntf = ns.itap ? cw.z : __int_as_float(0x4B000000 | int(tab.nt[e])) - 8388608.0f;
    const float We = ns.itap ? cw.y : __ldg(tab.W32 + e);
    const float E = 2.0f * (u * ((ntf + 4.0f) * S * 1.001f + 2.0f * fabsf(v)) + ns.Ef + eta * We) +
                    4.0f * u * fabsf(v);
    const float lb = v - E, ub = v + E;
    const float tw = a.tie2_32 * fmaxf(1.0f, fabsf(v)) + 4.0f * u * fabsf(v);
    Umin = fminf(Umin, ub);
    track_lb(ns, lb, k);
    if (ub + tw < Lmin) {
      ns.cand = (unsigned long long)k;
      ns.ncand = 1;
      ns.overflow = false;
      Lmin = lb;
    } else if (lb <= Umin + tw) {
      cand_push(ns.cand, ns.ncand, ns.overflow, k);
      Lmin = fminf(Lmin, lb);
    }
  }
  ns.umin = Umin;
}

__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }

// The paired screen of two interior-class nodes (the taps from the kernel parameter).
template <int TMAX>
__device__ __forceinline__ void screen_pair(const ArgminArgs &a, const ArgminITaps &it, const float *xs32,
                                            const float4 *ctl_phi, const float4 *ctl_cw, float eta,
                                            NodeScreen &n0, NodeScreen &n1) {
  const int K = a.tab.K, nf = a.nf;
  const float u = 5.9604645e-8f;
  const char *xb0 = reinterpret_cast<const char *>(xs32 + n0.sidx);
  const char *xb1 = reinterpret_cast<const char *>(xs32 + n1.sidx);
  const float2 nx0 = make_float2(-n0.x0, -n1.x0);
  const float2 xj = make_float2(n0.xj32, n1.xj32);
  const float2 F0 = make_float2(n0.Fv32[0], n1.Fv32[0]), F1 = make_float2(n0.Fv32[1], n1.Fv32[1]);
  const float2 F2 = make_float2(n0.Fv32[2], n1.Fv32[2]), F3 = make_float2(n0.Fv32[3], n1.Fv32[3]);
  const float2 Ef2 = make_float2(2.0f * n0.Ef, 2.0f * n1.Ef);
  const float eta2 = 2.0f * eta, tw_rel = a.tie2_32;
  float Umin[2] = {INFINITY, INFINITY}, Lmin[2] = {INFINITY, INFINITY};
  NodeScreen *ns[2] = {&n0, &n1};
  for (int k = 0; k < K; ++k) {
    float2 acc = f2(0.f), sa = f2(0.f);
#pragma unroll
    for (int t = 0; t < TMAX; ++t) {
      const int2 p = it.t[k * TMAX + t];
      const float2 w = f2(__int_as_float(p.y));
      const float2 d = make_float2(*reinterpret_cast<const float *>(xb0 + p.x),
                                   *reinterpret_cast<const float *>(xb1 + p.x));
      const float2 dd = __fadd2_rn(d, nx0);
      acc = __ffma2_rn(w, dd, acc);
      sa = __ffma2_rn(w, make_float2(fabsf(dd.x), fabsf(dd.y)), sa);
    }
    const float4 ph = ctl_phi[k], cw = ctl_cw[k];
    float2 f = __ffma2_rn(f2(ph.x), F0, f2(0.f));
    f = __ffma2_rn(f2(ph.y), F1, f);
    f = __ffma2_rn(f2(ph.z), F2, f);
    if (nf > 3) f = __ffma2_rn(f2(ph.w), F3, f);
    const float2 v = __fadd2_rn(acc, __ffma2_rn(f2(cw.x), xj, f));
    const float2 av = make_float2(fabsf(v.x), fabsf(v.y));
    // E = A_k S + 8 u |v| + 2 E_f + 2 eta W_k  (cw.w = A_k, cw.y = W_k)
    const float2 E = __ffma2_rn(f2(cw.w), sa, __ffma2_rn(f2(8.0f * u), av, __ffma2_rn(f2(eta2), f2(cw.y), Ef2)));
    const float2 lb = __fadd2_rn(v, make_float2(-E.x, -E.y)), ub = __fadd2_rn(v, E);
    const float2 tw = __ffma2_rn(f2(4.0f * u), av,
                                 __fmul2_rn(f2(tw_rel), make_float2(fmaxf(1.0f, av.x), fmaxf(1.0f, av.y))));
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float vq = q ? v.y : v.x;
      if (!(vq == vq)) continue;
      const float lbq = q ? lb.y : lb.x, ubq = q ? ub.y : ub.x, twq = q ? tw.y : tw.x;
      Umin[q] = fminf(Umin[q], ubq);
      track_lb(*ns[q], lbq, k);
      if (ubq + twq < Lmin[q]) {
        ns[q]->cand = (unsigned long long)k;
        ns[q]->ncand = 1;
        ns[q]->overflow = false;
        Lmin[q] = lbq;
      } else if (lbq <= Umin[q] + twq) {
        cand_push(ns[q]->cand, ns[q]->ncand, ns[q]->overflow, k);
        Lmin[q] = fminf(Lmin[q], lbq);
      }
    }
  }
  n0.umin = Umin[0];
  n1.umin = Umin[1];
}

// The exact FP64 decision among a node's screened candidates (all controls on overflow), as in
// k_argmin's pass 2: the lowest index within the tie window of the FP64 minimum; -1 if none.
__device__ __forceinline__ int decide_fp64(const ArgminArgs &a, const NodeScreen &ns, double &vbest) {
  vbest = __longlong_as_double(0x7ff8000000000000ll);  // NaN: not evaluated in FP64
  if (ns.ncand == 1 && !ns.overflow) return int(ns.cand & 0xffull);
  if (ns.ncand == 0 && !ns.overflow) return -1;
  const FineTab &tab = a.tab;
  const int nf = a.nf, j = ns.j;
  const size_t N = size_t(tab.n) * tab.n;
  double Fv[4];
#pragma unroll
  for (int mm = 0; mm < 4; ++mm) Fv[mm] = mm < nf ? a.F[mm * N + j] : 0.0;
  const double Xj = a.X[j];
  const int cnt = ns.overflow ? tab.K : ns.ncand;
  auto value = [&](int k) {
    const int e = (k * tab.Q + ns.q2) * tab.Q + ns.q1;
    double f = 0.0;
#pragma unroll
    for (int mm = 0; mm < 4; ++mm)
      if (mm < nf) f = fma(__ldg(a.phi + k * nf + mm), Fv[mm], f);
    return eval_global64(tab, e, a.X, j) + fma(tab.c64[k], Xj, f);
  };
  double vm = INFINITY;
  double vals[kMaxCand];
  for (int c = 0; c < cnt; ++c) {
    const int k = ns.overflow ? c : int((ns.cand >> (8 * c)) & 0xffull);
    const double v = value(k);
    if (c < kMaxCand) vals[c] = v;
    vm = fmin(vm, v);
  }
  const double thr = vm + a.tie_rel * fmax(1.0, fabs(vm));
  for (int c = 0; c < cnt; ++c) {
    const int k = ns.overflow ? c : int((ns.cand >> (8 * c)) & 0xffull);
    const double v = c < kMaxCand ? vals[c] : value(k);
    if (v <= thr) {
      vbest = v;
      return k;
    }
  }
  return -1;
}

// The margin of a node's decision for ArgminArgs::gap: every other control's value exceeds the
// chosen one's by at least this much more than four tie windows, in exact arithmetic, at the X
// of this improvement (the other controls' screen lower bounds against the chosen value: its
// FP64 value rounded up, or its screen upper bound when it was the only candidate).  -inf when
// no margin is known.
__device__ __forceinline__ float decision_gap(const ArgminArgs &a, const NodeScreen &ns, int best, double vbest) {
  if (best < 0 || ns.overflow) return -INFINITY;
  if (a.tab.K == 1) return INFINITY;
  const float others = best == ns.i1 ? ns.l2 : ns.l1;
  float vup;
  if (vbest == vbest) {
    const float vf = float(vbest);
    vup = vf + fabsf(vf) * 1.2e-7f + 1e-30f;
  } else {
    vup = ns.umin;
  }
  if (!(others == others) || !(vup == vup) || others == INFINITY) return -INFINITY;
  const float u = 5.9604645e-8f;
  const float g = others - vup;
  return g - fabsf(g) * 1e-6f - 8.0f * u * fmaxf(fabsf(others), fabsf(vup)) -
         2.0f * a.tie2_32 * fmaxf(1.0f, fabsf(vup));
}

// Capped at four blocks of 256 threads per SM (64 registers): the skip test's extra live values
// would otherwise take the kernel to 80 registers and three blocks per SM (10.12 against 9.95 ms
// per step at 2049^2, K = 65).
template <int TMAX>
__global__ void __launch_bounds__(kTX *kTY, 4) k_argmin2(const __grid_constant__ ArgminArgs a,
                                                      const __grid_constant__ ArgminITaps it) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned red_cnt[kTX * kTY / 32];
  __shared__ float red_max[kTX * kTY / 32];
  const int SH = kTY2 + 2 * a.halo;
  float *xs32 = reinterpret_cast<float *>(smem_raw);
  float4 *ctl_phi = reinterpret_cast<float4 *>(smem_raw + argmin_tile_bytes(a.SW, SH, true));
  float4 *ctl_cw = ctl_phi + a.tab.K;
  const FineTab &tab = a.tab;
  const int n = tab.n, m = tab.m;
  const int tid = threadIdx.y * kTX + threadIdx.x;
  const int i1 = 1 + blockIdx.x * kTX + threadIdx.x;
  // Nodes whose last decision cannot change.  Since the last improvement (this step, same
  // coefficients) X has moved by dX = X - Xprev; over this tile and its halo a control value
  // has moved by at most Wabs osc(dX) + cmax max|dX| (osc: max dX - min dX), so a node whose
  // margin exceeds twice that keeps its control and its margin shrinks by the same amount.  A
  // block whose nodes all keep theirs stages nothing.  dX is formed in FP64 and its extremes
  // are taken on ordered integer images of the values (the integer pipe, not the narrow FP64
  // one); a NaN anywhere in the window disables the test.
  bool warp_keeps = false;  // every node of this warp keeps its control (skip its screen)
  float kept_gap[2] = {0.f, 0.f};
  if (a.gap && a.skip_flag && *a.skip_flag) {
    __shared__ long long sk_max[kTX * kTY / 32], sk_min[kTX * kTY / 32];
    __shared__ int sk_nan[kTX * kTY / 32];
    __shared__ float sk_shrink;
    const int WW = kTX + 2 * a.halo, HH = kTY2 + 2 * a.halo;
    const int b1 = 1 + blockIdx.x * kTX - a.halo, b2 = 1 + blockIdx.y * kTY2 - a.halo;
    long long omax = LLONG_MIN, omin = LLONG_MAX;
    int nan = 0;
    for (int idx = tid; idx < WW * HH; idx += kTX * kTY) {
      const int r = idx / WW, cc = idx - r * WW;
      const int g1 = b1 + cc, g2 = b2 + r;
      if (g1 < 0 || g1 >= n || g2 < 0 || g2 >= n) continue;
      const size_t gj = size_t(g2) * n + g1;
      const long long bits = __double_as_longlong(a.X[gj] - a.Xprev[gj]);
      nan |= (bits & 0x7fffffffffffffffll) > 0x7ff0000000000000ll;
      const long long ord = bits >= 0 ? bits : (bits ^ 0x7fffffffffffffffll);
      omax = max(omax, ord);
      omin = min(omin, ord);
    }
    for (int o = 16; o > 0; o >>= 1) {
      omax = max(omax, __shfl_xor_sync(0xffffffffu, omax, o));
      omin = min(omin, __shfl_xor_sync(0xffffffffu, omin, o));
      nan |= __shfl_xor_sync(0xffffffffu, nan, o);
    }
    if ((tid & 31) == 0) {
      sk_max[tid >> 5] = omax;
      sk_min[tid >> 5] = omin;
      sk_nan[tid >> 5] = nan;
    }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < kTX * kTY / 32; ++w) {
        omax = max(omax, sk_max[w]);
        omin = min(omin, sk_min[w]);
        nan |= sk_nan[w];
      }
      const long long bmax = omax >= 0 ? omax : (omax ^ 0x7fffffffffffffffll);
      const long long bmin = omin >= 0 ? omin : (omin ^ 0x7fffffffffffffffll);
      const double dmax = __longlong_as_double(bmax), dmin = __longlong_as_double(bmin);
      // each dX is X - Xprev rounded (relative error <= 2^-53): widen by that much of max|dX|
      const double amax = fmax(fabs(dmax), fabs(dmin));
      const double osc = (dmax - dmin) * (1.0 + 1e-15) + 4.5e-16 * amax;
      const double sh = 2.0 * (a.Wabs * osc + a.cmax * amax) * (1.0 + 1e-12);
      sk_shrink = (nan || !(sh < 1e30)) ? INFINITY : float(sh) * 1.000001f + 1e-30f;
    }
    __syncthreads();
    const float shrink = sk_shrink;
    bool keep = shrink < INFINITY;
    float g[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i2 = 1 + blockIdx.y * kTY2 + threadIdx.y + 8 * q;
      g[q] = INFINITY;
      if (i1 <= m && i2 <= m) {
        g[q] = a.gap[(i2 - 1) * m + (i1 - 1)];
        keep = keep && g[q] > shrink;
      }
    }
    if (__syncthreads_and(keep)) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int i2 = 1 + blockIdx.y * kTY2 + threadIdx.y + 8 * q;
        if (i1 <= m && i2 <= m) a.gap[(i2 - 1) * m + (i1 - 1)] = g[q] - shrink;
      }
      return;
    }
    // the block stages its tile for the warps that must decide; a warp whose nodes all keep
    // their controls only shrinks their margins
    warp_keeps = __all_sync(0xffffffffu, keep);
    kept_gap[0] = g[0] - shrink;
    kept_gap[1] = g[1] - shrink;
  }
  const int o1 = 1 + blockIdx.x * kTX - a.halo, o2 = 1 + blockIdx.y * kTY2 - a.halo;
  const int c1 = min(1 + blockIdx.x * kTX + kTX / 2, n - 2), c2 = min(1 + blockIdx.y * kTY2 + kTY2 / 2, n - 2);
  const double xc = a.X[size_t(c2) * n + c1];
  const float u = 5.9604645e-8f;
  float dmax = 0.f;
  stage_window<4, float>(xs32, a.SW, SH, threadIdx.x, threadIdx.y, [&](int r, int cc) {
    const int g2 = o2 + r, g1 = o1 + cc;
    const bool in = g1 >= 0 && g1 < n && g2 >= 0 && g2 < n;
    const float xd = float((in ? a.X[size_t(g2) * n + g1] : 0.0) - xc);
    if (in) dmax = fmaxf(dmax, fabsf(xd));
    return xd;
  }, 32 + 2 * a.halo);
  for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if ((tid & 31) == 0) red_max[tid >> 5] = dmax;
  const bool inner_exists = n - 1 >= 2 * tab.B;
  for (int k = tid; k < tab.K; k += kTX * kTY) {
    float p[4];
#pragma unroll
    for (int mm = 0; mm < 4; ++mm) p[mm] = mm < a.nf ? __ldg(a.phi32 + k * a.nf + mm) : 0.f;
    ctl_phi[k] = make_float4(p[0], p[1], p[2], p[3]);
    const int ei = (k * tab.Q + tab.B) * tab.Q + tab.B;
    const float ntf = inner_exists ? float(tab.nt[ei]) : 0.f;
    ctl_cw[k] = make_float4(tab.c32[k], inner_exists ? tab.W32[ei] : 0.f, ntf, 2.0f * u * (ntf + 4.0f) * 1.001f);
  }
  __syncthreads();
  float Dmax = 0.f;
  for (int w = 0; w < kTX * kTY / 32; ++w) Dmax = fmaxf(Dmax, red_max[w]);
  const float eta = 2.0f * u * Dmax * 1.001f + 1e-30f;

  NodeScreen ns[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    NodeScreen &s = ns[q];
    const int i2 = 1 + blockIdx.y * kTY2 + threadIdx.y + 8 * q;
    s.valid = i1 <= m && i2 <= m;
    s.cand = 0ull;
    s.ncand = 0;
    s.overflow = false;
    s.itap = false;
    s.l1 = s.l2 = s.umin = INFINITY;
    s.i1 = -1;
    if (!s.valid) continue;
    s.j = i2 * n + i1;
    s.q1 = class_q(i1, n, tab.B);
    s.q2 = class_q(i2, n, tab.B);
    s.sidx = (threadIdx.y + 8 * q + a.halo) * a.SW + threadIdx.x + a.halo;
    const size_t N = size_t(n) * n;
    float Fabs = 0.f;
#pragma unroll
    for (int mm = 0; mm < 4; ++mm) {
      s.Fv32[mm] = mm < a.nf ? a.F32[mm * N + s.j] : 0.f;
      if (mm < a.nf) Fabs = fmaf(a.phimax32[mm], fabsf(s.Fv32[mm]), Fabs);
    }
    s.xj32 = float(a.X[s.j]);
    s.Ef = u * ((a.nf + 3.0f) * Fabs * 1.001f + 3.0f * a.cmax32 * fabsf(s.xj32) * 1.001f);
    s.x0 = xs32[s.sidx];
    s.itap = TMAX > 0 && it.n > 0 && s.q1 == tab.B && s.q2 == tab.B;
  }
  if (warp_keeps) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!ns[q].valid) continue;
      const int i2 = 1 + blockIdx.y * kTY2 + threadIdx.y + 8 * q;
      a.gap[(i2 - 1) * m + (i1 - 1)] = kept_gap[q];
      ns[q].valid = false;
    }
  } else if (ns[0].valid && ns[1].valid && ns[0].itap && ns[1].itap) {
    screen_pair<TMAX>(a, it, xs32, ctl_phi, ctl_cw, eta, ns[0], ns[1]);
  } else {
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if (ns[q].valid) screen_one<TMAX>(a, it, xs32, ctl_phi, ctl_cw, eta, ns[q]);
  }
  unsigned changed = 0;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (!ns[q].valid) continue;
    double vbest;
    const int best = decide_fp64(a, ns[q], vbest);
    const int i2 = 1 + blockIdx.y * kTY2 + threadIdx.y + 8 * q;
    const int pidx = (i2 - 1) * m + (i1 - 1);
    if (a.gap) a.gap[pidx] = decision_gap(a, ns[q], best, vbest);
    if (best < 0) {
      atomicOr(a.flags, 1);
    } else if (a.policy[pidx] != uint8_t(best)) {
      changed += 1;
      a.policy[pidx] = uint8_t(best);
    }
  }
  const unsigned c = __reduce_add_sync(0xffffffffu, changed);
  if ((tid & 31) == 0) red_cnt[tid >> 5] = c;
  __syncthreads();
  if (tid == 0) {
    unsigned tot = 0;
    for (int w = 0; w < kTX * kTY / 32; ++w) tot += red_cnt[w];
    if (tot) atomicAdd(a.changes, (unsigned long long)tot);
  }
}

template <int SCREEN, int TMAX>
cudaError_t argmin_launch(const ArgminArgs &a, const ArgminITaps &it, dim3 grd, dim3 blk, size_t bytes,
                          cudaStream_t s) {
  note_launch();
  k_argmin<SCREEN, TMAX><<<grd, blk, bytes, s>>>(a, it);
  return cudaGetLastError();
}

cudaError_t launch_argmin(const ArgminArgs &a, const ArgminITaps &it, cudaStream_t s) {
  if (a.screen && a.tab.tmax == 12 && it.n > 0) {
    // two nodes per thread on 32 x 16 tiles (k_argmin2)
    dim3 blk(kTX, kTY), grd((a.tab.m + kTX - 1) / kTX, (a.tab.m + kTY2 - 1) / kTY2);
    const size_t bytes = argmin_tile_bytes(a.SW, kTY2 + 2 * a.halo, true) + 2 * size_t(a.tab.K) * sizeof(float4);
    note_launch();
    k_argmin2<12><<<grd, blk, bytes, s>>>(a, it);
    return cudaGetLastError();
  }
  dim3 blk(kTX, kTY), grd((a.tab.m + kTX - 1) / kTX, (a.tab.m + kTY - 1) / kTY);
  const size_t bytes = argmin_tile_bytes(a.SW, a.SH, a.screen) + (a.screen ? 2 * size_t(a.tab.K) * sizeof(float4) : 0);
  if (!a.screen) return argmin_launch<0, 0>(a, it, grd, blk, bytes, s);
  switch (a.tab.tmax) {
    case 8: return argmin_launch<1, 8>(a, it, grd, blk, bytes, s);
    case 12: return argmin_launch<1, 12>(a, it, grd, blk, bytes, s);
    case 16: return argmin_launch<1, 16>(a, it, grd, blk, bytes, s);
    case 20: return argmin_launch<1, 20>(a, it, grd, blk, bytes, s);
    default: return argmin_launch<1, 0>(a, it, grd, blk, bytes, s);
  }
}

// ----------------------------------------------------------------------------- fine operator
// (A x)_j = (1 + dt (W - c_k)) x_j - dt sum_t w_t x_{j+o_t}  (Eq. 2.11, theta = 1; x has
// zero boundary entries, so boundary taps drop out as they belong to the right-hand side).
// Diagonal entry d_j = 1 + dt (W - c_k - w_self).
//
// Each block stages a 32 x 32 tile of x plus a halo of the longest tap in shared memory; each
// thread computes kFineRPT = 4 rows of one column (i2 = base + ty + 8 r) independently (the
// policy changes too often along a column for rows to share their taps).  With a halo of ten
// nodes the 32 x 32 tile stages 2.6 values per row against 3.7 for a 32 x 16 one, which took
// the FP32 apply at 2049^2 from 36 to 33 us.  The rows' controls are read before the tile is
// staged.  Taps are packed {tile offset, weight} and the loop runs over the padded table width
// TMAX (unused slots carry weight 0 at offset 0), fully unrolled, so all table loads of a row
// are issued together.
constexpr int kFineRPT = 4;  // rows per thread: a block covers 32 x (8 kFineRPT) rows

template <typename T, int OP>
__device__ __forceinline__ void fine_finish(T *y, const T *b, int j, T xj, T ax, T od) {
  if (OP == OP_APPLY) y[j] = ax;
  else if (OP == OP_RESID) y[j] = b[j] - ax;
  else y[j] = xj + od * (b[j] - ax);
}

// Stages rows [o2, o2 + SH) x columns [o1, o1 + SW) of a full-grid vector into shared memory,
// with zeros outside the grid; tiles whose halo lies inside the grid skip the bounds checks.
// SW is the pitch of xs; WD columns are staged.
template <typename T>
__device__ __forceinline__ void stage_tile(T *xs, const T *__restrict__ x, int n, int o1, int o2, int SW,
                                           int WD, int SH, int tx, int ty) {
  if (o1 >= 0 && o2 >= 0 && o1 + WD <= n && o2 + SH <= n) {
    const T *src = x + size_t(o2) * n + o1;
    stage_window<4, T>(xs, SW, SH, tx, ty, [&](int r, int c) { return src[size_t(r) * n + c]; }, WD);
  } else {
    stage_window<4, T>(xs, SW, SH, tx, ty, [&](int r, int c) {
      const int g2 = o2 + r, g1 = o1 + c;
      return (g2 >= 0 && g2 < n && g1 >= 0 && g1 < n) ? x[size_t(g2) * n + g1] : T(0);
    }, WD);
  }
}

// Sum of w_t x_{j+o_t} over the taps of control k's interior entry, from the tap-major table;
// the taps are added in the order of the entry (t = 0, 1, ...), as on the general path.
template <typename T, int TMAX> struct InnerTaps;
template <int TMAX> struct InnerTaps<float, TMAX> {
  static __device__ __forceinline__ float sum(const FineTab &tab, int k, const float *xs, int sidx) {
    const int4 *p = tab.ipk32 + k;
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < TMAX / 2; ++t) {
      const int4 q = __ldg(p + t * tab.K);
      acc = fmaf(__int_as_float(q.y), xs[sidx + q.x], acc);
      acc = fmaf(__int_as_float(q.w), xs[sidx + q.z], acc);
    }
    return acc;
  }
  static __device__ __forceinline__ float Wc(const FineTab &tab, int k) { return tab.iWc32[k]; }
  static __device__ __forceinline__ float od(const FineTab &tab, int k) { return tab.iod32[k]; }
};
template <int TMAX> struct InnerTaps<double, TMAX> {
  static __device__ __forceinline__ double sum(const FineTab &tab, int k, const double *xs, int sidx) {
    const longlong2 *p = tab.ipk64 + k;
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < TMAX; ++t) {
      const longlong2 q = __ldg(p + t * tab.K);
      acc = fma(__longlong_as_double(q.y), xs[sidx + int(q.x)], acc);
    }
    return acc;
  }
  static __device__ __forceinline__ double Wc(const FineTab &tab, int k) { return tab.iWc64[k]; }
  static __device__ __forceinline__ double od(const FineTab &tab, int k) { return tab.iod64[k]; }
};

// The rows of tile (bx, by) (32 columns x 8 RPT rows) from the staged tile xs (pitch SW; the
// tile's column 0 is grid column 1 + 32 bx - halo); kr: the rows' controls.  Every fine
// operator kernel calls this, so all of them compute each row the same way.
// color: -1 for every row; 0 or 1 for a half-sweep of the two-colour Gauss-Seidel smoother, in
// which the Jacobi ops update only the rows with (i1 + i2) mod 2 == color and pass the others
// through (x for OP_JACOBI, 0 for OP_JACOBI0, whose start is x = 0).
template <typename T, int OP, int TMAX, int RPT>
__device__ __forceinline__ void fine_tile_rows(const FineTab &tab, T dt, T omega, const T *xs,
                                               const T *__restrict__ b, T *__restrict__ y, int halo,
                                               int SW, int bx, int by, const int (&kr)[RPT], int color) {
  const int n = tab.n, m = tab.m;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i1 = 1 + bx * 32 + tx;
  if (i1 > m) return;
  // a block whose rows all lie in the interior class (q1 = q2 = B) reads the tap-major
  // interior table, indexed by the control alone
  const int B = tab.B;
  const int r1 = bx * 32, r2 = by * (8 * RPT);
  const bool inner = TMAX > 0 && tab.ipk32 != nullptr && !tab.general && n - 1 >= 2 * B &&
                     1 + r1 >= B && r1 + 32 <= n - 1 - B && 1 + r2 >= B && r2 + 8 * RPT <= n - 1 - B;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int i2 = 1 + by * (8 * RPT) + ty + 8 * r;
    if (i2 > m) continue;
    const int k = kr[r];
    const int j = i2 * n + i1;
    if ((OP == OP_JACOBI || OP == OP_JACOBI0) && color >= 0 && ((i1 + i2) & 1) != color) {
      y[j] = OP == OP_JACOBI ? xs[(ty + 8 * r + halo) * SW + tx + halo] : T(0);
      continue;
    }
    if (inner) {
      if (OP == OP_JACOBI0) {
        y[j] = InnerTaps<T, TMAX>::od(tab, k) * b[j];
        continue;
      }
      const int sidx = (ty + 8 * r + halo) * SW + tx + halo;
      const T acc = InnerTaps<T, TMAX>::sum(tab, k, xs, sidx);
      const T xj = xs[sidx];
      const T diag = T(1) + dt * InnerTaps<T, TMAX>::Wc(tab, k);
      fine_finish<T, OP>(y, b, j, xj, diag * xj - dt * acc,
                         OP == OP_JACOBI ? InnerTaps<T, TMAX>::od(tab, k) : T(0));
      continue;
    }
    const int e = fine_row_entry(tab, k, i1, i2);
    if (OP == OP_JACOBI0) {
      y[j] = tab_od<T>(tab)[e] * b[j];
      continue;
    }
    const int sidx = (ty + 8 * r + halo) * SW + tx + halo;
    T acc = T(0);
    if (TMAX > 0) {
#pragma unroll
      for (int t = 0; t < TMAX; ++t) {
        int off;
        T w;
        PackedTap<T>::get(tab, e * TMAX + t, off, w);
        acc = fma(w, xs[sidx + off], acc);
      }
    } else {
      const int nt = tab.nt[e];
      for (int t = 0; t < nt; ++t) {
        int off;
        T w;
        PackedTap<T>::get(tab, e * tab.tmax + t, off, w);
        acc = fma(w, xs[sidx + off], acc);
      }
    }
    const T xj = xs[sidx];
    const T diag = T(1) + dt * (tab_W<T>(tab)[e] - tab_c<T>(tab)[k]);
    fine_finish<T, OP>(y, b, j, xj, diag * xj - dt * acc, OP == OP_JACOBI ? tab_od<T>(tab)[e] : T(0));
  }
}


template <typename T, int OP, int TMAX, int RPT = kFineRPT>
__global__ void __launch_bounds__(256) k_fine_op(FineTab tab, const uint8_t *__restrict__ policy, T dt, T omega,
                                                 const T *__restrict__ x, const T *__restrict__ b,
                                                 T *__restrict__ y, int halo, int SW, int color) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  const int n = tab.n, m = tab.m;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i1 = 1 + blockIdx.x * 32 + tx;
  // the rows' controls are read before the tile is staged, so that both loads are in flight
  int kr[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int i2 = 1 + blockIdx.y * (8 * RPT) + ty + 8 * r;
    kr[r] = i1 <= m && i2 <= m ? int(policy[(i2 - 1) * m + (i1 - 1)]) : 0;
  }
  if (OP != OP_JACOBI0) {
    stage_tile<T>(xs, x, n, 1 + blockIdx.x * 32 - halo, 1 + blockIdx.y * (8 * RPT) - halo, SW,
                  32 + 2 * halo, (8 * RPT) + 2 * halo, tx, ty);
    __syncthreads();
  }
  fine_tile_rows<T, OP, TMAX, RPT>(tab, dt, omega, xs, b, y, halo, SW, blockIdx.x, blockIdx.y, kr, color);
}

// ----------------------------------------------------------------------------- TMA fine operator
// The FP32 fine operator (apply, residual, Jacobi sweep) as a persistent kernel whose tiles are
// moved by the TMA unit.  Each block walks the 32 x 32-row tiles t = blockIdx.x, + gridDim.x,
// ...; while it computes one tile, the rows of its next interior tile are in flight into the
// other of two shared buffers, one cp.async.bulk global -> shared copy per tile row, completing
// on that buffer's mbarrier.  A bulk copy needs 16-byte-aligned addresses and a length that is
// a multiple of 16 bytes; a grid row of n = 2^j + 1 values is not, so each row is copied from
// its 16-byte-aligned start with its length rounded up, and the tile pitch SW is congruent to n
// mod 4 (and at least 3 columns wider than the 32 + 2 halo staged ones) so that every row keeps
// the same offset a0 (0..3 values) inside its 16 bytes in shared memory as in global memory;
// the tile then starts at buffer + a0.  The extra values at both ends of a row land in columns
// the taps never read.  Tiles at the boundary, whose halo leaves the grid, are staged by the
// threads with zeros outside the grid, as in k_fine_op.  A wait that does not complete within
// kTmaSpin polls sets *err (reported by the solver as SL_ETIMEOUT) and the tile is computed
// from whatever arrived; no wait is unbounded.
constexpr unsigned kTmaSpin = 1u << 20;

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes,
                                              unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// orders this thread's earlier generic shared accesses before later async-proxy (TMA) ones
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

struct TmaTiles {
  int tiles_x, ntiles;  // tiles per grid row, total
  int buf_floats;       // floats per shared buffer (multiple of 32)
  int *err;             // set to 1 when a wait gave up
};

// Issues (warp 0) the bulk copies of the interior tile with origin (o1, o2) into bf; one copy
// per row, all completing on bar, whose expected byte count lane 0 raises first.
__device__ __forceinline__ void tma_issue_tile(const float *__restrict__ x, int n, int o1, int o2, int WD,
                                               int SH, int SW, float *bf, unsigned long long *bar) {
  const int lane = threadIdx.x;
  unsigned bytes = 0;
  for (int r = lane; r < SH; r += 32) {
    const int ar = int((size_t(o2 + r) * n + o1) & 3);
    bytes += unsigned(((ar + WD + 3) & ~3) * 4);
  }
  for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
  if (lane == 0) mbar_arrive_expect_tx(bar, bytes);
  __syncwarp();
  const int a0 = int((size_t(o2) * n + o1) & 3);
  for (int r = lane; r < SH; r += 32) {
    const size_t g = size_t(o2 + r) * n + o1;
    const int ar = int(g & 3);
    bulk_copy_g2s(bf + (a0 + r * SW - ar), x + (g - ar), unsigned(((ar + WD + 3) & ~3) * 4), bar);
  }
}

template <int OP, int TMAX>
__global__ void __launch_bounds__(256) k_fine_op_tma(FineTab tab, const uint8_t *__restrict__ policy, float dt,
                                                     float omega, const float *__restrict__ x,
                                                     const float *__restrict__ b, float *__restrict__ y,
                                                     int halo, int SW, TmaTiles tt, int color) {
  constexpr int RPT = kFineRPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bar[2];
  float *buf[2] = {reinterpret_cast<float *>(smem_raw), reinterpret_cast<float *>(smem_raw) + tt.buf_floats};
  const int n = tab.n, m = tab.m;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int WD = 32 + 2 * halo, SH = 8 * RPT + 2 * halo;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto origin = [&](int t, int &o1, int &o2) {
    o1 = 1 + (t % tt.tiles_x) * 32 - halo;
    o2 = 1 + (t / tt.tiles_x) * (8 * RPT) - halo;
  };
  // the row copies stay inside the array: 3 values of rounding at either end of each row
  // (and a bulk copy needs a 16-byte-aligned shared address: otherwise every tile is staged
  // by the threads)
  const bool smem16 = (smem_addr(smem_raw) & 15u) == 0u;
  auto interior = [&](int o1, int o2) {
    return smem16 && o1 >= 3 && o2 >= 0 && o1 + WD + 3 <= n && o2 + SH <= n;
  };
  unsigned parity[2] = {0u, 0u};
  int cur = 0;
  int t = blockIdx.x;
  if (t < tt.ntiles && ty == 0) {
    int o1, o2;
    origin(t, o1, o2);
    if (interior(o1, o2)) tma_issue_tile(x, n, o1, o2, WD, SH, SW, buf[0], &bar[0]);
  }
  bool failed = false;
  for (; t < tt.ntiles; t += gridDim.x) {
    const int tn = t + gridDim.x;
    // prefetch the next tile into the other buffer (its readers finished before the last
    // __syncthreads of the previous iteration)
    if (tn < tt.ntiles && ty == 0) {
      int p1, p2;
      origin(tn, p1, p2);
      if (interior(p1, p2)) {
        fence_proxy_async_smem();
        tma_issue_tile(x, n, p1, p2, WD, SH, SW, buf[cur ^ 1], &bar[cur ^ 1]);
      }
    }
    const int bx = t % tt.tiles_x, by = t / tt.tiles_x;
    const int i1 = 1 + bx * 32 + tx;
    int kr[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int i2 = 1 + by * (8 * RPT) + ty + 8 * r;
      kr[r] = i1 <= m && i2 <= m ? int(policy[(i2 - 1) * m + (i1 - 1)]) : 0;
    }
    int o1, o2;
    origin(t, o1, o2);
    const float *xs;
    if (interior(o1, o2)) {
      unsigned spins = 0;
      while (!mbar_try_wait(&bar[cur], parity[cur])) {
        if (++spins >= kTmaSpin) {
          failed = true;
          break;
        }
      }
      parity[cur] ^= 1u;
      xs = buf[cur] + int((size_t(o2) * n + o1) & 3);
    } else {
      stage_tile<float>(buf[cur], x, n, o1, o2, SW, WD, SH, tx, ty);
      __syncthreads();
      xs = buf[cur];
    }
    fine_tile_rows<float, OP, TMAX, RPT>(tab, dt, omega, xs, b, y, halo, SW, bx, by, kr, color);
    __syncthreads();
    cur ^= 1;
  }
  if (failed) atomicExch(tt.err, 1);
}

// The TMA kernel for the FP32 ops that stage x, on the common tap stride 12, when x is
// 16-byte aligned and the grid has interior tiles; false: the caller launches k_fine_op.
// One tile per block, as k_fine_op, with the interior tile's rows copied by the TMA unit
// instead of the threads (warp 0 issues them; every thread loads its rows' controls meanwhile).
template <int OP, int TMAX>
__global__ void __launch_bounds__(256) k_fine_op_tma1(FineTab tab, const uint8_t *__restrict__ policy,
                                                      float dt, float omega, const float *__restrict__ x,
                                                      const float *__restrict__ b, float *__restrict__ y,
                                                      int halo, int SW, TmaTiles tt, int color) {
  constexpr int RPT = kFineRPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bar;
  float *buf = reinterpret_cast<float *>(smem_raw);
  const int n = tab.n, m = tab.m;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int WD = 32 + 2 * halo, SH = 8 * RPT + 2 * halo;
  const int o1 = 1 + blockIdx.x * 32 - halo, o2 = 1 + blockIdx.y * (8 * RPT) - halo;
  const bool tma = (smem_addr(smem_raw) & 15u) == 0u && o1 >= 3 && o2 >= 0 && o1 + WD + 3 <= n && o2 + SH <= n;
  if (tma) {
    if (ty == 0) {
      if (tx == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
      }
      __syncwarp();
      tma_issue_tile(x, n, o1, o2, WD, SH, SW, buf, &bar);
    }
  }
  const int i1 = 1 + blockIdx.x * 32 + tx;
  int kr[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int i2 = 1 + blockIdx.y * (8 * RPT) + ty + 8 * r;
    kr[r] = i1 <= m && i2 <= m ? int(policy[(i2 - 1) * m + (i1 - 1)]) : 0;
  }
  const float *xs = buf;
  if (tma) {
    __syncthreads();  // the barrier is initialised before anyone polls it
    unsigned spins = 0;
    bool failed = false;
    while (!mbar_try_wait(&bar, 0u)) {
      if (++spins >= kTmaSpin) {
        failed = true;
        break;
      }
    }
    if (failed && tx == 0 && ty == 0) atomicExch(tt.err, 1);
    xs = buf + int((size_t(o2) * n + o1) & 3);
  } else {
    stage_tile<float>(buf, x, n, o1, o2, SW, WD, SH, tx, ty);
    __syncthreads();
  }
  fine_tile_rows<float, OP, TMAX, RPT>(tab, dt, omega, xs, b, y, halo, SW, blockIdx.x, blockIdx.y, kr, color);
}

template <typename T, int OP>
bool fine_op_tma(const FineTab &tab, const uint8_t *policy, T dt, T omega, const T *x, const T *b, T *y,
                 int halo, int SW, int color, cudaStream_t s) {
  if constexpr (!std::is_same<T, float>::value || OP == OP_JACOBI0) {
    return false;
  } else {
    if (!tab.tma || !tab.tma_err || tab.tmax != 12 || (reinterpret_cast<uintptr_t>(x) & 15) != 0 ||
        tab.n < 64 + 2 * halo + 8)
      return false;
    TmaTiles tt{};
    tt.tiles_x = (tab.m + 31) / 32;
    tt.ntiles = tt.tiles_x * ((tab.m + 8 * kFineRPT - 1) / (8 * kFineRPT));
    const int SH = 8 * kFineRPT + 2 * halo;
    tt.buf_floats = (SW * SH + 8 + 31) / 32 * 32;
    tt.err = tab.tma_err;
    note_launch();
    if (tab.tma == 2) {
      // persistent: four blocks per SM of the 152, or one per tile when there are fewer
      const size_t bytes = 2 * size_t(tt.buf_floats) * sizeof(float);
      const int grid = std::min(tt.ntiles, 4 * 152);
      k_fine_op_tma<OP, 12><<<grid, dim3(32, 8), bytes, s>>>(tab, policy, dt, omega, x, b, y, halo, SW, tt, color);
    } else {
      const size_t bytes = size_t(tt.buf_floats) * sizeof(float);
      dim3 grd(tt.tiles_x, tt.ntiles / tt.tiles_x);
      k_fine_op_tma1<OP, 12><<<grd, dim3(32, 8), bytes, s>>>(tab, policy, dt, omega, x, b, y, halo, SW, tt,
                                                             color);
    }
    return true;
  }
}

template <typename T, int OP>
void fine_op_dispatch(const FineTab &tab, const uint8_t *policy, T dt, T omega, const T *x, const T *b,
                      T *y, int halo, int SW, int color, cudaStream_t s) {
  if (fine_op_tma<T, OP>(tab, policy, dt, omega, x, b, y, halo, SW, color, s)) return;
  dim3 blk(32, 8), grd((tab.m + 31) / 32, (tab.m + 8 * kFineRPT - 1) / (8 * kFineRPT));
  const size_t bytes = OP == OP_JACOBI0 ? 0 : size_t(SW) * (8 * kFineRPT + 2 * halo) * sizeof(T);
  note_launch();
  switch (tab.tmax) {
    case 8: k_fine_op<T, OP, 8><<<grd, blk, bytes, s>>>(tab, policy, dt, omega, x, b, y, halo, SW, color); break;
    case 12: k_fine_op<T, OP, 12><<<grd, blk, bytes, s>>>(tab, policy, dt, omega, x, b, y, halo, SW, color); break;
    case 16: k_fine_op<T, OP, 16><<<grd, blk, bytes, s>>>(tab, policy, dt, omega, x, b, y, halo, SW, color); break;
    case 20: k_fine_op<T, OP, 20><<<grd, blk, bytes, s>>>(tab, policy, dt, omega, x, b, y, halo, SW, color); break;
    default: k_fine_op<T, OP, 0><<<grd, blk, bytes, s>>>(tab, policy, dt, omega, x, b, y, halo, SW, color); break;
  }
}

template <typename T>
void launch_fine_op(int op, const FineTab &tab, const int32_t *slin, const uint8_t *policy, T dt,
                    T omega, const T *x, const T *b, T *y, int halo, int SW, cudaStream_t s, int color) {
  (void)slin;
  switch (op) {
    case OP_APPLY: fine_op_dispatch<T, OP_APPLY>(tab, policy, dt, omega, x, b, y, halo, SW, -1, s); break;
    case OP_RESID: fine_op_dispatch<T, OP_RESID>(tab, policy, dt, omega, x, b, y, halo, SW, -1, s); break;
    case OP_JACOBI: fine_op_dispatch<T, OP_JACOBI>(tab, policy, dt, omega, x, b, y, halo, SW, color, s); break;
    default: fine_op_dispatch<T, OP_JACOBI0>(tab, policy, dt, omega, x, b, y, halo, SW, color, s); break;
  }
}
template void launch_fine_op<double>(int, const FineTab &, const int32_t *, const uint8_t *, double,
                                     double, const double *, const double *, double *, int, int,
                                     cudaStream_t, int);
template void launch_fine_op<float>(int, const FineTab &, const int32_t *, const uint8_t *, float,
                                    float, const float *, const float *, float *, int, int,
                                    cudaStream_t, int);

// omega / d_e for every fine table entry, d_e = 1 + dt (W_e - c_k - w_self,e) (the Jacobi scale).
// The interior entry of each control (q1 = q2 = B) also goes to iod[k] when iod64 is given.
__global__ void k_fine_od(FineTab tab, double dt, double omega, int E, double *od64, float *od32,
                          double *iod64, float *iod32) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    const int k = e / (tab.Q * tab.Q);
    const double d64 = 1.0 + dt * (tab.W64[e] - tab.c64[k] - tab.ws64[e]);
    const float d32 = 1.0f + float(dt) * (tab.W32[e] - tab.c32[k] - tab.ws32[e]);
    od64[e] = omega / d64;
    od32[e] = float(omega) / d32;
    if (iod64 && e % (tab.Q * tab.Q) == tab.B * tab.Q + tab.B) {
      iod64[k] = od64[e];
      iod32[k] = od32[e];
    }
  }
}
void launch_fine_od(const FineTab &tab, double dt, double omega, double *od64, float *od32,
                    double *iod64, float *iod32, cudaStream_t s) {
  const int E = tab.K * tab.Q * tab.Q;
  note_launch();
  k_fine_od<<<(E + 255) / 256, 256, 0, s>>>(tab, dt, omega, E, od64, od32, iod64, iod32);
}

// ----------------------------------------------------------------------------- HJB residual
// r_j = F_j - (A X)_j = U^{n-1}_j - X_j + dt (sum_t w_t (X_{j+o_t} - X_j) + c_k X_j + f_k(j)),
// X carrying psi on the boundary (the boundary columns of Remark 2.2 are included here).
//
// FP64 is thin on this GPU, so the differences X_{j+o_t} - X_j are not formed per tap.  The
// block stages x' = X - X_c on its 32 x 32 tile plus halo (X_c: X at the tile's centre node),
// one subtraction per staged value, and forms sum_t w_t x'_t - W x'_j: 12 + 1 FMAs instead of
// 12 subtractions and 12 FMAs.  In exact arithmetic this equals sum_t w_t (X_t - X_j), since
// sum_t w_t = W for every table entry.  The rounding error stays of the order of
// u W max_tile |X - X_c| (the variation of X over the tile), far below the u W |X| of the
// plain form W X_j - sum_t w_t X_t.
template <int TMAX>
__global__ void __launch_bounds__(256) k_hjb_resid(FineTab tab, const uint8_t *__restrict__ policy,
                                                   const double *__restrict__ X,
                                                   const double *__restrict__ U,
                                                   const double *__restrict__ F,
                                                   const double *__restrict__ phi, int nf, double dt,
                                                   double *__restrict__ r, int zero_inside, int halo,
                                                   int SW, double *__restrict__ ub_out,
                                                   const double *__restrict__ ub_in) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *xs = reinterpret_cast<double *>(smem_raw);
  constexpr int RPT = kFineRPT;
  const int n = tab.n, m = tab.m;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int r1 = blockIdx.x * 32, r2 = blockIdx.y * (8 * RPT);
  const int i1 = 1 + r1 + tx;
  // zero_inside = R > 0: X vanishes on the interior and no tap of a row farther than R from
  // the boundary reaches it, so L X + c X = 0 there (the right-hand side F of the step); a
  // block made only of such rows stages nothing
  const int R = zero_inside;
  const bool far_blk = R > 0 && 1 + r1 > R && r1 + 32 < n - 1 - R && 1 + r2 > R && r2 + 8 * RPT < n - 1 - R;
  double xc = 0.0;
  if (!far_blk) {
    const int c1 = min(1 + r1 + 16, n - 2), c2 = min(1 + r2 + 4 * RPT, n - 2);
    xc = X[size_t(c2) * n + c1];
    const int o1 = 1 + r1 - halo, o2 = 1 + r2 - halo, SH = 8 * RPT + 2 * halo;
    stage_window<4, double>(xs, SW, SH, tx, ty, [&](int rr, int cc) {
      const int g2 = o2 + rr, g1 = o1 + cc;
      return (g2 >= 0 && g2 < n && g1 >= 0 && g1 < n) ? X[size_t(g2) * n + g1] - xc : 0.0;
    }, 32 + 2 * halo);
  }
  __syncthreads();
  if (i1 > m) return;
  const bool inner = TMAX > 0 && tab.ipk64 != nullptr && !tab.general && n - 1 >= 2 * tab.B &&
                     1 + r1 >= tab.B && r1 + 32 <= n - 1 - tab.B && 1 + r2 >= tab.B &&
                     r2 + 8 * RPT <= n - 1 - tab.B;
  const size_t N = size_t(n) * n;
#pragma unroll
  for (int rr = 0; rr < RPT; ++rr) {
    const int i2 = 1 + r2 + ty + 8 * rr;
    if (i2 > m) continue;
    const int j = i2 * n + i1;
    const int k = policy[(i2 - 1) * m + (i1 - 1)];
    double f = 0.0, ub = 0.0;
    if (ub_in) {
      ub = ub_in[j];
    } else {
#pragma unroll
      for (int mm = 0; mm < 4; ++mm)
        if (mm < nf) f = fma(__ldg(phi + k * nf + mm), F[mm * N + j], f);
      if (ub_out || R > 0) ub = U[j] + dt * f;
      if (ub_out) ub_out[j] = ub;
    }
    if (R > 0 && i1 > R && i1 < n - 1 - R && i2 > R && i2 < n - 1 - R) {
      r[j] = ub;
      continue;
    }
    const int sidx = (ty + 8 * rr + halo) * SW + tx + halo;
    const int e = fine_row_entry(tab, k, i1, i2);
    double acc;
    if (inner) {
      acc = InnerTaps<double, TMAX>::sum(tab, k, xs, sidx);
    } else {
      acc = 0.0;
      const int nt = tab.nt[e];
      for (int t = 0; t < nt; ++t) {
        int off;
        double w;
        PackedTap<double>::get(tab, e * tab.tmax + t, off, w);
        acc = fma(w, xs[sidx + off], acc);
      }
    }
    const double Xj = X[j];
    if (ub_in) {
      const double v = fma(-tab.W64[e], xs[sidx], acc) + tab.c64[k] * Xj;
      r[j] = (ub - Xj) + dt * v;
    } else {
      const double v = fma(-tab.W64[e], xs[sidx], acc) + (f + tab.c64[k] * Xj);
      r[j] = (U[j] - Xj) + dt * v;
    }
  }
}

void launch_hjb_resid(const FineTab &tab, const uint8_t *policy, const double *X,
                      const double *Uprev, const double *F, const double *phi, int nf, double dt,
                      double *r, int halo, int SW, cudaStream_t s, int zero_inside, double *ub_out,
                      const double *ub_in) {
  dim3 blk(32, 8), grd((tab.m + 31) / 32, (tab.m + 8 * kFineRPT - 1) / (8 * kFineRPT));
  const size_t bytes = size_t(SW) * (8 * kFineRPT + 2 * halo) * sizeof(double);
  note_launch();
#define SL_RESID_ARGS tab, policy, X, Uprev, F, phi, nf, dt, r, zero_inside, halo, SW, ub_out, ub_in
  switch (tab.tmax) {
    case 8: k_hjb_resid<8><<<grd, blk, bytes, s>>>(SL_RESID_ARGS); break;
    case 12: k_hjb_resid<12><<<grd, blk, bytes, s>>>(SL_RESID_ARGS); break;
    case 16: k_hjb_resid<16><<<grd, blk, bytes, s>>>(SL_RESID_ARGS); break;
    case 20: k_hjb_resid<20><<<grd, blk, bytes, s>>>(SL_RESID_ARGS); break;
    default: k_hjb_resid<0><<<grd, blk, bytes, s>>>(SL_RESID_ARGS); break;
  }
#undef SL_RESID_ARGS
}

// ----------------------------------------------------------------------------- transfers
// Full weighting (restrict_point) and bilinear prolongation with correction (prolong_point).
template <typename T>
__global__ void k_restrict(const T *__restrict__ rf, int nf, T *__restrict__ bc, int nc) {
  const int I1 = 1 + blockIdx.x * 32 + threadIdx.x;
  const int I2 = 1 + blockIdx.y * 8 + threadIdx.y;
  if (I1 > nc - 2 || I2 > nc - 2) return;
  bc[size_t(I2) * nc + I1] = restrict_point<T>(rf, nf, I1, I2);
}

// One thread per coarse cell [J1, J1 + 1] x [J2, J2 + 1]: it reads the cell's four coarse
// values once and updates the fine nodes (2 J1 + a1, 2 J2 + a2), a in {0, 1}, with the
// weights and the order of additions of prolong_point (the same values bit for bit), instead
// of each fine node gathering its own one to four coarse values with parity branches.
template <typename T>
__global__ void k_prolong_add(const T *__restrict__ xc, int nc, T *__restrict__ xf, int nf) {
  const int J1 = blockIdx.x * 32 + threadIdx.x;
  const int J2 = blockIdx.y * 8 + threadIdx.y;
  if (J1 > nc - 2 || J2 > nc - 2) return;
  const T *c0 = xc + size_t(J2) * nc + J1;
  const T c00 = c0[0], c10 = c0[1], c01 = c0[nc], c11 = c0[nc + 1];
  const int i1 = 2 * J1, i2 = 2 * J2;
  T *f0 = xf + size_t(i2) * nf + i1;
  if (J2 > 0) {  // fine row 2 J2 (row 0 is the boundary)
    if (J1 > 0) f0[0] += c00;
    f0[1] += T(0.5) * (c00 + c10);
  }
  T *f1 = f0 + nf;  // fine row 2 J2 + 1 <= nf - 2
  if (J1 > 0) f1[0] += T(0.5) * (c00 + c01);
  f1[1] += T(0.25) * ((c00 + c10) + (c01 + c11));
}

template <typename T>
void launch_restrict(const T *rf, int nf, T *bc, int nc, cudaStream_t s) {
  dim3 blk(32, 8), grd((nc - 2 + 31) / 32, (nc - 2 + 7) / 8);
  note_launch();
  k_restrict<T><<<grd, blk, 0, s>>>(rf, nf, bc, nc);
}
template <typename T>
void launch_prolong_add(const T *xc, int nc, T *xf, int nf, cudaStream_t s) {
  dim3 blk(32, 8), grd((nc - 1 + 31) / 32, (nc - 1 + 7) / 8);
  note_launch();
  k_prolong_add<T><<<grd, blk, 0, s>>>(xc, nc, xf, nf);
}
template void launch_restrict<double>(const double *, int, double *, int, cudaStream_t);
template void launch_restrict<float>(const float *, int, float *, int, cudaStream_t);
template void launch_prolong_add<double>(const double *, int, double *, int, cudaStream_t);
template void launch_prolong_add<float>(const float *, int, float *, int, cudaStream_t);

// ----------------------------------------------------------------------------- attributes
template <typename T, int OP>
static cudaError_t prepare_fine_op() {
  const void *fs[] = {reinterpret_cast<const void *>(k_fine_op<T, OP, 8>),
                      reinterpret_cast<const void *>(k_fine_op<T, OP, 12>),
                      reinterpret_cast<const void *>(k_fine_op<T, OP, 16>),
                      reinterpret_cast<const void *>(k_fine_op<T, OP, 20>),
                      reinterpret_cast<const void *>(k_fine_op<T, OP, 0>)};
  for (const void *f : fs) {
    cudaError_t e = allow_dynamic_smem(f);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t prepare_fine_kernels() {
  const void *fs[] = {reinterpret_cast<const void *>(k_hjb_resid<8>),
                      reinterpret_cast<const void *>(k_hjb_resid<12>),
                      reinterpret_cast<const void *>(k_hjb_resid<16>),
                      reinterpret_cast<const void *>(k_hjb_resid<20>),
                      reinterpret_cast<const void *>(k_hjb_resid<0>),
                      reinterpret_cast<const void *>(k_argmin<0, 0>),
                      reinterpret_cast<const void *>(k_argmin<1, 8>),
                      reinterpret_cast<const void *>(k_argmin<1, 12>),
                      reinterpret_cast<const void *>(k_argmin<1, 16>),
                      reinterpret_cast<const void *>(k_argmin<1, 20>),
                      reinterpret_cast<const void *>(k_argmin<1, 0>),
                      reinterpret_cast<const void *>(k_argmin2<12>)};
  for (const void *f : fs) {
    cudaError_t e = allow_dynamic_smem(f);
    if (e != cudaSuccess) return e;
  }
  const void *tma[] = {reinterpret_cast<const void *>(k_fine_op_tma<OP_APPLY, 12>),
                       reinterpret_cast<const void *>(k_fine_op_tma<OP_RESID, 12>),
                       reinterpret_cast<const void *>(k_fine_op_tma<OP_JACOBI, 12>),
                       reinterpret_cast<const void *>(k_fine_op_tma1<OP_APPLY, 12>),
                       reinterpret_cast<const void *>(k_fine_op_tma1<OP_RESID, 12>),
                       reinterpret_cast<const void *>(k_fine_op_tma1<OP_JACOBI, 12>)};
  for (const void *f : tma) {
    cudaError_t e = allow_dynamic_smem(f);
    if (e != cudaSuccess) return e;
  }
  cudaError_t (*ops[])() = {prepare_fine_op<double, OP_APPLY>, prepare_fine_op<double, OP_RESID>,
                            prepare_fine_op<double, OP_JACOBI>, prepare_fine_op<double, OP_JACOBI0>,
                            prepare_fine_op<float, OP_APPLY>, prepare_fine_op<float, OP_RESID>,
                            prepare_fine_op<float, OP_JACOBI>, prepare_fine_op<float, OP_JACOBI0>};
  for (auto op : ops) {
    cudaError_t e = op();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sl
