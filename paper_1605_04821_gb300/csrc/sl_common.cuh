// sl_common.cuh - data layout shared by the host orchestration and the sm_103a kernels.
//
// Fine level (level 0): matrix-free.  Row j = (i1, i2) of A^alpha (Eq. 2.11, theta = 1)
// is described by its control k = alpha_j and its boundary-distance class (q1, q2):
//   (A x)_j = (1 + dt (W - c_k)) x_j - dt sum_t w_t x_{j + o_t}
// where the taps (o_t, w_t) are the bilinear interpolation weights of the truncated Scheme-2
// endpoints scaled by A_p/(2h), B_p/(2h) (Proposition 2.2, Eq. 2.9), and
// W = sum_p (A_p + B_p)/(2h).  Rows farther than B cells from the boundary in both
// dimensions are never truncated and share one table entry per control; rows in the band
// get one entry per (distance to the low side, distance to the high side) pair, so every
// row of the grid reads its stencil from a small table that stays in L1/L2.
//
// Coarse levels: row I of A_l = R A_{l-1} P is either "class k" (every row of level l-1 in
// the support of the full-weighting stencil at 2I is a class-k interior row, so the row is
// the translation-invariant Galerkin stencil S_k^l) or explicit (a dense window of
// (2 R_l + 1)^2 coefficients around I).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#define SL_HD __host__ __device__ __forceinline__

namespace sl {

constexpr int kMaxLevels = 16;
constexpr int kMaxCand = 8;       // argmin candidate list length (then full FP64 fallback)
constexpr int kRedBlocks = 608;   // 4 x 152 SMs: grid of the vector kernels / reductions
constexpr int kCoarsestMax = 256; // largest coarsest level solved by a dense inverse

// Boundary-distance class of a coordinate i in [1, n-2] (band width B).
SL_HD int class_q(int i, int n, int B) {
  if (n - 1 >= 2 * B) {
    if (i < B) return i;
    int e = n - 1 - i;
    if (e < B) return 2 * B - e;
    return B;
  }
  return i;
}

// A representative coordinate of class q.
SL_HD int class_rep(int q, int n, int B) {
  if (n - 1 >= 2 * B) {
    if (q <= B) return q;
    return n - 1 - (2 * B - q);
  }
  return q;
}

SL_HD int class_count(int n, int B) { return (n - 1 >= 2 * B) ? 2 * B : n - 1; }

// Device view of the fine-level stencil tables (entry e = (k*Q + q2)*Q + q1).
struct FineTab {
  int n, m, B, Q, tmax, K;
  const int32_t *lin;     // [e*tmax + t] linear offset dy*n + dx
  const double *w64;      // [e*tmax + t] tap weight (already / (2h))
  const float *w32;
  const uint8_t *nt;      // [e] number of taps
  const double *W64;      // [e] sum_p (A_p + B_p)/(2h)
  const float *W32;
  const double *ws64;     // [e] weight of the tap at offset 0 (node itself)
  const float *ws32;
  const double *c64;      // [K] discount
  const float *c32;
  const double *od64;     // [e] omega / d_e with d_e = 1 + dt (W - c - w_self) (per hierarchy dt)
  const float *od32;
  const int2 *pk32;       // [e*tmax + t] {staged-tile offset, fp32 weight bits}
  const longlong2 *pk64;  // [e*tmax + t] {staged-tile offset, fp64 weight bits}
  int general;            // 1: x-dependent sigma; entry e = interior row, assembled per policy
  // The interior class (q1 = q2 = B) of every control again, tap-major with the controls
  // adjacent, so that the rows of a warp, whose controls are few and close together, find
  // tap t of all their controls in one or two cache lines (null on a general level or for an
  // odd tap stride).
  const int4 *ipk32;      // [(t / 2) * K + k] {offset_t, w_t bits, offset_t+1, w_t+1 bits}
  const longlong2 *ipk64; // [t * K + k] {offset, w bits}
  const double *iWc64;    // [k] W_e - c_k of the interior entry e of control k
  const float *iWc32;     // [k] the same difference taken in FP32 (W32[e] - c32[k])
  const double *iod64;    // [k] od of the interior entry
  const float *iod32;
  // FP32 operator with TMA-staged tiles (k_fine_op_tma): 1 to use it where it applies; err is
  // set to 1 by a bounded wait that gave up
  int tma;
  int *tma_err;
};

// Table entry of row (i1, i2) whose control is k: the (control, boundary class) entry, or, on
// a general fine level (x-dependent diffusion), the row's own entry, which holds the taps of
// the row's current control.
SL_HD int fine_row_entry(const FineTab &t, int k, int i1, int i2) {
  if (t.general) return (i2 - 1) * t.m + (i1 - 1);
  return (k * t.Q + class_q(i2, t.n, t.B)) * t.Q + class_q(i1, t.n, t.B);
}



template <typename T> SL_HD const T *tab_w(const FineTab &t);
template <> SL_HD const double *tab_w<double>(const FineTab &t) { return t.w64; }
template <> SL_HD const float *tab_w<float>(const FineTab &t) { return t.w32; }
template <typename T> SL_HD const T *tab_W(const FineTab &t);
template <> SL_HD const double *tab_W<double>(const FineTab &t) { return t.W64; }
template <> SL_HD const float *tab_W<float>(const FineTab &t) { return t.W32; }
template <typename T> SL_HD const T *tab_ws(const FineTab &t);
template <> SL_HD const double *tab_ws<double>(const FineTab &t) { return t.ws64; }
template <> SL_HD const float *tab_ws<float>(const FineTab &t) { return t.ws32; }
template <typename T> SL_HD const T *tab_od(const FineTab &t);
template <> SL_HD const double *tab_od<double>(const FineTab &t) { return t.od64; }
template <> SL_HD const float *tab_od<float>(const FineTab &t) { return t.od32; }
template <typename T> SL_HD const T *tab_c(const FineTab &t);
template <> SL_HD const double *tab_c<double>(const FineTab &t) { return t.c64; }
template <> SL_HD const float *tab_c<float>(const FineTab &t) { return t.c32; }

// Device view of one coarse level.
template <typename T>
struct CoarseLev {
  int n, m, R, win;        // nodes per dim, interior per dim, window reach, (2R+1)^2
  const int32_t *cls;      // [m*m] >= 0: class k; < 0: explicit slot -cls-1
  // class tables: sparse taps of S_k (entry k), including the centre coefficient
  const int32_t *clin;     // [k*ctmax + t] linear offset dy*n + dx
  const int32_t *coff;     // [k*ctmax + t] packed (dy << 16) | (dx & 0xffff)
  const int2 *cpk32;       // [k*ctmax + t] {dy*(32+2R) + dx, fp32 weight bits} (staged tile)
  const longlong2 *cpk64;  // [k*ctmax + t] {dy*(32+2R) + dx, fp64 weight bits}
  const T *cw;             // [k*ctmax + t]
  const int32_t *cnt;      // [k]
  const T *cdiag;          // [k]
  int ctmax;
  int nk;                  // number of classes (controls): the class tables hold nk * ctmax taps
  // explicit rows
  const T *ewin;           // [e*cap + slot], e = (dy+R)*(2R+1) + (dx+R)
  const int32_t *erow;     // [slot] linear full-grid index of the row
  int cap;
};

#ifdef __CUDACC__
// One tap of a staged tile: offset in the tile and weight, loaded with a single vector load.
template <typename T> struct PackedTap;
template <> struct PackedTap<float> {
  static __device__ __forceinline__ void get(const FineTab &t, int ix, int &off, float &w) {
    const int2 p = __ldg(t.pk32 + ix);
    off = p.x;
    w = __int_as_float(p.y);
  }
};
template <> struct PackedTap<double> {
  static __device__ __forceinline__ void get(const FineTab &t, int ix, int &off, double &w) {
    const longlong2 p = __ldg(t.pk64 + ix);
    off = int(p.x);
    w = __longlong_as_double(p.y);
  }
};

// Copies the SH x SW window whose element (r, c) is load(r, c) into xs (row pitch SW) with a
// block of 32 x 8 threads (tx, ty).  Each pass covers 8 NR rows and the first 64 columns: a
// thread issues its 2 NR loads into registers before any of its stores, so one round of memory
// latency serves the whole pass.  (A loop that stores each value right after loading it makes
// every load wait for the previous one, since the store waits for its data and instructions
// issue in order; on a level with one block per SM nothing hides that.)  Columns from 64 on,
// for wide halos, are copied one by one.  SW is the row pitch of xs; the first `width` columns
// of each row are staged (width < 0: all SW).
template <int NR, typename T, typename Load>
__device__ __forceinline__ void stage_window(T *xs, int SW, int SH, int tx, int ty, Load load,
                                             int width = -1) {
  const int WD = width < 0 ? SW : width;
  for (int r0 = 0; r0 < SH; r0 += 8 * NR) {
    T v[NR][2];
#pragma unroll
    for (int i = 0; i < NR; ++i)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int r = r0 + ty + 8 * i, c = tx + 32 * q;
        v[i][q] = (r < SH && c < WD) ? load(r, c) : T(0);
      }
#pragma unroll
    for (int i = 0; i < NR; ++i)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int r = r0 + ty + 8 * i, c = tx + 32 * q;
        if (r < SH && c < WD) xs[r * SW + c] = v[i][q];
      }
  }
  for (int r = ty; r < SH; r += 8)
    for (int c = tx + 64; c < WD; c += 32) xs[r * SW + c] = load(r, c);
}

template <typename T> struct ClassTap;
template <> struct ClassTap<float> {
  using Packed = int2;
  static __device__ __forceinline__ const int2 *table(const CoarseLev<float> &L) { return L.cpk32; }
  static __device__ __forceinline__ void get(const CoarseLev<float> &L, int ix, int &off, float &w) {
    const int2 p = __ldg(L.cpk32 + ix);
    off = p.x;
    w = __int_as_float(p.y);
  }
  static __device__ __forceinline__ void unpack(const int2 &p, int &off, float &w) {
    off = p.x;
    w = __int_as_float(p.y);
  }
};
template <> struct ClassTap<double> {
  using Packed = longlong2;
  static __device__ __forceinline__ const longlong2 *table(const CoarseLev<double> &L) { return L.cpk64; }
  static __device__ __forceinline__ void get(const CoarseLev<double> &L, int ix, int &off, double &w) {
    const longlong2 p = __ldg(L.cpk64 + ix);
    off = int(p.x);
    w = __longlong_as_double(p.y);
  }
  static __device__ __forceinline__ void unpack(const longlong2 &p, int &off, double &w) {
    off = int(p.x);
    w = __longlong_as_double(p.y);
  }
};
#endif

// Full-weighting and bilinear 1-D weights: R uses (1, 2, 1)/4 per dimension, P uses 1 at
// even fine indices and (1/2, 1/2) at odd ones.
SL_HD double fw_weight(int a) { return a == 0 ? 0.5 : 0.25; }

// Scatters one level-(l-1) matrix entry v at column j (level-(l-1) coordinates) of the fine
// row 2I + a into the Galerkin window of coarse row I:
// window[J - I] += R_a * v * P_{j,J} over the bilinear parents J of j.
template <typename T>
SL_HD void rap_scatter(T *win, int R, int I1, int I2, int j1, int j2, T rv) {
  int W = 2 * R + 1;
  int J1a, J1b, J2a, J2b;
  T p1a, p1b, p2a, p2b;
  if ((j1 & 1) == 0) { J1a = j1 >> 1; J1b = J1a; p1a = T(1); p1b = T(0); }
  else { J1a = (j1 - 1) >> 1; J1b = J1a + 1; p1a = T(0.5); p1b = T(0.5); }
  if ((j2 & 1) == 0) { J2a = j2 >> 1; J2b = J2a; p2a = T(1); p2b = T(0); }
  else { J2a = (j2 - 1) >> 1; J2b = J2a + 1; p2a = T(0.5); p2b = T(0.5); }
  int d1a = J1a - I1 + R, d1b = J1b - I1 + R, d2a = J2a - I2 + R, d2b = J2b - I2 + R;
  win[d2a * W + d1a] += rv * p1a * p2a;
  if (p1b != T(0)) win[d2a * W + d1b] += rv * p1b * p2a;
  if (p2b != T(0)) {
    win[d2b * W + d1a] += rv * p1a * p2b;
    if (p1b != T(0)) win[d2b * W + d1b] += rv * p1b * p2b;
  }
}

// Row pitch of a staged coarse-level tile, and the pitch the packed class-table offsets assume:
// 32 columns plus a halo of R on each side, plus the one column of the residual ring that the
// fused residual-and-restriction kernel computes beyond its tile.
SL_HD int coarse_pitch(int R) { return 33 + 2 * R; }

// Full weighting at coarse interior node (I1, I2):
// b_c(I) = sum_{a in {-1,0,1}^2} w_a1 w_a2 r_f(2I + a), w = (1/4, 1/2, 1/4).
template <typename T>
SL_HD T restrict_point(const T *rf, int nf, int I1, int I2) {
  const T *r0 = rf + size_t(2 * I2) * nf + 2 * I1;
  const T rowm = T(0.25) * r0[-nf - 1] + T(0.5) * r0[-nf] + T(0.25) * r0[-nf + 1];
  const T row0 = T(0.25) * r0[-1] + T(0.5) * r0[0] + T(0.25) * r0[1];
  const T rowp = T(0.25) * r0[nf - 1] + T(0.5) * r0[nf] + T(0.25) * r0[nf + 1];
  return T(0.25) * rowm + T(0.5) * row0 + T(0.25) * rowp;
}

// Bilinear prolongation at fine interior node (i1, i2): sum_J P_{iJ} x_c(J).
template <typename T>
SL_HD T prolong_point(const T *xc, int nc, int i1, int i2) {
  const int J1 = i1 >> 1, J2 = i2 >> 1;
  const bool odd1 = i1 & 1, odd2 = i2 & 1;
  const T *c0 = xc + size_t(J2) * nc + J1;
  if (!odd1 && !odd2) return c0[0];
  if (odd1 && !odd2) return T(0.5) * (c0[0] + c0[1]);
  if (!odd1 && odd2) return T(0.5) * (c0[0] + c0[nc]);
  return T(0.25) * ((c0[0] + c0[1]) + (c0[nc] + c0[nc + 1]));
}

// Scalars of one BiCGSTAB run, kept in device memory so that no iteration needs the host.
struct BicgScalars {
  double rho, rho_old, alpha, omega;
  double rv, ts, tt, ss, rr;   // (r^, v), (t, s), (t, t), (s, s), (r, r)
  double bnorm2;               // ||b||^2 of the system
  double tolrel2;              // tol^2 (set by the host before the run)
  double tol2;                 // (tol ||b||)^2
  double rmax, bmax;           // ||r||_inf, ||b||_inf (true-residual checks)
  int first;                   // 1 until the first search direction has been formed
  int breakdown;               // 1: rho or (r^, v) or (t, t) vanished
  int nonfinite;               // 1: a NaN / Inf was seen
  int inject_bd;               // > 0: iterations left until one is marked as a breakdown
                               // (sl_hjb_inject_breakdown); kept across solves
};

}  // namespace sl
