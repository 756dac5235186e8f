// sl_geometry.h - host-side construction of the Scheme-2 stencil tables (FP64, at create
// time) and of the translation-invariant Galerkin class stencils (per hierarchy build).
#pragma once

#include <cstdint>
#include <vector>

namespace sl {

struct FineTabHost {
  int n = 0, m = 0, B = 0, Q = 0, tmax = 0, K = 0;
  int R0 = 0;                       // largest |dx|, |dy| of any tap
  std::vector<int32_t> dx, dy;      // [e*tmax + t]
  std::vector<double> w;            // [e*tmax + t]
  std::vector<uint8_t> nt;          // [e]
  std::vector<double> W, ws;        // [e]
  std::vector<double> c;            // [K]
  std::vector<double> Wmax_class;   // [q2*Q + q1] max_k W of that class (argmin screen bound)
  int entry(int k, int q1, int q2) const { return (k * Q + q2) * Q + q1; }
};

// sigma: K*2*P (column p of control k is (sigma[(k*2)*P+p], sigma[(k*2+1)*P+p])),
// b: K*2 or null, c: K or null; grid n x n with spacing h.
FineTabHost build_fine_tables(int n, double h, int K, int P, const double *sigma,
                              const double *b, const double *c);

// Diffusion taps of every interior row for an x-dependent sigma shared by all controls:
// field[((i2*n + i1)*2 + d)*P + p] is component d of column p at node (i1, i2).  Row
// I = (i2-1)(n-2) + (i1-1) has nt[I] taps (dy, dx, w) at [I*stride + t] and the weight sum
// W[I] = sum_p (A_p + B_p)/(2h) (Proposition 2.2, Eq. 2.9); R0 is the longest tap.
struct NodeTabHost {
  int stride = 0, R0 = 0;
  std::vector<int32_t> dx, dy;
  std::vector<double> w;
  std::vector<uint8_t> nt;
  std::vector<double> W;
};
NodeTabHost build_node_tables(int n, double h, int P, const double *field);

// Derivative of every fine table entry with respect to a scalar parameter theta of the
// diffusion coefficients (dsig = d sigma / d theta, laid out like sigma): taps (dy, dx, dw) of
// d(L^k)/d theta with dw = d w_t / d theta, and dW = d W / d theta, so that
//   (d L^k / d theta x)_j = sum_t dw_t x_{j + o_t} - dW x_j.
// Entry numbering is that of FineTabHost (same B and Q); `stride` is the tap stride.
struct FineDTabHost {
  int stride = 0;
  std::vector<int32_t> dx, dy;  // [e*stride + t]
  std::vector<double> dw;       // [e*stride + t]
  std::vector<uint8_t> nt;      // [e]
  std::vector<double> dW;       // [e]
};
FineDTabHost build_fine_dtables(const FineTabHost &t, double h, int P, const double *sigma,
                                const double *dsig);

// Dense (2R+1)^2 window of the level-l class-k Galerkin stencil, built from the level-(l-1)
// class-k row `prev` (dense window of reach Rprev; for level 1 the fine interior row).
std::vector<double> rap_class_window(const std::vector<double> &prev, int Rprev, int R);

// Fine interior row of control k as a dense window of reach R0 (matrix coefficients:
// centre 1 + dt (W - c) - dt w_self, off-centre -dt w).
std::vector<double> fine_interior_window(const FineTabHost &t, int k, double dt);

}  // namespace sl
