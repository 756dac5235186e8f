// sl_geometry.cpp - Scheme-2 stencils with boundary truncation, evaluated once in FP64.
//
// For control k and a node at integer grid index i = (i1, i2), every diffusion column
// sigma_p contributes the directions +-s_p with s_p = sigma_p / sqrt(h) in grid-index units
// (the stencil length of Eq. 3.2), and a drift b contributes s = b (y = h b).  The
// truncation factor mu in (0, 1] is the largest value keeping i + mu s inside [0, n-1]^2
// (Proposition 2.2); a component that hits the boundary is placed exactly on it.  Weights:
// A_p = 2/(mu+^2 + mu+ mu-), B_p = 2/(mu-^2 + mu- mu+) (Eq. 2.3), A = B = 1/mu for the
// drift (Eq. 2.2).  The endpoint value is the bilinear interpolant of the four nodes of
// its cell (Eq. 1.7); each tap weight is A_p w_i / (2h) (Eq. 2.9) and
// W = sum_p (A_p + B_p) / (2h).
#include "sl_geometry.h"

#include <algorithm>
#include <cmath>
#include <limits>
#include <map>
#include <stdexcept>
#include <utility>

#include "sl_common.cuh"

namespace sl {
namespace {

struct Endpoint {
  double mu, z1, z2;
};

Endpoint truncate_endpoint(double i1, double i2, double s1, double s2, int n) {
  const double top = double(n - 1);
  const double inf = std::numeric_limits<double>::infinity();
  double b1 = inf, b2 = inf;
  if (s1 > 0) b1 = (top - i1) / s1; else if (s1 < 0) b1 = (0.0 - i1) / s1;
  if (s2 > 0) b2 = (top - i2) / s2; else if (s2 < 0) b2 = (0.0 - i2) / s2;
  Endpoint e;
  e.mu = std::min(1.0, std::min(b1, b2));
  e.z1 = i1 + e.mu * s1;
  e.z2 = i2 + e.mu * s2;
  if (e.mu < 1.0) {
    if (b1 == e.mu) e.z1 = s1 > 0 ? top : 0.0;
    if (b2 == e.mu) e.z2 = s2 > 0 ? top : 0.0;
  }
  return e;
}

using TapMap = std::map<std::pair<int, int>, double>;  // (dy, dx) -> weight

void add_bilinear(TapMap &taps, int i1, int i2, double z1, double z2, int n, double scale) {
  double c1 = std::min(std::max(std::floor(z1), 0.0), double(n - 2));
  double c2 = std::min(std::max(std::floor(z2), 0.0), double(n - 2));
  double t1 = z1 - c1, t2 = z2 - c2;
  int a1 = int(c1) - i1, a2 = int(c2) - i2;
  const double wts[4] = {(1 - t1) * (1 - t2), t1 * (1 - t2), (1 - t1) * t2, t1 * t2};
  const int o1[4] = {0, 1, 0, 1}, o2[4] = {0, 0, 1, 1};
  for (int c = 0; c < 4; ++c) {
    if (wts[c] == 0.0) continue;
    taps[{a2 + o2[c], a1 + o1[c]}] += wts[c] * scale;
  }
}

}  // namespace

FineTabHost build_fine_tables(int n, double h, int K, int P, const double *sigma,
                              const double *b, const double *c) {
  FineTabHost t;
  t.n = n;
  t.m = n - 2;
  t.K = K;
  const double sqh = std::sqrt(h);
  // band width: one more than the longest untruncated displacement component
  double reach = 0.0;
  for (int k = 0; k < K; ++k) {
    for (int p = 0; p < P; ++p)
      for (int d = 0; d < 2; ++d)
        reach = std::max(reach, std::fabs(sigma[(k * 2 + d) * P + p]) / sqh);
    if (b)
      for (int d = 0; d < 2; ++d) reach = std::max(reach, std::fabs(b[k * 2 + d]));
  }
  t.B = int(std::ceil(reach)) + 1;
  t.Q = class_count(n, t.B);
  t.tmax = 4 * (2 * P + (b ? 1 : 0));
  const int E = K * t.Q * t.Q;
  t.dx.assign(size_t(E) * t.tmax, 0);
  t.dy.assign(size_t(E) * t.tmax, 0);
  t.w.assign(size_t(E) * t.tmax, 0.0);
  t.nt.assign(E, 0);
  t.W.assign(E, 0.0);
  t.ws.assign(E, 0.0);
  t.c.assign(K, 0.0);
  t.Wmax_class.assign(size_t(t.Q) * t.Q, 0.0);
  if (c)
    for (int k = 0; k < K; ++k) t.c[k] = c[k];
  const int qlo = 1;  // class 0 is never used by an interior coordinate
  for (int k = 0; k < K; ++k) {
    for (int q2 = qlo; q2 < t.Q; ++q2) {
      for (int q1 = qlo; q1 < t.Q; ++q1) {
        const int i1 = class_rep(q1, n, t.B), i2 = class_rep(q2, n, t.B);
        if (i1 < 1 || i1 > n - 2 || i2 < 1 || i2 > n - 2) continue;
        TapMap taps;
        double W = 0.0;
        for (int p = 0; p < P; ++p) {
          const double s1 = sigma[(k * 2 + 0) * P + p] / sqh;
          const double s2 = sigma[(k * 2 + 1) * P + p] / sqh;
          Endpoint ep = truncate_endpoint(i1, i2, s1, s2, n);
          Endpoint em = truncate_endpoint(i1, i2, -s1, -s2, n);
          const double A = 2.0 / (ep.mu * ep.mu + ep.mu * em.mu);
          const double Bw = 2.0 / (em.mu * em.mu + em.mu * ep.mu);
          add_bilinear(taps, i1, i2, ep.z1, ep.z2, n, A / (2.0 * h));
          add_bilinear(taps, i1, i2, em.z1, em.z2, n, Bw / (2.0 * h));
          W += (A + Bw) / (2.0 * h);
        }
        if (b) {
          Endpoint e = truncate_endpoint(i1, i2, b[k * 2 + 0], b[k * 2 + 1], n);
          const double AB = 2.0 / e.mu;
          add_bilinear(taps, i1, i2, e.z1, e.z2, n, AB / (2.0 * h));
          W += AB / (2.0 * h);
        }
        const int e = t.entry(k, q1, q2);
        if (int(taps.size()) > t.tmax) throw std::runtime_error("stencil table overflow");
        int slot = 0;
        for (const auto &kv : taps) {
          const int ddy = kv.first.first, ddx = kv.first.second;
          t.dy[size_t(e) * t.tmax + slot] = ddy;
          t.dx[size_t(e) * t.tmax + slot] = ddx;
          t.w[size_t(e) * t.tmax + slot] = kv.second;
          if (ddx == 0 && ddy == 0) t.ws[e] = kv.second;
          t.R0 = std::max(t.R0, std::max(std::abs(ddx), std::abs(ddy)));
          ++slot;
        }
        t.nt[e] = uint8_t(slot);
        t.W[e] = W;
        double &wm = t.Wmax_class[size_t(q2) * t.Q + q1];
        wm = std::max(wm, W);
      }
    }
  }
  // Shrink the table stride to the longest actual tap list (rounded up to a multiple of 4), so
  // that kernels looping over the padded width do no work on slots that are always empty.
  int maxnt = 1;
  for (uint8_t v : t.nt) maxnt = std::max(maxnt, int(v));
  const int stride = (maxnt + 3) / 4 * 4;
  if (stride < t.tmax) {
    std::vector<int32_t> dx(size_t(E) * stride, 0), dy(size_t(E) * stride, 0);
    std::vector<double> w(size_t(E) * stride, 0.0);
    for (int e = 0; e < E; ++e)
      for (int s = 0; s < t.nt[e]; ++s) {
        dx[size_t(e) * stride + s] = t.dx[size_t(e) * t.tmax + s];
        dy[size_t(e) * stride + s] = t.dy[size_t(e) * t.tmax + s];
        w[size_t(e) * stride + s] = t.w[size_t(e) * t.tmax + s];
      }
    t.dx.swap(dx);
    t.dy.swap(dy);
    t.w.swap(w);
    t.tmax = stride;
  }
  return t;
}

// ---------------------------------------------------------------------- derivative tables
// Forward-mode differentiation of the construction above: every quantity carries its value
// and its derivative in theta.  Branches (which side truncates, which cell an endpoint falls
// in) follow the values, so the result is the derivative of the piecewise-smooth map on the
// piece the current sigma lies in.  A component placed exactly on the boundary by the
// truncation has derivative zero.
namespace {

struct Dual {
  double v, d;
};
Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
Dual cst(double v) { return {v, 0.0}; }

struct DEndpoint {
  Dual mu, z1, z2;
};

DEndpoint dtruncate_endpoint(double i1, double i2, Dual s1, Dual s2, int n) {
  const double top = double(n - 1);
  const double inf = std::numeric_limits<double>::infinity();
  Dual b1 = cst(inf), b2 = cst(inf);
  if (s1.v > 0) b1 = cst(top - i1) / s1; else if (s1.v < 0) b1 = cst(0.0 - i1) / s1;
  if (s2.v > 0) b2 = cst(top - i2) / s2; else if (s2.v < 0) b2 = cst(0.0 - i2) / s2;
  const Dual bmin = (b2.v < b1.v) ? b2 : b1;
  DEndpoint e;
  e.mu = (bmin.v < 1.0) ? bmin : cst(1.0);
  e.z1 = cst(i1) + e.mu * s1;
  e.z2 = cst(i2) + e.mu * s2;
  if (e.mu.v < 1.0) {
    if (b1.v == e.mu.v) e.z1 = cst(s1.v > 0 ? top : 0.0);
    if (b2.v == e.mu.v) e.z2 = cst(s2.v > 0 ? top : 0.0);
  }
  return e;
}

using DTapMap = std::map<std::pair<int, int>, Dual>;

void dadd_bilinear(DTapMap &taps, int i1, int i2, Dual z1, Dual z2, int n, Dual scale) {
  const double c1 = std::min(std::max(std::floor(z1.v), 0.0), double(n - 2));
  const double c2 = std::min(std::max(std::floor(z2.v), 0.0), double(n - 2));
  const Dual t1 = z1 - cst(c1), t2 = z2 - cst(c2);
  const int a1 = int(c1) - i1, a2 = int(c2) - i2;
  const Dual one = cst(1.0);
  const Dual wts[4] = {(one - t1) * (one - t2), t1 * (one - t2), (one - t1) * t2, t1 * t2};
  const int o1[4] = {0, 1, 0, 1}, o2[4] = {0, 0, 1, 1};
  for (int c = 0; c < 4; ++c) {
    const Dual w = wts[c] * scale;
    Dual &acc = taps.emplace(std::make_pair(a2 + o2[c], a1 + o1[c]), cst(0.0)).first->second;
    acc = acc + w;
  }
}

}  // namespace

FineDTabHost build_fine_dtables(const FineTabHost &t, double h, int P, const double *sigma,
                                const double *dsig) {
  const int n = t.n, K = t.K, E = K * t.Q * t.Q;
  const double sqh = std::sqrt(h);
  std::vector<std::vector<std::pair<std::pair<int, int>, double>>> rows(E);
  std::vector<double> dW(E, 0.0);
  int maxnt = 1;
  for (int k = 0; k < K; ++k)
    for (int q2 = 1; q2 < t.Q; ++q2)
      for (int q1 = 1; q1 < t.Q; ++q1) {
        const int i1 = class_rep(q1, n, t.B), i2 = class_rep(q2, n, t.B);
        if (i1 < 1 || i1 > n - 2 || i2 < 1 || i2 > n - 2) continue;
        DTapMap taps;
        Dual W = cst(0.0);
        for (int p = 0; p < P; ++p) {
          const size_t r1 = size_t(k * 2 + 0) * P + p, r2 = size_t(k * 2 + 1) * P + p;
          const Dual s1 = {sigma[r1] / sqh, dsig[r1] / sqh};
          const Dual s2 = {sigma[r2] / sqh, dsig[r2] / sqh};
          const DEndpoint ep = dtruncate_endpoint(i1, i2, s1, s2, n);
          const DEndpoint em = dtruncate_endpoint(i1, i2, cst(0.0) - s1, cst(0.0) - s2, n);
          const Dual A = cst(2.0) / (ep.mu * ep.mu + ep.mu * em.mu);
          const Dual Bw = cst(2.0) / (em.mu * em.mu + em.mu * ep.mu);
          dadd_bilinear(taps, i1, i2, ep.z1, ep.z2, n, A / cst(2.0 * h));
          dadd_bilinear(taps, i1, i2, em.z1, em.z2, n, Bw / cst(2.0 * h));
          W = W + (A + Bw) / cst(2.0 * h);
        }
        // the drift taps do not depend on sigma and have zero derivative
        const int e = t.entry(k, q1, q2);
        for (const auto &kv : taps)
          if (kv.second.d != 0.0) rows[e].push_back({kv.first, kv.second.d});
        dW[e] = W.d;
        maxnt = std::max(maxnt, int(rows[e].size()));
      }
  FineDTabHost d;
  d.stride = (maxnt + 3) / 4 * 4;
  d.dx.assign(size_t(E) * d.stride, 0);
  d.dy.assign(size_t(E) * d.stride, 0);
  d.dw.assign(size_t(E) * d.stride, 0.0);
  d.nt.assign(E, 0);
  d.dW = dW;
  for (int e = 0; e < E; ++e) {
    d.nt[e] = uint8_t(rows[e].size());
    for (size_t s = 0; s < rows[e].size(); ++s) {
      d.dy[size_t(e) * d.stride + s] = rows[e][s].first.first;
      d.dx[size_t(e) * d.stride + s] = rows[e][s].first.second;
      d.dw[size_t(e) * d.stride + s] = rows[e][s].second;
    }
  }
  return d;
}

NodeTabHost build_node_tables(int n, double h, int P, const double *field) {
  NodeTabHost t;
  const int m = n - 2;
  const double sqh = std::sqrt(h);
  t.stride = 4 * 2 * P;
  t.dx.assign(size_t(m) * m * t.stride, 0);
  t.dy.assign(t.dx.size(), 0);
  t.w.assign(t.dx.size(), 0.0);
  t.nt.assign(size_t(m) * m, 0);
  t.W.assign(size_t(m) * m, 0.0);
  for (int i2 = 1; i2 <= m; ++i2)
    for (int i1 = 1; i1 <= m; ++i1) {
      const size_t I = size_t(i2 - 1) * m + (i1 - 1);
      const double *sg = field + (size_t(i2) * n + i1) * 2 * P;
      TapMap taps;
      double W = 0.0;
      for (int p = 0; p < P; ++p) {
        const double s1 = sg[0 * P + p] / sqh, s2 = sg[1 * P + p] / sqh;
        Endpoint ep = truncate_endpoint(i1, i2, s1, s2, n);
        Endpoint em = truncate_endpoint(i1, i2, -s1, -s2, n);
        const double A = 2.0 / (ep.mu * ep.mu + ep.mu * em.mu);
        const double Bw = 2.0 / (em.mu * em.mu + em.mu * ep.mu);
        add_bilinear(taps, i1, i2, ep.z1, ep.z2, n, A / (2.0 * h));
        add_bilinear(taps, i1, i2, em.z1, em.z2, n, Bw / (2.0 * h));
        W += (A + Bw) / (2.0 * h);
      }
      if (int(taps.size()) > t.stride) throw std::runtime_error("node stencil table overflow");
      int slot = 0;
      for (const auto &kv : taps) {
        t.dy[I * t.stride + slot] = kv.first.first;
        t.dx[I * t.stride + slot] = kv.first.second;
        t.w[I * t.stride + slot] = kv.second;
        t.R0 = std::max(t.R0, std::max(std::abs(kv.first.first), std::abs(kv.first.second)));
        ++slot;
      }
      t.nt[I] = uint8_t(slot);
      t.W[I] = W;
    }
  return t;
}

std::vector<double> fine_interior_window(const FineTabHost &t, int k, double dt) {
  const int R = t.R0, Wd = 2 * R + 1;
  std::vector<double> win(size_t(Wd) * Wd, 0.0);
  const int e = t.entry(k, class_q(t.B, t.n, t.B), class_q(t.B, t.n, t.B));
  win[size_t(R) * Wd + R] = 1.0 + dt * (t.W[e] - t.c[k]);
  for (int s = 0; s < t.nt[e]; ++s) {
    const size_t ix = size_t(e) * t.tmax + s;
    win[size_t(t.dy[ix] + R) * Wd + (t.dx[ix] + R)] -= dt * t.w[ix];
  }
  return win;
}

std::vector<double> rap_class_window(const std::vector<double> &prev, int Rprev, int R) {
  // Coarse row I = (I0, I0) with all nine level-(l-1) rows 2I + a having the window `prev`.
  const int Wp = 2 * Rprev + 1, Wd = 2 * R + 1;
  std::vector<double> win(size_t(Wd) * Wd, 0.0);
  const int I0 = 4 * (R + Rprev + 4);
  for (int a2 = -1; a2 <= 1; ++a2)
    for (int a1 = -1; a1 <= 1; ++a1) {
      const double ra = fw_weight(a1) * fw_weight(a2);
      const int i1 = 2 * I0 + a1, i2 = 2 * I0 + a2;
      for (int o2 = -Rprev; o2 <= Rprev; ++o2)
        for (int o1 = -Rprev; o1 <= Rprev; ++o1) {
          const double v = prev[size_t(o2 + Rprev) * Wp + (o1 + Rprev)];
          if (v == 0.0) continue;
          rap_scatter<double>(win.data(), R, I0, I0, i1 + o1, i2 + o2, ra * v);
        }
    }
  return win;
}

}  // namespace sl
