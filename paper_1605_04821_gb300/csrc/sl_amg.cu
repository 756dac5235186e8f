// sl_amg.cu - aggregation-based AMG with a K-cycle (the paper's recommended class of solver,
// Section 3.4: aggregation multigrid as a Krylov preconditioner, justified by the M-matrix
// property with non-negative row and column sums of Prop. 3.1).
//
// Coarsening, one level = two pairwise passes (aggregates of at most four unknowns):
//   strength s_ij = -(a_ij + a_ji)/2, the off-diagonal part of the symmetric part of A on the
//   union of the patterns of A and A^T (zeros dropped); j is strong for i when
//   s_ij > 0 and s_ij >= 0.25 max_k s_ik; in each of kAmgRounds rounds every unmatched
//   unknown proposes its strong unmatched neighbour that is largest in the edge order
//   (exponent of s_ij, fmix32(min ^ fmix32(max)), -j) (fmix32: MurmurHash3's 32-bit
//   finalizer; strengths within a factor two rank equal and the hash orders them), and two
//   unknowns that propose each other pair up; aggregates are numbered in the order of their
//   lowest member; the coarse matrix is the Galerkin product P^T A P with piecewise-constant P.
//   Coarsening stops at kAmgCoarsest unknowns or when a level keeps more than 3/4 of the
//   unknowns above it; a last level above kAmgCoarsest is solved by kAmgCoarseSweeps damped
//   Jacobi sweeps instead of a dense solve.
// Cycle: damped Jacobi smoothing; the coarse correction of level l is approximated by GCR on
//   level l+1 preconditioned by the cycle of level l+1 (two GCR steps on levels 1..k_levels,
//   one below), with an exact dense solve on the coarsest level.
// All scalars of the cycle stay on the device and every reduction is in a fixed order, so a
// cycle is deterministic and can be captured in a CUDA graph.
#include "sl_amg.h"

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/sl_hjb.h"

namespace sl {

namespace {
constexpr int kAT = 256;
constexpr int kDotBlocks = 608;
inline int nblk(long long n) { return int((n + kAT - 1) / kAT); }
}  // namespace

// ----------------------------------------------------------------------------- level 0
// Row I of the step matrix from the fine tables, columns sorted, equal columns merged (in tap
// order).  PASS 0 counts, PASS 1 writes.
template <int PASS>
__global__ void __launch_bounds__(kAT) k_amg_csr0(FineTab tab, const int32_t *__restrict__ off,
                                                   const uint8_t *__restrict__ policy, double dt,
                                                   const int32_t *__restrict__ rowptr, int *__restrict__ cnt,
                                                   int32_t *__restrict__ col, double *__restrict__ val) {
  const int m = tab.m;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= m * m) return;
  const int i1 = 1 + I % m, i2 = 1 + I / m;
  const int k = policy[I];
  const int e = fine_row_entry(tab, k, i1, i2);
  int c[64];
  double v[64];
  int len = 1;
  c[0] = I;
  v[0] = 1.0 + dt * (tab.W64[e] - tab.c64[k]) - dt * tab.ws64[e];
  for (int t = 0; t < tab.nt[e]; ++t) {
    const int o = off[e * tab.tmax + t];
    const int dx = int(int16_t(o & 0xffff)), dy = o >> 16;
    const int j1 = i1 + dx, j2 = i2 + dy;
    if ((dx | dy) == 0 || j1 < 1 || j1 > m || j2 < 1 || j2 > m) continue;
    const int J = (j2 - 1) * m + (j1 - 1);
    const double w = -dt * tab.w64[e * tab.tmax + t];
    int p = len - 1;
    while (p >= 0 && c[p] > J) --p;
    if (p >= 0 && c[p] == J) {
      v[p] += w;
    } else if (len < 64) {
      for (int q = len; q > p + 1; --q) { c[q] = c[q - 1]; v[q] = v[q - 1]; }
      c[p + 1] = J;
      v[p + 1] = w;
      ++len;
    }
  }
  if (PASS == 0) {
    cnt[I] = len;
  } else {
    const int base = rowptr[I];
    for (int a = 0; a < len; ++a) { col[base + a] = c[a]; val[base + a] = v[a]; }
  }
}

// ----------------------------------------------------------------------------- matching
__device__ __forceinline__ unsigned fmix32(unsigned x) {
  x ^= x >> 16;
  x *= 0x85ebca6bu;
  x ^= x >> 13;
  x *= 0xc2b2ae35u;
  x ^= x >> 16;
  return x;
}
__device__ __forceinline__ unsigned edge_hash(int i, int j) {
  const unsigned a = unsigned(min(i, j)), b = unsigned(max(i, j));
  return fmix32(a ^ fmix32(b));
}

// A^T of a CSR matrix: count per column, then scatter (atomic slots), then order every row.
__global__ void k_amg_tr_count(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                               int *__restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) atomicAdd(cnt + col[p], 1);
}

__global__ void k_amg_tr_fill(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                              const double *__restrict__ v, const int32_t *__restrict__ rpT,
                              int *__restrict__ fill, int32_t *__restrict__ colT, double *__restrict__ vT) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
    const int j = col[p];
    const int pos = rpT[j] + atomicAdd(fill + j, 1);
    colT[pos] = i;
    vT[pos] = v[p];
  }
}

// Stable insertion sort of one segment by column (values carried along): in registers when
// the segment is short, in place otherwise.
__device__ void sort_segment(int32_t *__restrict__ col, double *__restrict__ val, int lo, int len) {
  if (len <= kAmgRowMax) {
    int c[kAmgRowMax];
    double w[kAmgRowMax];
    for (int a = 0; a < len; ++a) {
      const int ca = col[lo + a];
      const double wa = val[lo + a];
      int b = a - 1;
      while (b >= 0 && c[b] > ca) { c[b + 1] = c[b]; w[b + 1] = w[b]; --b; }
      c[b + 1] = ca;
      w[b + 1] = wa;
    }
    for (int a = 0; a < len; ++a) { col[lo + a] = c[a]; val[lo + a] = w[a]; }
    return;
  }
  for (int a = lo + 1; a < lo + len; ++a) {
    const int ca = col[a];
    const double wa = val[a];
    int b = a - 1;
    while (b >= lo && col[b] > ca) { col[b + 1] = col[b]; val[b + 1] = val[b]; --b; }
    col[b + 1] = ca;
    val[b + 1] = wa;
  }
}

__global__ void __launch_bounds__(kAT) k_amg_tr_sort(int n, const int32_t *__restrict__ rpT,
                                                      int32_t *__restrict__ colT, double *__restrict__ vT) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  sort_segment(colT, vT, rpT[j], rpT[j + 1] - rpT[j]);
}

// Row i of the strength matrix: union of row i of A and of A^T (both sorted), value
// -(a_ij + a_ji)/2, the diagonal and zero values dropped; PASS 1 also writes the row maximum.
template <int PASS>
__global__ void __launch_bounds__(kAT) k_amg_sym(int n, const int32_t *__restrict__ rowptr,
                                                 const int32_t *__restrict__ col, const double *__restrict__ v,
                                                 const int32_t *__restrict__ rpT, const int32_t *__restrict__ colT,
                                                 const double *__restrict__ vT, const int32_t *__restrict__ rpS,
                                                 int *__restrict__ cnt, int32_t *__restrict__ colS,
                                                 double *__restrict__ s, double *__restrict__ smax) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int p = rowptr[i], pe = rowptr[i + 1], q = rpT[i], qe = rpT[i + 1];
  int len = 0;
  double mx = 0.0;
  const int base = PASS ? rpS[i] : 0;
  while (p < pe || q < qe) {
    const int cp = p < pe ? col[p] : INT32_MAX, cq = q < qe ? colT[q] : INT32_MAX;
    const int j = min(cp, cq);
    const double a = (cp == j) ? v[p] : 0.0;
    const double b = (cq == j) ? vT[q] : 0.0;
    if (cp == j) ++p;
    if (cq == j) ++q;
    if (j == i) continue;
    const double sv = -(a + b) / 2.0;
    if (sv == 0.0) continue;
    if (PASS) {
      colS[base + len] = j;
      s[base + len] = sv;
      mx = len ? fmax(mx, sv) : sv;
    }
    ++len;
  }
  if (PASS == 0) cnt[i] = len;
  else smax[i] = len ? mx : 0.0;
}

__global__ void __launch_bounds__(kAT) k_amg_propose(int n, const int32_t *__restrict__ rowptr,
                                                      const int32_t *__restrict__ col,
                                                      const double *__restrict__ s,
                                                      const double *__restrict__ smax,
                                                      const int *__restrict__ partner, int *__restrict__ prop) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (partner[i] >= 0) {
    prop[i] = -1;
    return;
  }
  const double thr = 0.25 * smax[i];
  int best = -1, be = 0;
  unsigned bh = 0u;
  for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {  // the strength pattern (no diagonal)
    const int j = col[p];
    const double sv = s[p];
    if (partner[j] >= 0 || !(sv > 0.0) || sv < thr) continue;
    int e;
    frexp(sv, &e);  // sv = m 2^e, m in [0.5, 1): exact
    const unsigned h = edge_hash(i, j);
    if (best < 0 || e > be || (e == be && (h > bh || (h == bh && j < best)))) {
      best = j;
      be = e;
      bh = h;
    }
  }
  prop[i] = best;
}

__global__ void k_amg_accept(int n, const int *__restrict__ prop, int *__restrict__ partner) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int j = prop[i];
  if (j >= 0 && prop[j] == i) partner[i] = j;
}

__global__ void k_amg_leader(int n, const int *__restrict__ partner, int *__restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int j = partner[i];
  flag[i] = (j < 0 || i < j) ? 1 : 0;
}

// agg[i] and the (at most two) members of every aggregate, leader first.
__global__ void k_amg_assign(int n, const int *__restrict__ partner, const int32_t *__restrict__ ids,
                             int32_t *__restrict__ agg, int32_t *__restrict__ mem) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int j = partner[i];
  if (!(j < 0 || i < j)) return;
  const int id = ids[i];
  agg[i] = id;
  mem[2 * id] = i;
  mem[2 * id + 1] = j;
  if (j >= 0) agg[j] = id;
}

// Composes two passes: agg[i] = a2[a1[i]], members of every final aggregate ascending.
__global__ void k_amg_compose(int n, int nc, const int32_t *__restrict__ a1, const int32_t *__restrict__ a2,
                              const int32_t *__restrict__ mem1, const int32_t *__restrict__ mem2,
                              int32_t *__restrict__ agg, int32_t *__restrict__ mem4) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) agg[t] = a2[a1[t]];
  if (t < nc) {
    int m[4] = {-1, -1, -1, -1};
    int c = 0;
    for (int q = 0; q < 2; ++q) {
      const int A = mem2[2 * t + q];
      if (A < 0) continue;
      for (int r = 0; r < 2; ++r) {
        const int i = mem1[2 * A + r];
        if (i >= 0) m[c++] = i;
      }
    }
    for (int a = 1; a < c; ++a) {  // ascending
      const int x = m[a];
      int b = a - 1;
      while (b >= 0 && m[b] > x) { m[b + 1] = m[b]; --b; }
      m[b + 1] = x;
    }
    for (int q = 0; q < 4; ++q) mem4[4 * t + q] = m[q];
  }
}

// Galerkin product P^T A P.  The entries of coarse row I are those of its member rows
// (members ascending, entries in column order) with columns mapped to aggregates; they are
// written unmerged (their total is nnz(A)), ordered by a stable sort, and merged, so equal
// columns are summed in that order.
template <int MS>
__global__ void k_gal_rawcount(int nc, const int32_t *__restrict__ mem, const int32_t *__restrict__ rowptr,
                               int *__restrict__ cnt) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  int c = 0;
  for (int q = 0; q < MS; ++q) {
    const int i = mem[MS * I + q];
    if (i >= 0) c += rowptr[i + 1] - rowptr[i];
  }
  cnt[I] = c;
}

template <int MS>
__global__ void k_gal_rawfill(int nc, const int32_t *__restrict__ mem, const int32_t *__restrict__ agg,
                              const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                              const double *__restrict__ v, const int32_t *__restrict__ rawptr,
                              int32_t *__restrict__ rawcol, double *__restrict__ rawval) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  int o = rawptr[I];
  for (int q = 0; q < MS; ++q) {
    const int i = mem[MS * I + q];
    if (i < 0) continue;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p, ++o) {
      rawcol[o] = agg[col[p]];
      rawval[o] = v[p];
    }
  }
}

__global__ void __launch_bounds__(kAT) k_gal_sort(int nc, const int32_t *__restrict__ rawptr,
                                                   int32_t *__restrict__ rawcol, double *__restrict__ rawval) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  sort_segment(rawcol, rawval, rawptr[I], rawptr[I + 1] - rawptr[I]);
}

template <int PASS>
__global__ void k_gal_merge(int nc, const int32_t *__restrict__ rawptr, const int32_t *__restrict__ rawcol,
                            const double *__restrict__ rawval, const int32_t *__restrict__ rowptr_c,
                            int *__restrict__ cnt_c, int32_t *__restrict__ col_c, double *__restrict__ v_c) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  int len = 0;
  const int base = PASS ? rowptr_c[I] : 0;
  for (int p = rawptr[I]; p < rawptr[I + 1];) {
    const int c = rawcol[p];
    double acc = rawval[p];
    for (++p; p < rawptr[I + 1] && rawcol[p] == c; ++p) acc += rawval[p];
    if (PASS) {
      col_c[base + len] = c;
      v_c[base + len] = acc;
    }
    ++len;
  }
  if (!PASS) cnt_c[I] = len;
}

__global__ void k_amg_diag(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                           const double *__restrict__ v, double *__restrict__ d64, float *__restrict__ d32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0;
  for (int p = rowptr[i]; p < rowptr[i + 1]; ++p)
    if (col[p] == i) d = v[p];
  d64[i] = d;
  d32[i] = float(d);
}

__global__ void k_amg_f32(long long nnz, const double *__restrict__ v, float *__restrict__ v32) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nnz; p += (long long)gridDim.x * blockDim.x)
    v32[p] = float(v[p]);
}

// Dense inverse of the coarsest matrix (n <= kAmgCoarsest) by Gauss-Jordan elimination with
// partial pivoting, in one thread block.
__global__ void k_amg_dense_inverse(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                    const double *__restrict__ v, double *__restrict__ work,
                                    double *__restrict__ Ainv64, float *__restrict__ Ainv32) {
  double *A = work, *Inv = work + size_t(n) * n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    A[idx] = 0.0;
    Inv[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x)
    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) A[size_t(r) * n + col[p]] += v[p];
  __syncthreads();
  __shared__ int piv;
  for (int c = 0; c < n; ++c) {
    if (threadIdx.x == 0) {
      int p = c;
      double best = fabs(A[size_t(c) * n + c]);
      for (int r = c + 1; r < n; ++r) {
        const double a = fabs(A[size_t(r) * n + c]);
        if (a > best) { best = a; p = r; }
      }
      piv = p;
    }
    __syncthreads();
    const int p = piv;
    if (p != c)
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double t0 = A[size_t(c) * n + k]; A[size_t(c) * n + k] = A[size_t(p) * n + k]; A[size_t(p) * n + k] = t0;
        double t1 = Inv[size_t(c) * n + k]; Inv[size_t(c) * n + k] = Inv[size_t(p) * n + k]; Inv[size_t(p) * n + k] = t1;
      }
    __syncthreads();
    const double inv = 1.0 / A[size_t(c) * n + c];
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      A[size_t(c) * n + k] *= inv;
      Inv[size_t(c) * n + k] *= inv;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      if (r == c) continue;
      const double f = A[size_t(r) * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        A[size_t(r) * n + k] -= f * A[size_t(c) * n + k];
        Inv[size_t(r) * n + k] -= f * Inv[size_t(c) * n + k];
      }
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    Ainv64[idx] = Inv[idx];
    Ainv32[idx] = float(Inv[idx]);
  }
}

// ----------------------------------------------------------------------------- cycle kernels
template <typename T, int OP>
__global__ void __launch_bounds__(kAT) k_amg_op(int n, const int32_t *__restrict__ rowptr,
                                                 const int32_t *__restrict__ col, const T *__restrict__ v,
                                                 const T *__restrict__ d, T omega, const T *__restrict__ x,
                                                 const T *__restrict__ b, T *__restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (OP == OP_JACOBI0) {
    y[i] = omega * b[i] / d[i];
    return;
  }
  // eight entries per pass, their columns and values and then the x values loaded before the
  // FMAs (chaining column -> x -> FMA per entry cost two memory round trips per entry); the
  // entries are added in the same order
  T acc = T(0);
  const int lo = rowptr[i], hi = rowptr[i + 1];
  for (int p0 = lo; p0 < hi; p0 += 8) {
    int cj[8];
    T vv[8], xv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const bool in = p0 + u < hi;
      cj[u] = in ? col[p0 + u] : i;
      vv[u] = in ? v[p0 + u] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) xv[u] = p0 + u < hi ? x[cj[u]] : T(0);
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (p0 + u < hi) acc = fma(vv[u], xv[u], acc);
  }
  if (OP == OP_APPLY) y[i] = acc;
  else if (OP == OP_RESID) y[i] = b[i] - acc;
  else y[i] = x[i] + omega * (b[i] - acc) / d[i];
}

template <typename T>
__global__ void k_amg_restrict(int nc, const int32_t *__restrict__ mem4, const T *__restrict__ r,
                               T *__restrict__ bc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  T acc = T(0);
  for (int q = 0; q < 4; ++q) {
    const int i = mem4[4 * I + q];
    if (i >= 0) acc += r[i];
  }
  bc[I] = acc;
}

template <typename T>
__global__ void k_amg_prolong(int n, const int32_t *__restrict__ agg, const T *__restrict__ e, T *__restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] += e[agg[i]];
}

template <typename T>
__global__ void k_amg_dense(int n, const T *__restrict__ Ainv, const T *__restrict__ b, T *__restrict__ x) {
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    T acc = T(0);
    for (int c0 = 0; c0 < n; c0 += 8) {  // eight loads in flight, then the FMAs in order
      T av[8], bv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        av[u] = c0 + u < n ? Ainv[size_t(r) * n + c0 + u] : T(0);
        bv[u] = c0 + u < n ? b[c0 + u] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (c0 + u < n) acc = fma(av[u], bv[u], acc);
    }
    x[r] = acc;
  }
}

template <typename T>
__global__ void k_amg_copy(int n, const T *__restrict__ a, T *__restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

// partials[2 blk + {0,1}] = block sums of a.b and c.d (FP64 accumulation), fixed grid.
template <typename T>
__global__ void __launch_bounds__(kAT) k_amg_dots(int n, const T *__restrict__ a, const T *__restrict__ b,
                                                   const T *__restrict__ c, const T *__restrict__ d,
                                                   double *__restrict__ partials) {
  double s0 = 0.0, s1 = 0.0;
  const int st = gridDim.x * blockDim.x;
  for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += 4 * st) {
    T av[4], bv[4], cv[4], dv[4];  // four elements' loads, then the sums in the same order
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * st;
      const bool in = i < n;
      av[u] = in ? a[i] : T(0);
      bv[u] = in ? b[i] : T(0);
      cv[u] = in ? c[i] : T(0);
      dv[u] = in ? d[i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (i0 + u * st < n) {
        s0 = fma(double(av[u]), double(bv[u]), s0);
        s1 = fma(double(cv[u]), double(dv[u]), s1);
      }
    }
  }
  __shared__ double sh[2][kAT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sh[0][wid] = s0; sh[1][wid] = s1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < kAT / 32; ++w) { t0 += sh[0][w]; t1 += sh[1][w]; }
    partials[2 * blockIdx.x] = t0;
    partials[2 * blockIdx.x + 1] = t1;
  }
}

__global__ void k_amg_dots_final(int nb, const double *__restrict__ partials, double *__restrict__ out) {
  double s0 = 0.0, s1 = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) { s0 += partials[2 * b]; s1 += partials[2 * b + 1]; }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if (threadIdx.x == 0) { out[0] = s0; out[1] = s1; }
}

// e = a1 v1 with a1 = (w1.r)/(w1.w1) (0 for a zero denominator); with a second step also
// r2 = r - a1 w1.
template <typename T>
__global__ void k_gcr_first(int n, const T *__restrict__ v1, const T *__restrict__ w1, const T *__restrict__ r,
                            T *__restrict__ e, T *__restrict__ r2, const double *__restrict__ scal, int two) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a1 = scal[1] > 0.0 ? scal[0] / scal[1] : 0.0;
  e[i] = T(a1) * v1[i];
  if (two) r2[i] = r[i] - T(a1) * w1[i];
}

// g = (w2.w1)/(w1.w1); w2 -= g w1; v2 -= g v1.
template <typename T>
__global__ void k_gcr_orth(int n, T *__restrict__ v2, T *__restrict__ w2, const T *__restrict__ v1,
                           const T *__restrict__ w1, const double *__restrict__ scal) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double g = scal[1] > 0.0 ? scal[2] / scal[1] : 0.0;
  w2[i] -= T(g) * w1[i];
  v2[i] -= T(g) * v1[i];
}

// e += a2 v2 with a2 = (w2.r2)/(w2.w2).
template <typename T>
__global__ void k_gcr_second(int n, T *__restrict__ e, const T *__restrict__ v2, const double *__restrict__ scal) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a2 = scal[4] > 0.0 ? scal[3] / scal[4] : 0.0;
  e[i] += T(a2) * v2[i];
}

template <typename T>
__global__ void k_amg_gather(int n, const T *__restrict__ full, T *__restrict__ compact) {
  const int m = n - 2;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I < m * m) compact[I] = full[(1 + I / m) * n + 1 + I % m];
}

template <typename T>
__global__ void k_amg_scatter(int n, const T *__restrict__ compact, T *__restrict__ full) {
  const int m = n - 2;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I < m * m) full[(1 + I / m) * n + 1 + I % m] = compact[I];
}

// ----------------------------------------------------------------------------- host side
namespace {

template <typename P>
cudaError_t grow(AmgEngine &E, P **p, size_t *cap, size_t count) {
  if (*p && *cap >= count) return cudaSuccess;
  if (*p) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    E.allocs.erase(std::find(E.allocs.begin(), E.allocs.end(), static_cast<void *>(*p)));
    cudaFree(*p);
    *p = nullptr;
  }
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(P));
  if (e != cudaSuccess) return e;
  E.allocs.push_back(*p);
  *cap = count;
  return cudaMemset(*p, 0, count * sizeof(P));
}

#define AMG_CK(call)                         \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return e_;        \
  } while (0)

template <typename T> T *vec(AmgLevel &L, int k);
template <> double *vec<double>(AmgLevel &L, int k) { return L.vec64[k]; }
template <> float *vec<float>(AmgLevel &L, int k) { return L.vec32[k]; }
template <typename T> const T *vals(const AmgLevel &L);
template <> const double *vals<double>(const AmgLevel &L) { return L.v64; }
template <> const float *vals<float>(const AmgLevel &L) { return L.v32; }
template <typename T> const T *diag(const AmgLevel &L);
template <> const double *diag<double>(const AmgLevel &L) { return L.d64; }
template <> const float *diag<float>(const AmgLevel &L) { return L.d32; }
template <typename T> const T *ainv(const AmgEngine &E);
template <> const double *ainv<double>(const AmgEngine &E) { return E.Ainv64; }
template <> const float *ainv<float>(const AmgEngine &E) { return E.Ainv32; }

cudaError_t read_int(AmgEngine &E, const int *dev, int *out, cudaStream_t s) {
  AMG_CK(cudaMemcpyAsync(E.h_int, dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  AMG_CK(cudaStreamSynchronize(s));
  *out = *E.h_int;
  return cudaSuccess;
}

// One pairwise pass on the CSR (n, rowptr, col, v): partner via kAmgRounds rounds, then the
// aggregate numbering (agg, two members each).  Returns the number of aggregates in *nc.
cudaError_t pairwise_pass(AmgEngine &E, int n, const int32_t *rowptr, const int32_t *col, const double *v,
                          int32_t *agg, int32_t *mem, int *nc, cudaStream_t s) {
  // A^T, then the strength matrix on the union pattern
  AMG_CK(cudaMemsetAsync(E.cnt, 0, size_t(n) * sizeof(int), s));
  AMG_CK(cudaMemsetAsync(E.err, 0, sizeof(int32_t), s));
  note_launch(1);
  k_amg_tr_count<<<nblk(n), kAT, 0, s>>>(n, rowptr, col, E.cnt);
  launch_exclusive_scan(E.cnt, n, E.rpT, E.scan, s);
  AMG_CK(cudaMemsetAsync(E.cnt, 0, size_t(n) * sizeof(int), s));
  note_launch(4);
  k_amg_tr_fill<<<nblk(n), kAT, 0, s>>>(n, rowptr, col, v, E.rpT, E.cnt, E.colT, E.vT);
  k_amg_tr_sort<<<nblk(n), kAT, 0, s>>>(n, E.rpT, E.colT, E.vT);
  k_amg_sym<0><<<nblk(n), kAT, 0, s>>>(n, rowptr, col, v, E.rpT, E.colT, E.vT, nullptr, E.cnt, nullptr, nullptr,
                                       nullptr);
  launch_exclusive_scan(E.cnt, n, E.rpS, E.scan, s);
  k_amg_sym<1><<<nblk(n), kAT, 0, s>>>(n, rowptr, col, v, E.rpT, E.colT, E.vT, E.rpS, nullptr, E.colS, E.s,
                                       E.smax);
  AMG_CK(cudaMemsetAsync(E.partner, 0xff, size_t(n) * sizeof(int), s));
  for (int r = 0; r < kAmgRounds; ++r) {
    note_launch(2);
    k_amg_propose<<<nblk(n), kAT, 0, s>>>(n, E.rpS, E.colS, E.s, E.smax, E.partner, E.prop);
    k_amg_accept<<<nblk(n), kAT, 0, s>>>(n, E.prop, E.partner);
  }
  note_launch(1);
  k_amg_leader<<<nblk(n), kAT, 0, s>>>(n, E.partner, E.flag);
  launch_exclusive_scan(E.flag, n, E.ids, E.scan, s);
  AMG_CK(read_int(E, E.ids + n, nc, s));
  note_launch(1);
  k_amg_assign<<<nblk(n), kAT, 0, s>>>(n, E.partner, E.ids, agg, mem);
  return cudaGetLastError();
}

// Galerkin product into (rowptr_c, col_c, v_c): own_storage grows the coarse level's arrays,
// otherwise they are scratch of capacity *cap_c.
template <int MS>
cudaError_t galerkin(AmgEngine &E, int nc, const int32_t *mem, const int32_t *agg, const int32_t *rowptr,
                     const int32_t *col, const double *v, int32_t *rowptr_c, int32_t **col_c, double **v_c,
                     float **v32_c, size_t *cap_c, long long *nnz, bool own_storage, cudaStream_t s) {
  note_launch(3);
  k_gal_rawcount<MS><<<nblk(nc), kAT, 0, s>>>(nc, mem, rowptr, E.cnt);
  launch_exclusive_scan(E.cnt, nc, E.rawptr, E.scan, s);
  k_gal_rawfill<MS><<<nblk(nc), kAT, 0, s>>>(nc, mem, agg, rowptr, col, v, E.rawptr, E.rawcol, E.rawval);
  k_gal_sort<<<nblk(nc), kAT, 0, s>>>(nc, E.rawptr, E.rawcol, E.rawval);
  note_launch(1);
  k_gal_merge<0><<<nblk(nc), kAT, 0, s>>>(nc, E.rawptr, E.rawcol, E.rawval, nullptr, E.cnt, nullptr, nullptr);
  launch_exclusive_scan(E.cnt, nc, rowptr_c, E.scan, s);
  int total = 0;
  AMG_CK(read_int(E, rowptr_c + nc, &total, s));
  if (own_storage) {  // col, v64 and v32 share one capacity
    size_t c1 = *cap_c, c2 = *cap_c, c3 = *cap_c;
    AMG_CK(grow(E, col_c, &c1, size_t(total)));
    AMG_CK(grow(E, v_c, &c2, size_t(total)));
    AMG_CK(grow(E, v32_c, &c3, size_t(total)));
    *cap_c = std::min(c1, std::min(c2, c3));
  } else if (size_t(total) > *cap_c) {
    E.err_msg = "pass-1 coarse matrix larger than its scratch";
    return cudaErrorInvalidValue;
  }
  note_launch(1);
  k_gal_merge<1><<<nblk(nc), kAT, 0, s>>>(nc, E.rawptr, E.rawcol, E.rawval, rowptr_c, nullptr, *col_c, *v_c);
  *nnz = total;
  return cudaGetLastError();
}

cudaError_t level_vectors(AmgEngine &E, AmgLevel &L, bool gcr) {
  const int kmax = gcr ? AV_COUNT : AV_V1;
  if (L.cap_vec >= size_t(L.n) && L.vec64[0] && (!gcr || L.vec64[AV_V1])) return cudaSuccess;
  size_t c0 = 0;
  for (int k = 0; k < kmax; ++k) {
    size_t ca = 0, cb = 0;
    if (L.vec64[k]) { E.allocs.erase(std::find(E.allocs.begin(), E.allocs.end(), (void *)L.vec64[k])); cudaFree(L.vec64[k]); L.vec64[k] = nullptr; }
    if (L.vec32[k]) { E.allocs.erase(std::find(E.allocs.begin(), E.allocs.end(), (void *)L.vec32[k])); cudaFree(L.vec32[k]); L.vec32[k] = nullptr; }
    AMG_CK(grow(E, &L.vec64[k], &ca, size_t(L.n)));
    AMG_CK(grow(E, &L.vec32[k], &cb, size_t(L.n)));
    c0 = ca;
  }
  L.cap_vec = c0;
  if (!L.scal) {
    size_t cs = 0;
    AMG_CK(grow(E, &L.scal, &cs, 8));
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t amg_reserve_level0(AmgEngine &E, int n, long long nnz) {
  AmgLevel &L = E.lev[0];
  size_t c1 = L.cap_nnz, c2 = L.cap_nnz, c3 = L.cap_nnz, cn2 = L.cap_n, cn3 = L.cap_n;
  AMG_CK(grow(E, &L.rowptr, &L.cap_rp, size_t(n) + 1));
  AMG_CK(grow(E, &L.d64, &cn2, size_t(n)));
  AMG_CK(grow(E, &L.d32, &cn3, size_t(n)));
  AMG_CK(grow(E, &L.col, &c1, size_t(nnz)));
  AMG_CK(grow(E, &L.v64, &c2, size_t(nnz)));
  AMG_CK(grow(E, &L.v32, &c3, size_t(nnz)));
  L.cap_n = std::min(cn2, cn3);
  L.cap_nnz = std::min(c1, std::min(c2, c3));
  // setup scratch: every level is at most this large
  if (E.cap_n < size_t(n) || E.cap_nnz < size_t(nnz)) {
    size_t a = 2 * E.cap_nnz, b = E.cap_nnz, c = E.cap_nnz, d = 2 * E.cap_nnz, f = E.cap_nnz, g = E.cap_nnz;
    AMG_CK(grow(E, &E.s, &a, 2 * size_t(nnz)));
    AMG_CK(grow(E, &E.colS, &d, 2 * size_t(nnz)));
    AMG_CK(grow(E, &E.t_col, &b, size_t(nnz)));
    AMG_CK(grow(E, &E.t_v, &c, size_t(nnz)));
    AMG_CK(grow(E, &E.colT, &f, size_t(nnz)));
    AMG_CK(grow(E, &E.vT, &g, size_t(nnz)));
    size_t h1 = E.cap_nnz, h2 = E.cap_nnz, h3 = E.cap_n ? E.cap_n + 1 : 0;
    AMG_CK(grow(E, &E.rawcol, &h1, size_t(nnz)));
    AMG_CK(grow(E, &E.rawval, &h2, size_t(nnz)));
    AMG_CK(grow(E, &E.rawptr, &h3, size_t(n) + 1));
    size_t r1 = E.cap_n ? E.cap_n + 1 : 0, r2 = r1;
    AMG_CK(grow(E, &E.rpT, &r1, size_t(n) + 1));
    AMG_CK(grow(E, &E.rpS, &r2, size_t(n) + 1));
    size_t q[12] = {E.cap_n, E.cap_n, E.cap_n, E.cap_n, E.cap_n, E.cap_n, E.cap_n, E.cap_n, E.cap_n, E.cap_n, E.cap_n, E.cap_n};
    AMG_CK(grow(E, &E.smax, &q[0], size_t(n)));
    AMG_CK(grow(E, &E.partner, &q[1], size_t(n)));
    AMG_CK(grow(E, &E.prop, &q[2], size_t(n)));
    AMG_CK(grow(E, &E.flag, &q[3], size_t(n)));
    AMG_CK(grow(E, &E.cnt, &q[4], size_t(n)));
    AMG_CK(grow(E, &E.ids, &q[5], size_t(n) + 1));
    AMG_CK(grow(E, &E.a1, &q[6], size_t(n)));
    AMG_CK(grow(E, &E.mem1, &q[7], 2 * size_t(n)));
    AMG_CK(grow(E, &E.mem2, &q[8], 2 * size_t(n)));
    AMG_CK(grow(E, &E.t_rowptr, &q[9], size_t(n) + 1));
    AMG_CK(grow(E, &E.scan, &q[10], 2 * (size_t(n) + 1023) / 1024 + 4));
    E.cap_n = size_t(n);
    E.cap_nnz = size_t(nnz);
  }
  if (!E.err) {
    size_t c0 = 0, c1b = 0, c2b = 0, c3b = 0, c4b = 0;
    AMG_CK(grow(E, &E.err, &c0, 1));
    AMG_CK(grow(E, &E.partials, &c1b, 2 * size_t(kDotBlocks)));
    AMG_CK(grow(E, &E.Ainv64, &c2b, size_t(kAmgCoarsest) * kAmgCoarsest));
    AMG_CK(grow(E, &E.Ainv32, &c3b, size_t(kAmgCoarsest) * kAmgCoarsest));
    AMG_CK(grow(E, &E.work, &c4b, 2 * size_t(kAmgCoarsest) * kAmgCoarsest));
    AMG_CK(cudaMallocHost(reinterpret_cast<void **>(&E.h_int), sizeof(int)));
  }
  L.n = n;
  return cudaSuccess;
}

cudaError_t amg_level0_from_tables(AmgEngine &E, const FineTab &tab, const int32_t *off, const uint8_t *policy,
                                   double dt, cudaStream_t s) {
  const int n = tab.m * tab.m;
  AMG_CK(amg_reserve_level0(E, n, (long long)n * (1 + tab.tmax)));
  AmgLevel &L = E.lev[0];
  note_launch(1);
  k_amg_csr0<0><<<nblk(n), kAT, 0, s>>>(tab, off, policy, dt, nullptr, E.cnt, nullptr, nullptr);
  launch_exclusive_scan(E.cnt, n, L.rowptr, E.scan, s);
  note_launch(1);
  k_amg_csr0<1><<<nblk(n), kAT, 0, s>>>(tab, off, policy, dt, L.rowptr, nullptr, L.col, L.v64);
  int total = 0;
  AMG_CK(read_int(E, L.rowptr + n, &total, s));
  L.nnz = total;
  return cudaGetLastError();
}

cudaError_t amg_setup(AmgEngine &E, cudaStream_t s) {
  E.err_msg.clear();
  int l = 0;
  for (;;) {
    AmgLevel &A = E.lev[l];
    note_launch(2);
    k_amg_diag<<<nblk(A.n), kAT, 0, s>>>(A.n, A.rowptr, A.col, A.v64, A.d64, A.d32);
    k_amg_f32<<<std::max(1, std::min(nblk(A.nnz), 4 * 152)), kAT, 0, s>>>(A.nnz, A.v64, A.v32);
    AMG_CK(level_vectors(E, A, l > 0));
    if (A.n <= kAmgCoarsest || l + 1 >= kAmgMaxLevels) break;
    // pass 1 on A
    int n1 = 0, n2 = 0;
    AMG_CK(pairwise_pass(E, A.n, A.rowptr, A.col, A.v64, E.a1, E.mem1, &n1, s));
    long long nnz1 = 0;
    size_t capt = E.cap_nnz;
    AMG_CK(galerkin<2>(E, n1, E.mem1, E.a1, A.rowptr, A.col, A.v64, E.t_rowptr, &E.t_col, &E.t_v, nullptr,
                       &capt, &nnz1, false, s));
    // pass 2 on the pass-1 matrix
    AmgLevel &C = E.lev[l + 1];
    AMG_CK(grow(E, &A.agg, &A.cap_agg, size_t(A.n)));
    int32_t *a2 = E.flag;  // free after pass 1's numbering
    AMG_CK(pairwise_pass(E, n1, E.t_rowptr, E.t_col, E.t_v, a2, E.mem2, &n2, s));
    if (double(n2) > kAmgMinReduction * double(A.n)) break;  // coarsening stalls
    AMG_CK(grow(E, &A.mem, &A.cap_mem, 4 * size_t(n2)));
    note_launch(1);
    k_amg_compose<<<nblk(std::max(A.n, n2)), kAT, 0, s>>>(A.n, n2, E.a1, a2, E.mem1, E.mem2, A.agg, A.mem);
    // level l+1 = P^T A P from A with the composed aggregates
    AMG_CK(grow(E, &C.rowptr, &C.cap_rp, size_t(n2) + 1));
    {
      size_t cd1 = C.cap_n, cd2 = C.cap_n;
      AMG_CK(grow(E, &C.d64, &cd1, size_t(n2)));
      AMG_CK(grow(E, &C.d32, &cd2, size_t(n2)));
      C.cap_n = std::min(cd1, cd2);
    }
    long long nnzc = 0;
    AMG_CK(galerkin<4>(E, n2, A.mem, A.agg, A.rowptr, A.col, A.v64, C.rowptr, &C.col, &C.v64, &C.v32,
                       &C.cap_nnz, &nnzc, true, s));
    C.n = n2;
    C.nnz = nnzc;
    ++l;
  }
  E.L = l + 1;
  AmgLevel &Lc = E.lev[E.L - 1];
  E.dense_coarsest = Lc.n <= kAmgCoarsest;
  if (E.dense_coarsest) {
    note_launch(1);
    k_amg_dense_inverse<<<1, 256, 0, s>>>(Lc.n, Lc.rowptr, Lc.col, Lc.v64, E.work, E.Ainv64, E.Ainv32);
  } else if (!Lc.vec64[AV_T]) {
    AMG_CK(level_vectors(E, Lc, true));
  }
  return cudaGetLastError();
}

namespace {

template <typename T>
void amg_op(int op, const AmgLevel &L, T omega, const T *x, const T *b, T *y, cudaStream_t s) {
  note_launch();
  const int g = nblk(L.n);
  switch (op) {
    case OP_APPLY: k_amg_op<T, OP_APPLY><<<g, kAT, 0, s>>>(L.n, L.rowptr, L.col, vals<T>(L), diag<T>(L), omega, x, b, y); break;
    case OP_RESID: k_amg_op<T, OP_RESID><<<g, kAT, 0, s>>>(L.n, L.rowptr, L.col, vals<T>(L), diag<T>(L), omega, x, b, y); break;
    case OP_JACOBI: k_amg_op<T, OP_JACOBI><<<g, kAT, 0, s>>>(L.n, L.rowptr, L.col, vals<T>(L), diag<T>(L), omega, x, b, y); break;
    default: k_amg_op<T, OP_JACOBI0><<<g, kAT, 0, s>>>(L.n, L.rowptr, L.col, vals<T>(L), diag<T>(L), omega, x, b, y); break;
  }
}

template <typename T>
void dots(AmgEngine &E, int n, const T *a, const T *b, const T *c, const T *d, double *out, cudaStream_t s) {
  const int g = std::max(1, std::min(kDotBlocks, nblk(n)));
  note_launch(2);
  k_amg_dots<T><<<g, kAT, 0, s>>>(n, a, b, c, d, E.partials);
  k_amg_dots_final<<<1, 32, 0, s>>>(g, E.partials, out);
}

template <typename T>
void gcr(AmgEngine &E, int l, const T *r, T *e, cudaStream_t s);

// The last level: x = A^{-1} b (dense), or kAmgCoarseSweeps damped-Jacobi sweeps from zero.
template <typename T>
void coarsest(AmgEngine &E, const T *b, T *x, cudaStream_t s) {
  AmgLevel &A = E.lev[E.L - 1];
  if (E.dense_coarsest) {
    note_launch();
    k_amg_dense<T><<<1, 256, 0, s>>>(A.n, ainv<T>(E), b, x);
    return;
  }
  const T om = T(E.omega);
  T *cur = x, *oth = vec<T>(A, AV_T);
  amg_op<T>(OP_JACOBI0, A, om, nullptr, b, cur, s);
  for (int k = 1; k < kAmgCoarseSweeps; ++k) {
    amg_op<T>(OP_JACOBI, A, om, cur, b, oth, s);
    std::swap(cur, oth);
  }
  if (cur != x) {
    note_launch();
    k_amg_copy<T><<<nblk(A.n), kAT, 0, s>>>(A.n, cur, x);
  }
}

template <typename T>
void kcyc(AmgEngine &E, int l, const T *b, T *x, cudaStream_t s) {
  AmgLevel &A = E.lev[l];
  if (l == E.L - 1) {
    coarsest<T>(E, b, x, s);
    return;
  }
  const T om = T(E.omega);
  T *t = vec<T>(A, AV_T), *r = vec<T>(A, AV_R);
  amg_op<T>(OP_JACOBI0, A, om, nullptr, b, x, s);
  T *cur = x, *oth = t;
  for (int k = 1; k < E.nu1; ++k) {
    amg_op<T>(OP_JACOBI, A, om, cur, b, oth, s);
    std::swap(cur, oth);
  }
  amg_op<T>(OP_RESID, A, om, cur, b, r, s);
  AmgLevel &C = E.lev[l + 1];
  note_launch();
  k_amg_restrict<T><<<nblk(C.n), kAT, 0, s>>>(C.n, A.mem, r, vec<T>(C, AV_B));
  gcr<T>(E, l + 1, vec<T>(C, AV_B), vec<T>(C, AV_E), s);
  note_launch();
  k_amg_prolong<T><<<nblk(A.n), kAT, 0, s>>>(A.n, A.agg, vec<T>(C, AV_E), cur);
  for (int k = 0; k < E.nu2; ++k) {
    amg_op<T>(OP_JACOBI, A, om, cur, b, oth, s);
    std::swap(cur, oth);
  }
  if (cur != x) {
    note_launch();
    k_amg_copy<T><<<nblk(A.n), kAT, 0, s>>>(A.n, cur, x);
  }
}

template <typename T>
void gcr(AmgEngine &E, int l, const T *r, T *e, cudaStream_t s) {
  AmgLevel &A = E.lev[l];
  if (l == E.L - 1) {
    coarsest<T>(E, r, e, s);
    return;
  }
  T *v1 = vec<T>(A, AV_V1), *w1 = vec<T>(A, AV_W1), *v2 = vec<T>(A, AV_V2), *w2 = vec<T>(A, AV_W2),
    *r2 = vec<T>(A, AV_R2);
  const int g = nblk(A.n);
  kcyc<T>(E, l, r, v1, s);
  amg_op<T>(OP_APPLY, A, T(0), v1, nullptr, w1, s);
  dots<T>(E, A.n, w1, r, w1, w1, A.scal, s);
  const int two = l <= E.k_levels;
  note_launch();
  k_gcr_first<T><<<g, kAT, 0, s>>>(A.n, v1, w1, r, e, r2, A.scal, two);
  if (!two) return;
  kcyc<T>(E, l, r2, v2, s);
  amg_op<T>(OP_APPLY, A, T(0), v2, nullptr, w2, s);
  dots<T>(E, A.n, w2, w1, w2, w1, A.scal + 2, s);
  note_launch();
  k_gcr_orth<T><<<g, kAT, 0, s>>>(A.n, v2, w2, v1, w1, A.scal);
  dots<T>(E, A.n, w2, r2, w2, w2, A.scal + 3, s);
  note_launch();
  k_gcr_second<T><<<g, kAT, 0, s>>>(A.n, e, v2, A.scal);
}

}  // namespace

template <typename T>
void amg_cycle(AmgEngine &E, const T *b, T *x, cudaStream_t s) {
  kcyc<T>(E, 0, b, x, s);
}
template void amg_cycle<double>(AmgEngine &, const double *, double *, cudaStream_t);
template void amg_cycle<float>(AmgEngine &, const float *, float *, cudaStream_t);

template <typename T>
void amg_full_to_compact(int n, const T *full, T *compact, cudaStream_t s) {
  note_launch();
  k_amg_gather<T><<<nblk((long long)(n - 2) * (n - 2)), kAT, 0, s>>>(n, full, compact);
}
template <typename T>
void amg_compact_to_full(int n, const T *compact, T *full, cudaStream_t s) {
  note_launch();
  k_amg_scatter<T><<<nblk((long long)(n - 2) * (n - 2)), kAT, 0, s>>>(n, compact, full);
}
template void amg_full_to_compact<double>(int, const double *, double *, cudaStream_t);
template void amg_full_to_compact<float>(int, const float *, float *, cudaStream_t);
template void amg_compact_to_full<double>(int, const double *, double *, cudaStream_t);
template void amg_compact_to_full<float>(int, const float *, float *, cudaStream_t);

void amg_free(AmgEngine &E) {
  for (void *p : E.allocs) cudaFree(p);
  E.allocs.clear();
  if (E.h_int) cudaFreeHost(E.h_int);
  E.h_int = nullptr;
}

}  // namespace sl

// ----------------------------------------------------------------------------- C ABI
struct sl_amg {
  sl::AmgEngine E;
  std::string err;
};

namespace {
sl_status amg_fail(sl_amg *a, sl_status st, const std::string &msg) {
  if (a) a->err = msg;
  return st;
}
}  // namespace

extern "C" {

sl_status sl_amg_create(sl_amg **out, int n, const int *rowptr, const int *col, const double *val,
                        const sl_opts *opts) {
  if (!out) return SL_EINVAL;
  *out = nullptr;
  if (n < 1 || !rowptr || !col || !val) return SL_EINVAL;
  // the matrix: sorted columns, no repeats, a diagonal entry in every row
  for (int i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) return SL_EINVAL;
    bool diag = false;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      if (col[p] < 0 || col[p] >= n || (p > rowptr[i] && col[p] <= col[p - 1])) return SL_EINVAL;
      diag |= col[p] == i;
    }
    if (!diag) return SL_EINVAL;
  }
  sl_amg *a = new (std::nothrow) sl_amg();
  if (!a) return SL_ENOMEM;
  sl_opts o;
  if (opts) o = *opts; else sl_opts_default(&o);
  a->E.nu1 = o.nu1;
  a->E.nu2 = o.nu2;
  a->E.omega = o.omega;
  a->E.k_levels = o.amg_k_levels;
  if (o.nu1 < 1 || o.nu2 < 0 || !(o.omega > 0) || o.amg_k_levels < 0) {
    delete a;
    return SL_EINVAL;
  }
  const long long nnz = rowptr[n];
  cudaError_t e = sl::amg_reserve_level0(a->E, n, nnz);
  sl::AmgLevel &L = a->E.lev[0];
  if (e == cudaSuccess) e = cudaMemcpy(L.rowptr, rowptr, (size_t(n) + 1) * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(L.col, col, size_t(nnz) * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(L.v64, val, size_t(nnz) * sizeof(double), cudaMemcpyHostToDevice);
  L.nnz = nnz;
  if (e == cudaSuccess) e = sl::amg_setup(a->E, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    const sl_status st = (e == cudaErrorInvalidValue && !a->E.err_msg.empty()) ? SL_EINVAL : SL_ECUDA;
    std::fprintf(stderr, "sl_amg_create: %s\n",
                 a->E.err_msg.empty() ? cudaGetErrorString(e) : a->E.err_msg.c_str());
    sl::amg_free(a->E);
    delete a;
    return st;
  }
  *out = a;
  return SL_OK;
}

int sl_amg_num_levels(const sl_amg *a) { return a ? a->E.L : 0; }

sl_status sl_amg_level(const sl_amg *a, int level, int *n, long long *nnz, int *agg, int *rowptr, int *col,
                       double *val) {
  if (!a || level < 0 || level >= a->E.L) return SL_EINVAL;
  const sl::AmgLevel &L = a->E.lev[level];
  if (n) *n = L.n;
  if (nnz) *nnz = L.nnz;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && agg) {
    if (level == a->E.L - 1) return SL_EINVAL;
    e = cudaMemcpy(agg, L.agg, size_t(L.n) * sizeof(int), cudaMemcpyDeviceToHost);
  }
  if (e == cudaSuccess && rowptr) e = cudaMemcpy(rowptr, L.rowptr, (size_t(L.n) + 1) * sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && col) e = cudaMemcpy(col, L.col, size_t(L.nnz) * sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && val) e = cudaMemcpy(val, L.v64, size_t(L.nnz) * sizeof(double), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SL_OK : SL_ECUDA;
}

sl_status sl_amg_apply(sl_amg *a, int precision, const void *b, void *x, void *stream) {
  if (!a || !b || !x || (precision != 0 && precision != 1)) return SL_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == 0)
    sl::amg_cycle<double>(a->E, static_cast<const double *>(b), static_cast<double *>(x), s);
  else
    sl::amg_cycle<float>(a->E, static_cast<const float *>(b), static_cast<float *>(x), s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SL_OK : amg_fail(a, SL_ECUDA, cudaGetErrorString(e));
}

const char *sl_amg_last_error(const sl_amg *a) { return a ? a->err.c_str() : "null AMG"; }

void sl_amg_destroy(sl_amg *a) {
  if (!a) return;
  cudaDeviceSynchronize();
  sl::amg_free(a->E);
  delete a;
}

}  // extern "C"
