// sl_adjoint.cu - transposed operators for the backward solves of the discrete adjoint, and
// the gradient accumulations.
//
// At a fixed policy the implicit step is the linear system A^alpha U^n = F^alpha (Eq.
// 2.11, theta = 1).  The adjoint recursion solves A_n^T mu_n = lambda_n, so every
// operator of the V-cycle is needed transposed:
//   - fine level: an explicit transpose in CSR form (rows = interior columns of A), built once
//     per step from the stencil tables and the policy.  Entries are scattered with atomics
//     and then sorted by source row, so the row contents and their order are deterministic;
//   - coarse levels: A_l^T = R A_{l-1}^T P is the Galerkin operator of A^T with the same
//     transfers (P^T = 4R), so its rows are read from the forward windows: row J of A_l^T
//     holds, at offset o, the coefficient of row J + o at offset -o.  These rows are gathered
//     into dense (2R_l + 1)^2 windows, one per coarse row;
//   - coarsest level: the transpose of the dense inverse.
#include "sl_launch.h"

namespace sl {

constexpr int kAdjThreads = 256;
constexpr int kScanChunk = 1024;

__device__ __forceinline__ int fine_entry(const FineTab &tab, int k, int i1, int i2) {
  return fine_row_entry(tab, k, i1, i2);
}

// ----------------------------------------------------------------------------- CSR transpose
// Counts the off-diagonal interior entries of every column of A (= row of A^T).
__global__ void __launch_bounds__(kAdjThreads) k_csrT_count(FineTab tab, const int32_t *__restrict__ off,
                                                             const uint8_t *__restrict__ policy,
                                                             int *__restrict__ cnt) {
  const int m = tab.m;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= m * m) return;
  const int i1 = 1 + I % m, i2 = 1 + I / m;
  const int e = fine_entry(tab, policy[I], i1, i2);
  for (int t = 0; t < tab.nt[e]; ++t) {
    const int o = off[e * tab.tmax + t];
    const int dx = int(int16_t(o & 0xffff)), dy = o >> 16;
    const int j1 = i1 + dx, j2 = i2 + dy;
    if ((dx | dy) == 0 || j1 < 1 || j1 > m || j2 < 1 || j2 > m) continue;
    atomicAdd(cnt + (j2 - 1) * m + (j1 - 1), 1);
  }
}

// Exclusive block scan of kScanChunk ints (one per thread); returns the block total.
__device__ __forceinline__ int block_exclusive_scan(int v, int *total) {
  __shared__ int warp_tot[kScanChunk / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int w = warp_tot[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    warp_tot[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const int base = wid > 0 ? warp_tot[wid - 1] : 0;
  *total = warp_tot[kScanChunk / 32 - 1];
  return base + inc - v;
}

__global__ void __launch_bounds__(kScanChunk) k_scan_chunk_sums(const int *__restrict__ cnt, int M,
                                                                 int *__restrict__ chunk_sum) {
  const int i = blockIdx.x * kScanChunk + threadIdx.x;
  int tot;
  block_exclusive_scan(i < M ? cnt[i] : 0, &tot);
  if (threadIdx.x == 0) chunk_sum[blockIdx.x] = tot;
}

// Exclusive scan of the chunk sums in one block (segments of `per` chunks per thread).
__global__ void __launch_bounds__(kScanChunk) k_scan_chunk_offsets(const int *__restrict__ chunk_sum,
                                                                    int nchunks, int *__restrict__ chunk_off) {
  const int per = (nchunks + kScanChunk - 1) / kScanChunk;
  const int lo = threadIdx.x * per, hi = min(nchunks, lo + per);
  int sum = 0;
  for (int c = lo; c < hi; ++c) sum += chunk_sum[c];
  int tot;
  int run = block_exclusive_scan(sum, &tot);
  for (int c = lo; c < hi; ++c) {
    chunk_off[c] = run;
    run += chunk_sum[c];
  }
}

__global__ void __launch_bounds__(kScanChunk) k_scan_apply(const int *__restrict__ cnt, int M,
                                                            const int *__restrict__ chunk_off,
                                                            int32_t *__restrict__ rowptr) {
  const int i = blockIdx.x * kScanChunk + threadIdx.x;
  const int v = i < M ? cnt[i] : 0;
  int tot;
  const int ex = block_exclusive_scan(v, &tot);
  if (i < M) rowptr[i] = chunk_off[blockIdx.x] + ex;
  if (i == M - 1) rowptr[M] = chunk_off[blockIdx.x] + ex + v;
}

// out[0..n] = exclusive prefix sums of in[0..n-1] (out[n] = total); scratch: 2 ceil(n/1024) ints.
void launch_exclusive_scan(const int *in, int n, int32_t *out, int *scratch, cudaStream_t s) {
  const int nchunks = (n + kScanChunk - 1) / kScanChunk;
  note_launch(3);
  k_scan_chunk_sums<<<nchunks, kScanChunk, 0, s>>>(in, n, scratch);
  k_scan_chunk_offsets<<<1, kScanChunk, 0, s>>>(scratch, nchunks, scratch + nchunks);
  k_scan_apply<<<nchunks, kScanChunk, 0, s>>>(in, n, scratch + nchunks, out);
}

// Scatters the entries A[i, j] (i = source row) into row j of A^T and writes the diagonal.
__global__ void __launch_bounds__(kAdjThreads) k_csrT_fill(FineTab tab, const int32_t *__restrict__ off,
                                                            const uint8_t *__restrict__ policy, double dt,
                                                            const int32_t *__restrict__ rowptr,
                                                            int *__restrict__ fillc, int32_t *__restrict__ col,
                                                            double *__restrict__ vtmp,
                                                            double *__restrict__ d64, float *__restrict__ d32) {
  const int m = tab.m, n = tab.n;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= m * m) return;
  const int i1 = 1 + I % m, i2 = 1 + I / m;
  const int k = policy[I];
  const int e = fine_entry(tab, k, i1, i2);
  const double d = 1.0 + dt * (tab.W64[e] - tab.c64[k]) - dt * tab.ws64[e];
  d64[I] = d;
  d32[I] = float(d);
  for (int t = 0; t < tab.nt[e]; ++t) {
    const int ix = e * tab.tmax + t;
    const int o = off[ix];
    const int dx = int(int16_t(o & 0xffff)), dy = o >> 16;
    const int j1 = i1 + dx, j2 = i2 + dy;
    if ((dx | dy) == 0 || j1 < 1 || j1 > m || j2 < 1 || j2 > m) continue;
    const int J = (j2 - 1) * m + (j1 - 1);
    const int pos = rowptr[J] + atomicAdd(fillc + J, 1);
    col[pos] = i2 * n + i1;
    vtmp[pos] = -dt * tab.w64[ix];
  }
}

// Orders every row by source index.  A row holds a few dozen entries whose sources lie
// within the stencil reach of j, so each entry is keyed by (i - j + kOff) << 6 | slot in one
// int; each thread sorts its row's keys in a local array (insertion sort) and writes the
// sorted columns and the permuted values (from the staging array vtmp) once.  A row longer
// than the local array is sorted in place in global memory.
constexpr int kSortMax = 64;

__global__ void __launch_bounds__(kAdjThreads) k_csrT_sort(int M, int m, int n, int koff,
                                                            const int32_t *__restrict__ rowptr,
                                                            int32_t *__restrict__ col,
                                                            const double *__restrict__ vtmp,
                                                            double *__restrict__ v64, float *__restrict__ v32) {
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= M) return;
  const int j = (1 + J / m) * n + 1 + J % m;
  const int lo = rowptr[J], hi = rowptr[J + 1], len = hi - lo;
  if (len <= kSortMax) {
    int key[kSortMax];
    for (int a = 0; a < len; ++a) {
      const int ka = ((col[lo + a] - j + koff) << 6) | a;
      int b = a - 1;
      while (b >= 0 && key[b] > ka) {
        key[b + 1] = key[b];
        --b;
      }
      key[b + 1] = ka;
    }
    for (int a = 0; a < len; ++a) {
      const double v = vtmp[lo + (key[a] & 63)];
      col[lo + a] = j + (key[a] >> 6) - koff;
      v64[lo + a] = v;
      v32[lo + a] = float(v);
    }
    return;
  }
  for (int a = lo; a < hi; ++a) v64[a] = vtmp[a];
  for (int a = lo + 1; a < hi; ++a) {
    const int c = col[a];
    const double w = v64[a];
    int b = a - 1;
    while (b >= lo && col[b] > c) {
      col[b + 1] = col[b];
      v64[b + 1] = v64[b];
      --b;
    }
    col[b + 1] = c;
    v64[b + 1] = w;
  }
  for (int a = lo; a < hi; ++a) v32[a] = float(v64[a]);
}

void launch_csrT_build(const FineTab &tab, const int32_t *off, const uint8_t *policy, double dt, int R0,
                       int *cnt, int *scan_scratch, int32_t *rowptr, int32_t *col, double *vtmp,
                       double *v64, float *v32, double *d64, float *d32, cudaStream_t s) {
  const int M = tab.m * tab.m;
  const int g = (M + kAdjThreads - 1) / kAdjThreads;
  const int nchunks = (M + kScanChunk - 1) / kScanChunk;
  note_launch(6);
  cudaMemsetAsync(cnt, 0, size_t(M) * sizeof(int), s);
  k_csrT_count<<<g, kAdjThreads, 0, s>>>(tab, off, policy, cnt);
  k_scan_chunk_sums<<<nchunks, kScanChunk, 0, s>>>(cnt, M, scan_scratch);
  k_scan_chunk_offsets<<<1, kScanChunk, 0, s>>>(scan_scratch, nchunks, scan_scratch + nchunks);
  k_scan_apply<<<nchunks, kScanChunk, 0, s>>>(cnt, M, scan_scratch + nchunks, rowptr);
  cudaMemsetAsync(cnt, 0, size_t(M) * sizeof(int), s);
  k_csrT_fill<<<g, kAdjThreads, 0, s>>>(tab, off, policy, dt, rowptr, cnt, col, vtmp, d64, d32);
  // sources i of row j satisfy |i - j| <= R0 (n + 1)
  k_csrT_sort<<<g, kAdjThreads, 0, s>>>(M, tab.m, tab.n, R0 * (tab.n + 1), rowptr, col, vtmp, v64, v32);
}

// ----------------------------------------------------------------------------- transposed ops
template <typename T, int OP>
__device__ __forceinline__ void finishT(T *y, const T *x, const T *b, int j, T acc, T d, T omega) {
  if (OP == OP_APPLY) y[j] = acc;
  else if (OP == OP_RESID) y[j] = b[j] - acc;
  else y[j] = x[j] + omega * (b[j] - acc) / d;
}

template <typename T, int OP>
__global__ void __launch_bounds__(kAdjThreads) k_fineT_op(CsrTView<T> A, T omega, const T *__restrict__ x,
                                                           const T *__restrict__ b, T *__restrict__ y) {
  const int m = A.m;
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= m * m) return;
  const int j = (1 + J / m) * A.n + 1 + J % m;
  const T d = A.d[J];
  if (OP == OP_JACOBI0) {
    y[j] = omega * b[j] / d;
    return;
  }
  T acc = d * x[j];
  const int lo = A.rowptr[J], hi = A.rowptr[J + 1];
  // eight entries per pass: their columns and values, then the eight x values, are loaded
  // before the FMAs (a loop that chained column -> x -> FMA per entry paid two memory round
  // trips for every entry); the entries are added in the same order
  for (int e0 = lo; e0 < hi; e0 += 8) {
    int cj[8];
    T vv[8], xv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const bool in = e0 + u < hi;
      cj[u] = in ? A.col[e0 + u] : j;
      vv[u] = in ? A.v[e0 + u] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) xv[u] = e0 + u < hi ? __ldg(x + cj[u]) : T(0);
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (e0 + u < hi) acc = fma(vv[u], xv[u], acc);
  }
  finishT<T, OP>(y, x, b, j, acc, d, omega);
}

template <typename T>
void launch_fineT_op(int op, const CsrTView<T> &A, T omega, const T *x, const T *b, T *y, cudaStream_t s) {
  const int g = (A.m * A.m + kAdjThreads - 1) / kAdjThreads;
  note_launch();
  switch (op) {
    case OP_APPLY: k_fineT_op<T, OP_APPLY><<<g, kAdjThreads, 0, s>>>(A, omega, x, b, y); break;
    case OP_RESID: k_fineT_op<T, OP_RESID><<<g, kAdjThreads, 0, s>>>(A, omega, x, b, y); break;
    case OP_JACOBI: k_fineT_op<T, OP_JACOBI><<<g, kAdjThreads, 0, s>>>(A, omega, x, b, y); break;
    default: k_fineT_op<T, OP_JACOBI0><<<g, kAdjThreads, 0, s>>>(A, omega, x, b, y); break;
  }
}
template void launch_fineT_op<double>(int, const CsrTView<double> &, double, const double *,
                                      const double *, double *, cudaStream_t);
template void launch_fineT_op<float>(int, const CsrTView<float> &, float, const float *, const float *,
                                     float *, cudaStream_t);

// Row J of A_l^T as a dense window: WT[e * m^2 + J], e = (oy + R)(2R + 1) + (ox + R), holds
// A_l[J + o, J] (zero where J + o is not an interior row).
template <typename T>
__global__ void __launch_bounds__(kAdjThreads) k_denseT_build(CoarseLev<T> L, const T *__restrict__ cdense,
                                                               T *__restrict__ WT) {
  const int m = L.m, R = L.R, Wd = 2 * R + 1;
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= m * m) return;
  const int J1 = 1 + J % m, J2 = 1 + J / m;
  for (int e = 0; e < L.win; ++e) {
    const int oy = e / Wd - R, ox = e % Wd - R;
    const int I1 = J1 + ox, I2 = J2 + oy;
    T v = T(0);
    if (I1 >= 1 && I1 <= m && I2 >= 1 && I2 <= m) {
      const int c = L.cls[(I2 - 1) * m + (I1 - 1)];
      const int eo = (R - oy) * Wd + (R - ox);
      v = c >= 0 ? cdense[size_t(c) * L.win + eo] : L.ewin[size_t(eo) * L.cap + (-c - 1)];
    }
    WT[size_t(e) * m * m + J] = v;
  }
}

template <typename T>
void launch_denseT_build(const CoarseLev<T> &L, const T *cdense, T *WT, cudaStream_t s) {
  note_launch();
  k_denseT_build<T><<<(L.m * L.m + kAdjThreads - 1) / kAdjThreads, kAdjThreads, 0, s>>>(L, cdense, WT);
}
template void launch_denseT_build<double>(const CoarseLev<double> &, const double *, double *, cudaStream_t);
template void launch_denseT_build<float>(const CoarseLev<float> &, const float *, float *, cudaStream_t);

// With RR > 0 the reach is a compile-time constant and each window row is unrolled with a
// predicate per entry, so its weight and value loads are in flight together (same order of
// summation as the runtime loop, which serves other reaches).
template <typename T, int OP, int RR>
__global__ void __launch_bounds__(kAdjThreads) k_denseT_op(int n, int Rrt, const T *__restrict__ WT, T omega,
                                                            const T *__restrict__ x, const T *__restrict__ b,
                                                            T *__restrict__ y) {
  const int R = RR > 0 ? RR : Rrt;
  const int m = n - 2, mm = m * m, Wd = 2 * R + 1;
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= mm) return;
  const int J1 = 1 + J % m, J2 = 1 + J / m;
  const int j = J2 * n + J1;
  const T d = WT[size_t(R * Wd + R) * mm + J];
  if (OP == OP_JACOBI0) {
    y[j] = omega * b[j] / d;
    return;
  }
  const int ylo = max(-R, -J2), yhi = min(R, n - 1 - J2);
  const int xlo = max(-R, -J1), xhi = min(R, n - 1 - J1);
  T acc = T(0);
  for (int oy = ylo; oy <= yhi; ++oy) {
    const T *wrow = WT + size_t((oy + R) * Wd + R) * mm + J;
    const T *xrow = x + j + oy * n;
    if (RR > 0) {
#pragma unroll
      for (int ox = -RR; ox <= RR; ++ox)
        if (ox >= xlo && ox <= xhi) acc = fma(wrow[ptrdiff_t(ox) * mm], __ldg(xrow + ox), acc);
    } else {
      for (int ox = xlo; ox <= xhi; ++ox) acc = fma(wrow[ptrdiff_t(ox) * mm], __ldg(xrow + ox), acc);
    }
  }
  finishT<T, OP>(y, x, b, j, acc, d, omega);
}

template <typename T, int RR>
void denseT_dispatch(int op, int g, int n, int R, const T *WT, T omega, const T *x, const T *b, T *y,
                     cudaStream_t s) {
  switch (op) {
    case OP_APPLY: k_denseT_op<T, OP_APPLY, RR><<<g, kAdjThreads, 0, s>>>(n, R, WT, omega, x, b, y); break;
    case OP_RESID: k_denseT_op<T, OP_RESID, RR><<<g, kAdjThreads, 0, s>>>(n, R, WT, omega, x, b, y); break;
    case OP_JACOBI: k_denseT_op<T, OP_JACOBI, RR><<<g, kAdjThreads, 0, s>>>(n, R, WT, omega, x, b, y); break;
    default: k_denseT_op<T, OP_JACOBI0, RR><<<g, kAdjThreads, 0, s>>>(n, R, WT, omega, x, b, y); break;
  }
}

template <typename T>
void launch_denseT_op(int op, int n, int R, const T *WT, T omega, const T *x, const T *b, T *y,
                      cudaStream_t s) {
  const int g = ((n - 2) * (n - 2) + kAdjThreads - 1) / kAdjThreads;
  note_launch();
  switch (R) {
    case 1: denseT_dispatch<T, 1>(op, g, n, R, WT, omega, x, b, y, s); break;
    case 2: denseT_dispatch<T, 2>(op, g, n, R, WT, omega, x, b, y, s); break;
    case 3: denseT_dispatch<T, 3>(op, g, n, R, WT, omega, x, b, y, s); break;
    case 4: denseT_dispatch<T, 4>(op, g, n, R, WT, omega, x, b, y, s); break;
    case 5: denseT_dispatch<T, 5>(op, g, n, R, WT, omega, x, b, y, s); break;
    case 6: denseT_dispatch<T, 6>(op, g, n, R, WT, omega, x, b, y, s); break;
    case 7: denseT_dispatch<T, 7>(op, g, n, R, WT, omega, x, b, y, s); break;
    case 8: denseT_dispatch<T, 8>(op, g, n, R, WT, omega, x, b, y, s); break;
    default: denseT_dispatch<T, 0>(op, g, n, R, WT, omega, x, b, y, s); break;
  }
}
template void launch_denseT_op<double>(int, int, int, const double *, double, const double *,
                                       const double *, double *, cudaStream_t);
template void launch_denseT_op<float>(int, int, int, const float *, float, const float *, const float *,
                                      float *, cudaStream_t);

// ----------------------------------------------------------------------------- gradients
// y = x on interior nodes, 0 on the boundary.
__global__ void k_interior_copy(int n, const double *__restrict__ x, double *__restrict__ y) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n * n) return;
  const int j1 = j % n, j2 = j / n;
  y[j] = (j1 > 0 && j1 < n - 1 && j2 > 0 && j2 < n - 1) ? x[j] : 0.0;
}

void launch_interior_copy(int n, const double *x, double *y, cudaStream_t s) {
  note_launch();
  k_interior_copy<<<(n * n + kAdjThreads - 1) / kAdjThreads, kAdjThreads, 0, s>>>(n, x, y);
}

// dJ/dG[m][q](x) += dt tau_q(t_n) phi[alpha_n(x), m] mu_n(x): the source of step n enters
// F^alpha as dt f^alpha with f^k = sum_m phi[k, m] sum_q tau_q G[m][q].
__global__ void __launch_bounds__(kAdjThreads) k_adj_dG(int n, int nf, int nq, const uint8_t *__restrict__ policy,
                                                         const double *__restrict__ phi,
                                                         const double *__restrict__ tau, double dt,
                                                         const double *__restrict__ mu, double *__restrict__ dG) {
  const int m = n - 2;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= m * m) return;
  const int j = (1 + I / m) * n + 1 + I % m;
  const int k = policy[I];
  const double mj = mu[j];
  const size_t N = size_t(n) * n;
  for (int f = 0; f < nf; ++f) {
    const double pm = dt * phi[k * nf + f] * mj;
    for (int q = 0; q < nq; ++q) dG[size_t(f * nq + q) * N + j] += tau[q] * pm;
  }
}

void launch_adj_dG(int n, int nf, int nq, const uint8_t *policy, const double *phi, const double *tau,
                   double dt, const double *mu, double *dG, cudaStream_t s) {
  note_launch();
  const int m = n - 2;
  k_adj_dG<<<(m * m + kAdjThreads - 1) / kAdjThreads, kAdjThreads, 0, s>>>(n, nf, nq, policy, phi, tau, dt, mu, dG);
}

// partial[p][block] = sum over the block's nodes of mu_j (dL^alpha/dtheta_p U)_j, with
// (dL/dtheta U)_j = sum_t dw_t U_{j + o_t} - dW U_j (U carries psi on the boundary).
__global__ void __launch_bounds__(kAdjThreads) k_adj_dtheta(FineTab tab, DTabView d,
                                                             const uint8_t *__restrict__ policy,
                                                             const double *__restrict__ mu,
                                                             const double *__restrict__ U,
                                                             double *__restrict__ partials) {
  const int m = tab.m, n = tab.n;
  double acc[kMaxParams];
#pragma unroll
  for (int p = 0; p < kMaxParams; ++p) acc[p] = 0.0;
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < m * m; I += gridDim.x * blockDim.x) {
    const int i1 = 1 + I % m, i2 = 1 + I / m;
    const int j = i2 * n + i1;
    const int e = fine_entry(tab, policy[I], i1, i2);
    const double mj = mu[j], uj = U[j];
#pragma unroll
    for (int p = 0; p < kMaxParams; ++p) {
      if (p >= d.np) break;
      const size_t pe = size_t(p) * d.E + e;
      double v = -d.dW[pe] * uj;
      for (int t = 0; t < d.nt[pe]; ++t) {
        const size_t ix = pe * d.stride + t;
        v = fma(d.dw[ix], U[j + d.lin[ix]], v);
      }
      acc[p] = fma(mj, v, acc[p]);
    }
  }
  __shared__ double sh[kMaxParams][kAdjThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int p = 0; p < kMaxParams; ++p) {
    double v = acc[p];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[p][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < d.np) {
    double s = 0.0;
    for (int w = 0; w < kAdjThreads / 32; ++w) s += sh[threadIdx.x][w];
    partials[size_t(threadIdx.x) * gridDim.x + blockIdx.x] = s;
  }
}

// out[p] += dt * sum_b partials[p][b], one warp per parameter, fixed summation order.
__global__ void k_adj_dtheta_final(int np, int nblocks, const double *__restrict__ partials, double dt,
                                   double *__restrict__ out) {
  const int p = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (p >= np) return;
  double v = 0.0;
  for (int b = lane; b < nblocks; b += 32) v += partials[size_t(p) * nblocks + b];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) out[p] += dt * v;
}

void launch_adj_dtheta(const FineTab &tab, const DTabView &d, const uint8_t *policy, const double *mu,
                       const double *U, double dt, double *partials, double *out, cudaStream_t s) {
  note_launch(2);
  k_adj_dtheta<<<kRedBlocks, kAdjThreads, 0, s>>>(tab, d, policy, mu, U, partials);
  k_adj_dtheta_final<<<1, 32 * kMaxParams, 0, s>>>(d.np, kRedBlocks, partials, dt, out);
}

}  // namespace sl
