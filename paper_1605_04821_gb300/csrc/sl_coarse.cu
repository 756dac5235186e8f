// sl_coarse.cu - Galerkin coarse levels A_l = R A_{l-1} P (Section 3.3) on the device.
#include <algorithm>
#include <climits>
#include <cmath>

#include "sl_launch.h"

namespace sl {

// ----------------------------------------------------------------------------- classification
// Coarse row I is class k when all nine rows 2I + a of the previous level are class-k interior
// rows (level 0: untruncated band-free rows with control k); otherwise it is stored explicitly.
// Explicit rows get their slots in row-major order (count per 256-row chunk, scan, assign), so
// the slot order is deterministic and neighbouring slots are neighbouring rows.
constexpr int kChunk = 256;
constexpr int kPending = INT32_MIN;

__device__ __forceinline__ int coarse_class_of(int level, const FineTab &tab, const uint8_t *policy,
                                               const int32_t *cls_prev, int n_prev, int I1, int I2) {
  int k0 = -1;
  for (int a2 = -1; a2 <= 1; ++a2)
    for (int a1 = -1; a1 <= 1; ++a1) {
      const int i1 = 2 * I1 + a1, i2 = 2 * I2 + a2;
      int k;
      if (level == 1) {
        // rows of a general fine level (x-dependent diffusion) are all different
        const bool interior = !tab.general && (tab.n - 1 >= 2 * tab.B) &&
                              class_q(i1, tab.n, tab.B) == tab.B && class_q(i2, tab.n, tab.B) == tab.B;
        k = interior ? int(policy[(i2 - 1) * tab.m + (i1 - 1)]) : -1;
      } else {
        k = cls_prev[(i2 - 1) * (n_prev - 2) + (i1 - 1)];
      }
      if (k < 0) return -1;
      if (k0 < 0) k0 = k;
      else if (k != k0) return -1;
    }
  return k0;
}

__global__ void __launch_bounds__(kChunk) k_classify_count(int level, FineTab tab, const uint8_t *__restrict__ policy,
                                                           const int32_t *__restrict__ cls_prev, int n_prev,
                                                           int32_t *__restrict__ cls, int n,
                                                           int *__restrict__ chunk_count) {
  const int m = n - 2;
  const int I = blockIdx.x * kChunk + threadIdx.x;
  int flag = 0;
  if (I < m * m) {
    const int k = coarse_class_of(level, tab, policy, cls_prev, n_prev, 1 + I % m, 1 + I / m);
    cls[I] = k >= 0 ? k : kPending;
    flag = k < 0;
  }
  const int c = __syncthreads_count(flag);
  if (threadIdx.x == 0) chunk_count[blockIdx.x] = c;
}

// Exclusive scan of the chunk counts in one block; the total goes to *total.
__global__ void __launch_bounds__(1024) k_scan_counts(const int *__restrict__ count, int nchunks,
                                                      int *__restrict__ offset, int *__restrict__ total) {
  __shared__ int part[1024];
  const int per = (nchunks + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(nchunks, lo + per);
  int sum = 0;
  for (int c = lo; c < hi; ++c) sum += count[c];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan of the segment sums
    const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - sum;
  for (int c = lo; c < hi; ++c) {
    offset[c] = run;
    run += count[c];
  }
  if (threadIdx.x == 1023) *total = part[1023];
}

__global__ void __launch_bounds__(kChunk) k_classify_assign(int32_t *__restrict__ cls, int n,
                                                            int32_t *__restrict__ erow,
                                                            const int *__restrict__ offset) {
  __shared__ int warp_base[kChunk / 32];
  const int m = n - 2;
  const int I = blockIdx.x * kChunk + threadIdx.x;
  const bool pend = I < m * m && cls[I] == kPending;
  const unsigned mask = __ballot_sync(0xffffffffu, pend);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_base[wid] = __popc(mask);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int w = 0; w < kChunk / 32; ++w) {
      const int c = warp_base[w];
      warp_base[w] = run;
      run += c;
    }
  }
  __syncthreads();
  if (pend) {
    const int slot = offset[blockIdx.x] + warp_base[wid] + __popc(mask & ((1u << lane) - 1u));
    cls[I] = -slot - 1;
    erow[slot] = (1 + I / m) * n + 1 + I % m;
  }
}

void launch_classify(int level, const FineTab &tab, const uint8_t *policy, const int32_t *cls_prev,
                     int n_prev, int32_t *cls, int n, int32_t *erow, int *count, int *chunk_scratch,
                     cudaStream_t s) {
  const int m = n - 2;
  const int nchunks = (m * m + kChunk - 1) / kChunk;
  note_launch(3);
  k_classify_count<<<nchunks, kChunk, 0, s>>>(level, tab, policy, cls_prev, n_prev, cls, n, chunk_scratch);
  k_scan_counts<<<1, 1024, 0, s>>>(chunk_scratch, nchunks, chunk_scratch + nchunks, count);
  k_classify_assign<<<nchunks, kChunk, 0, s>>>(cls, n, erow, chunk_scratch + nchunks);
}

// ----------------------------------------------------------------------------- explicit RAP
// Thread per explicit coarse row; the (2R+1)^2 window accumulates in shared memory.  Row
// 2I + a of the previous level contributes R_a * (its coefficient at column j) * P_{jJ}.
// The window of one explicit coarse row (slot), accumulated in `win` (cur.win entries).
template <typename T>
__device__ void rap_explicit_row(int level, const FineTab &tab, const int32_t *__restrict__ fine_off,
                                 const uint8_t *__restrict__ policy, T dt, const CoarseLev<T> &prev,
                                 const int32_t *__restrict__ prev_coff, const CoarseLev<T> &cur,
                                 int slot, T *win, T *__restrict__ ewin_out);

template <typename T>
__global__ void k_rap_explicit(int level, FineTab tab, const int32_t *__restrict__ fine_off,
                               const uint8_t *__restrict__ policy, T dt, CoarseLev<T> prev,
                               const int32_t *__restrict__ prev_coff, CoarseLev<T> cur, int count,
                               T *__restrict__ ewin_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= count) return;
  T *win = reinterpret_cast<T *>(smem_raw) + size_t(threadIdx.x) * cur.win;
  rap_explicit_row<T>(level, tab, fine_off, policy, dt, prev, prev_coff, cur, slot, win, ewin_out);
}

// The same rows with their number read from device memory, over a grid-stride loop: the launch
// shape depends only on the capacity, so a CUDA graph can rebuild the hierarchy on the device.
template <typename T>
__global__ void k_rap_explicit_dev(int level, FineTab tab, const int32_t *__restrict__ fine_off,
                                   const uint8_t *__restrict__ policy, T dt, CoarseLev<T> prev,
                                   const int32_t *__restrict__ prev_coff, CoarseLev<T> cur,
                                   const int *__restrict__ count_dev, T *__restrict__ ewin_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int count = *count_dev;
  T *win = reinterpret_cast<T *>(smem_raw) + size_t(threadIdx.x) * cur.win;
  for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < count; slot += gridDim.x * blockDim.x)
    rap_explicit_row<T>(level, tab, fine_off, policy, dt, prev, prev_coff, cur, slot, win, ewin_out);
}

template <typename T>
__device__ void rap_explicit_row(int level, const FineTab &tab, const int32_t *__restrict__ fine_off,
                                 const uint8_t *__restrict__ policy, T dt, const CoarseLev<T> &prev,
                                 const int32_t *__restrict__ prev_coff, const CoarseLev<T> &cur,
                                 int slot, T *win, T *__restrict__ ewin_out) {
  for (int e = 0; e < cur.win; ++e) win[e] = T(0);
  const int jr = cur.erow[slot];
  const int I1 = jr % cur.n, I2 = jr / cur.n;
  const int R = cur.R;
  for (int a2 = -1; a2 <= 1; ++a2)
    for (int a1 = -1; a1 <= 1; ++a1) {
      const T ra = T(fw_weight(a1) * fw_weight(a2));
      const int i1 = 2 * I1 + a1, i2 = 2 * I2 + a2;
      if (level == 1) {
        const int k = policy[(i2 - 1) * tab.m + (i1 - 1)];
        const int e = fine_row_entry(tab, k, i1, i2);
        const T W = tab_W<T>(tab)[e], c = tab_c<T>(tab)[k];
        rap_scatter<T>(win, R, I1, I2, i1, i2, ra * (T(1) + dt * (W - c)));
        const T *w = tab_w<T>(tab);
        for (int t = 0; t < tab.nt[e]; ++t) {
          const int ix = e * tab.tmax + t;
          const int off = fine_off[ix];
          const int dx = int(int16_t(off & 0xffff)), dy = off >> 16;
          rap_scatter<T>(win, R, I1, I2, i1 + dx, i2 + dy, -ra * dt * w[ix]);
        }
      } else {
        const int cp = prev.cls[(i2 - 1) * prev.m + (i1 - 1)];
        if (cp >= 0) {
          for (int t = 0; t < prev.cnt[cp]; ++t) {
            const int off = prev_coff[cp * prev.ctmax + t];
            const int dx = int(int16_t(off & 0xffff)), dy = off >> 16;
            rap_scatter<T>(win, R, I1, I2, i1 + dx, i2 + dy, ra * prev.cw[cp * prev.ctmax + t]);
          }
        } else {
          const int ps = -cp - 1;
          const int Wp = 2 * prev.R + 1;
          for (int e = 0; e < prev.win; ++e) {
            const T v = prev.ewin[size_t(e) * prev.cap + ps];
            if (v == T(0)) continue;
            const int dy = e / Wp - prev.R, dx = e % Wp - prev.R;
            rap_scatter<T>(win, R, I1, I2, i1 + dx, i2 + dy, ra * v);
          }
        }
      }
    }
  for (int e = 0; e < cur.win; ++e) ewin_out[size_t(e) * cur.cap + slot] = win[e];
}

template <typename T>
cudaError_t launch_rap_explicit_dev(int level, const FineTab &tab, const int32_t *fine_off,
                                    const uint8_t *policy, T dt, const CoarseLev<T> &prev,
                                    const int32_t *prev_coff, const CoarseLev<T> &cur,
                                    const int *count_dev, int cap, T *ewin_out, cudaStream_t s) {
  if (cap <= 0) return cudaSuccess;
  const size_t per = size_t(cur.win) * sizeof(T);
  int threads = int((200 * 1024) / per);
  threads = threads > 128 ? 128 : threads;
  if (threads < 1) return cudaErrorInvalidValue;
  const size_t bytes = per * threads;
  // two resident blocks per SM at most (the windows take up to 200 KB); a grid of that size
  // strides over the rows, and blocks beyond the row count exit at once
  int blocks = (cap + threads - 1) / threads;
  blocks = blocks > 2 * 152 ? 2 * 152 : blocks;
  note_launch();
  k_rap_explicit_dev<T><<<blocks, threads, bytes, s>>>(level, tab, fine_off, policy, dt, prev,
                                                       prev_coff, cur, count_dev, ewin_out);
  return cudaGetLastError();
}
template cudaError_t launch_rap_explicit_dev<double>(int, const FineTab &, const int32_t *,
                                                     const uint8_t *, double, const CoarseLev<double> &,
                                                     const int32_t *, const CoarseLev<double> &,
                                                     const int *, int, double *, cudaStream_t);
template cudaError_t launch_rap_explicit_dev<float>(int, const FineTab &, const int32_t *,
                                                    const uint8_t *, float, const CoarseLev<float> &,
                                                    const int32_t *, const CoarseLev<float> &,
                                                    const int *, int, float *, cudaStream_t);

template <typename T>
cudaError_t launch_rap_explicit(int level, const FineTab &tab, const int32_t *fine_off,
                                const uint8_t *policy, T dt, const CoarseLev<T> &prev,
                                const int32_t *prev_coff, const CoarseLev<T> &cur, int count,
                                T *ewin_out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const size_t per = size_t(cur.win) * sizeof(T);
  int threads = int((200 * 1024) / per);
  threads = threads > 128 ? 128 : threads;
  if (threads < 1) return cudaErrorInvalidValue;
  const size_t bytes = per * threads;
  note_launch();
  k_rap_explicit<T><<<(count + threads - 1) / threads, threads, bytes, s>>>(
      level, tab, fine_off, policy, dt, prev, prev_coff, cur, count, ewin_out);
  return cudaGetLastError();
}
template cudaError_t launch_rap_explicit<double>(int, const FineTab &, const int32_t *, const uint8_t *,
                                                 double, const CoarseLev<double> &, const int32_t *,
                                                 const CoarseLev<double> &, int, double *, cudaStream_t);
template cudaError_t launch_rap_explicit<float>(int, const FineTab &, const int32_t *, const uint8_t *,
                                                float, const CoarseLev<float> &, const int32_t *,
                                                const CoarseLev<float> &, int, float *, cudaStream_t);

// ----------------------------------------------------------------------------- coarse operator
// One launch per operator application: the first blocks take the class rows in 32 x 8 tiles
// (stencil S_k from the per-control table), the remaining blocks stride over the explicit
// rows (dense window), whose number is read from device memory so that the launch shape does
// not depend on the current hierarchy.
template <typename T, int OP>
__device__ __forceinline__ void coarse_finish(T *y, const T *x, const T *b, int j, T acc, T d, T omega) {
  if (OP == OP_APPLY) y[j] = acc;
  else if (OP == OP_RESID) y[j] = b[j] - acc;
  else y[j] = x[j] + omega * (b[j] - acc) / d;
}

template <typename T, int OP>
__device__ __forceinline__ void coarse_class_row(const CoarseLev<T> &L, int k, int j, T omega,
                                                 const T *__restrict__ x, const T *__restrict__ b,
                                                 T *__restrict__ y, int color = -1) {
  if ((OP == OP_JACOBI || OP == OP_JACOBI0) && color >= 0 && (((j % L.n) + (j / L.n)) & 1) != color) {
    y[j] = OP == OP_JACOBI ? x[j] : T(0);
    return;
  }
  const T d = L.cdiag[k];
  if (OP == OP_JACOBI0) {
    y[j] = omega * b[j] / d;
    return;
  }
  T acc = T(0);
  const int nt = L.cnt[k];
  for (int t = 0; t < nt; ++t) {
    const int ix = k * L.ctmax + t;
    acc = fma(__ldg(L.cw + ix), __ldg(x + j + __ldg(L.clin + ix)), acc);
  }
  coarse_finish<T, OP>(y, x, b, j, acc, d, omega);
}

// Partial product of explicit row `slot` (centre j = (I1, I2)) with x over the window rows
// dy = ylo + part, ylo + part + step, ...: sum of w(dy, dx) x_{j + dy n + dx}, dx ascending
// within a row.  With RR > 0 the reach is a compile-time constant and each window row is
// unrolled with a predicate per entry, so its 2 RR + 1 weight and value loads are in flight
// together (with runtime bounds every FMA waited for its own pair of loads); RR = 0 reads the
// reach from the level.  Both orders of summation are the same.
template <typename T, int RR>
__device__ __forceinline__ T expl_window_sum(const CoarseLev<T> &L, int slot, int j, int I1, int I2,
                                             const T *__restrict__ x, int part, int step) {
  const int R = RR > 0 ? RR : L.R, Wd = 2 * R + 1;
  const int ylo = max(-R, -I2), yhi = min(R, L.n - 1 - I2);
  const int xlo = max(-R, -I1), xhi = min(R, L.n - 1 - I1);
  T acc = T(0);
  for (int dy = ylo + part; dy <= yhi; dy += step) {
    const T *wrow = L.ewin + size_t((dy + R) * Wd + R) * L.cap + slot;
    const T *xrow = x + j + dy * L.n;
    if (RR > 0) {
#pragma unroll
      for (int dx = -RR; dx <= RR; ++dx)
        if (dx >= xlo && dx <= xhi) acc = fma(wrow[ptrdiff_t(dx) * L.cap], __ldg(xrow + dx), acc);
    } else {
      for (int dx = xlo; dx <= xhi; ++dx) acc = fma(wrow[ptrdiff_t(dx) * L.cap], __ldg(xrow + dx), acc);
    }
  }
  return acc;
}

template <typename T>
__device__ __forceinline__ T expl_window_sum_any(const CoarseLev<T> &L, int slot, int j, int I1, int I2,
                                                 const T *__restrict__ x, int part, int step) {
  switch (L.R) {
    case 1: return expl_window_sum<T, 1>(L, slot, j, I1, I2, x, part, step);
    case 2: return expl_window_sum<T, 2>(L, slot, j, I1, I2, x, part, step);
    case 3: return expl_window_sum<T, 3>(L, slot, j, I1, I2, x, part, step);
    case 4: return expl_window_sum<T, 4>(L, slot, j, I1, I2, x, part, step);
    case 5: return expl_window_sum<T, 5>(L, slot, j, I1, I2, x, part, step);
    case 6: return expl_window_sum<T, 6>(L, slot, j, I1, I2, x, part, step);
    case 7: return expl_window_sum<T, 7>(L, slot, j, I1, I2, x, part, step);
    case 8: return expl_window_sum<T, 8>(L, slot, j, I1, I2, x, part, step);
    default: return expl_window_sum<T, 0>(L, slot, j, I1, I2, x, part, step);
  }
}

template <typename T, int OP>
__device__ __forceinline__ void coarse_expl_row(const CoarseLev<T> &L, int slot, T omega,
                                                const T *__restrict__ x, const T *__restrict__ b,
                                                T *__restrict__ y, int color = -1) {
  const int j = L.erow[slot];
  const int I1 = j % L.n, I2 = j / L.n;
  if ((OP == OP_JACOBI || OP == OP_JACOBI0) && color >= 0 && ((I1 + I2) & 1) != color) {
    y[j] = OP == OP_JACOBI ? x[j] : T(0);
    return;
  }
  const int R = L.R, Wd = 2 * R + 1;
  const T d = L.ewin[size_t(R * Wd + R) * L.cap + slot];
  if (OP == OP_JACOBI0) {
    y[j] = omega * b[j] / d;
    return;
  }
  const T acc = expl_window_sum_any<T>(L, slot, j, I1, I2, x, 0, 1);
  coarse_finish<T, OP>(y, x, b, j, acc, d, omega);
}

// Class rows from a shared-memory tile of x: 32 x 32 rows per block (four per thread, one
// column) plus a halo of R (the level's stencil reach).  Class taps are packed {tile offset,
// weight}.  With STAB the block first copies the level's whole class table (nk * ctmax taps,
// 12-21 KB in FP32 at 2049^2) into shared memory beside the tile, in the same pass as the
// staging: on the small levels, where an SM runs one or two tiles, the table is cold in L1
// and every group of global tap loads cost an L2 round trip.
constexpr int kCRowsY = 32;
constexpr size_t kClassTabSmemMax = 48 * 1024;  // larger tables stay in global memory
constexpr int kClassTabSmemTiles = 256;          // only levels with at most this many tiles

template <typename T>
__host__ __device__ inline size_t coarse_tile_bytes(int R) {
  return (size_t(coarse_pitch(R)) * (kCRowsY + 2 * R) * sizeof(T) + 15) / 16 * 16;
}

// Capped at six blocks of 256 threads per SM (40 registers): the explicit rows' unrolled
// windows alone would take 62, which halved the residency of the class-row tiles that share
// the launch; the cap costs a few bytes of spill and measured faster over a whole step.
template <typename T, int OP, int STAB>
__global__ void __launch_bounds__(256, 6) k_coarse_op(CoarseLev<T> L, const int *__restrict__ nexpl_dev,
                                                   int tiles_x, int tiles, T omega, const T *__restrict__ x,
                                                   const T *__restrict__ b, T *__restrict__ y, int color) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (int(blockIdx.x) < tiles) {
    using PK = typename ClassTap<T>::Packed;
    T *xs = reinterpret_cast<T *>(smem_raw);
    PK *ts = reinterpret_cast<PK *>(smem_raw + coarse_tile_bytes<T>(L.R));
    const int R = L.R, SW = coarse_pitch(R), SH = kCRowsY + 2 * R;
    const int bx = blockIdx.x % tiles_x, by = blockIdx.x / tiles_x;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (STAB && OP != OP_JACOBI0) {
      const PK *src = ClassTap<T>::table(L);
      const int nt_all = L.nk * L.ctmax;
      for (int i0 = threadIdx.x; i0 < nt_all; i0 += 4 * blockDim.x) {  // four loads, then four stores
        PK v[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int i = i0 + b * blockDim.x;
          if (i < nt_all) v[b] = src[i];
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int i = i0 + b * blockDim.x;
          if (i < nt_all) ts[i] = v[b];
        }
      }
    }
    if (OP != OP_JACOBI0) {
      const int o1 = 1 + bx * 32 - R, o2 = 1 + by * kCRowsY - R;
      stage_window<4, T>(xs, SW, SH, tx, ty, [&](int r, int c) {
        const int g2 = o2 + r, g1 = o1 + c;
        return (g2 >= 0 && g2 < L.n && g1 >= 0 && g1 < L.n) ? x[size_t(g2) * L.n + g1] : T(0);
      }, 32 + 2 * R);
      __syncthreads();
    }
    const int I1 = 1 + bx * 32 + tx;
    if (I1 > L.m) return;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int I2 = 1 + by * kCRowsY + ty + 8 * r;
      if (I2 > L.m) continue;
      const int k = L.cls[(I2 - 1) * L.m + (I1 - 1)];
      if (k < 0) continue;
      const int j = I2 * L.n + I1;
      const int sidx = (ty + 8 * r + R) * SW + tx + R;
      if ((OP == OP_JACOBI || OP == OP_JACOBI0) && color >= 0 && ((I1 + I2) & 1) != color) {
        y[j] = OP == OP_JACOBI ? xs[sidx] : T(0);
        continue;
      }
      const T d = L.cdiag[k];
      if (OP == OP_JACOBI0) {
        y[j] = omega * b[j] / d;
        continue;
      }
      T acc = T(0);
      const int nt = L.cnt[k];
      if (STAB) {
        const PK *tk = ts + k * L.ctmax;
#pragma unroll 4
        for (int t = 0; t < nt; ++t) {
          int off;
          T w;
          ClassTap<T>::unpack(tk[t], off, w);
          acc = fma(w, xs[sidx + off], acc);
        }
      } else {
#pragma unroll 4
        for (int t = 0; t < nt; ++t) {
          int off;
          T w;
          ClassTap<T>::get(L, k * L.ctmax + t, off, w);
          acc = fma(w, xs[sidx + off], acc);
        }
      }
      if (OP == OP_APPLY) y[j] = acc;
      else if (OP == OP_RESID) y[j] = b[j] - acc;
      else y[j] = xs[sidx] + omega * (b[j] - acc) / d;
    }
    return;
  }
  // Explicit rows: four threads per row, each taking every fourth row of the window, then a
  // shuffle reduction.  Four threads keep four times as many loads in flight with the same
  // sectors (neighbouring slots stay neighbours in memory), and each window row issues all of
  // its loads at once (expl_window_sum).
  const int nexpl = *nexpl_dev;
  const int nb = gridDim.x - tiles;
  const int part = threadIdx.x & 3;
  const int stride = (nb * blockDim.x) >> 2;
  for (int slot = ((blockIdx.x - tiles) * blockDim.x + threadIdx.x) >> 2;
       __any_sync(0xffffffffu, slot < nexpl); slot += stride) {
    const bool act = slot < nexpl;
    T acc = T(0), d = T(1);
    int j = 0;
    bool pass = false;  // a row of the other colour in a Gauss-Seidel half-sweep
    if (act) {
      j = L.erow[slot];
      const int I1 = j % L.n, I2 = j / L.n;
      pass = (OP == OP_JACOBI || OP == OP_JACOBI0) && color >= 0 && ((I1 + I2) & 1) != color;
      const int R = L.R, Wd = 2 * R + 1;
      d = L.ewin[size_t(R * Wd + R) * L.cap + slot];
      if (OP != OP_JACOBI0 && !pass) acc = expl_window_sum_any<T>(L, slot, j, I1, I2, x, part, 4);
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (act && part == 0) {
      if (pass) y[j] = OP == OP_JACOBI ? x[j] : T(0);
      else if (OP == OP_JACOBI0) y[j] = omega * b[j] / d;
      else coarse_finish<T, OP>(y, x, b, j, acc, d, omega);
    }
  }
}

template <typename T>
void launch_coarse_op(int op, const CoarseLev<T> &L, const int *nexpl_dev, T omega, const T *x,
                      const T *b, T *y, cudaStream_t s, int color) {
  const int tx = (L.m + 31) / 32, tiles = tx * ((L.m + kCRowsY - 1) / kCRowsY);
  const int eg = std::max(1, std::min(2 * kRedBlocks, (4 * L.cap + 255) / 256));  // 4 threads per explicit row
  const int grid = tiles + eg;
  const size_t tab_bytes = size_t(L.nk) * L.ctmax * sizeof(typename ClassTap<T>::Packed);
  const bool stab = op != OP_JACOBI0 && L.nk > 0 && tab_bytes <= kClassTabSmemMax && tiles <= kClassTabSmemTiles;
  const size_t bytes = op == OP_JACOBI0 ? 0 : coarse_tile_bytes<T>(L.R) + (stab ? tab_bytes : 0);
  note_launch();
#define SL_COARSE_LAUNCH(OPV, ST) \
  k_coarse_op<T, OPV, ST><<<grid, 256, bytes, s>>>(L, nexpl_dev, tx, tiles, omega, x, b, y, color)
  switch (op) {
    case OP_APPLY: if (stab) SL_COARSE_LAUNCH(OP_APPLY, 1); else SL_COARSE_LAUNCH(OP_APPLY, 0); break;
    case OP_RESID: if (stab) SL_COARSE_LAUNCH(OP_RESID, 1); else SL_COARSE_LAUNCH(OP_RESID, 0); break;
    case OP_JACOBI: if (stab) SL_COARSE_LAUNCH(OP_JACOBI, 1); else SL_COARSE_LAUNCH(OP_JACOBI, 0); break;
    default: SL_COARSE_LAUNCH(OP_JACOBI0, 0); break;
  }
#undef SL_COARSE_LAUNCH
}
template void launch_coarse_op<double>(int, const CoarseLev<double> &, const int *, double,
                                       const double *, const double *, double *, cudaStream_t, int);
template void launch_coarse_op<float>(int, const CoarseLev<float> &, const int *, float, const float *,
                                      const float *, float *, cudaStream_t, int);

// ----------------------------------------------------------------------------- fused level passes
// The V-cycle's passes over one coarse level l >= 1 with the Jacobi smoother, two launches per
// level instead of five:
//   k_coarse_down: x = omega D^-1 b (the first pre-smoothing sweep from zero) or x as given,
//                  r = b - A_l x, and b_{l+1} = R r (full weighting);
//   k_coarse_up:   v = x + P x_{l+1} (the coarse-grid correction), then one Jacobi sweep
//                  y = v + omega D^-1 (b - A_l v).
// A block owns a tile of 32 x TH rows and stages its values plus a halo of R in shared memory,
// computing the staged values (omega b / d, or x + P x_c) for the halo itself, so no pass
// needs another block's output.  Class rows sum their taps from the tile; the tile's explicit
// rows go to a shared list that the whole block then works through in the order of
// k_coarse_op's explicit blocks (four threads per row, each summing the window
// rows dy = ylo + p mod 4, then two shuffles), so each value equals that of the one-pass
// kernels bit for bit.  The restriction needs the residuals of one row and one column past the tile
// (its last coarse node's full-weighting stencil), which the down pass computes as well.

// Diagonal of interior row (g1, g2): the class table's centre, or the explicit window's.
template <typename T>
__device__ __forceinline__ T coarse_diag(const CoarseLev<T> &L, int g1, int g2) {
  const int k = L.cls[(g2 - 1) * L.m + (g1 - 1)];
  if (k >= 0) return L.cdiag[k];
  return L.ewin[size_t(L.R * (2 * L.R + 1) + L.R) * L.cap + (-k - 1)];
}

template <typename T, int STAB>
__device__ __forceinline__ T class_sum_staged(const CoarseLev<T> &L, const typename ClassTap<T>::Packed *ts,
                                              int k, const T *xs, int sidx) {
  T acc = T(0);
  const int nt = L.cnt[k];
  if (STAB) {
    const typename ClassTap<T>::Packed *tk = ts + k * L.ctmax;
#pragma unroll 4
    for (int t = 0; t < nt; ++t) {
      int off;
      T w;
      ClassTap<T>::unpack(tk[t], off, w);
      acc = fma(w, xs[sidx + off], acc);
    }
  } else {
#pragma unroll 4
    for (int t = 0; t < nt; ++t) {
      int off;
      T w;
      ClassTap<T>::get(L, k * L.ctmax + t, off, w);
      acc = fma(w, xs[sidx + off], acc);
    }
  }
  return acc;
}

// Partial window sum of explicit row `slot`, centre (I1, I2) staged at xs[sidx] (pitch P): the
// window rows dy = ylo + part, ylo + part + 4, ..., each in ascending dx, as one of the four
// threads of k_coarse_op's explicit blocks computes it; four threads per row then add their
// parts with the same two shuffles, so the row's value is that of the one-pass kernel.
template <typename T, int RR>
__device__ __forceinline__ T expl_part_staged(const CoarseLev<T> &L, int slot, int I1, int I2, const T *xs,
                                              int sidx, int P, int part) {
  const int R = RR > 0 ? RR : L.R, Wd = 2 * R + 1;
  const int ylo = max(-R, -I2), yhi = min(R, L.n - 1 - I2);
  const int xlo = max(-R, -I1), xhi = min(R, L.n - 1 - I1);
  T acc = T(0);
  for (int dy = ylo + part; dy <= yhi; dy += 4) {
    const T *wrow = L.ewin + size_t((dy + R) * Wd + R) * L.cap + slot;
    const T *xrow = xs + sidx + dy * P;
    if (RR > 0) {
#pragma unroll
      for (int dx = -RR; dx <= RR; ++dx)
        if (dx >= xlo && dx <= xhi) acc = fma(__ldg(wrow + ptrdiff_t(dx) * L.cap), xrow[dx], acc);
    } else {
      for (int dx = xlo; dx <= xhi; ++dx) acc = fma(__ldg(wrow + ptrdiff_t(dx) * L.cap), xrow[dx], acc);
    }
  }
  return acc;
}

template <typename T>
__device__ __forceinline__ T expl_part_staged_any(const CoarseLev<T> &L, int slot, int I1, int I2, const T *xs,
                                                  int sidx, int P, int part) {
  switch (L.R) {
    case 1: return expl_part_staged<T, 1>(L, slot, I1, I2, xs, sidx, P, part);
    case 2: return expl_part_staged<T, 2>(L, slot, I1, I2, xs, sidx, P, part);
    case 3: return expl_part_staged<T, 3>(L, slot, I1, I2, xs, sidx, P, part);
    case 4: return expl_part_staged<T, 4>(L, slot, I1, I2, xs, sidx, P, part);
    case 5: return expl_part_staged<T, 5>(L, slot, I1, I2, xs, sidx, P, part);
    case 6: return expl_part_staged<T, 6>(L, slot, I1, I2, xs, sidx, P, part);
    default: return expl_part_staged<T, 0>(L, slot, I1, I2, xs, sidx, P, part);
  }
}

// Shared-memory layout of the fused passes: [class table (STAB)] [tile] [residuals (down)]
// [explicit list: local row index, slot].
template <typename T>
struct FusedSmem {
  size_t tab, tile, res, list;
  __host__ __device__ FusedSmem(int R, int TH, int nk, int ctmax, bool stab, bool down) {
    tab = stab ? (size_t(nk) * ctmax * sizeof(typename ClassTap<T>::Packed) + 15) / 16 * 16 : 0;
    const int rows = down ? TH + 1 : TH, cols = down ? 33 : 32;
    tile = (size_t(coarse_pitch(R)) * (rows + 2 * R) * sizeof(T) + 15) / 16 * 16;
    res = down ? (size_t(rows) * cols * sizeof(T) + 15) / 16 * 16 : 0;
    list = size_t(rows) * cols * 2 * sizeof(int);
  }
  __host__ __device__ size_t total() const { return tab + tile + res + list; }
};

template <typename T, int STAB>
__device__ __forceinline__ void stage_class_table(const CoarseLev<T> &L, typename ClassTap<T>::Packed *ts) {
  if (!STAB) return;
  using PK = typename ClassTap<T>::Packed;
  const PK *src = ClassTap<T>::table(L);
  const int nt_all = L.nk * L.ctmax;
  for (int i0 = threadIdx.x; i0 < nt_all; i0 += 4 * blockDim.x) {  // four loads, then four stores
    PK v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + q * blockDim.x;
      if (i < nt_all) v[q] = src[i];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + q * blockDim.x;
      if (i < nt_all) ts[i] = v[q];
    }
  }
}

template <typename T, int TH, int STAB, int FROM_ZERO>
__global__ void __launch_bounds__(256) k_coarse_down(CoarseLev<T> L, int tiles_x, T omega,
                                                     const T *__restrict__ b, const T *__restrict__ xin,
                                                     T *__restrict__ xout, T *__restrict__ bc, int nc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int ecount;
  using PK = typename ClassTap<T>::Packed;
  constexpr int RW = 33, NQ = (TH + 1) * RW;  // residual rows: the tile plus its ring
  const int R = L.R, P = coarse_pitch(R);
  const FusedSmem<T> lay(R, TH, L.nk, L.ctmax, STAB != 0, true);
  PK *ts = reinterpret_cast<PK *>(smem_raw);
  T *xs = reinterpret_cast<T *>(smem_raw + lay.tab);
  T *rs = reinterpret_cast<T *>(smem_raw + lay.tab + lay.tile);
  int *eq = reinterpret_cast<int *>(smem_raw + lay.tab + lay.tile + lay.res);
  int *eslot = eq + NQ;
  const int bx = blockIdx.x % tiles_x, by = blockIdx.x / tiles_x;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (threadIdx.x == 0) ecount = 0;
  stage_class_table<T, STAB>(L, ts);
  const int o1 = 1 + bx * 32, o2 = 1 + by * TH;
  // staged node (r, c) is grid node (o1 - R + c, o2 - R + r); boundary and outside nodes are 0
  stage_window<(TH >= 16 ? 4 : 2), T>(xs, P, TH + 1 + 2 * R, tx, ty, [&](int r, int c) {
    const int g2 = o2 - R + r, g1 = o1 - R + c;
    if (g2 < 1 || g2 > L.m || g1 < 1 || g1 > L.m) return T(0);
    if (FROM_ZERO) return omega * b[size_t(g2) * L.n + g1] / coarse_diag<T>(L, g1, g2);
    return xin[size_t(g2) * L.n + g1];
  });
  __syncthreads();
  for (int q = threadIdx.x; q < NQ; q += blockDim.x) {
    const int r = q / RW, c = q - r * RW;
    const int g1 = o1 + c, g2 = o2 + r;
    T res = T(0);
    if (g1 <= L.m && g2 <= L.m) {
      const int sidx = (r + R) * P + c + R;
      const size_t j = size_t(g2) * L.n + g1;
      if (FROM_ZERO && r < TH && c < 32) xout[j] = xs[sidx];
      const int k = L.cls[(g2 - 1) * L.m + (g1 - 1)];
      if (k < 0) {
        const int e = atomicAdd(&ecount, 1);
        eq[e] = q;
        eslot[e] = -k - 1;
        continue;
      }
      res = b[j] - class_sum_staged<T, STAB>(L, ts, k, xs, sidx);
    }
    rs[q] = res;
  }
  __syncthreads();
  // explicit rows: four threads per row (window rows dy = ylo + part mod 4), then two shuffles
  const int ne4 = 4 * ecount;
  for (int base = 0; base < ne4; base += blockDim.x) {
    const int idx = base + threadIdx.x, part = idx & 3;
    T acc = T(0);
    int q = 0, g1 = 0, g2 = 0;
    if (idx < ne4) {
      q = eq[idx >> 2];
      const int r = q / RW, c = q - r * RW;
      g1 = o1 + c;
      g2 = o2 + r;
      acc = expl_part_staged_any<T>(L, eslot[idx >> 2], g1, g2, xs, (r + R) * P + c + R, P, part);
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (idx < ne4 && part == 0) rs[q] = b[size_t(g2) * L.n + g1] - acc;
  }
  __syncthreads();
  // full weighting: this tile's coarse nodes I1 = 16 bx + 1 + c1, I2 = (TH / 2) by + 1 + c2 sit at
  // residual rows 1 + 2 c2, columns 1 + 2 c1
  constexpr int CH = TH / 2;
  const int c1 = threadIdx.x & 15, c2 = threadIdx.x >> 4;
  if (c2 < CH) {
    const int I1 = 16 * bx + 1 + c1, I2 = CH * by + 1 + c2;
    if (I1 <= nc - 2 && I2 <= nc - 2) bc[size_t(I2) * nc + I1] = restrict_point<T>(rs + RW + 1, RW, c1, c2);
  }
}

template <typename T, int TH, int STAB>
__global__ void __launch_bounds__(256) k_coarse_up(CoarseLev<T> L, int tiles_x, T omega, const T *__restrict__ b,
                                                   const T *__restrict__ cur, const T *__restrict__ xc, int nc,
                                                   T *__restrict__ y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int ecount;
  using PK = typename ClassTap<T>::Packed;
  constexpr int NQ = TH * 32;
  const int R = L.R, P = coarse_pitch(R), Wd = 2 * R + 1;
  const FusedSmem<T> lay(R, TH, L.nk, L.ctmax, STAB != 0, false);
  PK *ts = reinterpret_cast<PK *>(smem_raw);
  T *xs = reinterpret_cast<T *>(smem_raw + lay.tab);
  int *eq = reinterpret_cast<int *>(smem_raw + lay.tab + lay.tile);
  int *eslot = eq + NQ;
  const int bx = blockIdx.x % tiles_x, by = blockIdx.x / tiles_x;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (threadIdx.x == 0) ecount = 0;
  stage_class_table<T, STAB>(L, ts);
  const int o1 = 1 + bx * 32, o2 = 1 + by * TH;
  stage_window<(TH >= 16 ? 4 : 2), T>(xs, P, TH + 2 * R, tx, ty, [&](int r, int c) {
    const int g2 = o2 - R + r, g1 = o1 - R + c;
    if (g2 < 1 || g2 > L.m || g1 < 1 || g1 > L.m) return T(0);
    return cur[size_t(g2) * L.n + g1] + prolong_point<T>(xc, nc, g1, g2);
  }, 32 + 2 * R);
  __syncthreads();
  for (int q = threadIdx.x; q < NQ; q += blockDim.x) {
    const int r = q >> 5, c = q & 31;
    const int g1 = o1 + c, g2 = o2 + r;
    if (g1 > L.m || g2 > L.m) continue;
    const int k = L.cls[(g2 - 1) * L.m + (g1 - 1)];
    if (k < 0) {
      const int e = atomicAdd(&ecount, 1);
      eq[e] = q;
      eslot[e] = -k - 1;
      continue;
    }
    const int sidx = (r + R) * P + c + R;
    const size_t j = size_t(g2) * L.n + g1;
    const T acc = class_sum_staged<T, STAB>(L, ts, k, xs, sidx);
    y[j] = xs[sidx] + omega * (b[j] - acc) / L.cdiag[k];
  }
  __syncthreads();
  const int ne4 = 4 * ecount;
  for (int base = 0; base < ne4; base += blockDim.x) {
    const int idx = base + threadIdx.x, part = idx & 3;
    T acc = T(0);
    int slot = 0, sidx = 0;
    size_t j = 0;
    if (idx < ne4) {
      const int q = eq[idx >> 2];
      slot = eslot[idx >> 2];
      const int r = q >> 5, c = q & 31;
      const int g1 = o1 + c, g2 = o2 + r;
      sidx = (r + R) * P + c + R;
      j = size_t(g2) * L.n + g1;
      acc = expl_part_staged_any<T>(L, slot, g1, g2, xs, sidx, P, part);
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (idx < ne4 && part == 0) {
      const T d = L.ewin[size_t(R * Wd + R) * L.cap + slot];
      y[j] = xs[sidx] + omega * (b[j] - acc) / d;
    }
  }
}

// Tile height of the fused passes: the tallest of 32, 16 rows that still gives at least 512
// tiles (about three per SM); smaller levels take 8, and 4 when 8 would give fewer than 512
// tiles (their passes are latency-bound: more, smaller blocks run their phases in parallel).
static int fused_tile_rows(int m) {
  const int tx = (m + 31) / 32;
  for (int th : {32, 16})
    if (tx * ((m + th - 1) / th) >= 512) return th;
  return tx * ((m + 7) / 8) >= 512 ? 8 : 4;
}

template <typename T>
static bool fused_stab(const CoarseLev<T> &L, int blocks) {
  const size_t tab_bytes = size_t(L.nk) * L.ctmax * sizeof(typename ClassTap<T>::Packed);
  return L.nk > 0 && tab_bytes <= kClassTabSmemMax && blocks <= kClassTabSmemTiles;
}

template <typename T>
void launch_coarse_down(const CoarseLev<T> &L, T omega, const T *b, const T *xin, T *xout, T *bc, int nc,
                        cudaStream_t s) {
  const int th = fused_tile_rows(L.m);
  const int tx = (L.m + 31) / 32, blocks = tx * ((L.m + th - 1) / th);
  const bool stab = fused_stab(L, blocks);
  const size_t bytes = FusedSmem<T>(L.R, th, L.nk, L.ctmax, stab, true).total();
  const bool z = xin == nullptr;
  note_launch();
#define SL_DOWN(TH, ST, Z) \
  k_coarse_down<T, TH, ST, Z><<<blocks, 256, bytes, s>>>(L, tx, omega, b, xin, xout, bc, nc)
#define SL_DOWN_TH(TH) \
  if (stab) { if (z) SL_DOWN(TH, 1, 1); else SL_DOWN(TH, 1, 0); } \
  else { if (z) SL_DOWN(TH, 0, 1); else SL_DOWN(TH, 0, 0); }
  if (th == 32) { SL_DOWN_TH(32) }
  else if (th == 16) { SL_DOWN_TH(16) }
  else if (th == 8) { SL_DOWN_TH(8) }
  else { SL_DOWN_TH(4) }
#undef SL_DOWN_TH
#undef SL_DOWN
}

template <typename T>
void launch_coarse_up(const CoarseLev<T> &L, T omega, const T *b, const T *cur, const T *xc, int nc, T *y,
                      cudaStream_t s) {
  const int th = fused_tile_rows(L.m);
  const int tx = (L.m + 31) / 32, blocks = tx * ((L.m + th - 1) / th);
  const bool stab = fused_stab(L, blocks);
  const size_t bytes = FusedSmem<T>(L.R, th, L.nk, L.ctmax, stab, false).total();
  note_launch();
#define SL_UP(TH, ST) k_coarse_up<T, TH, ST><<<blocks, 256, bytes, s>>>(L, tx, omega, b, cur, xc, nc, y)
  if (th == 32) { if (stab) SL_UP(32, 1); else SL_UP(32, 0); }
  else if (th == 16) { if (stab) SL_UP(16, 1); else SL_UP(16, 0); }
  else if (th == 8) { if (stab) SL_UP(8, 1); else SL_UP(8, 0); }
  else { if (stab) SL_UP(4, 1); else SL_UP(4, 0); }
#undef SL_UP
}
template void launch_coarse_down<double>(const CoarseLev<double> &, double, const double *, const double *,
                                         double *, double *, int, cudaStream_t);
template void launch_coarse_down<float>(const CoarseLev<float> &, float, const float *, const float *, float *,
                                        float *, int, cudaStream_t);
template void launch_coarse_up<double>(const CoarseLev<double> &, double, const double *, const double *,
                                       const double *, int, double *, cudaStream_t);
template void launch_coarse_up<float>(const CoarseLev<float> &, float, const float *, const float *,
                                      const float *, int, float *, cudaStream_t);

// ----------------------------------------------------------------------------- V-cycle tail
// The coarse end of the V-cycle (every level from l0 down, each with at most a few thousand
// rows) in one thread block: on these levels a grid-wide launch per operation costs more
// than the work, so one CTA walks the levels with __syncthreads between phases.  Each row
// uses the same device functions as the grid-wide kernels.
template <typename T>
__device__ void tail_op(const CoarseLev<T> &L, int op, T omega, const T *x, const T *b, T *y, int color = -1) {
  const int rows = L.m * L.m;
  for (int I = threadIdx.x; I < rows; I += blockDim.x) {
    const int j = (1 + I / L.m) * L.n + 1 + I % L.m;
    const int c = L.cls[I];
    if (c >= 0) {
      switch (op) {
        case OP_RESID: coarse_class_row<T, OP_RESID>(L, c, j, omega, x, b, y); break;
        case OP_JACOBI: coarse_class_row<T, OP_JACOBI>(L, c, j, omega, x, b, y, color); break;
        default: coarse_class_row<T, OP_JACOBI0>(L, c, j, omega, x, b, y, color); break;
      }
    } else {
      switch (op) {
        case OP_RESID: coarse_expl_row<T, OP_RESID>(L, -c - 1, omega, x, b, y); break;
        case OP_JACOBI: coarse_expl_row<T, OP_JACOBI>(L, -c - 1, omega, x, b, y, color); break;
        default: coarse_expl_row<T, OP_JACOBI0>(L, -c - 1, omega, x, b, y, color); break;
      }
    }
  }
  __syncthreads();
}

// nu sweeps of the tail's smoother on level L from *c (from_zero: the first sweep starts at
// x = 0 and writes *c), ping-ponging between *c and *o; the order of kernels of the grid-wide
// path (sl_api.cu's smooth()).
template <typename T>
__device__ void tail_smooth(const CoarseLev<T> &L, const TailArgs<T> &a, const T *b, T *&c, T *&o,
                            int sweeps, bool from_zero) {
  for (int it = 0; it < sweeps; ++it) {
    if (a.rbgs) {
      for (int col = 0; col < 2; ++col) {
        if (from_zero && it == 0 && col == 0) {
          tail_op<T>(L, OP_JACOBI0, a.omega, nullptr, b, c, 0);
        } else {
          tail_op<T>(L, OP_JACOBI, a.omega, c, b, o, col);
          T *sw = c; c = o; o = sw;
        }
      }
    } else if (from_zero && it == 0) {
      tail_op<T>(L, OP_JACOBI0, a.omega, nullptr, b, c);
    } else {
      tail_op<T>(L, OP_JACOBI, a.omega, c, b, o);
      T *sw = c; c = o; o = sw;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_vcycle_tail(TailArgs<T> a) {
  T *cur[kMaxLevels];
  for (int l = a.l0; l < a.L - 1; ++l) {
    const CoarseLev<T> &L = a.lev[l];
    T *c = a.x[l], *o = a.t[l];
    if (a.nu1 == 0) {
      for (int I = threadIdx.x; I < L.m * L.m; I += blockDim.x) c[(1 + I / L.m) * L.n + 1 + I % L.m] = T(0);
      __syncthreads();
    } else {
      tail_smooth<T>(L, a, a.b[l], c, o, a.nu1, true);
    }
    tail_op<T>(L, OP_RESID, a.omega, c, a.b[l], a.r[l]);
    const CoarseLev<T> &C = a.lev[l + 1];
    for (int I = threadIdx.x; I < C.m * C.m; I += blockDim.x) {
      const int I1 = 1 + I % C.m, I2 = 1 + I / C.m;
      a.b[l + 1][I2 * C.n + I1] = restrict_point<T>(a.r[l], L.n, I1, I2);
    }
    __syncthreads();
    cur[l] = c;
  }
  {  // coarsest: x = A^{-1} b
    const CoarseLev<T> &C = a.lev[a.L - 1];
    const int N = C.m * C.m;
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      T acc = T(0);
      for (int c = 0; c < N; ++c) acc = fma(a.Ainv[size_t(r) * N + c], a.b[a.L - 1][(1 + c / C.m) * C.n + 1 + c % C.m], acc);
      a.x[a.L - 1][(1 + r / C.m) * C.n + 1 + r % C.m] = acc;
    }
    __syncthreads();
    cur[a.L - 1] = a.x[a.L - 1];
  }
  for (int l = a.L - 2; l >= a.l0; --l) {
    const CoarseLev<T> &L = a.lev[l];
    const CoarseLev<T> &C = a.lev[l + 1];
    T *c = cur[l], *o = (c == a.x[l]) ? a.t[l] : a.x[l];
    for (int I = threadIdx.x; I < L.m * L.m; I += blockDim.x) {
      const int i1 = 1 + I % L.m, i2 = 1 + I / L.m;
      c[i2 * L.n + i1] += prolong_point<T>(cur[l + 1], C.n, i1, i2);
    }
    __syncthreads();
    tail_smooth<T>(L, a, a.b[l], c, o, a.nu2, false);
    cur[l] = c;
  }
  if (cur[a.l0] != a.x[a.l0]) {
    const CoarseLev<T> &L = a.lev[a.l0];
    for (int I = threadIdx.x; I < L.m * L.m; I += blockDim.x) {
      const int j = (1 + I / L.m) * L.n + 1 + I % L.m;
      a.x[a.l0][j] = cur[a.l0][j];
    }
  }
}

// The same tail with every level's vectors and stencils in shared memory.  Each row's stencil
// is a dense (2R+1)^2 window ([e][I]: window entry e of row I; a class row's taps scattered
// into its window, zeros elsewhere), packed once per hierarchy into a device image
// (k_tail_pack) in exactly the shared-memory layout, so the block copies it with 16-byte loads
// (a few hundred KB from L2); after that every phase reads shared memory only, with the window
// loops unrolled on the reach, so a phase costs a few hundred cycles instead of the chain of
// L2 round trips (row class, then taps and values) of the global form.  Each row sums its
// window in the order of the explicit rows of tail_op (dy, then dx ascending); a class row's
// added zeros leave its sum unchanged.  Launched when the levels fit (launch_vcycle_tail).
struct TailSmem {
  int win[kMaxLevels];  // byte offsets of the windows of level l (first, contiguous: the image)
  int vec[kMaxLevels];  // x, t, r, b (n^2 values each) of level l
  int wbytes, bytes;    // windows only (the image), and everything
};

template <typename T>
static bool tail_smem_layout(const TailArgs<T> &a, TailSmem &lay, int limit) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 15) / 16 * 16;
    return o;
  };
  for (int l = a.l0; l < a.L; ++l) {
    const CoarseLev<T> &L = a.lev[l];
    lay.win[l] = l < a.L - 1 ? int(take(size_t(L.win) * L.m * L.m * sizeof(T))) : 0;
  }
  lay.wbytes = int(off);
  for (int l = a.l0; l < a.L; ++l) lay.vec[l] = int(take(4 * size_t(a.lev[l].n) * a.lev[l].n * sizeof(T)));
  lay.bytes = int(off);
  return off <= size_t(limit);
}

static int tail_smem_limit() {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  return optin - 1024;
}

template <typename T>
size_t tail_image_bytes(const TailArgs<T> &a) {
  TailSmem lay{};
  return tail_smem_layout<T>(a, lay, tail_smem_limit()) ? size_t(lay.wbytes) : 0;
}
template size_t tail_image_bytes<double>(const TailArgs<double> &);
template size_t tail_image_bytes<float>(const TailArgs<float> &);

// Window entry e of row I of level L: the explicit row's own window, or the class row's tap at
// that offset (0 where it has none).  Indices are checked, so a hierarchy that was never built
// packs garbage values but reads nothing out of bounds.
template <typename T>
__device__ T tail_window_entry(const CoarseLev<T> &L, int e, int I) {
  const int c = L.cls[I];
  if (c < 0) {
    const int slot = -c - 1;
    return slot < L.cap ? L.ewin[size_t(e) * L.cap + slot] : T(0);
  }
  if (c >= L.nk || !L.cnt || !L.coff || !L.cw) return T(0);
  const int Wd = 2 * L.R + 1, dy = e / Wd - L.R, dx = e % Wd - L.R;
  const int nt = min(L.cnt[c], L.ctmax);
  for (int t = 0; t < nt; ++t) {
    const int o = L.coff[c * L.ctmax + t];
    if (int(int16_t(o & 0xffff)) == dx && (o >> 16) == dy) return L.cw[c * L.ctmax + t];
  }
  return T(0);
}

template <typename T>
__global__ void k_tail_pack(TailArgs<T> a, TailSmem lay, T *__restrict__ img) {
  for (int l = a.l0; l < a.L - 1; ++l) {
    const CoarseLev<T> &L = a.lev[l];
    const int m2 = L.m * L.m, tot = L.win * m2;
    T *W = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(img) + lay.win[l]);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += gridDim.x * blockDim.x) {
      const int e = idx / m2, I = idx - e * m2;
      W[idx] = tail_window_entry<T>(L, e, I);
    }
  }
}

template <typename T>
void launch_tail_pack(const TailArgs<T> &a, T *img, cudaStream_t s) {
  TailSmem lay{};
  if (!img || !tail_smem_layout<T>(a, lay, tail_smem_limit())) return;
  note_launch();
  k_tail_pack<T><<<2 * 152, 256, 0, s>>>(a, lay, img);
}
template void launch_tail_pack<double>(const TailArgs<double> &, double *, cudaStream_t);
template void launch_tail_pack<float>(const TailArgs<float> &, float *, cudaStream_t);

template <typename T, int RR>
__device__ __forceinline__ T stail_window(const T *W, int m2, int I, int Rl, const T *x, int j, int n, int I1,
                                          int I2) {
  const int R = RR > 0 ? RR : Rl, Wd = 2 * R + 1;
  const int ylo = max(-R, -I2), yhi = min(R, n - 1 - I2);
  const int xlo = max(-R, -I1), xhi = min(R, n - 1 - I1);
  T acc = T(0);
  if (RR > 0) {
#pragma unroll
    for (int dy = -RR; dy <= RR; ++dy) {
      if (dy < ylo || dy > yhi) continue;
      const T *wrow = W + size_t((dy + RR) * Wd + RR) * m2 + I;
      const T *xrow = x + j + dy * n;
#pragma unroll
      for (int dx = -RR; dx <= RR; ++dx)
        if (dx >= xlo && dx <= xhi) acc = fma(wrow[dx * m2], xrow[dx], acc);
    }
  } else {
    for (int dy = ylo; dy <= yhi; ++dy) {
      const T *wrow = W + size_t((dy + R) * Wd + R) * m2 + I;
      const T *xrow = x + j + dy * n;
      for (int dx = xlo; dx <= xhi; ++dx) acc = fma(wrow[dx * m2], xrow[dx], acc);
    }
  }
  return acc;
}

template <typename T>
__device__ void stail_op(const CoarseLev<T> &L, const T *W, int op, T omega, const T *x, const T *b, T *y,
                         int color) {
  const int m2 = L.m * L.m, R = L.R, Wd = 2 * R + 1;
  for (int I = threadIdx.x; I < m2; I += blockDim.x) {
    const int I1 = 1 + I % L.m, I2 = 1 + I / L.m;
    const int j = I2 * L.n + I1;
    if (op != OP_RESID && color >= 0 && ((I1 + I2) & 1) != color) {
      y[j] = op == OP_JACOBI ? x[j] : T(0);
      continue;
    }
    const T d = W[size_t(R * Wd + R) * m2 + I];
    if (op == OP_JACOBI0) {
      y[j] = omega * b[j] / d;
      continue;
    }
    T acc;
    switch (R) {
      case 1: acc = stail_window<T, 1>(W, m2, I, R, x, j, L.n, I1, I2); break;
      case 2: acc = stail_window<T, 2>(W, m2, I, R, x, j, L.n, I1, I2); break;
      case 3: acc = stail_window<T, 3>(W, m2, I, R, x, j, L.n, I1, I2); break;
      default: acc = stail_window<T, 0>(W, m2, I, R, x, j, L.n, I1, I2); break;
    }
    if (op == OP_RESID) y[j] = b[j] - acc;
    else y[j] = x[j] + omega * (b[j] - acc) / d;
  }
  __syncthreads();
}

template <typename T>
__device__ void stail_smooth(const CoarseLev<T> &L, const T *W, const TailArgs<T> &a, const T *b, T *&c,
                             T *&o, int sweeps, bool from_zero) {
  for (int it = 0; it < sweeps; ++it) {
    if (a.rbgs) {
      for (int col = 0; col < 2; ++col) {
        if (from_zero && it == 0 && col == 0) {
          stail_op<T>(L, W, OP_JACOBI0, a.omega, nullptr, b, c, 0);
        } else {
          stail_op<T>(L, W, OP_JACOBI, a.omega, c, b, o, col);
          T *sw = c; c = o; o = sw;
        }
      }
    } else if (from_zero && it == 0) {
      stail_op<T>(L, W, OP_JACOBI0, a.omega, nullptr, b, c, -1);
    } else {
      stail_op<T>(L, W, OP_JACOBI, a.omega, c, b, o, -1);
      T *sw = c; c = o; o = sw;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_vcycle_tail_smem(TailArgs<T> a, TailSmem lay) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto vec = [&](int l, int q) {
    return reinterpret_cast<T *>(smem_raw + lay.vec[l]) + size_t(q) * a.lev[l].n * a.lev[l].n;
  };
  auto wins = [&](int l) { return reinterpret_cast<const T *>(smem_raw + lay.win[l]); };
  // the packed stencils (16-byte pieces, eight loads in flight per thread before their stores)
  {
    const float4 *src = reinterpret_cast<const float4 *>(a.img);
    float4 *dst = reinterpret_cast<float4 *>(smem_raw);
    const int n16 = lay.wbytes / 16;
    for (int i0 = threadIdx.x; i0 < n16; i0 += 8 * blockDim.x) {
      float4 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (i0 + q * int(blockDim.x) < n16) v[q] = __ldg(src + i0 + q * blockDim.x);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (i0 + q * int(blockDim.x) < n16) dst[i0 + q * blockDim.x] = v[q];
    }
  }
  // the vectors: zero (boundary entries stay zero), then b of the first level
  {
    T *v0 = reinterpret_cast<T *>(smem_raw + lay.wbytes);
    const int nv = (lay.bytes - lay.wbytes) / int(sizeof(T));
    for (int i = threadIdx.x; i < nv; i += blockDim.x) v0[i] = T(0);
  }
  __syncthreads();
  {
    const CoarseLev<T> &L = a.lev[a.l0];
    T *b0 = vec(a.l0, 3);
    for (int i = threadIdx.x; i < L.n * L.n; i += blockDim.x) b0[i] = a.b[a.l0][i];
  }
  __syncthreads();
  T *cur[kMaxLevels];
  for (int l = a.l0; l < a.L - 1; ++l) {
    const CoarseLev<T> &L = a.lev[l];
    const T *W = wins(l);
    T *c = vec(l, 0), *o = vec(l, 1), *r = vec(l, 2), *b = vec(l, 3);
    if (a.nu1 > 0) stail_smooth<T>(L, W, a, b, c, o, a.nu1, true);  // nu1 = 0: x = 0, the zeroed vector
    stail_op<T>(L, W, OP_RESID, a.omega, c, b, r, -1);
    const CoarseLev<T> &Cl = a.lev[l + 1];
    T *bn = vec(l + 1, 3);
    for (int I = threadIdx.x; I < Cl.m * Cl.m; I += blockDim.x) {
      const int I1 = 1 + I % Cl.m, I2 = 1 + I / Cl.m;
      bn[I2 * Cl.n + I1] = restrict_point<T>(r, L.n, I1, I2);
    }
    __syncthreads();
    cur[l] = c;
  }
  {  // coarsest: x = A^{-1} b
    const CoarseLev<T> &Cl = a.lev[a.L - 1];
    const int N = Cl.m * Cl.m;
    const T *bc = vec(a.L - 1, 3);
    T *xc = vec(a.L - 1, 0);
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      T acc = T(0);
      for (int c = 0; c < N; ++c) acc = fma(__ldg(a.Ainv + size_t(r) * N + c), bc[(1 + c / Cl.m) * Cl.n + 1 + c % Cl.m], acc);
      xc[(1 + r / Cl.m) * Cl.n + 1 + r % Cl.m] = acc;
    }
    __syncthreads();
    cur[a.L - 1] = xc;
  }
  for (int l = a.L - 2; l >= a.l0; --l) {
    const CoarseLev<T> &L = a.lev[l];
    const CoarseLev<T> &Cl = a.lev[l + 1];
    const T *W = wins(l);
    T *c = cur[l], *o = (c == vec(l, 0)) ? vec(l, 1) : vec(l, 0);
    for (int I = threadIdx.x; I < L.m * L.m; I += blockDim.x) {
      const int i1 = 1 + I % L.m, i2 = 1 + I / L.m;
      c[i2 * L.n + i1] += prolong_point<T>(cur[l + 1], Cl.n, i1, i2);
    }
    __syncthreads();
    stail_smooth<T>(L, W, a, vec(l, 3), c, o, a.nu2, false);
    cur[l] = c;
  }
  const CoarseLev<T> &L = a.lev[a.l0];
  for (int I = threadIdx.x; I < L.m * L.m; I += blockDim.x) {
    const int j = (1 + I / L.m) * L.n + 1 + I % L.m;
    a.x[a.l0][j] = cur[a.l0][j];
  }
}

template <typename T>
void launch_vcycle_tail(const TailArgs<T> &a, cudaStream_t s) {
  note_launch();
  TailSmem lay{};
  if (a.img && tail_smem_layout<T>(a, lay, tail_smem_limit())) {
    k_vcycle_tail_smem<T><<<1, 1024, lay.bytes, s>>>(a, lay);
    return;
  }
  k_vcycle_tail<T><<<1, 1024, 0, s>>>(a);
}
template void launch_vcycle_tail<double>(const TailArgs<double> &, cudaStream_t);
template void launch_vcycle_tail<float>(const TailArgs<float> &, cudaStream_t);

// ----------------------------------------------------------------------------- coarsest level
// Dense matrix of the coarsest level (interior unknowns, row-major) and its inverse by
// Gauss-Jordan elimination with partial pivoting in one thread block; the V-cycle then
// applies x = A^{-1} b.
template <typename T>
__global__ void k_coarsest_setup(int level, FineTab tab, const uint8_t *__restrict__ policy, T dt,
                                 CoarseLev<T> L, const int32_t *__restrict__ coff,
                                 double *__restrict__ work, T *__restrict__ Ainv) {
  const int m = (level == 0) ? tab.m : L.m;
  const int n = (level == 0) ? tab.n : L.n;
  const int N = m * m;
  double *A = work;            // N x N
  double *Inv = work + N * N;  // N x N
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    A[idx] = 0.0;
    Inv[idx] = (idx / N == idx % N) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    const int i1 = 1 + r % m, i2 = 1 + r / m;
    auto put = [&](int dx, int dy, double v) {
      const int c1 = i1 + dx, c2 = i2 + dy;
      if (c1 < 1 || c1 > m || c2 < 1 || c2 > m) return;  // boundary columns multiply zero
      A[size_t(r) * N + (c2 - 1) * m + (c1 - 1)] += v;
    };
    if (level == 0) {
      const int k = policy[r];
      const int e = fine_row_entry(tab, k, i1, i2);
      put(0, 0, 1.0 + double(dt) * (double(tab_W<T>(tab)[e]) - double(tab_c<T>(tab)[k])));
      for (int t = 0; t < tab.nt[e]; ++t) {
        const int ix = e * tab.tmax + t;
        const int off = coff[ix];
        put(int(int16_t(off & 0xffff)), off >> 16, -double(dt) * double(tab_w<T>(tab)[ix]));
      }
    } else {
      const int c = L.cls[r];
      if (c >= 0) {
        for (int t = 0; t < L.cnt[c]; ++t) {
          const int off = coff[c * L.ctmax + t];
          put(int(int16_t(off & 0xffff)), off >> 16, double(L.cw[c * L.ctmax + t]));
        }
      } else {
        const int s = -c - 1, Wd = 2 * L.R + 1;
        for (int e = 0; e < L.win; ++e)
          put(e % Wd - L.R, e / Wd - L.R, double(L.ewin[size_t(e) * L.cap + s]));
      }
    }
  }
  __syncthreads();
  __shared__ int piv;
  for (int col = 0; col < N; ++col) {
    if (threadIdx.x == 0) {
      int p = col;
      double best = fabs(A[size_t(col) * N + col]);
      for (int r = col + 1; r < N; ++r) {
        const double v = fabs(A[size_t(r) * N + col]);
        if (v > best) { best = v; p = r; }
      }
      piv = p;
    }
    __syncthreads();
    const int p = piv;
    if (p != col) {
      for (int c = threadIdx.x; c < N; c += blockDim.x) {
        double t0 = A[size_t(col) * N + c]; A[size_t(col) * N + c] = A[size_t(p) * N + c]; A[size_t(p) * N + c] = t0;
        double t1 = Inv[size_t(col) * N + c]; Inv[size_t(col) * N + c] = Inv[size_t(p) * N + c]; Inv[size_t(p) * N + c] = t1;
      }
    }
    __syncthreads();
    const double inv = 1.0 / A[size_t(col) * N + col];
    __syncthreads();
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
      A[size_t(col) * N + c] *= inv;
      Inv[size_t(col) * N + c] *= inv;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      if (r == col) continue;
      const double f = A[size_t(r) * N + col];
      if (f == 0.0) continue;
      for (int c = 0; c < N; ++c) {
        A[size_t(r) * N + c] -= f * A[size_t(col) * N + c];
        Inv[size_t(r) * N + c] -= f * Inv[size_t(col) * N + c];
      }
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) Ainv[idx] = T(Inv[idx]);
}

template <typename T>
void launch_coarsest_setup(int level, const FineTab &tab, const uint8_t *policy, T dt,
                           const CoarseLev<T> &L, const int32_t *coff, double *work, T *Ainv,
                           cudaStream_t s) {
  note_launch();
  k_coarsest_setup<T><<<1, 256, 0, s>>>(level, tab, policy, dt, L, coff, work, Ainv);
}
template void launch_coarsest_setup<double>(int, const FineTab &, const uint8_t *, double,
                                            const CoarseLev<double> &, const int32_t *, double *,
                                            double *, cudaStream_t);
template void launch_coarsest_setup<float>(int, const FineTab &, const uint8_t *, float,
                                           const CoarseLev<float> &, const int32_t *, double *,
                                           float *, cudaStream_t);

template <typename T>
__global__ void k_coarsest_apply(const T *__restrict__ Ainv, int n, const T *__restrict__ b,
                                 T *__restrict__ x, int trans) {
  const int m = n - 2, N = m * m;
  const size_t rs = trans ? 1 : size_t(N), cs = trans ? size_t(N) : 1;
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    T acc = T(0);
    for (int c = 0; c < N; ++c) acc = fma(Ainv[r * rs + c * cs], b[(1 + c / m) * n + 1 + c % m], acc);
    x[(1 + r / m) * n + 1 + r % m] = acc;
  }
}

template <typename T>
void launch_coarsest_apply(const T *Ainv, int n, const T *b, T *x, cudaStream_t s, int trans) {
  note_launch();
  k_coarsest_apply<T><<<1, 256, 0, s>>>(Ainv, n, b, x, trans);
}
template void launch_coarsest_apply<double>(const double *, int, const double *, double *, cudaStream_t, int);
template void launch_coarsest_apply<float>(const float *, int, const float *, float *, cudaStream_t, int);

// ----------------------------------------------------------------------------- attributes
template <typename T>
static cudaError_t prepare_coarse_T() {
  const void *fs[] = {reinterpret_cast<const void *>(k_rap_explicit<T>),
                      reinterpret_cast<const void *>(k_rap_explicit_dev<T>),
                      reinterpret_cast<const void *>(k_coarse_op<T, OP_APPLY, 0>),
                      reinterpret_cast<const void *>(k_coarse_op<T, OP_RESID, 0>),
                      reinterpret_cast<const void *>(k_coarse_op<T, OP_JACOBI, 0>),
                      reinterpret_cast<const void *>(k_coarse_op<T, OP_JACOBI0, 0>),
                      reinterpret_cast<const void *>(k_coarse_op<T, OP_APPLY, 1>),
                      reinterpret_cast<const void *>(k_coarse_op<T, OP_RESID, 1>),
                      reinterpret_cast<const void *>(k_coarse_op<T, OP_JACOBI, 1>),
#define SL_FUSED(TH) \
  reinterpret_cast<const void *>(k_coarse_down<T, TH, 0, 0>), \
  reinterpret_cast<const void *>(k_coarse_down<T, TH, 0, 1>), \
  reinterpret_cast<const void *>(k_coarse_down<T, TH, 1, 0>), \
  reinterpret_cast<const void *>(k_coarse_down<T, TH, 1, 1>), \
  reinterpret_cast<const void *>(k_coarse_up<T, TH, 0>), reinterpret_cast<const void *>(k_coarse_up<T, TH, 1>)
                      SL_FUSED(4), SL_FUSED(8), SL_FUSED(16), SL_FUSED(32),
                      reinterpret_cast<const void *>(k_vcycle_tail_smem<T>)};
#undef SL_FUSED
  for (const void *f : fs) {
    cudaError_t e = allow_dynamic_smem(f);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t prepare_coarse_kernels() {
  cudaError_t e = prepare_coarse_T<double>();
  return e != cudaSuccess ? e : prepare_coarse_T<float>();
}

}  // namespace sl
