// sl_krylov.cu - BiCGSTAB vector updates with fused dot products (van der Vorst's method,
// right preconditioning), conversions and norms.
//
// Every reduction writes one FP64 partial per block; the last block to finish (atomic ticket)
// adds the partials in block order, so results do not depend on scheduling, and then updates
// the scalars of the iteration in device memory (alpha, omega, rho), so that the host reads
// only the residual norm once per iteration.
#include <atomic>
#include <cmath>
#include <mutex>
#include <set>
#include <utility>

#include "sl_launch.h"

namespace sl {

constexpr int kVecThreads = 256;
// The grid-stride loops below take kU consecutive strides per pass and issue all of their
// loads before any arithmetic or store: a loop that computed and stored each element before
// loading the next made every load wait for the one before it (instructions issue in order).
// A thread still visits its elements in the same order, so every sum is unchanged.
constexpr int kU = 4;

static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;  // this host thread's launches (graph captures)
void note_launch(int n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  t_launches += n;
}
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
long long thread_launch_count() { return t_launches; }

cudaError_t allow_dynamic_smem(const void *func) {
  static std::mutex mu;
  static std::set<std::pair<const void *, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({func, dev})) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa{};
  e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - int(fa.sharedSizeBytes));
  if (e == cudaSuccess) done.insert({func, dev});
  return e;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of NF values in a fixed order; returns the sums in thread 0.
template <int NF>
__device__ __forceinline__ void block_sum(double (&v)[NF]) {
  __shared__ double sh[NF][kVecThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();  // sh may still be read by thread 0 from a previous call
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    v[f] = warp_sum(v[f]);
    if (lane == 0) sh[f][wid] = v[f];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      double s = 0.0;
      for (int w = 0; w < kVecThreads / 32; ++w) s += sh[f][w];
      v[f] = s;
    }
  }
}

__device__ void apply_post(int post, const double *tot, BicgScalars *S) {
  bool bad = false;
  switch (post) {
    case POST_RHO_INIT:
      S->rho = tot[0];
      S->rr = tot[1];
      S->rho_old = 1.0;
      S->alpha = 1.0;
      S->omega = 1.0;
      S->breakdown = 0;
      S->nonfinite = 0;
      S->first = 1;
      bad = !isfinite(tot[0]) || !isfinite(tot[1]);
      break;
    case POST_ALPHA:
      S->first = 0;
      S->rv = tot[0];
      bad = !isfinite(tot[0]);
      if (tot[0] == 0.0 || fabs(S->rho) < 1e-300) {
        S->breakdown = 1;
        S->alpha = 0.0;
      } else {
        S->alpha = S->rho / tot[0];
      }
      break;
    case POST_SS:
      S->ss = tot[0];
      bad = !isfinite(tot[0]);
      break;
    case POST_OMEGA:
      S->ts = tot[0];
      S->tt = tot[1];
      bad = !isfinite(tot[0]) || !isfinite(tot[1]);
      if (S->ss <= S->tol2) S->omega = 0.0;          // s already small: x += alpha p^, r = s
      else if (tot[1] == 0.0) { S->omega = 0.0; S->breakdown = 1; }
      else S->omega = tot[0] / tot[1];
      break;
    case POST_RHO:
      S->rho_old = S->rho;
      S->rho = tot[0];
      S->rr = tot[1];
      bad = !isfinite(tot[0]) || !isfinite(tot[1]);
      if (S->omega == 0.0 && S->ss > S->tol2) S->breakdown = 1;
      if (S->inject_bd > 0 && --S->inject_bd == 0) S->breakdown = 1;
      break;
    case POST_BNORM:
      S->bnorm2 = tot[0];
      S->tol2 = S->tolrel2 * tot[0];
      bad = !isfinite(tot[0]);
      break;
    case POST_RR:
      S->rr = tot[0];
      bad = !isfinite(tot[0]);
      break;
  }
  if (bad) S->nonfinite = 1;
}

// Each block writes its partial sums; the last block to arrive adds all partials with all of
// its threads (thread t takes blocks t, t + 256, ... in order, then a fixed-order tree), so
// the totals do not depend on which block finishes last.
template <int NF>
__device__ void finish(double (&v)[NF], int post, BicgScalars *S, double *partials,
                       unsigned *counter) {
  block_sum<NF>(v);
  __shared__ bool last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int f = 0; f < NF; ++f) partials[blockIdx.x * NF + f] = v[f];
    __threadfence();
    const unsigned ticket = atomicAdd(counter, 1u);
    last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double tot[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) tot[f] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
    for (int f = 0; f < NF; ++f) tot[f] += ((volatile double *)partials)[b * NF + f];
  block_sum<NF>(tot);
  if (threadIdx.x == 0) {
    apply_post(post, tot, S);
    *counter = 0u;
  }
}

// (a, b) and optionally (c, d)
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_dot2(const T *__restrict__ a, const T *__restrict__ b,
                                                      const T *__restrict__ c, const T *__restrict__ d,
                                                      size_t N, int post, BicgScalars *S,
                                                      double *partials, unsigned *counter) {
  double v[2] = {0.0, 0.0};
  T s0 = T(0), s1 = T(0);
  const size_t st = size_t(gridDim.x) * blockDim.x;
  for (size_t i0 = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i0 < N; i0 += kU * st) {
    T av[kU], bv[kU], cv[kU], dv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = i0 + u * st;
      av[u] = i < N ? a[i] : T(0);
      bv[u] = i < N ? b[i] : T(0);
      cv[u] = (c && i < N) ? c[i] : T(0);
      dv[u] = (c && i < N) ? d[i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      if (i0 + u * st < N) {
        s0 = fma(av[u], bv[u], s0);
        if (c) s1 = fma(cv[u], dv[u], s1);
      }
    }
  }
  v[0] = double(s0);
  v[1] = double(s1);
  finish<2>(v, post, S, partials, counter);
}

template <typename T>
void launch_dot2(const T *a, const T *b, const T *c, const T *d, size_t N, int post,
                 BicgScalars *S, double *partials, unsigned *counter, cudaStream_t s) {
  note_launch();
  k_dot2<T><<<kRedBlocks, kVecThreads, 0, s>>>(a, b, c, d, N, post, S, partials, counter);
}

// p = r + beta (p - omega v), beta = (rho / rho_old) (alpha / omega); first iteration p = r
// (the device flag S->first, so that one captured iteration serves every iteration).
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_bicg_p(T *__restrict__ p, const T *__restrict__ r,
                                                        const T *__restrict__ v, size_t N, int first_host,
                                                        const BicgScalars *S) {
  const int first = first_host || S->first;
  const double beta_d = first ? 0.0 : (S->rho / S->rho_old) * (S->alpha / S->omega);
  const T beta = T(beta_d), om = T(S->omega);
  const size_t st = size_t(gridDim.x) * blockDim.x;
  for (size_t i0 = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i0 < N; i0 += kU * st) {
    T rv[kU], pv[kU], vv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = i0 + u * st;
      rv[u] = i < N ? r[i] : T(0);
      pv[u] = (!first && i < N) ? p[i] : T(0);
      vv[u] = (!first && i < N) ? v[i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = i0 + u * st;
      if (i < N) p[i] = first ? rv[u] : rv[u] + beta * (pv[u] - om * vv[u]);
    }
  }
}

template <typename T>
void launch_bicg_p(T *p, const T *r, const T *v, size_t N, int first, const BicgScalars *S,
                   cudaStream_t s) {
  note_launch();
  k_bicg_p<T><<<kRedBlocks, kVecThreads, 0, s>>>(p, r, v, N, first, S);
}

// s = r - alpha v, (s, s)
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_bicg_s(T *__restrict__ sv, const T *__restrict__ r,
                                                        const T *__restrict__ v, size_t N, BicgScalars *S,
                                                        double *partials, unsigned *counter) {
  const T alpha = T(S->alpha);
  T acc = T(0);
  const size_t st = size_t(gridDim.x) * blockDim.x;
  for (size_t i0 = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i0 < N; i0 += kU * st) {
    T rv[kU], vv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = i0 + u * st;
      rv[u] = i < N ? r[i] : T(0);
      vv[u] = i < N ? v[i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = i0 + u * st;
      if (i < N) {
        const T si = rv[u] - alpha * vv[u];
        sv[i] = si;
        acc = fma(si, si, acc);
      }
    }
  }
  double vv[1] = {double(acc)};
  finish<1>(vv, POST_SS, S, partials, counter);
}

template <typename T>
void launch_bicg_s(T *sv, const T *r, const T *v, size_t N, BicgScalars *S, double *partials,
                   unsigned *counter, cudaStream_t s) {
  note_launch();
  k_bicg_s<T><<<kRedBlocks, kVecThreads, 0, s>>>(sv, r, v, N, S, partials, counter);
}

// x += alpha p^ + omega s^ ; r = s - omega t ; (r^, r), (r, r)
template <typename T, typename TX>
__global__ void __launch_bounds__(kVecThreads) k_bicg_xr(TX *__restrict__ x, const T *__restrict__ phat,
                                                         const T *__restrict__ shat, const T *__restrict__ sv,
                                                         const T *__restrict__ t, T *__restrict__ r,
                                                         const T *__restrict__ rhat, size_t N,
                                                         BicgScalars *S, double *partials,
                                                         unsigned *counter) {
  const double alpha = S->alpha, omega = S->omega;
  const T om = T(omega);
  T a0 = T(0), a1 = T(0);
  const size_t st = size_t(gridDim.x) * blockDim.x;
  for (size_t i0 = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i0 < N; i0 += kU * st) {
    TX xv[kU];
    T pv[kU], shv[kU], svv[kU], tv[kU], rhv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = i0 + u * st;
      const bool in = i < N;
      xv[u] = in ? x[i] : TX(0);
      pv[u] = in ? phat[i] : T(0);
      shv[u] = in ? shat[i] : T(0);
      svv[u] = in ? sv[i] : T(0);
      tv[u] = in ? t[i] : T(0);
      rhv[u] = in ? rhat[i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = i0 + u * st;
      if (i < N) {
        x[i] = xv[u] + TX(alpha) * TX(pv[u]) + TX(omega) * TX(shv[u]);
        const T ri = svv[u] - om * tv[u];
        r[i] = ri;
        a0 = fma(rhv[u], ri, a0);
        a1 = fma(ri, ri, a1);
      }
    }
  }
  double vv[2] = {double(a0), double(a1)};
  finish<2>(vv, POST_RHO, S, partials, counter);
}

template <typename T, typename TX>
void launch_bicg_xr(TX *x, const T *phat, const T *shat, const T *sv, const T *t, T *r,
                    const T *rhat, size_t N, BicgScalars *S, double *partials, unsigned *counter,
                    cudaStream_t s) {
  note_launch();
  k_bicg_xr<T, TX><<<kRedBlocks, kVecThreads, 0, s>>>(x, phat, shat, sv, t, r, rhat, N, S, partials,
                                                      counter);
}

__global__ void k_init_scalars(BicgScalars *S, double tolrel2) {
  BicgScalars z = {};
  z.rho_old = 1.0;
  z.alpha = 1.0;
  z.omega = 1.0;
  z.tolrel2 = tolrel2;
  z.inject_bd = S->inject_bd;
  *S = z;
}
void launch_init_scalars(BicgScalars *S, double tolrel2, cudaStream_t s) {
  note_launch();
  k_init_scalars<<<1, 1, 0, s>>>(S, tolrel2);
}

// k_init_scalars keeping the right-hand side's norms (||b||^2, ||b||_inf) of the solve: a
// refinement round's right-hand side is the same as the previous round's.
__global__ void k_init_scalars_keep_b(BicgScalars *S, double tolrel2) {
  BicgScalars z = {};
  z.rho_old = 1.0;
  z.alpha = 1.0;
  z.omega = 1.0;
  z.tolrel2 = tolrel2;
  z.bnorm2 = S->bnorm2;
  z.bmax = S->bmax;
  z.tol2 = tolrel2 * z.bnorm2;
  z.inject_bd = S->inject_bd;
  *S = z;
}
void launch_init_scalars_keep_b(BicgScalars *S, double tolrel2, cudaStream_t s) {
  note_launch();
  k_init_scalars_keep_b<<<1, 1, 0, s>>>(S, tolrel2);
}

template <typename T>
__global__ void k_fill(T *x, size_t N, T v) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < N; i += size_t(gridDim.x) * blockDim.x)
    x[i] = v;
}
template <typename T>
void launch_fill(T *x, size_t N, T v, cudaStream_t s) {
  note_launch();
  k_fill<T><<<kRedBlocks, kVecThreads, 0, s>>>(x, N, v);
}

template <typename Tin, typename Tout>
__global__ void k_convert(const Tin *__restrict__ x, Tout *__restrict__ y, size_t N, const int *flag) {
  if (flag && *flag == 0) return;  // the caller's device-side condition is off
  const size_t st = size_t(gridDim.x) * blockDim.x;
  for (size_t i0 = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i0 < N; i0 += kU * st) {
    Tin v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) v[u] = i0 + u * st < N ? x[i0 + u * st] : Tin(0);
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + u * st < N) y[i0 + u * st] = Tout(v[u]);
  }
}
template <typename Tin, typename Tout>
void launch_convert(const Tin *x, Tout *y, size_t N, cudaStream_t s, const int *flag) {
  note_launch();
  k_convert<Tin, Tout><<<kRedBlocks, kVecThreads, 0, s>>>(x, y, N, flag);
}

// X = 2 U - V on interior nodes (boundary of X untouched).
__global__ void k_extrapolate(double *__restrict__ X, const double *__restrict__ U,
                              const double *__restrict__ V, int n) {
  const size_t N = size_t(n) * n;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < N; i += size_t(gridDim.x) * blockDim.x) {
    const int i1 = int(i % n), i2 = int(i / n);
    if (i1 == 0 || i2 == 0 || i1 == n - 1 || i2 == n - 1) continue;
    X[i] = 2.0 * U[i] - V[i];
  }
}
void launch_extrapolate(double *X, const double *U, const double *V, int n, cudaStream_t s) {
  note_launch();
  k_extrapolate<<<kRedBlocks, kVecThreads, 0, s>>>(X, U, V, n);
}

__global__ void k_add_f32(double *__restrict__ x, const float *__restrict__ e, size_t N) {
  const size_t st = size_t(gridDim.x) * blockDim.x;
  for (size_t i0 = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i0 < N; i0 += kU * st) {
    double xv[kU];
    float ev[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      xv[u] = i0 + u * st < N ? x[i0 + u * st] : 0.0;
      ev[u] = i0 + u * st < N ? e[i0 + u * st] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + u * st < N) x[i0 + u * st] = xv[u] + double(ev[u]);
  }
}
void launch_add_f32_to_f64(double *x, const float *e, size_t N, cudaStream_t s) {
  note_launch();
  k_add_f32<<<kRedBlocks, kVecThreads, 0, s>>>(x, e, N);
}

// Sum of squares and max-abs of one vector: which = 0 stores (||b||^2, ||b||_inf) and the
// stop threshold; which = 1 stores (||r||^2, ||r||_inf).
// |a| as an ordered integer: the bit pattern with the sign cleared.  For non-NaN doubles the
// order of these integers is the order of the magnitudes, so their maximum is the bit pattern of
// max |a|; every NaN pattern lies above that of infinity.  The maxima below run on the integer
// pipe: fabs and fmax on doubles would take the narrow FP64 pipe beside the one FMA per value.
constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;
__device__ __forceinline__ unsigned long long abs_bits(double a) {
  return static_cast<unsigned long long>(__double_as_longlong(a)) & 0x7fffffffffffffffull;
}

__global__ void __launch_bounds__(kVecThreads) k_norms(const double *__restrict__ a, size_t N, int which,
                                                       BicgScalars *S, double *partials,
                                                       unsigned *counter) {
  double s2 = 0.0;
  unsigned long long mb = 0;
  const size_t st = size_t(gridDim.x) * blockDim.x;
  if (which == 1) {
    // The residual: its squares in FP32, each value turned into FP32 by integer operations
    // (its exponent moved by -e_b, e_b the exponent of ||b||_inf from the solve's first call,
    // the mantissa truncated to 24 bits) so that nothing of this loop runs on the narrow FP64
    // pipe; relative to ||b|| the scaled values neither overflow nor underflow FP32 in any
    // residual that the stop test can accept, and the 2^-23 truncation is far inside the test's
    // needs.  The sum is scaled back in FP64 per thread.
    const int eb = int((__double_as_longlong(S->bmax) >> 52) & 0x7ff);
    const int shift = eb > 0 ? 1023 - eb : 0;  // exponent offset that brings ||b||_inf to about 1
    float s2f = 0.f;
    for (size_t i0 = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i0 < N; i0 += kU * st) {
      double av[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) av[u] = i0 + u * st < N ? a[i0 + u * st] : 0.0;
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        if (i0 + u * st < N) {
          const unsigned long long b = abs_bits(av[u]);
          mb = max(mb, b);
          const int e = int(b >> 52) + shift - 1023 + 127;  // FP32 biased exponent of the scaled value
          const unsigned fb = e <= 0 ? 0u : (e >= 255 ? 0x7f7fffffu
                                                       : (unsigned(e) << 23) | unsigned((b >> 29) & 0x7fffffull));
          const float f = __uint_as_float(fb);
          s2f = fmaf(f, f, s2f);
        }
      }
    }
    s2 = double(s2f) * exp2(-2.0 * shift);
  } else {
    for (size_t i0 = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i0 < N; i0 += kU * st) {
      double av[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) av[u] = i0 + u * st < N ? a[i0 + u * st] : 0.0;
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        if (i0 + u * st < N) {
          s2 = fma(av[u], av[u], s2);
          mb = max(mb, abs_bits(av[u]));
        }
      }
    }
  }
  // max |a|, or infinity when a NaN was seen
  double mx = mb > kInfBits ? INFINITY : __longlong_as_double(static_cast<long long>(mb));
  s2 = warp_sum(s2);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ double ss[kVecThreads / 32], sm[kVecThreads / 32];
  __shared__ bool last;
  if ((threadIdx.x & 31) == 0) { ss[threadIdx.x >> 5] = s2; sm[threadIdx.x >> 5] = mx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    s2 = 0.0;
    for (int w = 0; w < kVecThreads / 32; ++w) { s2 += ss[w]; mx = fmax(mx, sm[w]); }
    partials[2 * blockIdx.x] = s2;
    partials[2 * blockIdx.x + 1] = mx;
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double T2 = 0.0, M = 0.0;
  for (unsigned b2 = threadIdx.x; b2 < gridDim.x; b2 += blockDim.x) {
    T2 += ((volatile double *)partials)[2 * b2];
    M = fmax(M, ((volatile double *)partials)[2 * b2 + 1]);
  }
  __syncthreads();
  T2 = warp_sum(T2);
  for (int o = 16; o > 0; o >>= 1) M = fmax(M, __shfl_xor_sync(0xffffffffu, M, o));
  if ((threadIdx.x & 31) == 0) { ss[threadIdx.x >> 5] = T2; sm[threadIdx.x >> 5] = M; }
  __syncthreads();
  if (threadIdx.x == 0) {
    T2 = 0.0;
    M = 0.0;
    for (int w = 0; w < kVecThreads / 32; ++w) { T2 += ss[w]; M = fmax(M, sm[w]); }
    if (which == 0) {
      S->bnorm2 = T2;
      S->bmax = M;
      S->tol2 = S->tolrel2 * T2;
    } else {
      S->rr = T2;
      S->rmax = M;
    }
    if (!isfinite(T2) || !isfinite(M)) S->nonfinite = 1;
    *counter = 0u;
  }
}
void launch_norms(const double *a, size_t N, int which, BicgScalars *S, double *partials,
                  unsigned *counter, cudaStream_t s) {
  note_launch();
  k_norms<<<kRedBlocks, kVecThreads, 0, s>>>(a, N, which, S, partials, counter);
}

// out[0] = max_j |a_j - b_j| over interior nodes, out[1] = max_j |a_j| (Howard stop test).
__global__ void __launch_bounds__(kVecThreads) k_maxabs_diff(const double *__restrict__ a,
                                                             const double *__restrict__ b, int n,
                                                             double *out, unsigned *counter,
                                                             double *partials) {
  // maxima as ordered bit patterns (abs_bits): a NaN difference or value is skipped, as fmax
  // skips it, and a NaN in a sets d to infinity
  unsigned long long db = 0, xb = 0;
  bool a_nan = false;
  const size_t N = size_t(n) * n;  // < 2^31 (sl_hjb_create limits n)
  const size_t st = size_t(gridDim.x) * blockDim.x;
  for (size_t i0 = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i0 < N; i0 += kU * st) {
    double av[kU], bv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = i0 + u * st;
      av[u] = i < N ? a[i] : 0.0;
      bv[u] = i < N ? b[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = i0 + u * st;
      if (i >= N) continue;
      const unsigned i2 = unsigned(i) / unsigned(n), i1 = unsigned(i) - i2 * unsigned(n);
      if (i1 == 0 || i2 == 0 || i1 == unsigned(n) - 1 || i2 == unsigned(n) - 1) continue;
      const unsigned long long dd = abs_bits(av[u] - bv[u]), aa = abs_bits(av[u]);
      if (dd <= kInfBits) db = max(db, dd);
      if (aa <= kInfBits) xb = max(xb, aa);
      else a_nan = true;
    }
  }
  double d = a_nan ? INFINITY : __longlong_as_double(static_cast<long long>(db));
  double x = __longlong_as_double(static_cast<long long>(xb));
  for (int o = 16; o > 0; o >>= 1) {
    d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
    x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  }
  __shared__ double sd[kVecThreads / 32], sx[kVecThreads / 32];
  __shared__ bool last;
  if ((threadIdx.x & 31) == 0) { sd[threadIdx.x >> 5] = d; sx[threadIdx.x >> 5] = x; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 0; w < kVecThreads / 32; ++w) { d = fmax(d, sd[w]); x = fmax(x, sx[w]); }
    partials[2 * blockIdx.x] = d;
    partials[2 * blockIdx.x + 1] = x;
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double D = 0.0, Xm = 0.0;
  for (unsigned b2 = threadIdx.x; b2 < gridDim.x; b2 += blockDim.x) {
    D = fmax(D, ((volatile double *)partials)[2 * b2]);
    Xm = fmax(Xm, ((volatile double *)partials)[2 * b2 + 1]);
  }
  __syncthreads();
  for (int o = 16; o > 0; o >>= 1) {
    D = fmax(D, __shfl_xor_sync(0xffffffffu, D, o));
    Xm = fmax(Xm, __shfl_xor_sync(0xffffffffu, Xm, o));
  }
  if ((threadIdx.x & 31) == 0) { sd[threadIdx.x >> 5] = D; sx[threadIdx.x >> 5] = Xm; }
  __syncthreads();
  if (threadIdx.x == 0) {
    D = 0.0;
    Xm = 0.0;
    for (int w = 0; w < kVecThreads / 32; ++w) { D = fmax(D, sd[w]); Xm = fmax(Xm, sx[w]); }
    out[0] = D;
    out[1] = Xm;
    *counter = 0u;
  }
}
void launch_maxabs_diff(const double *a, const double *b, int n, double *out2, unsigned *counter,
                        double *partials, cudaStream_t s) {
  note_launch();
  k_maxabs_diff<<<kRedBlocks, kVecThreads, 0, s>>>(a, b, n, out2, counter, partials);
}

#define SL_INST(T)                                                                                 \
  template void launch_dot2<T>(const T *, const T *, const T *, const T *, size_t, int,            \
                               BicgScalars *, double *, unsigned *, cudaStream_t);                 \
  template void launch_bicg_p<T>(T *, const T *, const T *, size_t, int, const BicgScalars *,      \
                                 cudaStream_t);                                                    \
  template void launch_bicg_s<T>(T *, const T *, const T *, size_t, BicgScalars *, double *,       \
                                 unsigned *, cudaStream_t);                                        \
  template void launch_fill<T>(T *, size_t, T, cudaStream_t);
SL_INST(double)
SL_INST(float)
template void launch_bicg_xr<double, double>(double *, const double *, const double *, const double *,
                                             const double *, double *, const double *, size_t,
                                             BicgScalars *, double *, unsigned *, cudaStream_t);
template void launch_bicg_xr<float, float>(float *, const float *, const float *, const float *,
                                           const float *, float *, const float *, size_t,
                                           BicgScalars *, double *, unsigned *, cudaStream_t);
template void launch_convert<double, float>(const double *, float *, size_t, cudaStream_t, const int *);
template void launch_convert<float, double>(const float *, double *, size_t, cudaStream_t, const int *);
template void launch_fill<int32_t>(int32_t *, size_t, int32_t, cudaStream_t);

}  // namespace sl
