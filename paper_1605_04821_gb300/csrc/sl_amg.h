// sl_amg.h - aggregation-based AMG with a K-cycle on compact CSR levels (host interface of
// sl_amg.cu).  Level 0 is the step matrix over the interior unknowns; every coarser level is
// the Galerkin product P^T A P of two passes of pairwise matching (aggregates of at most four
// unknowns).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "sl_launch.h"

namespace sl {

constexpr int kAmgMaxLevels = 16;
constexpr int kAmgRounds = 8;      // matching rounds per pass
constexpr int kAmgRowMax = 128;    // rows up to this length are sorted in registers, longer ones in place
constexpr int kAmgCoarsest = 256;  // dense solve at or below this many unknowns
constexpr double kAmgMinReduction = 0.75;  // a level keeps at most this fraction of the unknowns above
constexpr int kAmgCoarseSweeps = 16;        // Jacobi sweeps on a last level above kAmgCoarsest

enum AmgVec { AV_X = 0, AV_B, AV_R, AV_T, AV_V1, AV_W1, AV_V2, AV_W2, AV_E, AV_R2, AV_COUNT };

struct AmgLevel {
  int n = 0;
  long long nnz = 0;
  int32_t *rowptr = nullptr, *col = nullptr;
  double *v64 = nullptr, *d64 = nullptr;
  float *v32 = nullptr, *d32 = nullptr;
  int32_t *agg = nullptr;   // [n]: unknown of level l+1 that holds unknown i (levels < L-1)
  int32_t *mem = nullptr;   // [4 n_{l+1}]: members of each level-(l+1) unknown, ascending, -1 padded
  size_t cap_n = 0, cap_nnz = 0, cap_mem = 0, cap_rp = 0, cap_agg = 0;  // d / col,v64,v32 / mem / rowptr / agg
  double *vec64[AV_COUNT] = {};
  float *vec32[AV_COUNT] = {};
  size_t cap_vec = 0;
  double *scal = nullptr;   // GCR scalars of this level: [0] w1.r [1] w1.w1 [2] w2.w1 [3] w2.r2 [4] w2.w2
};

struct AmgEngine {
  int L = 0;
  bool dense_coarsest = true;  // false: the last level is solved by kAmgCoarseSweeps Jacobi sweeps
  AmgLevel lev[kAmgMaxLevels];
  int k_levels = 2, nu1 = 1, nu2 = 1;
  double omega = 0.8;
  // setup scratch (sized for the finest level)
  size_t cap_n = 0, cap_nnz = 0;
  double *s = nullptr, *smax = nullptr;
  int *partner = nullptr, *prop = nullptr, *flag = nullptr, *scan = nullptr, *cnt = nullptr;
  int32_t *ids = nullptr, *a1 = nullptr, *mem1 = nullptr, *mem2 = nullptr, *err = nullptr;
  int32_t *t_rowptr = nullptr, *t_col = nullptr;  // pass-1 coarse matrix
  double *t_v = nullptr;
  int32_t *rpT = nullptr, *colT = nullptr, *rpS = nullptr, *colS = nullptr;  // A^T; strength pattern
  double *vT = nullptr;
  int32_t *rawptr = nullptr, *rawcol = nullptr;  // Galerkin: unmerged entries of every coarse row
  double *rawval = nullptr;
  double *Ainv64 = nullptr, *work = nullptr, *partials = nullptr;
  float *Ainv32 = nullptr;
  int *h_int = nullptr;  // pinned
  std::vector<void *> allocs;
  std::string err_msg;
};

// Builds every level from lev[0] (n, nnz, rowptr, col, v64 on the device: sorted columns, no
// duplicates).  Returns cudaSuccess or the failing call's error; err_msg says which step failed
// on a non-CUDA failure (then cudaErrorInvalidValue).
cudaError_t amg_setup(AmgEngine &E, cudaStream_t s);
// Level 0 storage for n unknowns and nnz entries (grows only).
cudaError_t amg_reserve_level0(AmgEngine &E, int n, long long nnz);
// Level 0 from the fine stencil tables: row I = interior node, diagonal 1 + dt (W - c - w_self),
// off-diagonal -dt w at interior targets, columns sorted, equal columns merged.
cudaError_t amg_level0_from_tables(AmgEngine &E, const FineTab &tab, const int32_t *off,
                                   const uint8_t *policy, double dt, cudaStream_t s);
// x = K-cycle(b) on level 0 (compact vectors of lev[0].n entries).  Stream-ordered, no host
// synchronisation (capturable in a CUDA graph).
template <typename T>
void amg_cycle(AmgEngine &E, const T *b, T *x, cudaStream_t s);
// Gather / scatter between full-grid vectors (n x n, zero boundary) and compact interior ones.
template <typename T>
void amg_full_to_compact(int n, const T *full, T *compact, cudaStream_t s);
template <typename T>
void amg_compact_to_full(int n, const T *compact, T *full, cudaStream_t s);
void amg_free(AmgEngine &E);

}  // namespace sl
