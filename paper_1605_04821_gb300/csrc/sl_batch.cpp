// sl_batch.cpp - many independent HJB solves on one GPU.
//
// Instances are independent, so the batch needs no device-side exchange.  A host scheduler
// assigns them to worker threads by the longest-processing-time-first rule (LPT: sort by
// estimated cost, give each to the least-loaded worker), and every worker drives its own
// handles on its own CUDA stream.  The kernels of different instances then run concurrently
// on the device, which keeps the SMs busy even when one instance's grid is far too small to
// fill them, and every instance's own launch sequence stays exactly that of a single solve.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sl_hjb.h"

struct sl_batch {
  int device = 0;
  std::vector<sl_instance> inst;
  std::vector<sl_hjb *> handles;
  std::vector<std::vector<int>> queue;  // per worker: instance indices, in order
  std::vector<cudaStream_t> streams;
  std::string err;
};

namespace {

double instance_cost(const sl_instance &in) {
  // nodes x steps x (one argmin sweep over K controls + about 32 operator applications)
  const double nodes = double(in.grid.nx) * double(in.grid.ny);
  return nodes * std::max(1, in.n_steps) * (double(in.ctrl.K) + 32.0);
}

}  // namespace

extern "C" {

int sl_batch_plan(int n_items, const double *cost, int n_bins, int *bin_of) {
  if (n_items < 0 || n_bins < 1 || (n_items > 0 && (!cost || !bin_of))) return SL_EINVAL;
  std::vector<int> order(n_items);
  std::iota(order.begin(), order.end(), 0);
  // decreasing cost; equal costs keep their index order, so the plan is deterministic
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<double> load(n_bins, 0.0);
  for (int i : order) {
    int best = 0;
    for (int w = 1; w < n_bins; ++w)
      if (load[w] < load[best]) best = w;
    bin_of[i] = best;
    load[best] += cost[i];
  }
  return SL_OK;
}

sl_status sl_batch_create(sl_batch **out, int n_inst, const sl_instance *inst, const sl_opts *opts,
                          int n_workers) {
  if (!out) return SL_EINVAL;
  *out = nullptr;
  if (n_inst < 1 || !inst || n_workers < 1) return SL_EINVAL;
  for (int i = 0; i < n_inst; ++i)
    if (!inst[i].u_dev || inst[i].n_steps < 1 || !(inst[i].T > 0)) return SL_EINVAL;
  sl_batch *b = new (std::nothrow) sl_batch();
  if (!b) return SL_ENOMEM;
  cudaGetDevice(&b->device);
  b->inst.assign(inst, inst + n_inst);
  const int W = std::min(n_workers, n_inst);
  std::vector<double> cost(n_inst);
  for (int i = 0; i < n_inst; ++i) cost[i] = instance_cost(inst[i]);
  std::vector<int> bin(n_inst, 0);
  sl_batch_plan(n_inst, cost.data(), W, bin.data());
  b->queue.assign(W, {});
  // within a worker, largest first (the order in which LPT assigned them)
  std::vector<int> order(n_inst);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  for (int i : order) b->queue[bin[i]].push_back(i);
  b->streams.assign(W, nullptr);
  b->handles.assign(n_inst, nullptr);
  for (int w = 0; w < W; ++w) {
    if (cudaStreamCreateWithFlags(&b->streams[w], cudaStreamNonBlocking) != cudaSuccess) {
      sl_batch_destroy(b);
      return SL_ECUDA;
    }
  }
  // handles are created by their workers (the host-side table construction runs in parallel)
  std::vector<sl_status> st(n_inst, SL_OK);
  std::vector<std::thread> threads;
  for (int w = 0; w < W; ++w)
    threads.emplace_back([&, w]() {
      cudaSetDevice(b->device);
      for (int i : b->queue[w]) {
        const sl_instance &in = b->inst[i];
        st[i] = sl_hjb_create(&b->handles[i], &in.grid, &in.ctrl, &in.src, opts, b->streams[w]);
      }
    });
  for (auto &t : threads) t.join();
  for (int i = 0; i < n_inst; ++i)
    if (st[i] != SL_OK) {
      b->err = "sl_hjb_create failed for instance " + std::to_string(i);
      sl_status r = st[i];
      sl_batch_destroy(b);
      return r;
    }
  *out = b;
  return SL_OK;
}

sl_status sl_batch_run(sl_batch *b, sl_status *status_out, sl_stats *stats_out) {
  if (!b) return SL_EINVAL;
  const int n = int(b->inst.size()), W = int(b->queue.size());
  std::vector<sl_status> st(n, SL_OK);
  std::vector<std::thread> threads;
  for (int w = 0; w < W; ++w)
    threads.emplace_back([&, w]() {
      cudaSetDevice(b->device);
      for (int i : b->queue[w]) {
        const sl_instance &in = b->inst[i];
        sl_hjb_reset(b->handles[i]);
        st[i] = sl_hjb_solve(b->handles[i], in.u_dev, in.t0, in.T, in.n_steps, nullptr,
                             stats_out ? stats_out + i : nullptr, b->streams[w]);
      }
      cudaStreamSynchronize(b->streams[w]);
    });
  for (auto &t : threads) t.join();
  sl_status first = SL_OK;
  for (int i = 0; i < n; ++i) {
    if (status_out) status_out[i] = st[i];
    if (st[i] != SL_OK && first == SL_OK) {
      first = st[i];
      b->err = "instance " + std::to_string(i) + ": " + sl_hjb_last_error(b->handles[i]);
    }
  }
  return first;
}

int sl_batch_worker_of(const sl_batch *b, int i) {
  if (!b || i < 0 || i >= int(b->inst.size())) return -1;
  for (size_t w = 0; w < b->queue.size(); ++w)
    for (int j : b->queue[w])
      if (j == i) return int(w);
  return -1;
}

const char *sl_batch_last_error(const sl_batch *b) { return b ? b->err.c_str() : "null batch"; }

void sl_batch_destroy(sl_batch *b) {
  if (!b) return;
  for (sl_hjb *h : b->handles)
    if (h) sl_hjb_destroy(h);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  delete b;
}

}  // extern "C"
