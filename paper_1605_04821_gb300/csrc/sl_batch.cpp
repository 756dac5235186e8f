// sl_batch.cpp - many independent HJB solves on one GPU.
//
// Instances are independent, so the batch needs no device-side exchange.  A host scheduler
// assigns them to worker threads by the longest-processing-time-first rule (LPT: sort by
// estimated cost, give each to the least-loaded worker), and every worker drives its own
// handles on its own CUDA stream.  The kernels of different instances then run concurrently
// on the device, which keeps the SMs busy even when one instance's grid is far too small to
// fill them, and every instance's own launch sequence stays exactly that of a single solve.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
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
  sl_opts opts{};
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
  if (opts) b->opts = *opts;
  else sl_opts_default(&b->opts);
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

sl_status sl_batch_autotune(sl_batch *b, int probe_steps, int max_tail_rows, sl_tune_choice *out,
                            int max_out, int *n_out) {
  if (!b || probe_steps < 1 || (max_out > 0 && !out)) return SL_EINVAL;
  const int n = int(b->inst.size()), W = int(b->queue.size());
  cudaSetDevice(b->device);
  // size classes and their share of the work
  std::map<int, std::vector<int>> cls;
  std::map<int, double> work;
  for (int i = 0; i < n; ++i) {
    cls[b->inst[i].grid.nx].push_back(i);
    work[b->inst[i].grid.nx] += instance_cost(b->inst[i]);
  }
  std::vector<int> sizes;
  for (auto &kv : cls) sizes.push_back(kv.first);
  std::stable_sort(sizes.begin(), sizes.end(), [&](int a, int c) { return work[a] > work[c]; });
  // state copies, restored before every probe and at the end
  std::vector<double *> saved(n, nullptr);
  auto release = [&]() {
    for (double *p : saved)
      if (p) cudaFree(p);
  };
  for (int i = 0; i < n; ++i) {
    const size_t bytes = size_t(b->inst[i].grid.nx) * b->inst[i].grid.ny * sizeof(double);
    if (cudaMalloc(&saved[i], bytes) != cudaSuccess ||
        cudaMemcpy(saved[i], b->inst[i].u_dev, bytes, cudaMemcpyDeviceToDevice) != cudaSuccess) {
      release();
      b->err = "sl_batch_autotune: no device memory for the state copies";
      return SL_ENOMEM;
    }
  }
  // one probe: restore + reset + one untimed step (graph captures) on every instance, then
  // probe_steps timed steps of every instance, all workers concurrently
  sl_status probe_st = SL_OK;
  auto run_phase = [&](bool timed) {
    std::vector<std::thread> threads;
    std::vector<sl_status> st(n, SL_OK);
    for (int w = 0; w < W; ++w)
      threads.emplace_back([&, w]() {
        cudaSetDevice(b->device);
        for (int i : b->queue[w]) {
          const sl_instance &in = b->inst[i];
          const double dt = in.T / in.n_steps;
          const size_t bytes = size_t(in.grid.nx) * in.grid.ny * sizeof(double);
          if (!timed) {
            cudaMemcpyAsync(in.u_dev, saved[i], bytes, cudaMemcpyDeviceToDevice, b->streams[w]);
            sl_hjb_reset(b->handles[i]);
            st[i] = sl_hjb_solve(b->handles[i], in.u_dev, in.t0, dt, 1, nullptr, nullptr, b->streams[w]);
          } else {
            st[i] = sl_hjb_solve(b->handles[i], in.u_dev, in.t0 + dt, probe_steps * dt, probe_steps, nullptr,
                                 nullptr, b->streams[w]);
          }
        }
        cudaStreamSynchronize(b->streams[w]);
      });
    for (auto &t : threads) t.join();
    for (int i = 0; i < n; ++i)
      if (st[i] != SL_OK && probe_st == SL_OK) probe_st = st[i];
  };
  auto probe = [&]() {
    run_phase(false);
    const auto t0 = std::chrono::steady_clock::now();
    run_phase(true);
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  };
  std::map<int, int> choice;
  for (int nx : sizes) choice[nx] = -1;  // the handles' own setting until tuned
  std::map<int, double> best_sec;
  for (int nx : sizes) {
    sl_hjb *h0 = b->handles[cls[nx][0]];
    // candidate tails: none, and the row count of each level that can start the tail
    std::vector<int> cand = {0};
    const int L = sl_hjb_num_levels(h0);
    for (int l = 1; l < L - 1; ++l) {
      int nl = 0;
      sl_hjb_level_info(h0, l, &nl, nullptr, nullptr);
      const int rows = (nl - 2) * (nl - 2);
      if (rows <= max_tail_rows) cand.push_back(rows);
    }
    double best = 1e300;
    int pick = cand[0];
    for (int c : cand) {
      for (int i : cls[nx]) sl_hjb_set_launch(b->handles[i], b->opts.use_graphs, c);
      const double sec = probe();
      if (probe_st != SL_OK) break;
      if (sec < best) {
        best = sec;
        pick = c;
      }
    }
    if (probe_st != SL_OK) break;
    choice[nx] = pick;
    best_sec[nx] = best;
    for (int i : cls[nx]) sl_hjb_set_launch(b->handles[i], b->opts.use_graphs, pick);
  }
  for (int i = 0; i < n; ++i) {
    const size_t bytes = size_t(b->inst[i].grid.nx) * b->inst[i].grid.ny * sizeof(double);
    cudaMemcpy(b->inst[i].u_dev, saved[i], bytes, cudaMemcpyDeviceToDevice);
    sl_hjb_reset(b->handles[i]);
  }
  release();
  if (probe_st != SL_OK) {
    b->err = "sl_batch_autotune: a probe run failed";
    return probe_st;
  }
  int k = 0;
  for (int nx : sizes) {
    if (k < max_out) {
      out[k].n = nx;
      out[k].instances = int(cls[nx].size());
      out[k].coarse_tail_rows = choice[nx];
      out[k].probe_seconds = best_sec[nx];
    }
    ++k;
  }
  if (n_out) *n_out = k;
  return SL_OK;
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
