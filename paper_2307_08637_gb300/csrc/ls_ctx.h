// ls_ctx.h -- the library context (internal).
#pragma once

#include <cstdint>
#include <map>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ls.h"

// Parameters the autotuner picked for one (key type, floor(log2 n)) class.
struct ls_tuned_entry {
  uint32_t fanout = 0;
  uint32_t basecase_threshold = 0;
  double sample_rate = 0.0;
  int32_t recurse_model = 0;
  double ms = 0.0;  // sort time of the winner when it was tuned
};

// An instantiated CUDA graph of the device level loop (a while node around
// one batch's kernels), for the workspace, keys array and parameters in key.
struct ls_graph_entry {
  std::vector<uint64_t> key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t body_launches = 0;  // kernels per loop iteration
  bool pdl = false;            // captured with programmatic dependent launches
  uint64_t last_use = 0;
};

struct ls_ctx {
  int device = 0;
  unsigned int* d_status = nullptr;
  // cached device memory for ls_fit / ls_classify / ls_fit_grad / ls_sort_host
  void* d_cache = nullptr;
  size_t d_cache_bytes = 0;
  uint64_t launches = 0;
  // streams of ls_sort_host_batch (created on first use): sort, host->device,
  // device->host
  cudaStream_t s_sort = nullptr, s_in = nullptr, s_out = nullptr;
  // page-locked host buffer for the per-level readback of the sort, the
  // stream it is read on and the event (end of a level's K2) it waits for
  void* h_pin = nullptr;
  size_t h_pin_bytes = 0;
  cudaStream_t s_read = nullptr;
  cudaEvent_t ev_children = nullptr;
  // graphs of the device level loop (a few, least recently used first out)
  // and the stream they are captured on
  std::vector<ls_graph_entry> graphs;
  uint64_t graph_clock = 0;
  cudaStream_t s_cap = nullptr, s_cap_aux = nullptr;
  // autotuner results, keyed by dtype * 64 + floor(log2 n)
  std::map<int, ls_tuned_entry> tuned;
  std::mutex tuned_mu;
};

// Key of the tuning class of n keys of type dt.
inline int ls_tune_key(int dt, uint64_t n) {
  int lg = 0;
  while (lg < 63 && (n >> (lg + 1))) ++lg;
  return dt * 64 + lg;
}
