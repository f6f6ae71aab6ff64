// ls_tune.cu -- autotuner of the sort's parameters (fanout B, sample rate r,
// base-case threshold T, recursion mode) and its per-context table.
//
// The paper reports that adjusting the sample size improved the parallel
// performance of its learned sort (Sec. 5).  Here the tunable parameters are
// chosen by measurement: ls_sort is timed on copies of the caller's keys,
// one parameter at a time (coordinate descent from the caller's base
// parameters), and the fastest configuration is kept per (key type,
// floor(log2 n)).  Every candidate produces the same sorted output; only the
// speed differs.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ls_ctx.h"
#include "ls_kernels.h"

namespace {

const uint32_t kFanouts[] = {256, 512, 1000, 1024, 2048};
const uint32_t kThresholds[] = {1024, 2048, 4096, 8192};
const double kRates[] = {0.0025, 0.005, 0.01, 0.02};
const int32_t kRecurse[] = {LS_RECURSE_REFINE_GLOBAL, LS_RECURSE_RETRAIN};
// A candidate replaces the current configuration only when it is faster by
// this fraction: single sorts of a tuning array are short, and changes
// within the timing noise would otherwise decide (and a choice that wins by
// noise on one array can lose on the batched form it is tuned for).
constexpr double kMinGain = 0.05;
constexpr int kTimedReps = 5;  // timed sorts per configuration (median), after one warm-up

struct Scratch {
  void* keys = nullptr;
  void* ws = nullptr;
  ~Scratch() {
    if (keys) cudaFree(keys);
    if (ws) cudaFree(ws);
  }
};

// Median of kTimedReps timed sorts of a fresh copy of d_keys (after one
// warm-up sort), in ms; negative on failure (*st gets the failing status).
// h_off (nullable): the segments of a segmented sort (nseg + 1 offsets).
double time_config(ls_ctx* ctx, const void* d_keys, uint64_t n, const uint64_t* h_off, uint32_t nseg,
                   ls_dtype dtype, const ls_params& p, Scratch& s, size_t ws_bytes, cudaStream_t stream,
                   ls_status* st) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) {
    *st = LS_ECUDA;
    return -1.0;
  }
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    *st = LS_ECUDA;
    return -1.0;
  }
  double t[kTimedReps] = {};
  *st = LS_OK;
  for (int rep = 0; rep <= kTimedReps && *st == LS_OK; ++rep) {
    if (cudaMemcpyAsync(s.keys, d_keys, n * 8, cudaMemcpyDeviceToDevice, stream) != cudaSuccess) {
      *st = LS_ECUDA;
      break;
    }
    cudaEventRecord(e0, stream);
    ls_status r = h_off ? ls_sort_segmented(ctx, s.keys, h_off, nseg, dtype, &p, s.ws, ws_bytes, nullptr, nullptr,
                                            stream)
                        : ls_sort(ctx, s.keys, n, dtype, &p, s.ws, ws_bytes, nullptr, stream);
    cudaEventRecord(e1, stream);
    if (r != LS_OK) {
      *st = r;
      break;
    }
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      *st = LS_ECUDA;
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) t[rep - 1] = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (*st != LS_OK) return -1.0;
  std::sort(t, t + kTimedReps);
  return t[kTimedReps / 2];
}

// Coordinate descent over the candidate lists for one array (h_off null)
// or one batch of segments; the table key is floor(log2) of the array's
// length or of the mean segment length.
ls_status tune(ls_ctx* ctx, const void* d_keys, uint64_t n, const uint64_t* h_off, uint32_t nseg, ls_dtype dtype,
               const ls_params* base, ls_params* out, ls_tune_report* report, ls_stream_t stream) {
  if (!ctx || !base || !out || (!d_keys && n) || (dtype != LS_F64 && dtype != LS_U64) || n < 2) return LS_EINVAL;
  const uint32_t wseg = h_off ? nseg : 1u;
  ls_params cur = *base;
  cur.flags &= ~LS_FLAG_TUNED;  // time what is asked, not an earlier entry
  cur.flags &= ~LS_FLAG_TIME_PASSES;
  size_t ws_max = 0;
  {
    // workspace for the largest candidate in every dimension
    ls_params probe = cur;
    for (uint32_t f : kFanouts)
      for (double r : kRates)
        for (int32_t m : kRecurse) {
          probe.fanout = f;
          probe.sample_rate = r;
          probe.recurse_model = m;
          probe.basecase_threshold = cur.basecase_threshold;
          size_t b = 0;
          ls_status v = ls_workspace_size(ctx, n, wseg, dtype, &probe, &b);
          if (v != LS_OK) return v;
          ws_max = std::max(ws_max, b);
          for (uint32_t T : kThresholds) {
            probe.basecase_threshold = T;
            v = ls_workspace_size(ctx, n, wseg, dtype, &probe, &b);
            if (v != LS_OK) return v;
            ws_max = std::max(ws_max, b);
          }
        }
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LS_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch s;
  if (cudaMalloc(&s.keys, n * 8) != cudaSuccess) return LS_ENOMEM;
  if (cudaMalloc(&s.ws, ws_max) != cudaSuccess) return LS_ENOMEM;
  ls_status sv = LS_OK;
  double best = time_config(ctx, d_keys, n, h_off, nseg, dtype, cur, s, ws_max, st, &sv);
  if (best < 0.0) return sv;
  const double base_ms = best;
  uint32_t configs = 1;
  auto consider = [&](const ls_params& cand) -> ls_status {
    ls_status r = LS_OK;
    double ms = time_config(ctx, d_keys, n, h_off, nseg, dtype, cand, s, ws_max, st, &r);
    if (ms < 0.0) return r;
    ++configs;
    if (ms < best * (1.0 - kMinGain)) {
      best = ms;
      cur = cand;
    }
    return LS_OK;
  };
  for (uint32_t f : kFanouts) {
    if (f == cur.fanout) continue;
    ls_params c = cur;
    c.fanout = f;
    if (ls_status r = consider(c)) return r;
  }
  for (uint32_t T : kThresholds) {
    if (T == cur.basecase_threshold) continue;
    ls_params c = cur;
    c.basecase_threshold = T;
    if (ls_status r = consider(c)) return r;
  }
  for (double rr : kRates) {
    if (rr == cur.sample_rate) continue;
    ls_params c = cur;
    c.sample_rate = rr;
    if (ls_status r = consider(c)) return r;
  }
  for (int32_t m : kRecurse) {
    if (m == cur.recurse_model) continue;
    ls_params c = cur;
    c.recurse_model = m;
    if (ls_status r = consider(c)) return r;
  }
  *out = *base;
  out->fanout = cur.fanout;
  out->basecase_threshold = cur.basecase_threshold;
  out->sample_rate = cur.sample_rate;
  out->recurse_model = cur.recurse_model;
  {
    ls_tuned_entry e;
    e.fanout = cur.fanout;
    e.basecase_threshold = cur.basecase_threshold;
    e.sample_rate = cur.sample_rate;
    e.recurse_model = cur.recurse_model;
    e.ms = best;
    std::lock_guard<std::mutex> lk(ctx->tuned_mu);
    ctx->tuned[ls_tune_key(dtype, h_off ? n / nseg : n)] = e;
  }
  if (report) {
    report->configs = configs;
    report->base_ms = base_ms;
    report->best_ms = best;
  }
  return LS_OK;
}

}  // namespace

extern "C" {

ls_status ls_autotune(ls_ctx* ctx, const void* d_keys, uint64_t n, ls_dtype dtype, const ls_params* base,
                      ls_params* out, ls_tune_report* report, ls_stream_t stream) {
  return tune(ctx, d_keys, n, nullptr, 0, dtype, base, out, report, stream);
}

ls_status ls_autotune_segmented(ls_ctx* ctx, const void* d_keys, const uint64_t* h_offsets, uint32_t nseg,
                                ls_dtype dtype, const ls_params* base, ls_params* out, ls_tune_report* report,
                                ls_stream_t stream) {
  if (!h_offsets || nseg == 0) return LS_EINVAL;
  for (uint32_t i = 0; i < nseg; ++i)
    if (h_offsets[i + 1] < h_offsets[i]) return LS_EINVAL;
  if (h_offsets[0] != 0) return LS_EINVAL;  // the timed copies cover keys [0, h_offsets[nseg])
  return tune(ctx, d_keys, h_offsets[nseg], h_offsets, nseg, dtype, base, out, report, stream);
}

ls_status ls_tune_export(ls_ctx* ctx, char* buf, size_t* bytes) {
  if (!ctx || !bytes) return LS_EINVAL;
  std::string text;
  {
    std::lock_guard<std::mutex> lk(ctx->tuned_mu);
    char line[256];
    for (const auto& kv : ctx->tuned) {
      const ls_tuned_entry& e = kv.second;
      snprintf(line, sizeof line, "%d %d %u %u %.17g %d %.6f\n", kv.first / 64, kv.first % 64, e.fanout,
               e.basecase_threshold, e.sample_rate, e.recurse_model, e.ms);
      text += line;
    }
  }
  const size_t need = text.size() + 1;
  if (!buf) {
    *bytes = need;
    return LS_OK;
  }
  if (*bytes < need) {
    *bytes = need;
    return LS_ENOMEM;
  }
  memcpy(buf, text.c_str(), need);
  *bytes = need;
  return LS_OK;
}

ls_status ls_tune_import(ls_ctx* ctx, const char* text) {
  if (!ctx || !text) return LS_EINVAL;
  std::vector<std::pair<int, ls_tuned_entry>> add;
  const char* p = text;
  while (*p) {
    const char* eol = strchr(p, '\n');
    std::string line = eol ? std::string(p, eol - p) : std::string(p);
    p = eol ? eol + 1 : p + line.size();
    if (line.find_first_not_of(" \t\r") == std::string::npos) continue;
    int dt = -1, lg = -1, rm = -1;
    unsigned f = 0, T = 0;
    double r = 0.0, ms = 0.0;
    int used = 0;
    if (sscanf(line.c_str(), "%d %d %u %u %lf %d %lf %n", &dt, &lg, &f, &T, &r, &rm, &ms, &used) != 7)
      return LS_EINVAL;
    if (line.find_first_not_of(" \t\r", (size_t)used) != std::string::npos) return LS_EINVAL;
    if ((dt != LS_F64 && dt != LS_U64) || lg < 0 || lg > 63 || f < 2 || f > LS_MAX_FANOUT || T < 1 ||
        T > lsg::kMaxBaseCase ||
        !(r > 0.0 && r <= 1.0) || (rm != LS_RECURSE_REFINE_GLOBAL && rm != LS_RECURSE_RETRAIN))
      return LS_EINVAL;
    ls_tuned_entry e;
    e.fanout = f;
    e.basecase_threshold = T;
    e.sample_rate = r;
    e.recurse_model = rm;
    e.ms = ms;
    add.push_back({dt * 64 + lg, e});
  }
  std::lock_guard<std::mutex> lk(ctx->tuned_mu);
  for (const auto& kv : add) ctx->tuned[kv.first] = kv.second;
  return LS_OK;
}

}  // extern "C"
