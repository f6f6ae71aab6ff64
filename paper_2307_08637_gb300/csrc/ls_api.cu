// ls_api.cu -- C ABI and host orchestration of learned SampleSort on GB300.
//
// ls_sort runs the recursion of Sec. 2.2 / Sec. 4 level by level.  Each
// level's buckets that still need partitioning ("items") are planned on the
// host in batches; every per-key step runs in the kernels of ls_fit.cu and
// ls_partition.cu.  Per batch:
//   fresh items (their own sample: the root, RETRAIN buckets, buckets of a
//   splitter partition, no-progress redos): sample -> sort -> duplicate count
//   -> FP64 RMI fit -> exact learned pivots -> sample imbalance -> Alg. 5
//   decision -> splitter table when the tree is chosen;
//   refine items (LearnedSort 2.0's second round: same model, finer buckets):
//   exact pivots of floor(F(x) B^(k+1)) - B g, or direct FP64 for small items;
//   then K1 (classify + histogram), K2 (scan + children), K3 (scatter).
// After each level the finished spans are sorted (base case), copied home, or
// sorted by the depth-limit fallback.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <set>
#include <vector>

#include "ls_ctx.h"
#include "ls_kernels.h"

using namespace lsg;

namespace {
thread_local char g_error_detail[256] = "";
}  // namespace

void lsg::set_error_detail(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_error_detail, sizeof g_error_detail, fmt, ap);
  va_end(ap);
}

namespace {

constexpr uint64_t kPinItems = 4096;  // next-level items read back with the level counters
constexpr uint32_t kDirBits = 13;
constexpr size_t kAlign = 256;

inline size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }
inline uint32_t pow2ceil(uint32_t x) {
  uint32_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

#define CK(call)                                                        \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) {                                            \
      lsg::set_error_detail("CUDA error %s at %s:%d", cudaGetErrorString(e_), __FILE__, __LINE__); \
      return LS_ECUDA;                                                  \
    }                                                                   \
  } while (0)

ls_status validate_params(const ls_params* p) {
  if (!p) return LS_EINVAL;
  if (p->fanout < 2 || p->fanout > LS_MAX_FANOUT) return LS_EINVAL;
  if (p->splitter_fanout < 2 || p->splitter_fanout > LS_MAX_FANOUT / 2) return LS_EINVAL;
  if (p->auto_splitter_fanout < 2) return LS_EINVAL;
  if (p->basecase_threshold < 1 || p->basecase_threshold > kMaxBaseCase) return LS_EINVAL;
  if (p->max_depth >= LS_MAX_LEVELS - 2) return LS_EINVAL;
  if (p->min_sample < 2) return LS_EINVAL;
  if (!(p->sample_rate >= 0.0) || !(p->dup_frac >= 0.0) || !(p->imbalance_tau > 0.0)) return LS_EINVAL;
  if (p->partitioner < 0 || p->partitioner > 2) return LS_EINVAL;
  if (p->recurse_model < 0 || p->recurse_model > 1) return LS_EINVAL;
  if (p->classify_mode < 0 || p->classify_mode > 4) return LS_EINVAL;
  return LS_OK;
}

}  // namespace

// The parameters a sort really uses: with LS_FLAG_TUNED, the autotuner's
// entry for the key type and floor(log2) of the (mean segment) length
// replaces fanout, sample rate, base-case threshold and recursion mode.
static ls_params effective_params(ls_ctx* ctx, uint64_t n, uint32_t nseg, ls_dtype dtype, const ls_params& p) {
  ls_params e = p;
  if (!(p.flags & LS_FLAG_TUNED) || !ctx) return e;
  const uint64_t per = nseg ? n / nseg : n;
  std::lock_guard<std::mutex> lk(ctx->tuned_mu);
  auto it = ctx->tuned.find(ls_tune_key(dtype, per ? per : 1));
  if (it == ctx->tuned.end()) return e;
  e.fanout = it->second.fanout;
  e.basecase_threshold = it->second.basecase_threshold;
  e.sample_rate = it->second.sample_rate;
  e.recurse_model = it->second.recurse_model;
  return e;
}

namespace {

uint64_t sample_size(uint64_t n, const ls_params* p) {
  if (n == 0) return 0;
  double want = std::ceil(p->sample_rate * (double)n);
  uint64_t S;
  if (!(want < (double)n)) S = n;
  else if (want < 1.0) S = 0;
  else S = (uint64_t)want;
  if (S < p->min_sample) S = p->min_sample;
  if (S > n) S = n;
  return S;
}

// B^e in FP64, exact while it stays below 2^53.  The loop stops once the
// product passes the refinement limit (B >= 2, so it only grows): callers
// compare the result with that limit, and a huge e costs no more than ~50
// multiplications.
double pow_exact(uint32_t B, uint32_t e) {
  double P = 1.0;
  for (uint32_t i = 0; i < e && P <= kRefineLimit; ++i) P = P * (double)B;
  return P;
}

RunParams make_rp(const ls_params* p, int dt) {
  RunParams r;
  r.B = p->fanout;
  r.bs_max = p->splitter_fanout;
  r.bs_auto = p->auto_splitter_fanout;
  r.T = p->basecase_threshold;
  r.max_depth = p->max_depth;
  r.min_sample = p->min_sample;
  r.sample_rate = p->sample_rate;
  r.dup_frac = p->dup_frac;
  r.tau = p->imbalance_tau;
  r.min_learned_n = p->min_learned_n;
  r.seed = p->seed;
  r.partitioner = p->partitioner;
  r.recurse = p->recurse_model;
  r.classify_mode = p->classify_mode;
  r.dt = dt;
  r.tile = kTileKeys;
  r.dir_bits = kDirBits;
  return r;
}

// Workspace layout for n keys, nseg segments.
struct Layout {
  uint64_t n = 0;
  uint32_t L = 0, nbc = 0, cells = 0;
  uint64_t icap = 0, scap = 0, mcap = 0, base_cap = 0, mid_cap = 0, large_cap = 0, copy_cap = 0, fb_cap = 0;
  uint64_t rchunk_cap = 0, lchunk_cap = 0, chunk_cap = 0, seg_cap = 0, brun_cap = 0;
  size_t total = 0;
  size_t o_buf, o_cur, o_next, o_plans, o_counts, o_cursors, o_pivots, o_dirs, o_small, o_mid, o_large, o_copy, o_fb,
      o_models, o_leaves, o_leafcnt, o_samp0, o_samp1, o_rpart, o_lstart, o_lcnt, o_lpre, o_lpart, o_leafof,
      o_stmp, o_stats, o_ctr, o_rootplan, o_misc, o_agg, o_excl, o_segs, o_multi, o_chunkctr, o_chunkplan, o_fmodels, o_fleaves, o_fclamps, o_ids,
      o_vbuf, o_bruns, o_bitems, o_hostq, o_reflist, o_bdesc, o_queue;
  size_t stmp_elems = 0;
  size_t misc_bytes = 0;
};

Layout compute_layout(uint64_t n, uint32_t nseg, const ls_params* p, uint32_t vb = 0) {
  Layout l;
  l.n = n;
  l.L = p->fanout;
  uint32_t eqmax = 2 * p->splitter_fanout - 1;  // 2m+1 buckets, m <= B_s - 1 splitters
  // per-item bucket tables hold the learned fanout, the splitter tree with
  // equality buckets, or a radix split (2^kRadixBits buckets)
  l.nbc = pow2ceil(std::max<uint32_t>(std::max<uint32_t>(p->fanout, eqmax), 1u << kRadixBits));
  l.cells = 1u << kDirBits;
  uint64_t T = p->basecase_threshold;
  l.icap = n / (T + 1) + nseg + 16;
  uint64_t smax = sample_size(n ? n : 1, p);
  l.scap = std::max<uint64_t>(smax, 64ull * p->min_sample) + 1024;
  l.mcap = 1024 + n / 65536;
  l.base_cap = n / 2 + 1024;
  l.mid_cap = n / (kWarpSmallMax + 1) + 1024;
  l.large_cap = n / (kWarpSortMax + 1) + 1024;
  l.copy_cap = n / 2 + l.icap + 64 * 1024;  // <= one run of final buckets per non-final child + item
  l.fb_cap = n / (T + 1) + 1024;
  l.rchunk_cap = l.scap / kChunk + kBatchItems + 8;
  l.lchunk_cap = l.scap / kChunk + (uint64_t)kBatchItems * l.L + 8;
  l.stmp_elems = scan_tmp_elems((size_t)kBatchItems * l.L + 8) + 64;
  // chunks of a batch: at most n / 64Ki + one partial chunk per item, or
  // fewer than 2 kChunkSlots + one per item when the chunk size was reduced
  l.chunk_cap = n / kChunkKeys + kBatchItems + nseg + 8 + 2 * kChunkSlots;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t r = off;
    off = up(off + bytes);
    return r;
  };
  l.o_buf = take(n * 8);
  l.o_vbuf = vb ? take(n * vb) : 0;  // key-value sorts: ping-pong buffer of the values
  l.o_ids = take(n * 2);
  l.o_cur = take(l.icap * sizeof(Item));
  l.o_next = take(l.icap * sizeof(Item));
  l.o_plans = take(kBatchItems * sizeof(Plan));
  l.o_counts = take((size_t)kBatchItems * l.nbc * 8);
  l.o_cursors = take((size_t)kBatchItems * l.nbc * 8);
  l.o_pivots = take((size_t)kBatchItems * l.nbc * 8);
  l.o_dirs = take((size_t)kBatchItems * (l.cells + 1) * 2);
  l.o_small = take(l.base_cap * sizeof(Span));
  l.o_mid = take(l.mid_cap * sizeof(Span));
  l.o_large = take(l.large_cap * sizeof(Span));
  l.o_copy = take(l.copy_cap * sizeof(Span));
  l.o_fb = take(l.fb_cap * sizeof(Span));
  l.o_models = take(l.mcap * sizeof(DModel));
  l.o_leaves = take(l.mcap * l.L * sizeof(Leaf));
  l.o_leafcnt = take(l.mcap * l.L * 4);
  l.o_fmodels = take(l.mcap * sizeof(FModel));
  l.o_fleaves = take(l.mcap * l.L * sizeof(FLeaf));
  l.o_fclamps = take(l.mcap * l.L * sizeof(FClamp));
  l.o_samp0 = take(l.scap * 8);
  l.o_samp1 = take(l.scap * 8);
  l.o_rpart = take(8 * l.rchunk_cap * 8);
  l.o_lstart = take((size_t)kBatchItems * (l.L + 1) * 4);
  l.o_lcnt = take(((size_t)kBatchItems * l.L + 8) * 8);
  l.o_lpre = take(((size_t)kBatchItems * l.L + 8) * 8);
  l.o_lpart = take(4 * l.lchunk_cap * 8);
  l.o_leafof = take(l.scap * 4);
  l.o_stmp = take(l.stmp_elems * 8);
  l.o_stats = take(LS_MAX_LEVELS * sizeof(DevLevelStats));
  l.o_ctr = take(sizeof(LevelCounters));
  l.o_rootplan = take(sizeof(Plan));
  l.o_agg = take(l.chunk_cap * l.nbc * 4);
  l.o_excl = take(l.chunk_cap * l.nbc * 8);
  l.seg_cap = l.chunk_cap / kSegChunks + kBatchItems + 8;
  l.o_segs = take(l.seg_cap * sizeof(ChunkSeg));
  l.o_multi = take((size_t)kBatchItems * sizeof(uint2));
  l.o_chunkctr = take(16);
  // buffered-scatter runs: at most one per item plus the equal shares
  // (two per resident block; 4096 covers any part this library targets)
  l.brun_cap = kBatchItems + 4096;
  l.o_bruns = take(l.brun_cap * sizeof(BufRun));
  l.o_chunkplan = take(l.chunk_cap * 4);
  // device-planned levels: the batch's items, items handed back to the
  // host, the pivot list, the batch descriptor and the queue state
  l.o_bitems = take((size_t)kBatchItems * sizeof(Item));
  l.o_hostq = take(l.icap * sizeof(Item));
  l.o_reflist = take((size_t)kBatchItems * 4);
  l.o_bdesc = take(sizeof(BatchDesc));
  l.o_queue = take(sizeof(QueueState));
  l.misc_bytes = 16 * (kBatchItems + 8) * 8;
  l.o_misc = take(l.misc_bytes);
  l.total = off;
  return l;
}

template <typename T>
T* at(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

// Host mirror of one batch.
struct Batch {
  std::vector<Item> items;
  std::vector<Plan> plans;
  uint64_t ntiles = 0;
};

// CUDA-event timing of kernel classes (LS_FLAG_TIME_PASSES), recorded on
// the caller's stream around each launch group.
struct PassTimer {
  bool on = false;
  cudaStream_t st = nullptr;
  struct Rec {
    cudaEvent_t a, b;
    int cls;
    uint64_t keys;
  };
  std::vector<Rec> recs;
  Rec cur{};
  cudaEvent_t make() {
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void begin(int cls, uint64_t keys) {
    if (!on) return;
    cur = Rec{make(), make(), cls, keys};
    cudaEventRecord(cur.a, st);
  }
  void end() {
    if (!on) return;
    cudaEventRecord(cur.b, st);
    recs.push_back(cur);
  }
  void collect(ls_stats* s) {
    if (!on) return;
    cudaStreamSynchronize(st);
    for (Rec& r : recs) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess && s) {
        s->pass[r.cls].ms += ms;
        s->pass[r.cls].launches += 1;
        s->pass[r.cls].keys += r.keys;
      }
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    recs.clear();
  }
  ~PassTimer() {
    for (Rec& r : recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
  }
};

struct Sorter {
  PassTimer timer;
  ls_ctx* ctx;
  const ls_params* p;
  RunParams rp;
  Layout lay;
  void* ws;
  cudaStream_t st;
  uint64_t* A;
  uint64_t* Bb;
  void* VA = nullptr;   // key-value sorts: the caller's values ...
  void* VBb = nullptr;  // ... and their ping-pong buffer
  uint32_t vb = 0;      // bytes per value (0: keys only)
  int dt;
  std::vector<int> model_free;
  std::vector<uint8_t> model_used;
  uint64_t launches = 0;
  int32_t* seg_decision = nullptr;  // host, per segment
  uint32_t nseg = 0;
  bool root_copied = false;  // the root's plan waits in the workspace for the final readback
  uint64_t root_n = 0;
  uint64_t device_batches = 0;      // batches planned by the device work queue
  int32_t level_loop = LS_LOOP_HOST;  // the last form the levels below the root ran in

  int alloc_model() {
    if (model_free.empty()) return -1;
    int m = model_free.back();
    model_free.pop_back();
    return m;
  }
};

// Full range of ord values a key of dtype dt can have (NaN excluded).
void ord_range(int dt, uint64_t* lo, uint64_t* hi) {
  if (dt == LS_U64) {
    *lo = 0;
    *hi = ~0ull;
  } else {
    *lo = kOrdMinF64;
    *hi = kOrdMaxF64;
  }
}

// Plan and run one batch of items (all at the same level).
ls_status run_batch(Sorter& s, const Item* items, uint32_t nitems, bool level0, bool record_root,
                    ls_stats* stats, cudaEvent_t ev_children = nullptr) {
  const bool check_nan = level0;
  const ls_params* p = s.p;
  Layout& L = s.lay;
  cudaStream_t st = s.st;
  std::vector<Plan> plans(nitems);
  std::vector<uint32_t> fresh, cand, refine_tab;
  std::vector<uint64_t> samp_prefix(1, 0), cand_soff(1, 0), rchunk_prefix(1, 0), sort_off(1, 0),
      sort_cpre(1, 0);
  uint64_t tiles = 0;
  uint64_t max_s = 0;
  std::vector<Item> its(items, items + nitems);
  // Chunk size of the partition passes: 64Ki keys, halved (down to one tile)
  // while the batch would give fewer than kChunkSlots chunks, so that small
  // batches (deep levels, few small items) still spread over the GPU.
  // Every chunk size gives the same partition; only the work split differs.
  uint64_t batch_keys = 0;
  for (uint32_t i = 0; i < nitems; ++i) batch_keys += its[i].n;
  uint64_t ck = kChunkKeys;
  while (ck > kTileKeys && batch_keys / ck < kChunkSlots) ck >>= 1;
  for (uint32_t i = 0; i < nitems; ++i) {
    Item& it = its[i];
    Plan& pl = plans[i];
    memset(&pl, 0, sizeof pl);
    pl.chunk_begin = tiles;
    tiles += (it.n + ck - 1) / ck;
    pl.cnt_off = (uint64_t)i * L.nbc;
    pl.tab_off = (uint64_t)i * L.nbc;
    pl.dir_off = (uint64_t)i * (L.cells + 1);
    pl.mixed = 0;
    pl.model = -1;
    bool is_fresh = it.kind != KIND_REFINE && it.kind != KIND_RADIX;
    if (it.kind == KIND_RADIX) {
      // radix split of the bits [s, top) in which the item's keys may differ
      const uint32_t nb = radix_buckets(it.mk);
      pl.decision = LS_DEC_RADIX;
      pl.cls = CLS_RADIX;
      pl.nb = nb;
      pl.nb_pad = nb;
      pl.kmax = nb - 1;
      pl.dir_shift = radix_shift(it.mk);
    }
    if (it.kind == KIND_REFINE) {
      double P = pow_exact(p->fanout, it.mk + 1u);
      if (P > kRefineLimit) {
        is_fresh = true;
        it.kind = KIND_FRESH;  // beyond FP64 resolution: draw a new sample
        it.model = -1;
      } else {
        pl.P = P;
        pl.Bg = (double)((uint64_t)p->fanout * it.mg);
        pl.model = it.model;
        pl.decision = LS_DEC_LEARNED;
        pl.nb = p->fanout;
        pl.nb_pad = pow2ceil(p->fanout);
        pl.kmax = p->fanout - 1;
        bool direct = p->classify_mode == LS_CLASSIFY_DIRECT || it.n < 4ull * p->fanout;
        pl.cls = direct                                        ? CLS_DIRECT
                 : p->classify_mode == LS_CLASSIFY_TREE        ? CLS_TREE
                 : p->classify_mode == LS_CLASSIFY_DIRECTORY   ? CLS_DIR
                                                               : CLS_GUESS;
        if (!direct) refine_tab.push_back(i);
      }
    }
    if (is_fresh) {
      pl.fresh = 1;
      uint64_t S = sample_size(it.n, p);
      pl.S = (uint32_t)S;
      pl.sample_off = samp_prefix.back();
      fresh.push_back(i);
      samp_prefix.push_back(samp_prefix.back() + S);
      sort_off.push_back(sort_off.back() + S);
      sort_cpre.push_back(sort_cpre.back() + (S + kSortChunk - 1) / kSortChunk);
      max_s = std::max(max_s, S);
      bool want = it.kind != KIND_FORCE_SPLITTER &&
                  (p->partitioner == LS_PART_LEARNED ||
                   (p->partitioner == LS_PART_AUTO && it.n >= p->min_learned_n));
      if (want) {
        int m = s.alloc_model();
        if (m < 0) return LS_ENOMEM;
        pl.model = m;
        pl.want = 1;
        pl.P = (double)p->fanout;
        pl.Bg = 0.0;
        pl.nb_pad = pow2ceil(p->fanout);
        pl.fit_slot = (uint32_t)cand.size();
        cand.push_back(i);
        cand_soff.push_back(cand_soff.back() + S);
        rchunk_prefix.push_back(rchunk_prefix.back() + (S + kChunk - 1) / kChunk);
      }
    }
  }
  if (samp_prefix.back() > L.scap) return LS_ENOMEM;
  // upload items + plans + index lists
  Item* d_items = at<Item>(s.ws, L.o_cur);
  Plan* d_plans = at<Plan>(s.ws, L.o_plans);
  CK(cudaMemcpyAsync(d_items, its.data(), nitems * sizeof(Item), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_plans, plans.data(), nitems * sizeof(Plan), cudaMemcpyHostToDevice, st));
  uint64_t* misc = at<uint64_t>(s.ws, L.o_misc);
  const size_t M = kBatchItems + 8;
  uint32_t* d_fresh = reinterpret_cast<uint32_t*>(misc + 0 * M);
  uint64_t* d_sprefix = misc + 1 * M;
  uint32_t* d_cand = reinterpret_cast<uint32_t*>(misc + 2 * M);
  uint64_t* d_csoff = misc + 3 * M;
  uint64_t* d_rcp = misc + 4 * M;
  uint64_t* d_soff = misc + 5 * M;
  uint64_t* d_scpre = misc + 6 * M;
  uint32_t* d_reftab = reinterpret_cast<uint32_t*>(misc + 7 * M);
  if (!fresh.empty()) {
    CK(cudaMemcpyAsync(d_fresh, fresh.data(), fresh.size() * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_sprefix, samp_prefix.data(), samp_prefix.size() * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_soff, sort_off.data(), sort_off.size() * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_scpre, sort_cpre.data(), sort_cpre.size() * 8, cudaMemcpyHostToDevice, st));
  }
  if (!cand.empty()) {
    CK(cudaMemcpyAsync(d_cand, cand.data(), cand.size() * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_csoff, cand_soff.data(), cand_soff.size() * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_rcp, rchunk_prefix.data(), rchunk_prefix.size() * 8, cudaMemcpyHostToDevice, st));
  }
  if (!refine_tab.empty())
    CK(cudaMemcpyAsync(d_reftab, refine_tab.data(), refine_tab.size() * 4, cudaMemcpyHostToDevice, st));

  uint64_t* pivots = at<uint64_t>(s.ws, L.o_pivots);
  uint16_t* dirs = at<uint16_t>(s.ws, L.o_dirs);
  DModel* models = at<DModel>(s.ws, L.o_models);
  Leaf* leaves = at<Leaf>(s.ws, L.o_leaves);
  unsigned long long* counts = at<unsigned long long>(s.ws, L.o_counts);
  unsigned long long* cursors = at<unsigned long long>(s.ws, L.o_cursors);
  CK(cudaMemsetAsync(counts, 0, (size_t)nitems * L.nbc * 8, st));

  // ---- fresh items: sample, sort, dups, fit, pivots, decision
  const uint64_t* sorted = nullptr;
  if (!fresh.empty()) {
    FreshArgs f;
    f.items = d_items;
    f.plans = d_plans;
    f.fresh = d_fresh;
    f.samp_prefix = d_sprefix;
    f.nfresh = (uint32_t)fresh.size();
    f.total_samples = samp_prefix.back();
    f.keysA = s.A;
    f.keysB = s.Bb;
    uint64_t* samp0 = at<uint64_t>(s.ws, L.o_samp0);
    uint64_t* samp1 = at<uint64_t>(s.ws, L.o_samp1);
    s.timer.begin(LS_PASS_SAMPLE, samp_prefix.back());
    launch_sample_gather(f, s.rp, samp0, st);
    sorted = segmented_sort_u64(samp0, samp1, d_soff, d_scpre, (uint32_t)fresh.size(), sort_cpre.back(), max_s,
                                st, &s.launches);
    launch_dups(f, sorted, st);
    s.timer.end();
    s.launches += 2;
    if (!cand.empty()) {
      FitArgs fa{};
      fa.plans = d_plans;
      fa.items = d_items;
      fa.cand = d_cand;
      fa.cand_soff = d_csoff;
      fa.nbp_max = pow2ceil(p->fanout);
      fa.rchunk_prefix = d_rcp;
      fa.ncand = (uint32_t)cand.size();
      fa.total_rchunks = rchunk_prefix.back();
      fa.total_cand_samples = cand_soff.back();
      fa.lchunk_bound = cand_soff.back() / kChunk + (uint64_t)cand.size() * L.L + 8;
      fa.samp = sorted;
      fa.models = models;
      fa.leaves = leaves;
      fa.L = L.L;
      fa.rpart = at<double>(s.ws, L.o_rpart);
      fa.leaf_start = at<uint32_t>(s.ws, L.o_lstart);
      fa.lchunk_cnt = at<uint64_t>(s.ws, L.o_lcnt);
      fa.lchunk_prefix = at<uint64_t>(s.ws, L.o_lpre);
      fa.scan_tmp = at<uint64_t>(s.ws, L.o_stmp);
      fa.scan_tmp_elems = L.stmp_elems;
      fa.lpart = at<double>(s.ws, L.o_lpart);
      fa.leaf_of = at<uint32_t>(s.ws, L.o_leafof);
      fa.leaf_cnt = at<uint32_t>(s.ws, L.o_leafcnt);
      fa.fmodels = at<FModel>(s.ws, L.o_fmodels);
      fa.fleaves = at<FLeaf>(s.ws, L.o_fleaves);
      fa.fclamps = at<FClamp>(s.ws, L.o_fclamps);
      if (fa.total_rchunks > L.rchunk_cap || fa.lchunk_bound > L.lchunk_cap) return LS_ENOMEM;
      s.timer.begin(LS_PASS_FIT, cand_soff.back());
      launch_fit(fa, s.rp, st, &s.launches);
      s.timer.end();
      s.timer.begin(LS_PASS_PIVOTS, 0);
      launch_learned_pivots(d_plans, d_items, d_cand, fa.ncand, pow2ceil(p->fanout), models, leaves, pivots, s.rp,
                            st);
      launch_imbalance(fa, pivots, counts, s.rp, st, &s.launches);
      s.timer.end();
      s.launches += 1;
    }
    s.timer.begin(LS_PASS_PIVOTS, 0);
    launch_decide(f, models, s.rp, st);
    launch_splitter_build(f, sorted, pivots, s.rp, st);
    s.timer.end();
    s.launches += 2;
  }
  s.timer.begin(LS_PASS_PIVOTS, 0);
  if (!refine_tab.empty()) {
    launch_learned_pivots(d_plans, d_items, d_reftab, (uint32_t)refine_tab.size(), pow2ceil(p->fanout), models,
                          leaves, pivots, s.rp, st);
    s.launches += 1;
  }
  if (p->classify_mode == LS_CLASSIFY_DIRECTORY) {
    launch_dir_build(d_plans, nitems, L.cells, pivots, dirs, st);
    s.launches += 1;
  }
  s.timer.end();
  // shared memory of the passes is sized by what this batch really uses;
  // fresh items are decided on the device, so read their plans back
  uint32_t nbp_max = 2, cls_mask = 0;
  bool any_dir = false, any_guess = false;
  std::vector<Plan> hp;
  if (!fresh.empty()) {
    hp.resize(nitems);
    CK(cudaMemcpyAsync(hp.data(), d_plans, nitems * sizeof(Plan), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (const Plan& q : hp) {
      nbp_max = std::max(nbp_max, q.nb_pad);
      any_dir |= q.cls == CLS_DIR;
      any_guess |= q.cls == CLS_GUESS;
      cls_mask |= 1u << q.cls;
    }
  } else {
    for (const Plan& q : plans) {
      nbp_max = std::max(nbp_max, q.nb_pad);
      any_dir |= q.cls == CLS_DIR;
      any_guess |= q.cls == CLS_GUESS;
      cls_mask |= 1u << q.cls;
    }
  }
  uint32_t aux = 16;
  if (any_dir) aux = std::max<uint32_t>(aux, ((L.cells + 1) * 2 + 15) & ~15u);
  if (any_guess) aux = std::max<uint32_t>(aux, L.L * (uint32_t)(sizeof(FLeaf) + sizeof(FClamp)));

  // ---- partition passes
  PassArgs pa{};
  pa.items = d_items;
  pa.plans = d_plans;
  pa.nitems = nitems;
  pa.nchunks = tiles;
  if (tiles > L.chunk_cap) return LS_ENOMEM;
  {
    // the item of every chunk, for K1 and K3 (one load instead of a search
    // over the plans per chunk)
    std::vector<uint32_t> cp(tiles);
    for (uint32_t i = 0; i < nitems; ++i) {
      const uint64_t c1 = i + 1 < nitems ? plans[i + 1].chunk_begin : tiles;
      for (uint64_t c = plans[i].chunk_begin; c < c1; ++c) cp[c] = i;
    }
    uint32_t* d_cp = at<uint32_t>(s.ws, L.o_chunkplan);
    if (tiles) CK(cudaMemcpyAsync(d_cp, cp.data(), tiles * 4, cudaMemcpyHostToDevice, st));
    pa.chunk_plan = d_cp;
  }
  pa.agg = at<uint32_t>(s.ws, L.o_agg);
  pa.excl = at<unsigned long long>(s.ws, L.o_excl);
  pa.chunk_ctr = at<unsigned long long>(s.ws, L.o_chunkctr);
  pa.keysA = s.A;
  pa.keysB = s.Bb;
  pa.outA = s.A;
  pa.outB = s.Bb;
  pa.pivots = pivots;
  pa.dirs = dirs;
  pa.models = models;
  pa.leaves = leaves;
  pa.counts = counts;
  pa.cursors = cursors;
  pa.status = s.ctx->d_status;
  pa.check_nan = check_nan && s.dt == LS_F64;
  pa.nb_pad_max = nbp_max;
  pa.dir_cells_max = L.cells;
  pa.fmodels = at<FModel>(s.ws, L.o_fmodels);
  pa.fleaves = at<FLeaf>(s.ws, L.o_fleaves);
  pa.fclamps = at<FClamp>(s.ws, L.o_fclamps);
  pa.aux_bytes = aux;
  pa.cls_mask = cls_mask;
  pa.valsA = s.VA;
  pa.valsB = s.VBb;
  pa.vbytes = s.vb;
  pa.ids = at<uint16_t>(s.ws, L.o_ids);
  pa.chunk_keys = ck;
  CK(cudaMemsetAsync(pa.chunk_ctr, 0, 2 * sizeof(unsigned long long), st));
  // Runs of the buffered scatter for every item it may take (whether it
  // does is decided by K2 on the device): each candidate's keys split into
  // runs of about an equal share of two runs per resident block (whole items
  // when smaller), so that blocks get the same work and each bucket's region
  // of a run is long.  The stable K3 is launched as well and skips them.
  const std::vector<Plan>& dplans = fresh.empty() ? plans : hp;  // decisions as the device made them
  std::vector<BufRun> bruns;
  {
    uint64_t bkeys = 0;
    for (uint32_t i = 0; i < nitems; ++i)
      if (buffered_scatter_candidate(dplans[i], s.vb)) bkeys += its[i].n;
    const uint64_t slots = 2ull * buffered_scatter_slots();
    const uint64_t target = std::max<uint64_t>(kTileKeys, (bkeys + slots - 1) / slots);
    for (uint32_t i = 0; i < nitems; ++i) {
      const uint64_t n = its[i].n;
      if (!buffered_scatter_candidate(dplans[i], s.vb)) continue;
      const uint64_t nr = (n + target - 1) / target;
      for (uint64_t r = 0; r < nr; ++r) {
        BufRun br;
        memset(&br, 0, sizeof br);
        br.off = n * r / nr;
        br.len = n * (r + 1) / nr - br.off;
        br.plan = i;
        if (br.len) bruns.push_back(br);
      }
    }
    if (bruns.size() > L.brun_cap) return LS_ENOMEM;
    if (!bruns.empty())
      CK(cudaMemcpyAsync(at<BufRun>(s.ws, L.o_bruns), bruns.data(), bruns.size() * sizeof(BufRun),
                         cudaMemcpyHostToDevice, st));
  }
  s.timer.begin(LS_PASS_CLASSIFY, batch_keys);
  s.launches += launch_classify_hist(pa, s.rp, st);
  s.timer.end();

  ChildArgs ca{};
  ca.items = d_items;
  ca.plans = d_plans;
  ca.nitems = nitems;
  ca.pivots = pivots;
  ca.counts = counts;
  ca.cursors = cursors;
  ca.next = at<Item>(s.ws, L.o_next);
  ca.next_cap = L.icap;
  ca.base_small = at<Span>(s.ws, L.o_small);
  ca.base_mid = at<Span>(s.ws, L.o_mid);
  ca.base_large = at<Span>(s.ws, L.o_large);
  ca.base_cap = L.base_cap;
  ca.mid_cap = L.mid_cap;
  ca.large_cap = L.large_cap;
  ca.copy = at<Span>(s.ws, L.o_copy);
  ca.copy_cap = L.copy_cap;
  ca.fallback = at<Span>(s.ws, L.o_fb);
  ca.fallback_cap = L.fb_cap;
  ca.ctr = at<LevelCounters>(s.ws, L.o_ctr);
  ca.stats = at<DevLevelStats>(s.ws, L.o_stats);
  // per-chunk prefixes of the K1 counts, in runs of kSegChunks chunks
  std::vector<ChunkSeg> segs;
  std::vector<uint2> multi;  // items with several runs: (first run, runs)
  for (uint32_t i = 0; i < nitems; ++i) {
    uint64_t cb = plans[i].chunk_begin, nc = (its[i].n + ck - 1) / ck;
    uint32_t first = (uint32_t)segs.size();
    if (nc > kSegChunks) multi.push_back(make_uint2(first, (uint32_t)((nc + kSegChunks - 1) / kSegChunks)));
    for (uint64_t c = 0; c < nc; c += kSegChunks) {
      ChunkSeg g;
      g.c0 = cb + c;
      g.nch = (uint32_t)std::min<uint64_t>(kSegChunks, nc - c);
      g.plan = i;
      g.first = first;
      g.pad = 0;
      segs.push_back(g);
    }
  }
  if (segs.size() > L.seg_cap || multi.size() > kBatchItems) return LS_ENOMEM;
  ChunkSeg* d_segs = at<ChunkSeg>(s.ws, L.o_segs);
  uint2* d_multi = at<uint2>(s.ws, L.o_multi);
  if (!segs.empty())
    CK(cudaMemcpyAsync(d_segs, segs.data(), segs.size() * sizeof(ChunkSeg), cudaMemcpyHostToDevice, st));
  if (!multi.empty())
    CK(cudaMemcpyAsync(d_multi, multi.data(), multi.size() * sizeof(uint2), cudaMemcpyHostToDevice, st));
  s.timer.begin(LS_PASS_CHILDREN, 0);
  s.launches += launch_chunk_prefix(d_segs, (uint32_t)segs.size(), d_multi, (uint32_t)multi.size(), d_plans, pa.agg,
                                    pa.excl, nbp_max, st);
  launch_children(ca, s.rp, st);
  s.timer.end();
  // the level's counters and next items are final once K2 is done: the
  // host may read them back while the scatters run
  if (ev_children) CK(cudaEventRecord(ev_children, st));
  // The stable scatter is launched only when some item may need it: an item
  // whose decision already makes it order-free (a radix item, or a learned
  // item under REFINE_GLOBAL) is always taken by K3b.
  bool need_stable = false;
  for (uint32_t i = 0; i < nitems && !need_stable; ++i) {
    const Plan& q = dplans[i];
    const bool always_buffered =
        buffered_scatter_candidate(q, s.vb) &&
        (q.decision == LS_DEC_RADIX || (q.decision == LS_DEC_LEARNED && s.rp.recurse == LS_RECURSE_REFINE_GLOBAL));
    need_stable = !always_buffered;
  }
  s.timer.begin(LS_PASS_SCATTER, batch_keys);
  if (need_stable) launch_scatter(pa, s.rp, st);
  launch_scatter_buffered(pa, s.rp, at<BufRun>(s.ws, L.o_bruns), (uint32_t)bruns.size(), st);
  s.timer.end();
  s.launches += 1 + (tiles && need_stable ? 1 : 0) + (bruns.empty() ? 0 : 1);
  CK(cudaGetLastError());

  if (record_root && stats) {
    // keep the root's plan for the sort's final readback (no wait here)
    CK(cudaMemcpyAsync(at<Plan>(s.ws, L.o_rootplan), d_plans, sizeof(Plan), cudaMemcpyDeviceToDevice, st));
    s.root_copied = true;
    s.root_n = its[0].n;
  }
  if (s.seg_decision && level0) {
    // per-segment root decisions (level-0 batches)
    std::vector<Plan> hp(nitems);
    CK(cudaMemcpyAsync(hp.data(), d_plans, nitems * sizeof(Plan), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (uint32_t i = 0; i < nitems; ++i) {
      if (its[i].level != 0 || its[i].segment >= s.nseg) continue;
      s.seg_decision[its[i].segment] = (its[i].n > 0 && !hp[i].mixed) ? LS_DEC_HOMOGENEOUS : hp[i].decision;
    }
  }
  return LS_OK;
}

// Sort / copy the finished spans of one level.
ls_status finish_spans(Sorter& s, const LevelCounters& c) {
  Layout& L = s.lay;
  if (c.n_base_small || c.n_base_mid || c.n_base_large || c.n_fallback) {
    s.timer.begin(LS_PASS_BASE, 0);
    if (c.n_base_small)
      launch_base_small(at<Span>(s.ws, L.o_small), c.n_base_small, s.A, s.Bb, s.VA, s.VBb, s.vb, s.dt, s.st, false);
    if (c.n_base_mid)
      launch_base_small(at<Span>(s.ws, L.o_mid), c.n_base_mid, s.A, s.Bb, s.VA, s.VBb, s.vb, s.dt, s.st, true);
    if (c.n_base_large)
      s.launches += launch_base_large(at<Span>(s.ws, L.o_large), c.n_base_large, s.p->basecase_threshold, s.A, s.Bb,
                                      s.VA, s.VBb, s.vb, s.dt, s.st) - 1;
    if (c.n_fallback)
      launch_fallback(at<Span>(s.ws, L.o_fb), c.n_fallback, s.A, s.Bb, s.VA, s.VBb, s.vb, s.dt, s.st);
    s.timer.end();
  }
  if (c.n_copy) {
    s.timer.begin(LS_PASS_COPY, 0);
    launch_copy_spans(at<Span>(s.ws, L.o_copy), c.n_copy, s.A, s.Bb, s.VA, s.VBb, s.vb, s.st);
    s.timer.end();
  }
  s.launches += (c.n_base_small > 0) + (c.n_base_mid > 0) + (c.n_base_large > 0) + (c.n_copy > 0) + (c.n_fallback > 0);
  CK(cudaGetLastError());
  return LS_OK;
}

// ---- device-planned levels (ls_queue.cu), LS_FLAG_DEVICE_LEVELS
//
// Every level below the root is planned on the device when asked for and no
// bucket below the root can draw a sample: REFINE_GLOBAL (learned items refine the root's
// model, the others take the radix split), keys only (K3b takes every item),
// at most kBufMaxBuckets buckets, a classify mode without the radix
// directory, and a partitioner that is not the splitter tree everywhere.
// Items that do draw a sample (below a splitter tree) come back to the host
// planner.
bool device_levels_ok(const ls_params* p, uint32_t vb) {
  return vb == 0 && (p->flags & LS_FLAG_DEVICE_LEVELS) && p->recurse_model == LS_RECURSE_REFINE_GLOBAL &&
         p->partitioner != LS_PART_SPLITTER && p->classify_mode != LS_CLASSIFY_DIRECTORY &&
         pow2ceil(p->fanout) <= kBufMaxBuckets;
}

constexpr unsigned long long kMaxLoopIter = 1ull << 16;  // batches of one device loop (a safety bound)
constexpr size_t kMaxGraphs = 8;                         // graphs kept per context

// Where the kernels of one batch go: straight to a stream (launched from
// the host), or into the body of the level-loop graph being captured, with
// the optional groups in if nodes (their conditions set by the planner and
// the batch-end kernel).
struct BatchSink {
  cudaStream_t st = nullptr;   // stream of the kernels outside if nodes
  cudaStream_t aux = nullptr;  // capture of if-node bodies (graph only)
  bool graph = false;
  bool ok = true;
  LoopHandles h{};
  // Run fn(stream) under the condition hh (plain launch outside a graph).
  template <class F>
  uint64_t cond(cudaGraphConditionalHandle hh, F fn) {
    if (!graph) return fn(st);
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if (!ok || cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd) != cudaSuccess) {
      ok = false;
      return 0;
    }
    union NodeParams {  // the runtime's parameter union has no default constructor
      cudaGraphNodeParams p;
      unsigned char raw[sizeof(cudaGraphNodeParams)];
      NodeParams() { memset(raw, 0, sizeof raw); }
    } u;
    u.p.type = cudaGraphNodeTypeConditional;
    u.p.conditional.handle = hh;
    u.p.conditional.type = cudaGraphCondTypeIf;
    u.p.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (cudaGraphAddNode(&node, g, deps, nullptr, nd, &u.p) != cudaSuccess ||
        cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess ||
        cudaStreamBeginCaptureToGraph(aux, u.p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      ok = false;
      return 0;
    }
    const uint64_t n = fn(aux);
    cudaGraph_t got = nullptr;
    if (cudaStreamEndCapture(aux, &got) != cudaSuccess) ok = false;
    return n;
  }
};

// The kernels of one device-planned batch: planner, count reset, exact
// pivots, K1, chunk prefixes, K2, K3b, the batch-end kernel and the
// finished spans.  tm: pass timer (nullptr: untimed).  Returns the kernels
// launched (in a graph: the kernels of the body, if nodes included).
uint64_t launch_device_batch(Sorter& s, BatchSink& k, PassTimer* tm) {
  Layout& L = s.lay;
  const ls_params* p = s.p;
  cudaStream_t st = k.st;
  const uint32_t nbp = std::max<uint32_t>(pow2ceil(p->fanout), 1u << kRadixBits);
  BatchDesc* bd = at<BatchDesc>(s.ws, L.o_bdesc);
  QueueState* q = at<QueueState>(s.ws, L.o_queue);
  LevelCounters* ctr = at<LevelCounters>(s.ws, L.o_ctr);
  Item* bitems = at<Item>(s.ws, L.o_bitems);
  Plan* plans = at<Plan>(s.ws, L.o_plans);
  unsigned long long* counts = at<unsigned long long>(s.ws, L.o_counts);
  unsigned long long* cursors = at<unsigned long long>(s.ws, L.o_cursors);
  uint64_t* pivots = at<uint64_t>(s.ws, L.o_pivots);
  DModel* models = at<DModel>(s.ws, L.o_models);
  Leaf* leaves = at<Leaf>(s.ws, L.o_leaves);
  auto tb = [&](int cls) {
    if (tm) tm->begin(cls, 0);
  };
  auto te = [&]() {
    if (tm) tm->end();
  };
  uint64_t nl = 0;

  PlanArgs pg{};
  pg.level = at<Item>(s.ws, L.o_cur);
  pg.next = at<Item>(s.ws, L.o_next);
  pg.bitems = bitems;
  pg.plans = plans;
  pg.hostq = at<Item>(s.ws, L.o_hostq);
  pg.icap = L.icap;
  pg.chunk_plan = at<uint32_t>(s.ws, L.o_chunkplan);
  pg.chunk_cap = L.chunk_cap;
  pg.segs = at<ChunkSeg>(s.ws, L.o_segs);
  pg.seg_cap = L.seg_cap;
  pg.multi = at<uint2>(s.ws, L.o_multi);
  pg.runs = at<BufRun>(s.ws, L.o_bruns);
  pg.run_cap = L.brun_cap;
  pg.reflist = at<uint32_t>(s.ws, L.o_reflist);
  pg.bd = bd;
  pg.q = q;
  pg.ctr = ctr;
  pg.chunk_ctr = at<unsigned long long>(s.ws, L.o_chunkctr);
  pg.status = s.ctx->d_status;
  pg.nbc = L.nbc;
  pg.cells = L.cells;
  pg.slots = 2ull * buffered_scatter_slots();
  tb(LS_PASS_CHILDREN);
  launch_plan_batch(pg, s.rp, k.h, st);
  launch_zero_counts(bd, plans, counts, st);
  te();
  nl += 2;

  tb(LS_PASS_PIVOTS);
  nl += k.cond(k.h.pivots, [&](cudaStream_t cs) {
    launch_learned_pivots(plans, bitems, pg.reflist, kBatchItems, pow2ceil(p->fanout), models, leaves, pivots, s.rp,
                          cs, bd);
    return (uint64_t)1;
  });
  te();

  const bool guess = p->classify_mode == LS_CLASSIFY_AUTO || p->classify_mode == LS_CLASSIFY_GUESS;
  // queue items hold more than T keys, so the direct FP64 classifier (items
  // below 4 B keys) is needed only when T + 1 < 4 B or when it is the mode
  const bool direct = p->classify_mode == LS_CLASSIFY_DIRECT || (uint64_t)p->basecase_threshold + 1 < 4ull * p->fanout;
  if (k.graph && direct != (k.h.has_direct != 0)) k.ok = false;
  PassArgs pa{};
  pa.items = bitems;
  pa.plans = plans;
  pa.nitems = kBatchItems;
  pa.nchunks = L.chunk_cap;  // bounds the grids; the count is the planner's
  pa.keysA = s.A;
  pa.keysB = s.Bb;
  pa.outA = s.A;
  pa.outB = s.Bb;
  pa.pivots = pivots;
  pa.dirs = at<uint16_t>(s.ws, L.o_dirs);
  pa.models = models;
  pa.leaves = leaves;
  pa.fmodels = at<FModel>(s.ws, L.o_fmodels);
  pa.fleaves = at<FLeaf>(s.ws, L.o_fleaves);
  pa.fclamps = at<FClamp>(s.ws, L.o_fclamps);
  pa.aux_bytes = guess ? std::max<uint32_t>(16, L.L * (uint32_t)(sizeof(FLeaf) + sizeof(FClamp))) : 16;
  pa.ids = at<uint16_t>(s.ws, L.o_ids);
  pa.counts = counts;
  pa.cursors = cursors;
  pa.agg = at<uint32_t>(s.ws, L.o_agg);
  pa.excl = at<unsigned long long>(s.ws, L.o_excl);
  pa.chunk_ctr = pg.chunk_ctr;
  pa.chunk_plan = pg.chunk_plan;
  pa.chunk_keys = kChunkKeys;
  pa.status = s.ctx->d_status;
  pa.check_nan = 0;
  pa.nb_pad_max = nbp;
  pa.dir_cells_max = L.cells;
  pa.bd = bd;
  tb(LS_PASS_CLASSIFY);
  auto k1 = [&](uint32_t mask) {
    return [&, mask](cudaStream_t cs) {
      PassArgs a = pa;
      a.cls_mask = mask;
      return (uint64_t)launch_classify_hist(a, s.rp, cs);
    };
  };
  nl += k.cond(k.h.k1, k1(guess ? 1u << CLS_GUESS : p->classify_mode == LS_CLASSIFY_TREE ? 1u << CLS_TREE : 0u));
  if (direct) nl += k.cond(k.h.direct, k1(1u << CLS_DIRECT));
  nl += k.cond(k.h.radix, k1(1u << CLS_RADIX));
  te();

  ChildArgs ca{};
  ca.items = bitems;
  ca.plans = plans;
  ca.nitems = kBatchItems;  // the grid; the count is the planner's
  ca.pivots = pivots;
  ca.counts = counts;
  ca.cursors = cursors;
  ca.next = at<Item>(s.ws, L.o_next);
  ca.next_cap = L.icap;
  ca.base_small = at<Span>(s.ws, L.o_small);
  ca.base_mid = at<Span>(s.ws, L.o_mid);
  ca.base_large = at<Span>(s.ws, L.o_large);
  ca.base_cap = L.base_cap;
  ca.mid_cap = L.mid_cap;
  ca.large_cap = L.large_cap;
  ca.copy = at<Span>(s.ws, L.o_copy);
  ca.copy_cap = L.copy_cap;
  ca.fallback = at<Span>(s.ws, L.o_fb);
  ca.fallback_cap = L.fb_cap;
  ca.ctr = ctr;
  ca.stats = at<DevLevelStats>(s.ws, L.o_stats);
  ca.bd = bd;
  const uint32_t segs_grid = (uint32_t)std::min<uint64_t>(L.seg_cap, 1024);
  tb(LS_PASS_CHILDREN);
  nl += launch_chunk_prefix(pg.segs, segs_grid, pg.multi, 256, plans, pa.agg, pa.excl, nbp, st, bd, 1);
  nl += k.cond(k.h.multi, [&](cudaStream_t cs) {
    return (uint64_t)launch_chunk_prefix(pg.segs, segs_grid, pg.multi, 256, plans, pa.agg, pa.excl, nbp, cs, bd, 2);
  });
  launch_children(ca, s.rp, st);
  te();
  nl += 1;

  tb(LS_PASS_SCATTER);
  launch_scatter_buffered(pa, s.rp, pg.runs, (uint32_t)L.brun_cap, st);
  te();
  launch_batch_end(q, ctr, s.ctx->d_status, k.h, kMaxLoopIter, st);
  nl += 2;

  tb(LS_PASS_BASE);
  auto spans = [&](int which) {
    return [&, which](cudaStream_t cs) {
      return (uint64_t)launch_spans_device(which, ctr, ca.base_small, ca.base_mid, ca.base_large, ca.copy, ca.fallback,
                                           L.base_cap,
                                           p->basecase_threshold, s.A, s.Bb, s.dt, cs);
    };
  };
  nl += k.cond(k.h.small, spans(SPANS_SMALL));
  nl += k.cond(k.h.large, spans(SPANS_LARGE));
  nl += k.cond(k.h.copy, spans(SPANS_COPY));
  nl += k.cond(k.h.fallback, spans(SPANS_FALLBACK));
  te();
  return nl;
}

// What a captured graph depends on: the workspace, the keys, the layout and
// the run parameters (every kernel argument derives from these).
std::vector<uint64_t> graph_key(const Sorter& s) {
  const Layout& L = s.lay;
  const RunParams& r = s.rp;
  uint64_t sr, df, tau;
  memcpy(&sr, &r.sample_rate, 8);
  memcpy(&df, &r.dup_frac, 8);
  memcpy(&tau, &r.tau, 8);
  return {(uint64_t)(uintptr_t)s.ws, (uint64_t)(uintptr_t)s.A, (uint64_t)(uintptr_t)s.ctx->d_status, L.n, L.total,
          L.icap, L.chunk_cap, L.seg_cap, L.brun_cap, L.base_cap, L.mid_cap, L.large_cap, L.copy_cap, L.fb_cap, L.nbc,
          L.cells,
          L.L, r.B, r.bs_max, r.bs_auto, r.T, r.max_depth, r.min_sample, sr, df, tau, r.min_learned_n, r.seed,
          (uint64_t)(uint32_t)r.partitioner, (uint64_t)(uint32_t)r.recurse, (uint64_t)(uint32_t)r.classify_mode,
          (uint64_t)(uint32_t)r.dt, r.tile, r.dir_bits};
}

void drop_graph(ls_graph_entry& e) {
  if (e.exec) cudaGraphExecDestroy(e.exec);
  if (e.graph) cudaGraphDestroy(e.graph);
  e.exec = nullptr;
  e.graph = nullptr;
}

// Build (capture) the graph of the device level loop: a while node whose
// body is one batch.  plain: launch the body's kernels without the
// programmatic-serialization attribute.  Returns false if any step fails
// (the error is cleared; the caller launches the batches from the host).
bool build_graph(Sorter& s, bool plain, ls_graph_entry* out) {
  ls_ctx* ctx = s.ctx;
  if (!ctx->s_cap && cudaStreamCreateWithFlags(&ctx->s_cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  ls_graph_entry e;
  bool ok = cudaGraphCreate(&e.graph, 0) == cudaSuccess;
  cudaGraphConditionalHandle h = 0;
  cudaGraphNode_t node = nullptr;
  union NodeParams {  // the runtime's parameter union has no default constructor
    cudaGraphNodeParams p;
    unsigned char raw[sizeof(cudaGraphNodeParams)];
    NodeParams() { memset(raw, 0, sizeof raw); }
  } npu;
  cudaGraphNodeParams& np = npu.p;
  ok = ok && cudaGraphConditionalHandleCreate(&h, e.graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  if (ok) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    ok = cudaGraphAddNode(&node, e.graph, nullptr, nullptr, 0, &np) == cudaSuccess;
  }
  if (ok && !ctx->s_cap_aux && cudaStreamCreateWithFlags(&ctx->s_cap_aux, cudaStreamNonBlocking) != cudaSuccess)
    ok = false;
  if (ok) {
    cudaGraph_t body = np.conditional.phGraph_out[0];
    BatchSink k;
    k.st = ctx->s_cap;
    k.aux = ctx->s_cap_aux;
    k.graph = true;
    k.h.in_graph = 1;
    k.h.loop = h;
    // every handle must belong to one if node: the direct classifier's only
    // when the batch can use it
    const ls_params* p = s.p;
    k.h.has_direct = p->classify_mode == LS_CLASSIFY_DIRECT || (uint64_t)p->basecase_threshold + 1 < 4ull * p->fanout;
    for (cudaGraphConditionalHandle* c : {&k.h.pivots, &k.h.k1, &k.h.radix, &k.h.multi, &k.h.small, &k.h.large,
                                          &k.h.copy, &k.h.fallback})
      ok = ok && cudaGraphConditionalHandleCreate(c, body, 0, 0) == cudaSuccess;
    if (k.h.has_direct) ok = ok && cudaGraphConditionalHandleCreate(&k.h.direct, body, 0, 0) == cudaSuccess;
    ok = ok && cudaStreamBeginCaptureToGraph(ctx->s_cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) ==
                   cudaSuccess;
    if (ok) {
      const bool was = t_plain_launch;
      t_plain_launch = plain;
      e.body_launches = launch_device_batch(s, k, nullptr);
      t_plain_launch = was;
      cudaGraph_t got = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(ctx->s_cap, &got);
      ok = k.ok && ce == cudaSuccess && cudaGetLastError() == cudaSuccess;
    }
  }
  ok = ok && cudaGraphInstantiate(&e.exec, e.graph, 0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    drop_graph(e);
    return false;
  }
  e.pdl = !plain;
  *out = e;
  return true;
}

// Run the device level loop until the queue is empty; then one readback.
// handed_back: items that draw a sample (for the host planner).
ls_status run_device_levels(Sorter& s, std::vector<Item>* handed_back, bool* overflow, unsigned int* dstat) {
  Layout& L = s.lay;
  ls_ctx* ctx = s.ctx;
  cudaStream_t st = s.st;
  QueueState* q = at<QueueState>(s.ws, L.o_queue);
  BatchDesc* bd = at<BatchDesc>(s.ws, L.o_bdesc);
  CK(cudaMemsetAsync(q, 0, sizeof(QueueState), st));
  ls_graph_entry* ge = nullptr;
  if (!s.timer.on) {
    const std::vector<uint64_t> key = graph_key(s);
    for (ls_graph_entry& e : ctx->graphs)
      if (e.key == key) ge = &e;
    if (!ge) {
      if (ctx->graphs.size() >= kMaxGraphs) {
        size_t old = 0;
        for (size_t i = 1; i < ctx->graphs.size(); ++i)
          if (ctx->graphs[i].last_use < ctx->graphs[old].last_use) old = i;
        drop_graph(ctx->graphs[old]);
        ctx->graphs.erase(ctx->graphs.begin() + (long)old);
      }
      ls_graph_entry e;
      if (build_graph(s, false, &e) || build_graph(s, true, &e)) {
        e.key = key;
        ctx->graphs.push_back(e);
        ge = &ctx->graphs.back();
      }
    }
  }
  uint64_t iters = 0;
  if (ge) {
    ge->last_use = ++ctx->graph_clock;
    CK(cudaGraphLaunch(ge->exec, st));
  } else {
    // launched from the host, one batch at a time (pass timing, or no graph)
    BatchSink k;
    k.st = st;
    for (;;) {
      const size_t r0 = s.timer.recs.size();
      s.launches += launch_device_batch(s, k, s.timer.on ? &s.timer : nullptr);
      QueueState hq;
      BatchDesc hb;
      CK(cudaMemcpyAsync(&hq, q, sizeof hq, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(&hb, bd, sizeof hb, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (size_t i = r0; i < s.timer.recs.size(); ++i)
        if (s.timer.recs[i].cls == LS_PASS_CLASSIFY || s.timer.recs[i].cls == LS_PASS_SCATTER)
          s.timer.recs[i].keys = hb.keys;
      if (!hq.cont) break;
    }
  }
  QueueState hq;
  LevelCounters c;
  CK(cudaMemcpyAsync(&hq, q, sizeof hq, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&c, at<LevelCounters>(s.ws, L.o_ctr), sizeof c, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(dstat, ctx->d_status, sizeof *dstat, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  iters = hq.iter;
  if (ge) s.launches += ge->body_launches * iters;
  s.device_batches += iters;
  s.level_loop = ge ? (ge->pdl ? LS_LOOP_GRAPH_PDL : LS_LOOP_GRAPH) : LS_LOOP_DEVICE;
  *overflow = c.overflow != 0;
  if (hq.err) {
    lsg::set_error_detail("device level loop stopped after %llu batches", (unsigned long long)iters);
    return LS_EDEVICE;
  }
  handed_back->clear();
  const uint64_t nh = std::min<uint64_t>(hq.host_n, L.icap);
  if (nh) {
    handed_back->resize(nh);
    CK(cudaMemcpyAsync(handed_back->data(), at<Item>(s.ws, L.o_hostq), nh * sizeof(Item), cudaMemcpyDeviceToHost,
                       st));
    CK(cudaStreamSynchronize(st));
  }
  return LS_OK;
}

ls_status sort_impl(ls_ctx* ctx, uint64_t* d_keys, const uint64_t* h_off, uint32_t nseg, ls_dtype dtype,
                    const ls_params* p, void* ws, size_t ws_bytes, ls_stats* out_stats, int32_t* seg_dec,
                    cudaStream_t st, void* d_vals = nullptr, uint32_t vb = 0) {
  auto t0 = std::chrono::steady_clock::now();
  if (!ctx || !p || (!d_keys && h_off[nseg] > 0) || (dtype != LS_F64 && dtype != LS_U64)) return LS_EINVAL;
  const ls_params eff = effective_params(ctx, h_off[nseg], nseg, dtype, *p);
  p = &eff;
  ls_status vs = validate_params(p);
  if (vs != LS_OK) return vs;
  for (uint32_t s = 0; s < nseg; ++s)
    if (h_off[s + 1] < h_off[s]) return LS_EINVAL;
  uint64_t n = h_off[nseg];
  for (uint32_t s = 0; s < nseg; ++s)
    if (h_off[s + 1] - h_off[s] >= (1ull << 32)) return LS_EINVAL;
  if (vb != 0 && vb != 4 && vb != 8) return LS_EINVAL;
  if (vb && !d_vals && h_off[nseg] > 0) return LS_EINVAL;
  // keys (and values) must be naturally aligned 64-bit (32-bit) words
  if (reinterpret_cast<uintptr_t>(d_keys) % 8 || (vb && reinterpret_cast<uintptr_t>(d_vals) % vb)) return LS_EINVAL;
  Layout lay = compute_layout(n, nseg, p, vb);
  if (n > 0 && (!ws || ws_bytes < lay.total)) return LS_ENOMEM;
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return LS_EINVAL;
  CK(cudaSetDevice(ctx->device));
  ls_stats local;
  ls_stats* stats = out_stats ? out_stats : &local;
  memset(stats, 0, sizeof *stats);
  stats->root_decision = LS_DEC_NONE;
  if (seg_dec)
    for (uint32_t s = 0; s < nseg; ++s) seg_dec[s] = LS_DEC_NONE;
  if (n == 0) return LS_OK;

  Sorter s;
  s.ctx = ctx;
  s.p = p;
  s.dt = dtype;
  s.rp = make_rp(p, dtype);
  s.lay = lay;
  s.ws = ws;
  s.st = st;
  s.A = d_keys;
  s.Bb = at<uint64_t>(ws, lay.o_buf);
  s.VA = d_vals;
  s.VBb = vb ? static_cast<void*>(at<unsigned char>(ws, lay.o_vbuf)) : nullptr;
  s.vb = vb;
  s.seg_decision = seg_dec;
  s.nseg = nseg;
  s.timer.on = (p->flags & LS_FLAG_TIME_PASSES) != 0;
  s.timer.st = st;
  for (int m = (int)lay.mcap - 1; m >= 0; --m) s.model_free.push_back(m);

  CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned int), st));
  DevLevelStats* d_stats = at<DevLevelStats>(ws, lay.o_stats);
  LevelCounters* d_ctr = at<LevelCounters>(ws, lay.o_ctr);
  CK(cudaMemsetAsync(d_stats, 0, LS_MAX_LEVELS * sizeof(DevLevelStats), st));

  // level 0: one root item per segment; small roots straight to the base case
  uint64_t olo, ohi;
  ord_range(dtype, &olo, &ohi);
  std::vector<Item> items;
  std::vector<Span> small, mid, large;
  ls_level_stats root_base;
  memset(&root_base, 0, sizeof root_base);
  for (uint32_t sgi = 0; sgi < nseg; ++sgi) {
    uint64_t len = h_off[sgi + 1] - h_off[sgi];
    if (len <= 1) continue;
    if (len <= p->basecase_threshold) {
      Span sp{h_off[sgi], (uint32_t)len, 0u};
      (len <= kWarpSmallMax ? small : len <= kWarpSortMax ? mid : large).push_back(sp);
      root_base.base_items += 1;
      root_base.base_keys += len;
      continue;
    }
    Item it;
    memset(&it, 0, sizeof it);
    it.lo = h_off[sgi];
    it.n = len;
    it.segment = sgi;
    it.level = 0;
    it.kind = KIND_FRESH;
    it.model = -1;
    it.buf = 0;
    it.ord_lo = olo;
    it.ord_hi = ohi;
    items.push_back(it);
  }
  if (!small.empty() || !mid.empty() || !large.empty()) {
    CK(cudaMemcpyAsync(at<Span>(ws, lay.o_small), small.data(), small.size() * sizeof(Span), cudaMemcpyHostToDevice,
                       st));
    CK(cudaMemcpyAsync(at<Span>(ws, lay.o_mid), mid.data(), mid.size() * sizeof(Span), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(at<Span>(ws, lay.o_large), large.data(), large.size() * sizeof(Span), cudaMemcpyHostToDevice,
                       st));
    LevelCounters c;
    memset(&c, 0, sizeof c);
    c.n_base_small = small.size();
    c.n_base_mid = mid.size();
    c.n_base_large = large.size();
    ls_status r = finish_spans(s, c);
    if (r != LS_OK) return r;
    CK(cudaStreamSynchronize(st));
  }

  if (!ctx->s_read) CK(cudaStreamCreateWithFlags(&ctx->s_read, cudaStreamNonBlocking));
  if (!ctx->ev_children) CK(cudaEventCreateWithFlags(&ctx->ev_children, cudaEventDisableTiming));
  bool first = true;
  uint32_t level = 0;
  ls_status result = LS_OK;
  const bool dev_levels = device_levels_ok(p, vb);
  while (!items.empty()) {
    CK(cudaMemsetAsync(d_ctr, 0, sizeof(LevelCounters), st));
    // items of this level are replaced by the device list of the next level,
    // so keep a host copy and upload per batch into the "current" slot
    std::vector<Item> cur;
    cur.swap(items);
    for (size_t b0 = 0; b0 < cur.size();) {
      // batch by item count and by sample capacity
      size_t b1 = b0;
      uint64_t sacc = 0;
      while (b1 < cur.size() && b1 - b0 < kBatchItems) {
        const Item& it = cur[b1];
        bool fr = it.kind != KIND_REFINE || pow_exact(p->fanout, it.mk + 1u) > kRefineLimit;
        uint64_t S = fr ? sample_size(it.n, p) : 0;
        if (b1 > b0 && sacc + S > lay.scap) break;
        sacc += S;
        ++b1;
      }
      bool record = first && b0 == 0 && out_stats && cur[0].segment == 0;
      ls_status r = run_batch(s, cur.data() + b0, (uint32_t)(b1 - b0), level == 0, record, stats,
                              b1 == cur.size() ? ctx->ev_children : nullptr);
      if (r != LS_OK) return r;
      first = false;
      b0 = b1;
    }
    if (dev_levels) {
      // the next level's items and this level's finished spans stay on the
      // device: the device loop plans and sorts everything below; items
      // that draw a sample come back and are planned here
      bool ovf = false;
      unsigned int dstat = 0;
      ls_status r = run_device_levels(s, &items, &ovf, &dstat);
      if (r != LS_OK) return r;
      if (ovf) {
        lsg::set_error_detail("workspace list capacity exceeded below level %u", level);
        return LS_ENOMEM;
      }
      if (dstat != 0) {
        result = (ls_status)dstat;
        break;
      }
      // every item of the device queue is done: no model is referenced
      s.model_free.clear();
      for (int m = (int)lay.mcap - 1; m >= 0; --m) s.model_free.push_back(m);
      ++level;
      continue;
    }
    // one readback per level: counters, device status and the first
    // kPinItems next-level items (K2 wrote them), into page-locked memory,
    // on the side stream once the level's last K2 is done (the scatters
    // keep the GPU busy meanwhile; the status of the scatters themselves is
    // read with the final statistics)
    LevelCounters c;
    unsigned int dstat = 0;
    const uint64_t pin_items = std::min<uint64_t>(kPinItems, lay.icap);
    {
      const size_t need = sizeof(LevelCounters) + 16 + pin_items * sizeof(Item);
      if (ctx->h_pin_bytes < need) {
        if (ctx->h_pin) cudaFreeHost(ctx->h_pin);
        ctx->h_pin = nullptr;
        ctx->h_pin_bytes = 0;
        CK(cudaHostAlloc(&ctx->h_pin, need, cudaHostAllocDefault));
        ctx->h_pin_bytes = need;
      }
      char* hp = static_cast<char*>(ctx->h_pin);
      cudaStream_t rs = ctx->s_read;
      CK(cudaStreamWaitEvent(rs, ctx->ev_children, 0));
      CK(cudaMemcpyAsync(hp, d_ctr, sizeof(LevelCounters), cudaMemcpyDeviceToHost, rs));
      CK(cudaMemcpyAsync(hp + sizeof(LevelCounters), ctx->d_status, sizeof dstat, cudaMemcpyDeviceToHost, rs));
      CK(cudaMemcpyAsync(hp + sizeof(LevelCounters) + 16, at<Item>(ws, lay.o_next), pin_items * sizeof(Item),
                         cudaMemcpyDeviceToHost, rs));
      CK(cudaStreamSynchronize(rs));
      memcpy(&c, hp, sizeof c);
      memcpy(&dstat, hp + sizeof(LevelCounters), sizeof dstat);
    }
    if (c.overflow) {
      lsg::set_error_detail("workspace list capacity exceeded at level %u", level);
      return LS_ENOMEM;
    }
    if (dstat != 0) {
      result = (ls_status)dstat;
      break;
    }
    // the next level's items are complete (K2 wrote them): read them back
    // before the base case is launched, so the host plans the next level
    // while the GPU sorts this level's finished spans
    if (c.n_next) {
      items.resize(c.n_next);
      const uint64_t first = std::min<uint64_t>(c.n_next, pin_items);
      memcpy(items.data(), static_cast<char*>(ctx->h_pin) + sizeof(LevelCounters) + 16, first * sizeof(Item));
      if (c.n_next > first) {
        CK(cudaMemcpyAsync(items.data() + first, at<Item>(ws, lay.o_next) + first, (c.n_next - first) * sizeof(Item),
                           cudaMemcpyDeviceToHost, ctx->s_read));
        CK(cudaStreamSynchronize(ctx->s_read));
      }
    }
    ls_status r = finish_spans(s, c);
    if (r != LS_OK) return r;
    if (c.n_next) {
      // keep only models still referenced by refine items
      std::vector<uint8_t> live(lay.mcap, 0);
      for (const Item& it : items)
        if (it.kind == KIND_REFINE && it.model >= 0) live[it.model] = 1;
      s.model_free.clear();
      for (int m = (int)lay.mcap - 1; m >= 0; --m)
        if (!live[m]) s.model_free.push_back(m);
    }
    ++level;
  }
  // statistics
  std::vector<DevLevelStats> hs(LS_MAX_LEVELS);
  CK(cudaMemcpyAsync(hs.data(), d_stats, LS_MAX_LEVELS * sizeof(DevLevelStats), cudaMemcpyDeviceToHost, st));
  Plan rp0;
  if (s.root_copied) CK(cudaMemcpyAsync(&rp0, at<Plan>(ws, lay.o_rootplan), sizeof(Plan), cudaMemcpyDeviceToHost, st));
  unsigned int fstat = 0;  // the last level's scatters and base cases report here
  CK(cudaMemcpyAsync(&fstat, ctx->d_status, sizeof fstat, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (result == LS_OK && fstat != 0) result = (ls_status)fstat;
  if (s.root_copied) {
    if (s.root_n > 0 && !rp0.mixed) {
      // homogeneity is checked before any model is built (Sec. 2.2): the
      // sample the device drew speculatively is not part of the decision
      stats->root_decision = LS_DEC_HOMOGENEOUS;
    } else {
      stats->root_decision = rp0.decision;
      stats->root_nbuckets = rp0.nb;
      stats->root_sample_size = rp0.S;
      stats->root_dups = rp0.dups;
      stats->root_imbalance_max = rp0.imb;
    }
  }
  memcpy(stats->level, hs.data(), sizeof(stats->level));
  stats->level[0].base_items += root_base.base_items;
  stats->level[0].base_keys += root_base.base_keys;
  uint32_t used = 0;
  for (uint32_t l = 0; l < LS_MAX_LEVELS; ++l) {
    const ls_level_stats& q = stats->level[l];
    if (q.items || q.base_items || q.homogeneous || q.fallback_items) used = l + 1;
  }
  stats->levels_used = used;
  s.timer.collect(stats);
  for (uint32_t l = 0; l < LS_MAX_LEVELS; ++l)
    stats->pass[LS_PASS_BASE].keys += stats->level[l].base_keys + stats->level[l].fallback_keys;
  stats->status = result;
  stats->kernel_launches = s.launches;
  stats->device_batches = s.device_batches;
  stats->level_loop = s.level_loop;
  ctx->launches += s.launches;
  stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return result;
}

ls_status ensure_cache(ls_ctx* ctx, size_t bytes) {
  if (ctx->d_cache_bytes >= bytes) return LS_OK;
  if (ctx->d_cache) cudaFree(ctx->d_cache);
  ctx->d_cache = nullptr;
  ctx->d_cache_bytes = 0;
  if (cudaMalloc(&ctx->d_cache, bytes) != cudaSuccess) return LS_ENOMEM;
  ctx->d_cache_bytes = bytes;
  return LS_OK;
}

// Host model <-> device model (one slot).
void model_to_device_layout(const ls_model* m, DModel* dm, std::vector<Leaf>& lv) {
  memset(dm, 0, sizeof *dm);
  dm->xmin = m->xmin;
  dm->xmax = m->xmax;
  dm->rx0 = m->root_x0;
  dm->ra = m->root_a;
  dm->rb = m->root_b;
  dm->L = m->L;
  dm->S = m->S;
  dm->leaf_off = 0;
  dm->ok = 1;
  lv.resize(m->L);
  for (uint32_t i = 0; i < m->L; ++i) lv[i] = Leaf{m->leaf_x0[i], m->leaf_a[i], m->leaf_b[i], m->leaf_lo[i], m->leaf_hi[i]};
}

}  // namespace

// =============================================================== C ABI

extern "C" {

void ls_params_default(ls_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->fanout = 1000;
  p->splitter_fanout = 1024;
  p->basecase_threshold = 16;
  p->max_depth = 16;
  p->min_sample = 256;
  p->auto_splitter_fanout = 256;
  p->sample_rate = 0.01;
  p->dup_frac = 0.10;
  p->imbalance_tau = 8.0;
  p->min_learned_n = 100000;
  p->seed = 0x5EEDull;
  p->partitioner = LS_PART_AUTO;
  p->recurse_model = LS_RECURSE_REFINE_GLOBAL;
  p->classify_mode = LS_CLASSIFY_AUTO;
  p->tile_keys = 0;
}

ls_status ls_create(ls_ctx** out, int device) {
  if (!out) return LS_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return LS_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return LS_ECUDA;
  ls_ctx* c = new (std::nothrow) ls_ctx();
  if (!c) return LS_ENOMEM;
  c->device = device;
  if (cudaMalloc(&c->d_status, sizeof(unsigned int)) != cudaSuccess) {
    delete c;
    return LS_ECUDA;
  }
  cudaMemset(c->d_status, 0, sizeof(unsigned int));
  *out = c;
  return LS_OK;
}

void ls_destroy(ls_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_cache) cudaFree(ctx->d_cache);
  for (ls_graph_entry& e : ctx->graphs) drop_graph(e);
  for (cudaStream_t s : {ctx->s_sort, ctx->s_in, ctx->s_out, ctx->s_read, ctx->s_cap, ctx->s_cap_aux})
    if (s) cudaStreamDestroy(s);
  if (ctx->ev_children) cudaEventDestroy(ctx->ev_children);
  if (ctx->h_pin) cudaFreeHost(ctx->h_pin);
  delete ctx;
}

ls_status ls_workspace_size(ls_ctx* ctx, uint64_t n, uint32_t nseg, ls_dtype dtype, const ls_params* p,
                            size_t* bytes) {
  if (!bytes || !p || (dtype != LS_F64 && dtype != LS_U64)) return LS_EINVAL;
  const ls_params eff = effective_params(ctx, n, nseg ? nseg : 1, dtype, *p);
  ls_status vs = validate_params(&eff);
  if (vs != LS_OK) return vs;
  *bytes = compute_layout(n, nseg ? nseg : 1, &eff).total;
  return LS_OK;
}

ls_status ls_sort(ls_ctx* ctx, void* d_keys, uint64_t n, ls_dtype dtype, const ls_params* p, void* d_workspace,
                  size_t ws_bytes, ls_stats* out_stats, ls_stream_t stream) {
  uint64_t off[2] = {0, n};
  return sort_impl(ctx, static_cast<uint64_t*>(d_keys), off, 1, dtype, p, d_workspace, ws_bytes, out_stats,
                   nullptr, static_cast<cudaStream_t>(stream));
}

ls_status ls_sort_segmented(ls_ctx* ctx, void* d_keys, const uint64_t* h_offsets, uint32_t nseg, ls_dtype dtype,
                            const ls_params* p, void* d_workspace, size_t ws_bytes, ls_stats* out_stats,
                            int32_t* h_seg_decision, ls_stream_t stream) {
  if (!h_offsets || nseg == 0) return LS_EINVAL;
  return sort_impl(ctx, static_cast<uint64_t*>(d_keys), h_offsets, nseg, dtype, p, d_workspace, ws_bytes,
                   out_stats, h_seg_decision, static_cast<cudaStream_t>(stream));
}

ls_status ls_workspace_size_pairs(ls_ctx* ctx, uint64_t n, uint32_t val_bytes, ls_dtype dtype, const ls_params* p,
                                  size_t* bytes) {
  if (!bytes || !p || (dtype != LS_F64 && dtype != LS_U64) || (val_bytes != 4 && val_bytes != 8)) return LS_EINVAL;
  const ls_params eff = effective_params(ctx, n, 1, dtype, *p);
  ls_status vs = validate_params(&eff);
  if (vs != LS_OK) return vs;
  *bytes = compute_layout(n, 1, &eff, val_bytes).total;
  return LS_OK;
}

ls_status ls_sort_pairs(ls_ctx* ctx, void* d_keys, void* d_vals, uint32_t val_bytes, uint64_t n, ls_dtype dtype,
                        const ls_params* p, void* d_workspace, size_t ws_bytes, ls_stats* out_stats,
                        ls_stream_t stream) {
  if (val_bytes != 4 && val_bytes != 8) return LS_EINVAL;
  uint64_t off[2] = {0, n};
  return sort_impl(ctx, static_cast<uint64_t*>(d_keys), off, 1, dtype, p, d_workspace, ws_bytes, out_stats, nullptr,
                   static_cast<cudaStream_t>(stream), d_vals, val_bytes);
}

ls_status ls_sort_host(ls_ctx* ctx, void* h_keys, uint64_t n, ls_dtype dtype, const ls_params* p,
                       ls_stats* out_stats) {
  if (!ctx || (!h_keys && n)) return LS_EINVAL;
  size_t wsb = 0;
  ls_status vs = ls_workspace_size(ctx, n, 1, dtype, p, &wsb);  // tuned parameters included
  if (vs != LS_OK) return vs;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LS_ECUDA;
  size_t keyb = up(n * 8);
  ls_status r = ensure_cache(ctx, keyb + wsb + kAlign);
  if (r != LS_OK) return r;
  char* base = static_cast<char*>(ctx->d_cache);
  void* d_keys = base;
  void* d_ws = base + keyb;
  if (cudaMemcpy(d_keys, h_keys, n * 8, cudaMemcpyHostToDevice) != cudaSuccess) return LS_ECUDA;
  r = ls_sort(ctx, d_keys, n, dtype, p, d_ws, wsb, out_stats, nullptr);
  if (r != LS_OK) return r;
  if (cudaMemcpy(h_keys, d_keys, n * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return LS_ECUDA;
  return LS_OK;
}

ls_status ls_sort_host_batch(ls_ctx* ctx, void* const* h_keys, const uint64_t* n, uint32_t count, ls_dtype dtype,
                             const ls_params* p, ls_stats* out_stats) {
  if (!ctx || (count && (!h_keys || !n))) return LS_EINVAL;
  uint64_t nmax = 0;
  for (uint32_t i = 0; i < count; ++i) {
    if (!h_keys[i] && n[i]) return LS_EINVAL;
    nmax = std::max(nmax, n[i]);
  }
  size_t wsb = 0;
  ls_status vs = ls_workspace_size(ctx, nmax, 1, dtype, p, &wsb);  // grows with n: fits every array
  if (vs != LS_OK) return vs;
  if (count == 0) return LS_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LS_ECUDA;
  for (cudaStream_t* s : {&ctx->s_sort, &ctx->s_in, &ctx->s_out})
    if (!*s && cudaStreamCreateWithFlags(s, cudaStreamNonBlocking) != cudaSuccess) return LS_ECUDA;
  // three key buffers: array i sorts in slot i % 3 while i + 1 arrives and
  // i - 1 leaves
  const uint32_t nb = count < 3 ? count : 3;
  const size_t keyb = up(nmax * 8);
  ls_status r = ensure_cache(ctx, nb * keyb + wsb + kAlign);
  if (r != LS_OK) return r;
  char* base = static_cast<char*>(ctx->d_cache);
  void* ws = base + nb * keyb;
  cudaEvent_t ev[3][3];  // [slot][in, sorted, out]
  int made = 0;
  for (uint32_t q = 0; q < nb && r == LS_OK; ++q)
    for (int k = 0; k < 3 && r == LS_OK; ++k) {
      if (cudaEventCreateWithFlags(&ev[q][k], cudaEventDisableTiming) != cudaSuccess) r = LS_ECUDA;
      else ++made;
    }
  // big transfers go in pieces, so that the sort's own small per-level
  // copies (plans, counters) do not queue behind a whole array on the copy
  // engines
  static constexpr size_t kPiece = size_t(32) << 20;
  auto copy = [](void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t st) -> bool {
    for (size_t o = 0; o < bytes; o += kPiece)
      if (cudaMemcpyAsync(static_cast<char*>(dst) + o, static_cast<const char*>(src) + o,
                          std::min(kPiece, bytes - o), kind, st) != cudaSuccess)
        return false;
    return true;
  };
  // page-locked arrays mapped into the device's address space move through a
  // small copy kernel over the host link, which leaves the copy engines to
  // the sorts' own small copies; other arrays go through the engines
  std::vector<void*> mapped(count, nullptr);
  for (uint32_t i = 0; i < count; ++i) {
    cudaPointerAttributes at;
    if (h_keys[i] && cudaPointerGetAttributes(&at, h_keys[i]) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer)
      mapped[i] = at.devicePointer;
    else
      cudaGetLastError();  // clear a lookup failure of an unregistered pointer
  }
  auto h2d = [&](uint32_t i) -> bool {
    const uint32_t q = i % nb;
    if (i >= nb && cudaStreamWaitEvent(ctx->s_in, ev[q][2], 0) != cudaSuccess) return false;
    if (mapped[i]) {
      launch_link_copy(mapped[i], base + q * keyb, n[i] * 8, ctx->s_in);
      if (cudaGetLastError() != cudaSuccess) return false;
    } else if (!copy(base + q * keyb, h_keys[i], n[i] * 8, cudaMemcpyHostToDevice, ctx->s_in)) {
      return false;
    }
    return cudaEventRecord(ev[q][0], ctx->s_in) == cudaSuccess;
  };
  if (r == LS_OK && !h2d(0)) r = LS_ECUDA;
  for (uint32_t i = 0; i < count && r == LS_OK; ++i) {
    if (i + 1 < count && !h2d(i + 1)) {
      r = LS_ECUDA;
      break;
    }
    const uint32_t q = i % nb;
    if (cudaStreamWaitEvent(ctx->s_sort, ev[q][0], 0) != cudaSuccess) {
      r = LS_ECUDA;
      break;
    }
    r = ls_sort(ctx, base + q * keyb, n[i], dtype, p, ws, wsb, out_stats ? &out_stats[i] : nullptr, ctx->s_sort);
    if (r != LS_OK) break;
    if (cudaEventRecord(ev[q][1], ctx->s_sort) != cudaSuccess ||
        cudaStreamWaitEvent(ctx->s_out, ev[q][1], 0) != cudaSuccess ||
        (mapped[i] ? (launch_link_copy(base + q * keyb, mapped[i], n[i] * 8, ctx->s_out),
                      cudaGetLastError() != cudaSuccess)
                   : !copy(h_keys[i], base + q * keyb, n[i] * 8, cudaMemcpyDeviceToHost, ctx->s_out)) ||
        cudaEventRecord(ev[q][2], ctx->s_out) != cudaSuccess)
      r = LS_ECUDA;
  }
  // drain every stream before the buffers can be reused or the call returns
  for (cudaStream_t s : {ctx->s_in, ctx->s_sort, ctx->s_out})
    if (cudaStreamSynchronize(s) != cudaSuccess && r == LS_OK) r = LS_ECUDA;
  for (uint32_t q = 0; q < nb; ++q)
    for (int k = 0; k < 3; ++k)
      if (made-- > 0) cudaEventDestroy(ev[q][k]);
  return r;
}

ls_status ls_fit(ls_ctx* ctx, const void* d_keys, uint64_t n, ls_dtype dtype, const ls_params* p,
                 ls_model* out_model, ls_stats* out_stats, void* d_sorted_sample, ls_stream_t stream) {
  if (!ctx || !d_keys || n < 2 || !out_model || (dtype != LS_F64 && dtype != LS_U64)) return LS_EINVAL;
  ls_status vs = validate_params(p);
  if (vs != LS_OK) return vs;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LS_ECUDA;
  // a one-item "sort" workspace is enough for the fresh-item pipeline; the
  // partition passes are not run
  ls_params q = *p;
  if (q.partitioner == LS_PART_SPLITTER) q.partitioner = LS_PART_LEARNED;  // fit regardless
  Layout lay = compute_layout(n, 1, &q);
  ls_status r = ensure_cache(ctx, lay.total + kAlign);
  if (r != LS_OK) return r;
  void* ws = ctx->d_cache;
  Sorter s;
  s.ctx = ctx;
  s.p = &q;
  s.dt = dtype;
  s.rp = make_rp(&q, dtype);
  s.lay = lay;
  s.ws = ws;
  s.st = st;
  s.A = static_cast<uint64_t*>(const_cast<void*>(d_keys));
  s.Bb = at<uint64_t>(ws, lay.o_buf);
  s.model_free.push_back(0);
  // Run only the fresh pipeline of the root: reuse run_batch's planning by
  // hand (no partition passes).
  Item it;
  memset(&it, 0, sizeof it);
  it.n = n;
  it.kind = KIND_FRESH;
  it.model = -1;
  ord_range(dtype, &it.ord_lo, &it.ord_hi);
  uint64_t S = sample_size(n, &q);
  Plan pl;
  memset(&pl, 0, sizeof pl);
  pl.S = (uint32_t)S;
  pl.fresh = 1;
  pl.want = 1;
  pl.model = 0;
  pl.P = (double)q.fanout;
  pl.nb_pad = pow2ceil(q.fanout);
  pl.mixed = 0;
  Item* d_items = at<Item>(ws, lay.o_cur);
  Plan* d_plans = at<Plan>(ws, lay.o_plans);
  uint64_t* misc = at<uint64_t>(ws, lay.o_misc);
  const size_t M = kBatchItems + 8;
  uint32_t zero = 0;
  uint64_t pre[2] = {0, S};
  uint64_t rcp[2] = {0, (S + kChunk - 1) / kChunk};
  uint64_t scp[2] = {0, (S + kSortChunk - 1) / kSortChunk};
  CK(cudaMemcpyAsync(d_items, &it, sizeof it, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_plans, &pl, sizeof pl, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(misc, &zero, 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(misc + M, pre, 16, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(misc + 2 * M, &zero, 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(misc + 3 * M, pre, 16, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(misc + 4 * M, rcp, 16, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(misc + 5 * M, pre, 16, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(misc + 6 * M, scp, 16, cudaMemcpyHostToDevice, st));
  FreshArgs f;
  f.items = d_items;
  f.plans = d_plans;
  f.fresh = reinterpret_cast<uint32_t*>(misc);
  f.samp_prefix = misc + M;
  f.nfresh = 1;
  f.total_samples = S;
  f.keysA = s.A;
  f.keysB = s.Bb;
  uint64_t* samp0 = at<uint64_t>(ws, lay.o_samp0);
  uint64_t* samp1 = at<uint64_t>(ws, lay.o_samp1);
  launch_sample_gather(f, s.rp, samp0, st);
  const uint64_t* sorted = segmented_sort_u64(samp0, samp1, misc + 5 * M, misc + 6 * M, 1, scp[1], S, st,
                                              &s.launches);
  launch_dups(f, sorted, st);
  FitArgs fa{};
  fa.plans = d_plans;
  fa.items = d_items;
  fa.cand = reinterpret_cast<uint32_t*>(misc + 2 * M);
  fa.cand_soff = misc + 3 * M;
  fa.nbp_max = pow2ceil(q.fanout);
  fa.rchunk_prefix = misc + 4 * M;
  fa.ncand = 1;
  fa.total_rchunks = rcp[1];
  fa.total_cand_samples = S;
  fa.lchunk_bound = S / kChunk + lay.L + 8;
  fa.samp = sorted;
  fa.models = at<DModel>(ws, lay.o_models);
  fa.leaves = at<Leaf>(ws, lay.o_leaves);
  fa.L = lay.L;
  fa.rpart = at<double>(ws, lay.o_rpart);
  fa.leaf_start = at<uint32_t>(ws, lay.o_lstart);
  fa.lchunk_cnt = at<uint64_t>(ws, lay.o_lcnt);
  fa.lchunk_prefix = at<uint64_t>(ws, lay.o_lpre);
  fa.scan_tmp = at<uint64_t>(ws, lay.o_stmp);
  fa.scan_tmp_elems = lay.stmp_elems;
  fa.lpart = at<double>(ws, lay.o_lpart);
  fa.leaf_of = at<uint32_t>(ws, lay.o_leafof);
  fa.leaf_cnt = at<uint32_t>(ws, lay.o_leafcnt);
  fa.fmodels = at<FModel>(ws, lay.o_fmodels);
  fa.fleaves = at<FLeaf>(ws, lay.o_fleaves);
  fa.fclamps = at<FClamp>(ws, lay.o_fclamps);
  launch_fit(fa, s.rp, st, &s.launches);
  uint64_t* pivots = at<uint64_t>(ws, lay.o_pivots);
  unsigned long long* counts = at<unsigned long long>(ws, lay.o_counts);
  CK(cudaMemsetAsync(counts, 0, (size_t)lay.nbc * 8, st));
  launch_learned_pivots(d_plans, d_items, fa.cand, 1, pow2ceil(q.fanout), fa.models, fa.leaves, pivots, s.rp, st);
  launch_imbalance(fa, pivots, counts, s.rp, st, &s.launches);
  ls_params q2 = *p;  // decision with the caller's partitioner
  RunParams rp2 = make_rp(&q2, dtype);
  launch_decide(f, fa.models, rp2, st);
  CK(cudaGetLastError());
  // copy out
  DModel dm;
  std::vector<Leaf> lv(lay.L);
  std::vector<uint32_t> lc(lay.L);
  Plan hp;
  CK(cudaMemcpyAsync(&dm, fa.models, sizeof dm, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(lv.data(), fa.leaves, lay.L * sizeof(Leaf), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(lc.data(), fa.leaf_cnt, lay.L * 4, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&hp, d_plans, sizeof hp, cudaMemcpyDeviceToHost, st));
  if (d_sorted_sample) {
    // ord -> key bits on the host side of the copy is not possible on device
    // memory directly; copy through a host vector
    std::vector<uint64_t> hs(S);
    CK(cudaMemcpyAsync(hs.data(), sorted, S * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (auto& v : hs) v = unord(v, dtype);
    CK(cudaMemcpyAsync(d_sorted_sample, hs.data(), S * 8, cudaMemcpyHostToDevice, st));
  }
  CK(cudaStreamSynchronize(st));
  memset(out_model, 0, sizeof *out_model);
  out_model->L = dm.L;
  out_model->S = dm.S;
  out_model->xmin = dm.xmin;
  out_model->xmax = dm.xmax;
  out_model->root_x0 = dm.rx0;
  out_model->root_a = dm.ra;
  out_model->root_b = dm.rb;
  for (uint32_t i = 0; i < lay.L; ++i) {
    out_model->leaf_x0[i] = lv[i].x0;
    out_model->leaf_a[i] = lv[i].a;
    out_model->leaf_b[i] = lv[i].b;
    out_model->leaf_lo[i] = lv[i].lo;
    out_model->leaf_hi[i] = lv[i].hi;
    out_model->leaf_count[i] = lc[i];
  }
  if (out_stats) {
    memset(out_stats, 0, sizeof *out_stats);
    out_stats->root_sample_size = S;
    out_stats->root_dups = hp.dups;
    out_stats->root_imbalance_max = hp.imb;
    out_stats->root_decision = hp.decision == LS_DEC_LEARNED ? LS_DEC_LEARNED : LS_DEC_SPLITTER;
    out_stats->status = dm.ok ? LS_OK : LS_EDEVICE;
  }
  return LS_OK;
}

ls_status ls_classify(ls_ctx* ctx, const ls_model* model, const void* d_keys, uint64_t n, ls_dtype dtype, uint32_t k,
                      uint64_t g, int32_t mode, uint32_t* d_ids, uint64_t* d_hist, ls_stream_t stream) {
  if (!ctx || !model || (!d_keys && n) || (dtype != LS_F64 && dtype != LS_U64)) return LS_EINVAL;
  if (model->L < 2 || model->L > LS_MAX_FANOUT || mode < 0 || mode > 4) return LS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (k >= 50) return LS_EINVAL;  // B >= 2: B^(k+1) > 2^50 (and k + 1 cannot wrap)
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LS_ECUDA;
  uint32_t B = model->L;
  double P = pow_exact(B, k + 1);
  if (P > kRefineLimit) return LS_EINVAL;
  double Bg = (double)((uint64_t)B * g);
  uint32_t nbp = pow2ceil(B);
  uint32_t cells = 1u << kDirBits;
  size_t need = up(sizeof(DModel)) + up(B * sizeof(Leaf)) + up(sizeof(Item)) + up(sizeof(Plan)) + up(nbp * 8) +
                up((cells + 1) * 2) + up(8) + up(sizeof(FModel)) + up(B * sizeof(FLeaf)) + up(8);
  ls_status r = ensure_cache(ctx, need + kAlign);
  if (r != LS_OK) return r;
  char* b = static_cast<char*>(ctx->d_cache);
  DModel* d_m = reinterpret_cast<DModel*>(b);
  b += up(sizeof(DModel));
  Leaf* d_l = reinterpret_cast<Leaf*>(b);
  b += up(B * sizeof(Leaf));
  Item* d_it = reinterpret_cast<Item*>(b);
  b += up(sizeof(Item));
  Plan* d_pl = reinterpret_cast<Plan*>(b);
  b += up(sizeof(Plan));
  uint64_t* d_piv = reinterpret_cast<uint64_t*>(b);
  b += up(nbp * 8);
  uint16_t* d_dir = reinterpret_cast<uint16_t*>(b);
  b += up((cells + 1) * 2);
  uint32_t* d_list = reinterpret_cast<uint32_t*>(b);
  b += up(8);
  FModel* d_fm = reinterpret_cast<FModel*>(b);
  b += up(sizeof(FModel));
  FLeaf* d_fl = reinterpret_cast<FLeaf*>(b);
  b += up(B * sizeof(FLeaf));
  int32_t* d_slot = reinterpret_cast<int32_t*>(b);
  DModel dm;
  std::vector<Leaf> lv;
  model_to_device_layout(model, &dm, lv);
  CK(cudaMemcpyAsync(d_m, &dm, sizeof dm, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_l, lv.data(), B * sizeof(Leaf), cudaMemcpyHostToDevice, st));
  if (d_hist) CK(cudaMemsetAsync(d_hist, 0, B * 8, st));
  if (mode == LS_CLASSIFY_DIRECT) {
    launch_direct_classify(d_m, d_l, static_cast<const uint64_t*>(d_keys), n, dtype, P, Bg, B, d_ids,
                           reinterpret_cast<unsigned long long*>(d_hist), st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return LS_OK;
  }
  Item it;
  memset(&it, 0, sizeof it);
  ord_range(dtype, &it.ord_lo, &it.ord_hi);
  it.n = n;
  it.kind = KIND_REFINE;
  Plan pl;
  memset(&pl, 0, sizeof pl);
  pl.model = 0;
  pl.P = P;
  pl.Bg = Bg;
  pl.nb = B;
  pl.nb_pad = nbp;
  pl.decision = LS_DEC_LEARNED;
  pl.cls = (mode == LS_CLASSIFY_TREE) ? CLS_TREE : (mode == LS_CLASSIFY_GUESS) ? CLS_GUESS : CLS_DIR;
  uint32_t zero = 0;
  CK(cudaMemcpyAsync(d_it, &it, sizeof it, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_pl, &pl, sizeof pl, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_list, &zero, 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_slot, &zero, 4, cudaMemcpyHostToDevice, st));
  RunParams rp;
  memset(&rp, 0, sizeof rp);
  rp.B = B;
  rp.dt = dtype;
  launch_learned_pivots(d_pl, d_it, d_list, 1, nbp, d_m, d_l, d_piv, rp, st);
  launch_dir_build(d_pl, 1, cells, d_piv, d_dir, st);
  if (mode == LS_CLASSIFY_GUESS) launch_fmodel(d_m, d_l, d_slot, 1, B, d_fm, d_fl, st);
  launch_table_classify(d_pl, d_piv, d_dir, static_cast<const uint64_t*>(d_keys), n, dtype, d_ids,
                        reinterpret_cast<unsigned long long*>(d_hist), nbp, cells, st, d_fm, d_fl);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return LS_OK;
}

ls_status ls_sample(ls_ctx* ctx, const void* d_keys, uint64_t n, ls_dtype dtype, uint64_t S, uint64_t seed,
                    void* d_out, ls_stream_t stream) {
  if (!ctx || (dtype != LS_F64 && dtype != LS_U64)) return LS_EINVAL;
  if (S && (!d_keys || !d_out || n == 0)) return LS_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_keys) % 8 || reinterpret_cast<uintptr_t>(d_out) % 8) return LS_EINVAL;
  if (S > n) S = n;
  CK(cudaSetDevice(ctx->device));
  launch_sample_keys(static_cast<const uint64_t*>(d_keys), n, S, seed, static_cast<uint64_t*>(d_out),
                     static_cast<cudaStream_t>(stream));
  CK(cudaGetLastError());
  return LS_OK;
}

ls_status ls_fit_grad(ls_ctx* ctx, const ls_model* model, const void* d_sorted_sample, uint64_t S, ls_dtype dtype,
                      double* d_pred, double* d_resid, double* d_grad_a, double* d_grad_b, double* d_grad_root,
                      ls_stream_t stream) {
  if (!ctx || !model || !d_sorted_sample || S == 0 || S >= (1ull << 32)) return LS_EINVAL;
  if (model->L < 1 || model->L > LS_MAX_FANOUT || (dtype != LS_F64 && dtype != LS_U64)) return LS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LS_ECUDA;
  uint32_t L = model->L;
  size_t sb = fit_grad_scratch_bytes(S, L);
  size_t need = up(sizeof(DModel)) + up(L * sizeof(Leaf)) + up(sb);
  ls_status r = ensure_cache(ctx, need + kAlign);
  if (r != LS_OK) return r;
  char* b = static_cast<char*>(ctx->d_cache);
  DModel* d_m = reinterpret_cast<DModel*>(b);
  b += up(sizeof(DModel));
  Leaf* d_l = reinterpret_cast<Leaf*>(b);
  b += up(L * sizeof(Leaf));
  DModel dm;
  std::vector<Leaf> lv;
  model_to_device_layout(model, &dm, lv);
  CK(cudaMemcpyAsync(d_m, &dm, sizeof dm, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_l, lv.data(), L * sizeof(Leaf), cudaMemcpyHostToDevice, st));
  launch_fit_grad(d_m, d_l, static_cast<const uint64_t*>(d_sorted_sample), S, dtype, d_pred, d_resid, d_grad_a,
                  d_grad_b, d_grad_root, b, sb, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return LS_OK;
}

ls_status ls_last_device_status(ls_ctx* ctx, ls_stream_t stream) {
  if (!ctx) return LS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned int v = 0;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LS_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LS_ECUDA;
  if (cudaMemcpy(&v, ctx->d_status, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return LS_ECUDA;
  cudaMemset(ctx->d_status, 0, sizeof v);
  return (ls_status)v;
}

static uint64_t fnv1a(const void* p, size_t n) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  uint64_t h = 0xcbf29ce484222325ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 0x100000001b3ull;
  }
  return h;
}

ls_status ls_model_export(const ls_model* m, void* buf, size_t* bytes) {
  if (!m || !bytes) return LS_EINVAL;
  const size_t need = 16 + sizeof(ls_model) + 8;
  if (!buf) {
    *bytes = need;
    return LS_OK;
  }
  if (*bytes < need) return LS_ENOMEM;
  unsigned char* o = static_cast<unsigned char*>(buf);
  const uint64_t magic = 0x4C534D4F44454C31ull;  // "LSMODEL1"
  const uint64_t size = sizeof(ls_model);
  memcpy(o, &magic, 8);
  memcpy(o + 8, &size, 8);
  memcpy(o + 16, m, sizeof(ls_model));
  uint64_t h = fnv1a(m, sizeof(ls_model));
  memcpy(o + 16 + sizeof(ls_model), &h, 8);
  *bytes = need;
  return LS_OK;
}

ls_status ls_model_import(ls_model* m, const void* buf, size_t bytes) {
  if (!m || !buf) return LS_EINVAL;
  const size_t need = 16 + sizeof(ls_model) + 8;
  if (bytes < need) return LS_EINVAL;
  const unsigned char* o = static_cast<const unsigned char*>(buf);
  uint64_t magic, size, h;
  memcpy(&magic, o, 8);
  memcpy(&size, o + 8, 8);
  if (magic != 0x4C534D4F44454C31ull || size != sizeof(ls_model)) return LS_EINVAL;
  memcpy(&h, o + 16 + sizeof(ls_model), 8);
  if (h != fnv1a(o + 16, sizeof(ls_model))) return LS_EINVAL;
  memcpy(m, o + 16, sizeof(ls_model));
  if (m->L < 1 || m->L > LS_MAX_FANOUT) return LS_EINVAL;
  return LS_OK;
}

const char* ls_last_error_detail(void) { return g_error_detail; }

const char* ls_status_string(ls_status s) {
  switch (s) {
    case LS_OK: return "ok";
    case LS_EINVAL: return "invalid argument";
    case LS_ENOMEM: return "out of memory / workspace too small";
    case LS_ENAN: return "NaN key";
    case LS_ETIMEOUT: return "device wait timed out";
    case LS_ECUDA: return "CUDA error";
    case LS_ENOTIMPL: return "not implemented";
    case LS_EDEVICE: return "device consistency check failed";
  }
  return "unknown status";
}

}  // extern "C"
