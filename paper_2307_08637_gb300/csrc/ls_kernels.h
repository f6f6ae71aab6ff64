// ls_kernels.h -- host-side launch wrappers of the library's CUDA kernels
// (internal; not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "ls_common.cuh"

namespace lsg {

// Records a description of the last failure on this host thread (returned
// by ls_last_error_detail); the library never prints.
void set_error_detail(const char* fmt, ...);

// Programmatic dependent launch: a kernel launched this way may be set up
// while the previous kernel of its stream is still running; every kernel's
// first statement (pdl_wait) blocks until that kernel has finished and its
// writes are visible, so the stream order of the data is unchanged and only
// the launch latency between dependent kernels is hidden.
// t_plain_launch (this thread) turns the attribute off, e.g. while a graph
// is captured on a stream where it is not wanted.
inline thread_local bool t_plain_launch = false;
template <typename... KArgs, typename... Args>
inline void pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = t_plain_launch ? 0 : 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace lsg

namespace lsg {

// Run parameters copied into kernels by value.
struct RunParams {
  uint32_t B;             // learned fanout
  uint32_t bs_max;        // splitter fanout when forced / LEARNED fallback
  uint32_t bs_auto;       // splitter fanout when AUTO picks the tree
  uint32_t T;             // base-case threshold
  uint32_t max_depth;
  uint32_t min_sample;
  double sample_rate;
  double dup_frac;
  double tau;
  uint64_t min_learned_n;
  uint64_t seed;
  int32_t partitioner;    // ls_partitioner
  int32_t recurse;        // ls_recurse
  int32_t classify_mode;  // ls_classify_mode
  int32_t dt;             // 0 f64, 1 u64
  uint32_t tile;          // keys per partition tile
  uint32_t dir_bits;      // log2 of directory cells
};

// ---- device-planned batches (ls_queue.cu)
// The work of one batch that the planner kernel laid out on the device.
// Kernels of a device-planned batch read their counts from here (a null
// pointer: the host passed the counts by value).
struct BatchDesc {
  unsigned long long nchunks;     // chunks of the batch
  unsigned long long chunk_keys;  // keys per chunk
  unsigned long long keys;        // keys of the batch's items
  unsigned int nitems;            // items (plans) of the batch
  unsigned int nsegs, nmulti;     // chunk runs; items with several runs
  unsigned int nruns;             // buffered-scatter runs
  unsigned int nrefine;           // items whose exact pivots are searched
  unsigned int pad;
};

// The device work queue of the level loop: the current level's items (a
// prefix of which has been planned), the next level's items (appended by
// K2), and the items handed back to the host because they draw a sample.
struct QueueState {
  unsigned long long cur_n;   // items of the current level
  unsigned long long head;    // first item of the current level not yet planned
  unsigned long long host_n;  // items handed back to the host
  unsigned long long iter;    // loop iterations so far
  unsigned int cont;          // 1 while work remains (mirrors the graph's loop condition)
  unsigned int err;           // 1: the loop stopped at its iteration limit
  unsigned long long pad[2];
};

// ---- generic helpers (ls_partition.cu)
void launch_scan_exclusive_u64(const uint64_t* in, uint64_t* out, size_t n, uint64_t* tmp, size_t tmp_elems,
                               cudaStream_t st);
size_t scan_tmp_elems(size_t n);
void launch_fill_u64(uint64_t* p, uint64_t v, size_t n, cudaStream_t st);

// ---- segmented sort of u64 values (ls_fit.cu)
// Sorts each segment [off[s], off[s+1]) of `a` ascending.  `b` is scratch of
// the same size; returns the buffer that holds the result (a or b).
uint64_t* segmented_sort_u64(uint64_t* a, uint64_t* b, const uint64_t* d_off, const uint64_t* d_chunk_prefix,
                             uint32_t nseg, uint64_t total_chunks, uint64_t max_len, cudaStream_t st,
                             uint64_t* launches);

// ---- fresh-item pipeline (ls_fit.cu)
struct FreshArgs {
  const Item* items;       // batch items
  Plan* plans;             // batch plans
  const uint32_t* fresh;   // plan indices of fresh items
  const uint64_t* samp_prefix;  // nfresh+1 sample offsets
  uint32_t nfresh;
  uint64_t total_samples;
  const uint64_t* keysA;
  const uint64_t* keysB;
};
void launch_sample_gather(const FreshArgs& f, const RunParams& rp, uint64_t* samp, cudaStream_t st);
void launch_dups(const FreshArgs& f, const uint64_t* samp, cudaStream_t st);
// One array's sample (key bits) with stream seed h; see ls_sample.
void launch_sample_keys(const uint64_t* keys, uint64_t n, uint64_t S, uint64_t h, uint64_t* out, cudaStream_t st);

struct FitArgs {
  Plan* plans;
  const Item* items;
  const uint32_t* cand;        // plan indices of fit candidates
  const uint64_t* cand_soff;   // ncand+1 prefix of sample sizes (candidates only, offsets into samp)
  const uint64_t* rchunk_prefix; // ncand+1 prefix of root chunks
  uint32_t ncand;
  uint64_t total_rchunks;
  uint64_t total_cand_samples;
  uint64_t lchunk_bound;       // upper bound on leaf chunks
  const uint64_t* samp;        // sorted samples (ord), indexed by plan.sample_off
  DModel* models;
  Leaf* leaves;
  uint32_t L;
  uint32_t nbp_max;            // pivot table length of a learned candidate (L padded to a power of two)
  // scratch
  double* rpart;               // 4 * total_rchunks
  uint32_t* leaf_start;        // ncand * (L+1)
  uint64_t* lchunk_cnt;        // ncand*L + 1
  uint64_t* lchunk_prefix;     // ncand*L + 1
  uint64_t* scan_tmp;
  size_t scan_tmp_elems;
  double* lpart;               // 4 * lchunk_bound
  uint32_t* leaf_of;           // total_cand_samples
  uint32_t* leaf_cnt;          // per model slot * L (sample points per leaf)
  FModel* fmodels;             // per model slot: FP32 image header
  FLeaf* fleaves;              // per model slot * L: FP32 image leaves
  FClamp* fclamps;             // per model slot * L: FP32 image of the leaves' clamps
};
void launch_fit(const FitArgs& a, const RunParams& rp, cudaStream_t st, uint64_t* launches);

// FP32 images of the models of one slot list (used for bucket guesses).
void launch_fmodel(const DModel* models, const Leaf* leaves, const int32_t* slots, uint32_t nslots, uint32_t L,
                   FModel* fm, FLeaf* fl, cudaStream_t st, FClamp* fc = nullptr);
void launch_fmodel_for_fit(const FitArgs& a, cudaStream_t st);

// Exact learned pivots for items whose plan has decision candidate LEARNED:
// list of plan indices; thread per (item, j < nb_pad).
void launch_learned_pivots(Plan* plans, const Item* items, const uint32_t* list, uint32_t nlist, uint32_t nb_pad,
                           const DModel* models, const Leaf* leaves, uint64_t* pivots, const RunParams& rp,
                           cudaStream_t st, const BatchDesc* bd = nullptr);  // bd: list length from the device
// Sample-bucket maximum under the RMI (imbalance test) for fit candidates.
void launch_imbalance(const FitArgs& a, uint64_t* pivots, unsigned long long* cnt_pool, const RunParams& rp,
                      cudaStream_t st, uint64_t* launches);
// Alg. 5 decision for every fresh item; then splitter tables where needed.
void launch_decide(const FreshArgs& f, const DModel* models, const RunParams& rp, cudaStream_t st);
void launch_splitter_build(const FreshArgs& f, const uint64_t* samp, uint64_t* pivots, const RunParams& rp,
                           cudaStream_t st);
// Radix directory over every plan with cls == CLS_DIR (thread per cell).
void launch_dir_build(Plan* plans, uint32_t nplans, uint32_t cells, const uint64_t* pivots, uint16_t* dirs,
                      cudaStream_t st);

// ---- forward / backward of the fit objective (ls_fit.cu)
void launch_fit_grad(const DModel* model, const Leaf* leaves, const uint64_t* sample_bits, uint64_t S, int dt,
                     double* pred, double* resid, double* grad_a, double* grad_b, double* grad_root,
                     void* scratch, size_t scratch_bytes, cudaStream_t st);
size_t fit_grad_scratch_bytes(uint64_t S, uint32_t L);

// Items per batch (per-item tables in the workspace are sized for this many).
constexpr uint32_t kBatchItems = 2048;

// ---- partition passes (ls_partition.cu)
struct PassArgs {
  const Item* items;
  Plan* plans;
  uint32_t nitems;
  uint64_t nchunks;
  const uint64_t* keysA;
  const uint64_t* keysB;
  uint64_t* outA;
  uint64_t* outB;
  const uint64_t* pivots;
  const uint16_t* dirs;
  const DModel* models;
  const Leaf* leaves;
  const FModel* fmodels;
  const FLeaf* fleaves;
  const FClamp* fclamps;        // the leaves' clamps (beside the FP32 leaves)
  uint32_t aux_bytes;           // shared-memory bytes for a directory or the FP32 leaves and clamps
  uint32_t cls_mask;            // bit c set when some item of the batch uses classifier c
  uint16_t* ids;                // per key (same offsets as the keys): bucket id written by K1, read by K3
  unsigned long long* counts;   // per plan: nb counts
  unsigned long long* cursors;  // per plan: nb bucket bases in the destination
  uint32_t* agg;                // per chunk: nb_pad_max bucket counts (K1)
  unsigned long long* excl;     // per chunk: keys of each bucket in the item's earlier chunks
  unsigned long long* chunk_ctr;  // [0]: K3 dynamic chunk counter, [1]: K3b run counter (zeroed)
  const uint32_t* chunk_plan;   // per chunk: index of its item in the batch
  uint64_t chunk_keys;          // keys per chunk: a multiple of the tile, at most kChunkKeys
  void* valsA;                  // key-value sorts: payload of buffer A (caller's values) ...
  void* valsB;                  // ... and of the ping-pong buffer B
  uint32_t vbytes;              // bytes per value: 0 (keys only), 4 or 8
  unsigned int* status;         // device status word
  int check_nan;
  uint32_t nb_pad_max;
  uint32_t dir_cells_max;
  const BatchDesc* bd;          // device-planned batch: counts from here (nullptr: nchunks / chunk_keys above)
};
// Chunk count and chunk size of the batch a kernel works on.
__host__ __device__ inline uint64_t batch_chunks(const PassArgs& a) { return a.bd ? a.bd->nchunks : a.nchunks; }
__host__ __device__ inline uint64_t batch_chunk_keys(const PassArgs& a) {
  return a.bd ? a.bd->chunk_keys : a.chunk_keys;
}
int launch_classify_hist(const PassArgs& a, const RunParams& rp, cudaStream_t st);  // returns launches
// A batch with fewer chunks than this gets smaller chunks (about two per
// resident K1/K3 block on a 152-SM part; a constant so that workspace sizes
// do not depend on the device).
constexpr uint64_t kChunkSlots = 1024;

// A run of at most kSegChunks consecutive chunks of one item.
constexpr uint32_t kSegChunks = 16;
struct ChunkSeg {
  uint64_t c0;     // first chunk (global index)
  uint32_t nch;    // chunks in the run
  uint32_t plan;   // owning item / plan
  uint32_t first;  // index of the item's first run
  uint32_t pad;
};
// Per-chunk exclusive prefixes of the K1 counts within each item: one pass
// per run, then, for the items spanning several runs (multi: first run and
// run count per such item), a scan of the run totals and the carries.
// Returns launches.
// parts: 1 the run pass, 2 the carry scan and pass over items with several runs.
int launch_chunk_prefix(const ChunkSeg* segs, uint32_t nsegs, const uint2* multi, uint32_t nmulti,
                        const Plan* plans, uint32_t* agg, unsigned long long* excl, uint32_t nbp, cudaStream_t st,
                        const BatchDesc* bd = nullptr, int parts = 3);
void launch_scatter(const PassArgs& a, const RunParams& rp, cudaStream_t st);

// Buffered scatter (K3b).  An item none of whose descendants ever draws a
// sample needs no particular order of the keys inside its buckets: a learned
// item under REFINE_GLOBAL (its descendants refine the same model or take
// the radix split), a radix item, or any item none of whose children is
// partitioned again (K2 sets FLAG_ORDER_FREE).  Its keys go through
// per-bucket line buffers with atomic position claims (the buffered
// partitioning of Sec. 2.2 / Sec. 2.4) instead of the stable scatter.
// Key-only sorts with at most kBufMaxBuckets buckets.  The host plans runs
// for every candidate (the flag is set on the device after planning); each
// scatter kernel skips the items that belong to the other.
constexpr uint32_t kBufMaxBuckets = 1024;
__host__ __device__ inline bool buffered_scatter_candidate(const Plan& pl, uint32_t vbytes) {
  return vbytes == 0 && pl.nb_pad <= kBufMaxBuckets;
}
__host__ __device__ inline bool buffered_scatter_ok(const Plan& pl, const RunParams& rp, uint32_t vbytes) {
  return buffered_scatter_candidate(pl, vbytes) &&
         ((pl.flags & FLAG_ORDER_FREE) || pl.decision == LS_DEC_RADIX ||
          (pl.decision == LS_DEC_LEARNED && rp.recurse == LS_RECURSE_REFINE_GLOBAL));
}
// A range of one item's keys taken by one K3b block: keys [off, off + len)
// of the item (item-relative).
struct BufRun {
  uint64_t off, len;
  uint32_t plan, pad;
  uint64_t pad1;
};
static_assert(sizeof(BufRun) == 32, "BufRun layout");
// Number of K3b blocks that can be resident (the run list is sized for two
// runs per block).
uint32_t buffered_scatter_slots();
void launch_scatter_buffered(const PassArgs& a, const RunParams& rp, const BufRun* runs, uint32_t nruns,
                             cudaStream_t st);  // a.bd: the run count is read from the device

// The planner of a device-planned batch (ls_queue.cu).
struct PlanArgs {
  Item* level;                   // the current level's items (cur_n of them)
  const Item* next;              // the next level's items, appended by K2 (n_next of them)
  Item* bitems;                  // the batch's items
  Plan* plans;                   // the batch's plans
  Item* hostq;                   // items handed back to the host
  uint64_t icap;                 // capacity of level, next and hostq
  uint32_t* chunk_plan;          // per chunk: its item in the batch
  uint64_t chunk_cap;
  ChunkSeg* segs;                // runs of kSegChunks chunks
  uint64_t seg_cap;
  uint2* multi;                  // items with several chunk runs: (first run, runs)
  BufRun* runs;                  // buffered-scatter runs
  uint64_t run_cap;
  uint32_t* reflist;             // items whose exact pivots are searched
  BatchDesc* bd;
  QueueState* q;
  LevelCounters* ctr;
  unsigned long long* chunk_ctr;  // the scatters' work counters (zeroed)
  unsigned int* status;
  uint32_t nbc;                  // per-item stride of the count / cursor / pivot tables
  uint32_t cells;                // directory cells per item
  uint64_t slots;                // buffered-scatter run slots (two per resident block)
};
// Conditions of the level-loop graph: the while node (loop) and if nodes
// around the kernels a batch may not need.  All zero outside a graph.
struct LoopHandles {
  unsigned int in_graph;              // 1: the batch runs inside the graph and sets these
  unsigned int has_direct;            // the graph has an if node for the direct classifier
  cudaGraphConditionalHandle loop;    // another batch follows
  cudaGraphConditionalHandle pivots;  // some item's exact pivots are searched
  cudaGraphConditionalHandle k1;      // some item uses the table classifier (guess or tree)
  cudaGraphConditionalHandle direct;  // some item uses the direct FP64 classifier
  cudaGraphConditionalHandle radix;   // some item takes the radix split
  cudaGraphConditionalHandle multi;   // some item has several chunk runs
  cudaGraphConditionalHandle small, large, copy, fallback;  // span lists that are not empty
};
void launch_plan_batch(const PlanArgs& a, const RunParams& rp, const LoopHandles& h, cudaStream_t st);
void launch_zero_counts(const BatchDesc* bd, const Plan* plans, unsigned long long* counts, cudaStream_t st);
// After the batch's scatter: the loop condition and the span conditions.
// max_iter bounds the loop; the flag in q is what the host reads outside a graph.
void launch_batch_end(QueueState* q, const LevelCounters* ctr, const unsigned int* status, const LoopHandles& h,
                      unsigned long long max_iter, cudaStream_t st);

struct ChildArgs {
  const Item* items;
  Plan* plans;
  uint32_t nitems;
  const uint64_t* pivots;
  unsigned long long* counts;
  unsigned long long* cursors;
  Item* next;
  uint64_t next_cap;
  Span* base_small;
  Span* base_mid;
  Span* base_large;
  uint64_t base_cap;
  uint64_t mid_cap;
  uint64_t large_cap;
  Span* copy;
  uint64_t copy_cap;
  Span* fallback;
  uint64_t fallback_cap;
  LevelCounters* ctr;
  DevLevelStats* stats;
  const BatchDesc* bd;  // device-planned batch: item count from here (the grid covers kBatchItems)
};
void launch_children(const ChildArgs& a, const RunParams& rp, cudaStream_t st);

// Copy bytes (a multiple of 8) between device memory and mapped page-locked
// host memory with a small kernel (16 blocks) instead of a copy engine.
void launch_link_copy(const void* src, void* dst, size_t bytes, cudaStream_t st);

// Base cases, copies home and the depth-limit fallback.  VA / VBuf / vb:
// values of a key-value sort (vb = 4 or 8 bytes; 0 for keys only).
// mid: the list of spans longer than kWarpSmallMax keys (its own kernel instance).
void launch_base_small(const Span* spans, uint64_t n, uint64_t* A, const uint64_t* Bbuf, void* VA, const void* VBuf,
                       uint32_t vb, int dt, cudaStream_t st, bool mid);
// Returns the kernels launched (one per span size class).
int launch_base_large(const Span* spans, uint64_t n, uint32_t max_len, uint64_t* A, const uint64_t* Bbuf, void* VA,
                      const void* VBuf, uint32_t vb, int dt, cudaStream_t st);
void launch_copy_spans(const Span* spans, uint64_t n, uint64_t* A, const uint64_t* Bbuf, void* VA, const void* VBuf,
                       uint32_t vb, cudaStream_t st);
void launch_fallback(const Span* spans, uint64_t n, uint64_t* A, uint64_t* Bbuf, void* VA, void* VBuf, uint32_t vb,
                     int dt, cudaStream_t st);
// The same for keys only, with the span counts read from the device
// (the level counters); n_max bounds them (grid sizing).  which: SPANS_*.
// Returns the kernels launched.
enum { SPANS_SMALL = 1, SPANS_LARGE = 2, SPANS_COPY = 4, SPANS_FALLBACK = 8 };
int launch_spans_device(int which, const LevelCounters* ctr, const Span* small, const Span* mid, const Span* large,
                        const Span* copy, const Span* fallback, uint64_t n_max, uint32_t max_len, uint64_t* A,
                        uint64_t* Bbuf, int dt, cudaStream_t st);

// ls_classify helpers
void launch_direct_classify(const DModel* m, const Leaf* leaves, const uint64_t* keys, uint64_t n, int dt, double P,
                            double Bg, uint32_t B, uint32_t* ids, unsigned long long* hist, cudaStream_t st);
void launch_table_classify(const Plan* plan, const uint64_t* pivots, const uint16_t* dirs, const uint64_t* keys,
                           uint64_t n, int dt, uint32_t* ids, unsigned long long* hist, uint32_t nb_pad,
                           uint32_t cells, cudaStream_t st, const FModel* fm = nullptr, const FLeaf* fl = nullptr);

}  // namespace lsg
