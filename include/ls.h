/*
 * ls.h -- C ABI of the GB300 (sm_103a) learned SampleSort library.
 *
 * The library sorts arrays of 64-bit keys (IEEE doubles or unsigned 64-bit
 * integers) in ascending order on one GPU, following arxiv 2307.08637
 * ("LearnedSort as a learning-augmented SampleSort"):
 *   - a two-layer RMI F(x) = f2^{floor(B f1(x))}(x) with a linear root and B
 *     linear leaves (Sec. 2.1), trained in FP64 on a sorted random sample
 *     (Sec. 2.2, 1% by default), made monotone by per-leaf clamps (Sec. 4);
 *   - each key goes to bucket floor(B F(x)) (Sec. 2.2 partitioning), which is
 *     the SampleSort partition of the B-1 implicit learned pivots of Alg. 4;
 *   - the SampleSort splitter tree with IPS4o equality buckets (Sec. 2.4) is
 *     the alternative partitioner, chosen by Alg. 5 (BuildPartitionModel)
 *     or forced through ls_params.partitioner;
 *   - oversized buckets are partitioned again, all-equal buckets are left as
 *     they are (homogeneity check, Sec. 2.2), small buckets are sorted by a
 *     shared-memory base case.
 *
 * Keys are ordered by ord(x): for doubles IEEE totalOrder (-0.0 < +0.0),
 * for u64 the integer order.  NaN keys are rejected.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are device pointers on the context's device; h_*
 *     are host pointers.  The caller owns every buffer it passes in.
 *   - Calls are asynchronous on the given stream unless stated otherwise.
 *     Errors that can be seen on the host (bad arguments, too-small
 *     workspace) are returned before anything is launched and leave the
 *     buffers untouched.  Errors found on the device (NaN key, a failed
 *     consistency check) are recorded in a device status word; read it with
 *     ls_last_device_status().  After such an error the contents of d_keys
 *     are unspecified (still a permutation of some of the input's bytes).
 *   - No exceptions cross this boundary.  A context is not thread-safe: use
 *     one context per host thread.
 */
#ifndef LS_H
#define LS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* CUDA stream handle (cudaStream_t), passed as an opaque pointer so this
 * header needs no CUDA include.  NULL is the legacy default stream. */
typedef void* ls_stream_t;

typedef enum {
  LS_OK = 0,
  LS_EINVAL = 1,    /* bad argument (null pointer, bad dtype, fanout range) */
  LS_ENOMEM = 2,    /* workspace too small, or host/device allocation failed */
  LS_ENAN = 3,      /* a key is NaN (f64 only) */
  LS_ETIMEOUT = 4,  /* a bounded device wait ran out (no kernel of this version waits) */
  LS_ECUDA = 5,     /* a CUDA runtime call failed */
  LS_ENOTIMPL = 6,  /* option not implemented */
  LS_EDEVICE = 7    /* device-side consistency check failed */
} ls_status;

typedef enum { LS_F64 = 0, LS_U64 = 1 } ls_dtype;

/* Partition model choice (Alg. 5). */
typedef enum {
  LS_PART_AUTO = 0,     /* RMI if n >= min_learned_n, sample dups <= dup_frac
                           and the sample is not imbalanced; else the tree */
  LS_PART_LEARNED = 1,  /* always the RMI (tree only if the fit is not finite) */
  LS_PART_SPLITTER = 2  /* always the splitter tree */
} ls_partitioner;

/* How a bucket of a learned partition is split again (Sec. 3.3). */
typedef enum {
  LS_RECURSE_REFINE_GLOBAL = 0, /* LearnedSort 2.0: sample once, reuse the
                                   model: child = floor(F B^(k+1)) - B g */
  LS_RECURSE_RETRAIN = 1        /* AIPS2o: new sample and model per bucket */
} ls_recurse;

/* Per-key bucket search used by the partition passes.  Every mode gives
 * identical bucket ids; they differ only in speed. */
typedef enum {
  LS_CLASSIFY_AUTO = 0,      /* learned: FP32 guess; splitter: tree search */
  LS_CLASSIFY_DIRECTORY = 1, /* radix directory over the pivots + <=k compares */
  LS_CLASSIFY_TREE = 2,      /* branchless binary search over the pivots */
  LS_CLASSIFY_DIRECT = 3,    /* learned only: FP64 RMI per key (diagnostic) */
  LS_CLASSIFY_GUESS = 4      /* learned only: FP32 image of the RMI guesses the
                                bucket, exact pivots correct it */
} ls_classify_mode;

#define LS_MAX_FANOUT 4096
#define LS_MAX_LEVELS 48

typedef struct {
  uint32_t fanout;               /* B = RMI leaves = learned buckets, 2..4096 (1000) */
  uint32_t splitter_fanout;      /* largest splitter-tree fanout B_s, 2..4096 (1024) */
  uint32_t basecase_threshold;   /* T: buckets with <= T keys go to the base case (16) */
  uint32_t max_depth;            /* deeper buckets are sorted directly (16) */
  uint32_t min_sample;           /* sample size floor (256) */
  uint32_t auto_splitter_fanout; /* B_s when AUTO falls back to the tree (256) */
  double sample_rate;            /* S = ceil(r n) (0.01) */
  double dup_frac;               /* Alg. 5 duplicate bound (0.10) */
  double imbalance_tau;          /* reject the RMI if a sample bucket > tau S/B (8) */
  uint64_t min_learned_n;        /* Alg. 5 size bound (1e5) */
  uint64_t seed;                 /* sampling seed */
  int32_t partitioner;           /* ls_partitioner */
  int32_t recurse_model;         /* ls_recurse */
  int32_t classify_mode;         /* ls_classify_mode (speed only) */
  uint32_t tile_keys;            /* reserved (0): the tile size is fixed at 4096 keys */
  uint32_t flags;                /* LS_FLAG_* */
} ls_params;

/* ls_params.flags: record CUDA events around every kernel launch class and
 * report their device time in ls_stats.pass[] (adds one event pair per
 * launch; off by default). */
#define LS_FLAG_TIME_PASSES 1u
/* ls_params.flags: take fanout, sample_rate, basecase_threshold and
 * recurse_model from the context's autotuner entry for this key type and
 * floor(log2 n) (of the mean segment length for ls_sort_segmented), when
 * there is one; ls_workspace_size applies the same substitution. */
#define LS_FLAG_TUNED 2u
/* ls_params.flags: plan the recursion levels below the root on the device.
 * Without it every level is planned on the host (one readback per level,
 * overlapped with the level's scatter).  With it, when buckets below the
 * root are refined rather than resampled (REFINE_GLOBAL, partitioner not
 * LS_PART_SPLITTER, keys only, fanout <= 1024, not LS_CLASSIFY_DIRECTORY),
 * the levels below the root come from a device work queue and run as one
 * CUDA graph (launched batch by batch from the host when
 * LS_FLAG_TIME_PASSES is set), with one readback at the end; buckets that
 * do draw a sample are planned on the host.  The graph is captured once per
 * (keys, workspace, parameters) and kept in the context.  Results are
 * identical either way. */
#define LS_FLAG_DEVICE_LEVELS 4u

/* The trained two-layer RMI (all FP64), as exported by ls_fit. */
typedef struct {
  uint32_t L;          /* number of leaves (= fanout B) */
  uint32_t S;          /* sample size it was trained on */
  double xmin, xmax;   /* clamp range: smallest and largest sample key */
  double root_x0, root_a, root_b;
  double leaf_x0[LS_MAX_FANOUT];
  double leaf_a[LS_MAX_FANOUT];
  double leaf_b[LS_MAX_FANOUT];
  double leaf_lo[LS_MAX_FANOUT];
  double leaf_hi[LS_MAX_FANOUT];
  uint32_t leaf_count[LS_MAX_FANOUT]; /* sample points routed to each leaf */
} ls_model;

/* Decision codes (per partitioned bucket). */
#define LS_DEC_NONE 0
#define LS_DEC_LEARNED 1
#define LS_DEC_SPLITTER 2
#define LS_DEC_SPLITTER_EQ 3
#define LS_DEC_HOMOGENEOUS 4
#define LS_DEC_RADIX 5 /* radix split of the bits where the bucket's keys differ (no model,
                        * no sample): below a REFINE_GLOBAL model, for a bucket the model
                        * did not split or one past the FP64 refinement limit */

typedef struct {
  uint64_t items, learned, splitter, splitter_eq, homogeneous, noprogress;
  uint64_t base_items, base_keys, fallback_items, fallback_keys;
  uint64_t keys, max_child, sumsq_child, eq_keys;
  uint64_t radix; /* items partitioned by the radix split */
} ls_level_stats;

/* Kernel classes timed with LS_FLAG_TIME_PASSES. */
#define LS_PASS_SAMPLE 0    /* sample gather + sample sort + duplicate count */
#define LS_PASS_FIT 1       /* RMI fit (sums, leaves, monotone clamps) */
#define LS_PASS_PIVOTS 2    /* exact pivots, imbalance test, decision, splitter tables, directory */
#define LS_PASS_CLASSIFY 3  /* K1: classify + histogram (reads 8 B/key) */
#define LS_PASS_CHILDREN 4  /* K2: bucket scan + children */
#define LS_PASS_SCATTER 5   /* K3: stable scatter (reads and writes 8 B/key) */
#define LS_PASS_BASE 6      /* base case and depth-limit fallback (8 B/key each way) */
#define LS_PASS_COPY 7      /* copy of finished buckets back into the keys array */
#define LS_NPASS 8

typedef struct {
  double ms;          /* summed device time of the class's launches */
  uint64_t launches;
  uint64_t keys;      /* keys the launches processed */
} ls_pass_time;

typedef struct {
  int32_t status;               /* device status of the call (LS_OK, LS_ENAN, ...) */
  int32_t root_decision;        /* LS_DEC_* of the first array's root */
  uint64_t root_sample_size;
  uint64_t root_dups;           /* #{j >= 1 : ord(s_j) == ord(s_{j-1})} of the root sample */
  uint64_t root_imbalance_max;  /* largest root-sample bucket under the RMI */
  uint32_t root_nbuckets;
  uint32_t levels_used;
  ls_level_stats level[LS_MAX_LEVELS];
  double ms_total;              /* host-observed time of the call (stats only) */
  uint64_t kernel_launches;     /* kernels this call launched */
  ls_pass_time pass[LS_NPASS];  /* filled when LS_FLAG_TIME_PASSES is set */
  uint64_t device_batches;      /* batches planned by the device work queue */
  int32_t level_loop;           /* how the levels below the root ran: LS_LOOP_* */
  int32_t reserved;
} ls_stats;

/* ls_stats.level_loop */
#define LS_LOOP_HOST 0          /* planned on the host, one readback per level (default) */
#define LS_LOOP_DEVICE 1        /* device work queue, batches launched from the host */
#define LS_LOOP_GRAPH 2         /* device work queue in one CUDA graph (while node) */
#define LS_LOOP_GRAPH_PDL 3     /* the same, with programmatic dependent launches in the graph */

typedef struct ls_ctx ls_ctx;

/* Fill *p with the defaults listed beside each field of ls_params. */
void ls_params_default(ls_params* p);

/* Create a context bound to CUDA device `device` (made current inside every
 * call).  The context owns small pinned host buffers and an optional cached
 * device buffer for ls_sort_host.  *out is NULL on failure. */
ls_status ls_create(ls_ctx** out, int device);
void ls_destroy(ls_ctx* ctx);

/* Bytes of device workspace ls_sort / ls_sort_segmented need for n keys in
 * nseg segments with these parameters.  The workspace holds an n-key
 * ping-pong buffer plus tables; it is caller-owned device memory. */
ls_status ls_workspace_size(ls_ctx* ctx, uint64_t n, uint32_t nseg, ls_dtype dtype, const ls_params* p,
                            size_t* bytes);

/* Sort d_keys[0..n) ascending by ord (the sorting problem of Sec. 1-2).
 * d_keys must be 8-byte aligned (LS_EINVAL otherwise).  In place from the
 * caller's view; the library ping-pongs through d_workspace
 * (>= ls_workspace_size bytes, 256-byte aligned).  Stream ordered; the
 * host plans each level from a readback of the previous one (or, with
 * LS_FLAG_DEVICE_LEVELS, the device plans the levels below the root), so
 * the call returns after the sort is complete.  out_stats (nullable)
 * receives the decisions and per-level statistics. */
ls_status ls_sort(ls_ctx* ctx, void* d_keys, uint64_t n, ls_dtype dtype, const ls_params* p, void* d_workspace,
                  size_t ws_bytes, ls_stats* out_stats, ls_stream_t stream);

/* Sort nseg independent arrays: segment s is d_keys[h_offsets[s] ..
 * h_offsets[s+1]) (host array of nseg+1 non-decreasing offsets).  Every
 * segment gets its own sample, model and decisions (Alg. 5 per segment).
 * h_seg_decision (nullable, nseg entries) receives each root decision. */
ls_status ls_sort_segmented(ls_ctx* ctx, void* d_keys, const uint64_t* h_offsets, uint32_t nseg, ls_dtype dtype,
                            const ls_params* p, void* d_workspace, size_t ws_bytes, ls_stats* out_stats,
                            int32_t* h_seg_decision, ls_stream_t stream);

/* Key-value sort (a payload carried with each key, e.g. row ids of a
 * database column; argsort when the values are 0..n-1): sorts d_keys[0..n)
 * ascending by ord exactly as ls_sort does and applies the same permutation
 * to d_vals[0..n) (val_bytes = 4 or 8 bytes each).  Stable: values of equal
 * keys keep their input order.  The workspace (ls_workspace_size_pairs)
 * also holds a ping-pong buffer of the values.  Same conventions as ls_sort. */
ls_status ls_workspace_size_pairs(ls_ctx* ctx, uint64_t n, uint32_t val_bytes, ls_dtype dtype, const ls_params* p,
                                  size_t* bytes);
ls_status ls_sort_pairs(ls_ctx* ctx, void* d_keys, void* d_vals, uint32_t val_bytes, uint64_t n, ls_dtype dtype,
                        const ls_params* p, void* d_workspace, size_t ws_bytes, ls_stats* out_stats,
                        ls_stream_t stream);

/* End-to-end sort of a HOST array: copies h_keys to the device, sorts, and
 * copies the result back (h_keys is overwritten).  Device memory is cached
 * in the context between calls.  Synchronous. */
ls_status ls_sort_host(ls_ctx* ctx, void* h_keys, uint64_t n, ls_dtype dtype, const ls_params* p, ls_stats* out_stats);

/* ls_sort_host for `count` host arrays (array i: h_keys[i], n[i] keys, each
 * overwritten with its sorted keys).  The copies are pipelined with the
 * sorts on three context streams: array i + 1 is copied in while array i
 * is sorted and array i - 1 is copied out (the host link carries both
 * directions at once).  The overlap needs page-locked host arrays
 * (cudaMallocHost / cudaHostRegister); pageable arrays are still sorted
 * correctly.  Device memory (three arrays of the largest size plus one
 * workspace) is cached in the context.  out_stats (nullable) receives one
 * ls_stats per array.  Synchronous: returns when every array is back. */
ls_status ls_sort_host_batch(ls_ctx* ctx, void* const* h_keys, const uint64_t* n, uint32_t count, ls_dtype dtype,
                             const ls_params* p, ls_stats* out_stats);

/* Sample(A) of Alg. 2-5 (Sec. 2.2: the model is trained on a random
 * sample): writes min(S, n) keys of d_keys[0..n) to d_out, drawn with
 * replacement, key j from position floor(u_j * n / 2^64) where u_j is the
 * SplitMix64 output at state seed + (j+1) * 0x9E3779B97F4A7C15; S >= n
 * copies the keys in order.  Key bits are copied unchanged (dtype only
 * checks the type).  Both pointers 8-byte aligned, device memory owned by
 * the caller.  Stream ordered and asynchronous; allocates nothing. */
ls_status ls_sample(ls_ctx* ctx, const void* d_keys, uint64_t n, ls_dtype dtype, uint64_t S, uint64_t seed,
                    void* d_out, ls_stream_t stream);

/* Train the root model exactly as ls_sort would (sample with the root's
 * seed, sort the sample, fit; Sec. 2.2 / Alg. 5) and copy it to *out_model.
 * Also returns the root decision inputs in *out_stats (nullable).
 * d_sorted_sample (nullable, >= sample size keys) receives the sorted
 * sample as key bits.  Synchronous. */
ls_status ls_fit(ls_ctx* ctx, const void* d_keys, uint64_t n, ls_dtype dtype, const ls_params* p,
                 ls_model* out_model, ls_stats* out_stats, void* d_sorted_sample, ls_stream_t stream);

/* Bucket ids of d_keys[0..n) under a given model (host struct, copied to
 * the device): id = clamp(floor(F(x) B^(k+1)) - B g, 0, B-1) with B =
 * model->L (k = 0, g = 0 is floor(B F(x)) of Sec. 2.2).  d_ids (nullable)
 * gets n uint32 ids, d_hist (nullable) B uint64 counts (overwritten).  mode
 * picks the evaluation: LS_CLASSIFY_DIRECT evaluates the FP64 RMI per key;
 * the others compile the model into its B-1 exact pivots (Alg. 4) first.
 * Asynchronous. */
ls_status ls_classify(ls_ctx* ctx, const ls_model* model, const void* d_keys, uint64_t n, ls_dtype dtype,
                      uint32_t k, uint64_t g, int32_t mode, uint32_t* d_ids, uint64_t* d_hist, ls_stream_t stream);

/* Forward and backward pass of the RMI's least-squares objective on a
 * sorted sample (key bits, S keys): pred_j = f_leaf(s_j)(s_j) (raw linear
 * leaf), resid_j = pred_j - j/S, and the gradient of MSE = (1/S) sum resid^2
 * with respect to every leaf's (a_i, b_i) and the root's (a, b).  Outputs
 * are device arrays (nullable): d_pred[S], d_resid[S], d_grad_a[L],
 * d_grad_b[L], d_grad_root[2].  Asynchronous. */
ls_status ls_fit_grad(ls_ctx* ctx, const ls_model* model, const void* d_sorted_sample, uint64_t S, ls_dtype dtype,
                      double* d_pred, double* d_resid, double* d_grad_a, double* d_grad_b, double* d_grad_root,
                      ls_stream_t stream);

/* ls_classify without any device allocation (the paper has no counterpart:
 * this is a deployment variant of ls_classify).  For callers that cannot call
 * cudaMalloc where they classify -- an application whose own memory pool
 * owns the device memory, or a path that must not risk cudaMalloc's
 * device-wide synchronisation.  Same arguments and results as ls_classify,
 * without a context: it classifies on the current device and stream.
 * Every mode is accepted (k >= 50 is rejected with LS_EINVAL, as by
 * ls_classify).  Scratch is one fixed 288 KB device array inside the library
 * (enough for every mode at every fanout up to LS_MAX_FANOUT; present on
 * every GPU that loads it, until the process exits); it holds the model and
 * pivot tables of the last call, is fully rewritten by each call, and is
 * shared by all calls: calls that overlap on the GPU race, so serialise them.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress).
 * Fanouts up to LS_MAX_FANOUT fit; a model that needs more scratch than the
 * array holds is rejected with LS_ENOMEM.  Synchronous on `stream`. */
ls_status ls_classify_static(const ls_model* model, const void* d_keys, uint64_t n, ls_dtype dtype, uint32_t k,
                             uint64_t g, int32_t mode, uint32_t* d_ids, uint64_t* d_hist, ls_stream_t stream);

/* Autotuner.  The paper notes that adjusting the sample size improved its
 * parallel performance (Sec. 5); here the fanout B, the sample rate r, the
 * base-case threshold T and the recursion mode are chosen by timing ls_sort
 * on copies of the caller's keys: coordinate descent over the candidate
 * lists below, starting from *base, each configuration timed as the median
 * of five sorts after one warm-up sort (CUDA events on `stream`); a
 * candidate replaces the current configuration only when it is at least 5 %
 * faster, so that timing noise does not decide.
 *   fanout             256, 512, 1000, 1024, 2048
 *   basecase_threshold 1024, 2048, 4096, 8192
 *   sample_rate        0.0025, 0.005, 0.01, 0.02
 *   recurse_model      REFINE_GLOBAL, RETRAIN
 * The winner is written to *out (the other fields are *base's) and stored in
 * the context for (dtype, floor(log2 n)), where LS_FLAG_TUNED finds it.
 * d_keys is not modified.  The tuner allocates its own device scratch (n
 * keys plus the largest workspace of the candidates) and frees it before
 * returning.  report (nullable) receives the timings.  Synchronous. */
typedef struct {
  uint32_t configs;   /* configurations timed */
  double base_ms;     /* median sort time with *base */
  double best_ms;     /* median sort time with *out */
} ls_tune_report;

ls_status ls_autotune(ls_ctx* ctx, const void* d_keys, uint64_t n, ls_dtype dtype, const ls_params* base,
                      ls_params* out, ls_tune_report* report, ls_stream_t stream);

/* ls_autotune for a batch of segments (the form ls_sort_segmented sorts):
 * each candidate is timed on ls_sort_segmented of copies of d_keys[0 ..
 * h_offsets[nseg]) split at h_offsets (host array, h_offsets[0] = 0), so
 * the choice reflects the batch's mix of segment lengths.  The winner is
 * stored under floor(log2) of the mean segment length, where
 * ls_sort_segmented with LS_FLAG_TUNED finds it.  Same conventions as
 * ls_autotune. */
ls_status ls_autotune_segmented(ls_ctx* ctx, const void* d_keys, const uint64_t* h_offsets, uint32_t nseg,
                                ls_dtype dtype, const ls_params* base, ls_params* out, ls_tune_report* report,
                                ls_stream_t stream);

/* The context's tuning table as text, one entry per line:
 *   "<dtype> <log2n> <fanout> <basecase_threshold> <sample_rate> <recurse_model> <ms>\n"
 * ls_tune_export: *bytes is the buffer size on input and the bytes written
 * (including the terminating NUL) on output; buf = NULL queries the size.
 * ls_tune_import adds / replaces entries from such text (NUL-terminated);
 * malformed lines or out-of-range values give LS_EINVAL and change nothing. */
ls_status ls_tune_export(ls_ctx* ctx, char* buf, size_t* bytes);
ls_status ls_tune_import(ls_ctx* ctx, const char* text);

/* Synchronise `stream` and return the device status word of the last call
 * on this context (LS_OK, LS_ENAN, LS_ETIMEOUT or LS_EDEVICE), then clear it. */
ls_status ls_last_device_status(ls_ctx* ctx, ls_stream_t stream);

/* Serialise / load a model (versioned POD with a checksum).  *bytes is the
 * buffer size on input and the bytes used on output; pass buf = NULL to
 * query the size. */
ls_status ls_model_export(const ls_model* m, void* buf, size_t* bytes);
ls_status ls_model_import(ls_model* m, const void* buf, size_t bytes);

/* Human-readable name of a status code (static string). */
const char* ls_status_string(ls_status s);

/* Description of the last LS_ECUDA / LS_ENOMEM failure raised on the calling
 * host thread ("" if none): the CUDA error and where it was seen, or which
 * workspace list ran out.  The library never prints; this is its only
 * diagnostic channel.  The string is owned by the library and valid until
 * the thread's next failing call. */
const char* ls_last_error_detail(void);

#ifdef __cplusplus
}
#endif
#endif /* LS_H */
