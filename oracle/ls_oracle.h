/*
 * ls_oracle.h -- plain single-threaded CPU LearnedSort (test infrastructure).
 *
 * THIS IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only tests/, the
 * smoke check in __graft_entry__.py and the cpu_baseline / reference leg of
 * bench.py may load it.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * What it computes (arxiv 2307.08637, "LearnedSort as a learning-augmented
 * SampleSort"):
 *   - the ascending order of 64-bit keys (the sorting problem of Sec. 1/2.2);
 *   - the two-layer RMI  F(x) = f2^{floor(B f1(x))}(x)  of Sec. 2.1, linear
 *     root and B linear leaves, trained on a sorted random sample (Sec. 2.2),
 *     made monotone by per-leaf min/max clamps (Sec. 4, monotone RMI);
 *   - bucket b(x) = floor(B * F(x)) (Sec. 2.2, partitioning routine);
 *   - the splitter-tree SampleSort classifier with equality buckets
 *     (Sec. 2.4, IPS4o) and the model choice of Alg. 5 (BuildPartitionModel);
 *   - recursion on oversized buckets, homogeneity check (Sec. 2.2) and a
 *     base case (Sec. 2.2 / Sec. 4).
 * Every FP64 step is a single correctly rounded IEEE operation in a fixed
 * order; the file is compiled with -ffp-contract=off so no FMA is formed.
 *
 * Keys are 64-bit: doubles (LSREF_F64) or unsigned integers (LSREF_U64).
 * All comparisons use ord(x), an order-preserving map to uint64; the model
 * reads the key as a double.
 */
#ifndef LS_ORACLE_H
#define LS_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LSREF_F64 0
#define LSREF_U64 1

#define LSREF_OK 0
#define LSREF_EINVAL 1
#define LSREF_ENOMEM 2
#define LSREF_ENAN 3

#define LSREF_PART_AUTO 0
#define LSREF_PART_LEARNED 1
#define LSREF_PART_SPLITTER 2

#define LSREF_RECURSE_REFINE_GLOBAL 0
#define LSREF_RECURSE_RETRAIN 1

#define LSREF_MAX_FANOUT 4096
#define LSREF_MAX_LEVELS 48

/* Decision codes recorded per partitioned item. */
#define LSREF_DEC_NONE 0        /* not partitioned (n <= T, n <= 1) */
#define LSREF_DEC_LEARNED 1     /* RMI classifier */
#define LSREF_DEC_SPLITTER 2    /* splitter tree, no equality buckets */
#define LSREF_DEC_SPLITTER_EQ 3 /* splitter tree with equality buckets */
#define LSREF_DEC_HOMOGENEOUS 4 /* all keys equal: left as is */
#define LSREF_DEC_RADIX 5       /* radix split of the bits where the keys differ */

typedef struct {
  uint32_t fanout;             /* B = number of RMI leaves = learned buckets */
  uint32_t splitter_fanout;    /* B_s upper bound for the splitter tree */
  uint32_t basecase_threshold; /* T: items with n <= T go to the base case */
  uint32_t max_depth;          /* items at a deeper level are sorted directly */
  uint32_t min_sample;         /* lower bound on the sample size */
  uint32_t auto_splitter_fanout; /* B_s when Alg. 5 falls back to the tree */
  double sample_rate;          /* r: S = ceil(r n) */
  double dup_frac;             /* Alg. 5 TooManyDuplicates bound (0.10) */
  double imbalance_tau;        /* sample imbalance bound tau */
  uint64_t min_learned_n;      /* Alg. 5 InputSizeIsLarge bound (1e5) */
  uint64_t seed;
  int32_t partitioner;         /* LSREF_PART_* */
  int32_t recurse_model;       /* LSREF_RECURSE_* */
} lsref_params;

/* Two-layer RMI with per-leaf monotonicity clamps (all FP64). */
typedef struct {
  uint32_t L;        /* number of leaves (= B) */
  uint32_t S;        /* sample size it was trained on (informative) */
  double xmin, xmax; /* clamp range: first and last sorted sample key */
  double root_x0, root_a, root_b;
  double leaf_x0[LSREF_MAX_FANOUT];
  double leaf_a[LSREF_MAX_FANOUT];
  double leaf_b[LSREF_MAX_FANOUT];
  double leaf_lo[LSREF_MAX_FANOUT];
  double leaf_hi[LSREF_MAX_FANOUT];
  uint32_t leaf_count[LSREF_MAX_FANOUT]; /* sample points routed to each leaf */
} lsref_model;

/* Splitter classifier.  Without equality buckets: bucket = #{k: t_k < ord}.
 * With equality buckets over unique splitters u_0 < ... < u_{m-1}:
 * bucket 2k+1 = {ord == u_k}, bucket 2k = {u_{k-1} < ord < u_k}. */
typedef struct {
  uint32_t nsplit;     /* number of splitters (B_s - 1, or m unique) */
  uint32_t nbuckets;   /* B_s, or 2m+1 with equality buckets */
  int32_t equality;    /* 1 if equality buckets are used */
  uint64_t split[LSREF_MAX_FANOUT]; /* ord values, ascending */
} lsref_splitter;

typedef struct {
  uint64_t items;          /* items partitioned at this level */
  uint64_t learned;        /* ... with the RMI */
  uint64_t splitter;       /* ... with the splitter tree (no eq buckets) */
  uint64_t splitter_eq;    /* ... with equality buckets */
  uint64_t homogeneous;    /* items found all-equal (left as is) */
  uint64_t noprogress;     /* partitioned items whose keys all fell in one bucket */
  uint64_t base_items;     /* items sorted by the base case */
  uint64_t base_keys;
  uint64_t fallback_items; /* items past max_depth, sorted directly */
  uint64_t fallback_keys;
  uint64_t keys;           /* keys in partitioned items */
  uint64_t max_child;      /* largest bucket produced at this level */
  uint64_t sumsq_child;    /* sum of squared bucket sizes */
  uint64_t eq_keys;        /* keys that landed in equality buckets */
  uint64_t radix;          /* items partitioned by a radix split (no model, no sample) */
} lsref_level_stats;

typedef struct {
  int32_t status;
  int32_t root_decision;        /* LSREF_DEC_* of the (first) root item */
  uint64_t root_sample_size;
  uint64_t root_dups;           /* #{j>=1: ord(s_j) == ord(s_{j-1})} */
  uint64_t root_imbalance_max;  /* max sample-bucket count under the RMI */
  uint32_t root_nbuckets;
  uint32_t levels_used;
  lsref_level_stats level[LSREF_MAX_LEVELS];
} lsref_trace;

/* ---- primitives ---- */
uint64_t lsref_ord(uint64_t bits, int dtype);
uint64_t lsref_unord(uint64_t ord, int dtype);
double lsref_key_value(uint64_t bits, int dtype);
uint64_t lsref_splitmix64(uint64_t state);
uint64_t lsref_seed_item(uint64_t seed, uint64_t segment, uint32_t level, uint64_t gidx);
uint64_t lsref_sample_size(uint64_t n, const lsref_params* p);
void lsref_sample_positions(uint64_t seed_item, uint64_t n, uint64_t S, uint64_t* pos);
void lsref_params_default(lsref_params* p);

/* ---- model ---- */
/* Fit the RMI on a sample sorted by ord (bits, dtype).  L leaves. */
int lsref_fit(const uint64_t* sorted_sample, uint64_t S, int dtype, uint32_t L, lsref_model* m);
double lsref_model_F(const lsref_model* m, double x);
uint32_t lsref_model_leaf(const lsref_model* m, double x);
/* Bucket of one key at refinement level k with global parent index g
 * (k = 0, g = 0 gives floor(B F(x)) clamped to B-1). */
uint32_t lsref_refine_id(const lsref_model* m, uint64_t bits, int dtype, uint32_t B, uint32_t k, uint64_t g);
void lsref_classify(const lsref_model* m, const uint64_t* keys, uint64_t n, int dtype, uint32_t B,
                    uint32_t k, uint64_t g, uint32_t* ids, uint64_t* hist);
/* Forward (prediction, residual) and backward (d MSE / d(a,b)) of the raw
 * linear leaves and the root on the sorted sample. */
void lsref_fit_forward(const lsref_model* m, const uint64_t* sorted_sample, uint64_t S, int dtype,
                       double* pred, double* resid);
void lsref_fit_backward(const lsref_model* m, const uint64_t* sorted_sample, uint64_t S, int dtype,
                        double* grad_a, double* grad_b, double* grad_root);

/* ---- splitter ---- */
void lsref_splitter_build(const uint64_t* sorted_sample, uint64_t S, int dtype, uint32_t bs_max,
                          int force_equality, lsref_splitter* t);
uint32_t lsref_splitter_bucket(const lsref_splitter* t, uint64_t ord);
void lsref_splitter_classify(const lsref_splitter* t, const uint64_t* keys, uint64_t n, int dtype,
                             uint32_t* ids, uint64_t* hist);

/* ---- full sorts ---- */
/* Sort in place (ascending ord).  trace may be NULL.  root_model/root_hist
 * (nullable) receive the first root item's model and bucket histogram. */
int lsref_sort(uint64_t* keys, uint64_t n, int dtype, const lsref_params* p, lsref_trace* trace,
               lsref_model* root_model, uint64_t* root_hist);
/* Independent segments [off[s], off[s+1]).  seg_decision (nullable) gets each
 * root's decision code. */
int lsref_sort_segmented(uint64_t* keys, const uint64_t* off, uint32_t nseg, int dtype,
                         const lsref_params* p, lsref_trace* trace, int32_t* seg_decision);

/* Root-item decision only (sample, sort, dup count, Alg. 5, fit), no partitioning. */
int lsref_root_decision(const uint64_t* keys, uint64_t n, int dtype, const lsref_params* p,
                        uint64_t segment, lsref_trace* trace, lsref_model* m, lsref_splitter* t,
                        uint64_t* sorted_sample_out);

size_t lsref_sizeof_model(void);
size_t lsref_sizeof_trace(void);
size_t lsref_sizeof_params(void);
size_t lsref_sizeof_splitter(void);

#ifdef __cplusplus
}
#endif
#endif
