// ls_common.cuh -- device data structures and FP64 model arithmetic shared by
// the CUDA translation units of the learned SampleSort library.
//
// Notation follows arxiv 2307.08637: B buckets (= L RMI leaves), S sample
// size, F(x) the two-layer RMI of Sec. 2.1, b(x) = floor(B F(x)) (Sec. 2.2).
// Every FP64 step of the model is one explicitly rounded operation
// (__dadd_rn / __dsub_rn / __dmul_rn / __ddiv_rn), never contracted into an
// FMA, in a fixed order; max(p,q) = p < q ? q : p, min(p,q) = q < p ? q : p.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ls.h"

namespace lsg {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;  // SplitMix64 increment
constexpr uint32_t kChunk = 256;                      // FP64 summation chunk
constexpr double kRefineLimit = 1125899906842624.0;   // 2^50: deepest B^(k+1) refined
constexpr uint64_t kOrdMinF64 = 0x000FFFFFFFFFFFFFull; // ord(-inf)
constexpr uint64_t kOrdMaxF64 = 0xFFF0000000000000ull; // ord(+inf)
constexpr uint32_t kMaxBaseCase = 8192;               // largest shared-memory base case
constexpr uint32_t kWarpSortMax = 256;                // warp-register base case size
constexpr uint32_t kWarpSmallMax = 128;               // spans up to this size: the warp base case's short class
constexpr uint32_t kSortChunk = 2048;                 // segmented sample sort chunk
constexpr uint32_t kTileKeys = 4096;                  // keys per partition tile (256 threads x 16)
constexpr uint32_t kChunkTiles = 16;                  // tiles per chunk (one lookback unit)
constexpr uint64_t kChunkKeys = (uint64_t)kTileKeys * kChunkTiles;

enum : uint8_t { KIND_FRESH = 0, KIND_FORCE_SPLITTER = 1, KIND_REFINE = 2, KIND_RADIX = 3 };
enum : uint8_t { CLS_DIRECT = 0, CLS_TREE = 1, CLS_DIR = 2, CLS_GUESS = 3, CLS_RADIX = 4 };
enum : uint8_t { FLAG_SKIP_SCATTER = 1, FLAG_HOMOGENEOUS = 2, FLAG_NOPROGRESS = 4, FLAG_ORDER_FREE = 8 };

// One RMI leaf f2^(i)(x) = a (x - x0) + b, clamped to [lo, hi] (Sec. 4).
struct Leaf {
  double x0, a, b, lo, hi;
};

// Device-resident RMI header; leaves live in a pool at leaf_off.
struct DModel {
  double xmin, xmax;   // clamp range (first / last sorted sample key)
  double rx0, ra, rb;  // root f1(x) = ra (x - rx0) + rb
  uint32_t L, S;
  uint64_t leaf_off;
  uint32_t ok;         // 1 if every parameter is finite
  uint32_t pad;
};

// FP32 image of a model, used only to guess a bucket that exact pivots then
// correct: root r = raL (xf - rx0f) + rbL gives the leaf, leaf i is
// F ~ a_i (xf - x0_i) + b_i (FLeaf = {x0, a, b, unused}).
struct FModel {
  float xminf, xmaxf, rx0f, raL, rbL;
  uint32_t L;
  uint64_t leaf_off;  // offset into the FLeaf pool (same as the FP64 leaves)
};
typedef float4 FLeaf;
// FP32 image of a leaf's monotone clamps [lo, hi] (Sec. 4).
typedef float2 FClamp;

// A range of keys still to be partitioned (a bucket of the previous level).
struct Item {
  uint64_t lo, n;          // keys [lo, lo + n) of buffer `buf`
  uint64_t gidx;           // global bucket index (sampling seed)
  uint64_t mg;             // refine: parent index g inside the model
  uint64_t ord_lo, ord_hi; // every key of the item has ord in [ord_lo, ord_hi]
  uint32_t segment;
  uint16_t level, mk;      // recursion level; refine depth k below the model (radix: keys agree above bit mk)
  int32_t model;           // refine: model slot
  uint8_t kind, buf;       // KIND_*; 0 = keys array, 1 = workspace buffer
  uint16_t pad;
};
static_assert(sizeof(Item) == 64, "Item layout");

// Per-item plan of one batch: host fills offsets, device fills the rest.
struct Plan {
  uint64_t chunk_begin; // first chunk of the item in this batch's chunk space
  uint64_t sample_off;  // fresh items: offset in the sample pool
  uint64_t cnt_off;     // offset in the count / cursor pools (nb_cap entries)
  uint64_t tab_off;     // offset in the pivot pool (nb_pad_cap entries)
  uint64_t dir_off;     // offset in the directory pool
  uint64_t dir_lo;      // ord at directory cell 0
  uint64_t dir_hi;      // last pivot; keys >= dir_hi are in bucket kmax
  unsigned int mixed;   // K1: 1 when some key of the item differs from its first key
  unsigned int pad0;
  unsigned long long odiff;  // K1: OR over the keys of ord(x) ^ ord(first key)
  unsigned long long dups;        // fresh: sample duplicates
  unsigned long long imb;         // fresh: largest sample bucket under the RMI
  double P, Bg;         // refine scale B^(k+1) and offset B g
  uint32_t S;           // fresh: sample size
  uint32_t nb;          // buckets
  uint32_t nb_pad;      // pivot table length (power of two)
  uint32_t kmax;        // largest bucket a key of the item can get
  uint32_t dir_shift;
  uint32_t dir_cells;
  int32_t model;        // model used to classify (learned), -1 otherwise
  uint32_t fit_slot;    // fresh learned candidates: index in the fit arrays
  uint8_t cls;          // CLS_*
  uint8_t decision;     // LS_DEC_*
  uint8_t fresh;        // 1 if the item drew its own sample
  uint8_t flags;        // FLAG_*
  uint8_t want;         // fresh: fit attempted
  uint8_t pad[3];
};

// A finished range: sort it (base case / fallback) or copy it home.
struct Span {
  uint64_t lo;
  uint32_t n;
  uint32_t buf;
};

// Device counters of one level (reset per level by the host).
struct LevelCounters {
  unsigned long long n_next;       // items appended for the next level
  unsigned long long n_base_small; // spans for the warp base case
  unsigned long long n_base_large; // spans for the CTA base case
  unsigned long long n_copy;       // spans to copy from the buffer
  unsigned long long n_fallback;   // spans past max_depth
  unsigned long long overflow;     // a list ran out of capacity
  unsigned long long n_base_mid;   // spans for the warp base case's long class (kWarpSmallMax, kWarpSortMax]
};

// Device-side level statistics (mirrors ls_level_stats field order).
struct DevLevelStats {
  unsigned long long items, learned, splitter, splitter_eq, homogeneous, noprogress;
  unsigned long long base_items, base_keys, fallback_items, fallback_keys;
  unsigned long long keys, max_child, sumsq_child, eq_keys;
  unsigned long long radix;
};
static_assert(sizeof(DevLevelStats) == sizeof(ls_level_stats), "stats layout");

// ------------------------------------------------------------------ keys

__host__ __device__ __forceinline__ uint64_t ord_of(uint64_t bits, int dt) {
  return dt ? bits : ((bits >> 63) ? ~bits : (bits ^ 0x8000000000000000ull));
}
__host__ __device__ __forceinline__ uint64_t unord(uint64_t u, int dt) {
  return dt ? u : ((u >> 63) ? (u ^ 0x8000000000000000ull) : ~u);
}
__device__ __forceinline__ double key_value(uint64_t bits, int dt) {
  return dt ? __ull2double_rn(bits) : __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double ord_value(uint64_t u, int dt) { return key_value(unord(u, dt), dt); }

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t seed_item(uint64_t seed, uint64_t segment, uint32_t level,
                                                       uint64_t gidx) {
  uint64_t tag = (segment << 40) + ((uint64_t)level << 32) + (gidx & 0xFFFFFFFFull);
  return splitmix64(seed ^ tag);
}

// ------------------------------------------------------------- FP64 model

// First statement of every kernel: wait for the stream's previous kernel
// when this one was launched as a programmatic dependent (no-op otherwise).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ double dmax(double p, double q) { return (p < q) ? q : p; }
__device__ __forceinline__ double dmin(double p, double q) { return (q < p) ? q : p; }

// Integer index from a floored double: values that are not > 0 (negatives,
// zeros, NaN from a non-finite model) give 0, values >= hi give hi; equal to
// min(max(t, 0), hi) for every non-NaN t.  No NaN ever reaches a conversion.
__device__ __forceinline__ uint32_t clamp_index(double t, uint32_t hi) {
  if (!(t > 0.0)) return 0;
  if (!(t < (double)hi)) return hi;
  return (uint32_t)t;
}

// Root routing: leaf floor(L f1(xc)) clamped to [0, L-1] (Sec. 2.1).
__device__ __forceinline__ uint32_t root_leaf(const DModel& m, double xc) {
  double t = __dsub_rn(xc, m.rx0);
  t = __dmul_rn(m.ra, t);
  t = __dadd_rn(t, m.rb);
  t = __dmul_rn(t, (double)m.L);
  t = floor(t);
  return clamp_index(t, m.L - 1);
}

// Raw linear leaf f2^(i)(xc).
__device__ __forceinline__ double leaf_eval(const Leaf& l, double xc) {
  double f = __dsub_rn(xc, l.x0);
  f = __dmul_rn(l.a, f);
  f = __dadd_rn(f, l.b);
  return f;
}

// F(x): clamp x to the sample range, route, evaluate the leaf, clamp to the
// leaf's monotone [lo, hi] (Sec. 2.1 + Sec. 4).
__device__ __forceinline__ double model_F(const DModel& m, const Leaf* __restrict__ leaves, double x) {
  double xc = dmax(x, m.xmin);
  xc = dmin(xc, m.xmax);
  uint32_t i = root_leaf(m, xc);
  Leaf l = leaves[i];
  double f = leaf_eval(l, xc);
  f = dmax(f, l.lo);
  f = dmin(f, l.hi);
  return f;
}

// True when B^e exceeds the FP64 refinement limit 2^50 (B >= 2; the
// product stops growing once it is past the limit).
__host__ __device__ __forceinline__ bool beyond_refine_limit(uint32_t B, uint32_t e) {
  double P = 1.0;
  for (uint32_t i = 0; i < e && P <= kRefineLimit; ++i) P = P * (double)B;
  return P > kRefineLimit;
}

// Radix split of a bucket whose keys agree above bit `top`: the window of
// ord bits [shift, top), at most kRadixBits wide.
constexpr uint32_t kRadixBits = 10;
__host__ __device__ __forceinline__ uint32_t radix_shift(uint32_t top) {
  return top > kRadixBits ? top - kRadixBits : 0;
}
__host__ __device__ __forceinline__ uint32_t radix_buckets(uint32_t top) {
  const uint32_t s = radix_shift(top);
  return top > s ? 1u << (top - s) : 2u;
}

// Refinement bucket (k levels below the model's item, parent index g):
// id = clamp(floor(F(x) P) - Bg, 0, B-1), P = B^(k+1), Bg = B g.
__device__ __forceinline__ uint32_t refine_id(const DModel& m, const Leaf* __restrict__ leaves, double x, double P,
                                              double Bg, uint32_t B) {
  double F = model_F(m, leaves, x);
  double t = __dmul_rn(F, P);
  t = floor(t);
  t = __dsub_rn(t, Bg);
  return clamp_index(t, B - 1);
}

// --------------------------------------------------- pivot-table search

// Bucket of ord value u from an exact pivot table: T[j] (j = 1..nb_pad-1,
// non-decreasing) is the smallest ord with bucket >= j, so the bucket is
// #{j : T[j] <= u}, clamped to kmax (pivots past kmax are padding).
// Branchless binary search; nb_pad is a power of two.
__device__ __forceinline__ uint32_t pivot_count(const uint64_t* __restrict__ T, uint32_t nb_pad, uint64_t u) {
  uint32_t c = 0;
#pragma unroll 1
  for (uint32_t s = nb_pad >> 1; s >= 1; s >>= 1) {
    uint32_t c2 = c + s;
    c = (T[c2] <= u) ? c2 : c;
  }
  return c;
}

// Same result through a radix directory over [dir_lo, dir_hi]: D[c] is the
// bucket at the start of cell c, so u's bucket lies in [D[c], D[c+1]].
__device__ __forceinline__ uint32_t pivot_count_dir(const uint64_t* __restrict__ T, const uint16_t* __restrict__ D,
                                                    uint64_t dir_lo, uint64_t dir_hi, uint32_t shift,
                                                    uint32_t kmax, uint64_t u) {
  if (u < dir_lo) return 0;
  if (u >= dir_hi) return kmax;
  uint32_t c = (uint32_t)((u - dir_lo) >> shift);
  uint32_t b = D[c];
  uint32_t e = D[c + 1];
  // narrow [b, e] with a short binary search, then step
  while (e - b > 4) {
    uint32_t mid = (b + e + 1) >> 1;
    if (T[mid] <= u) b = mid;
    else e = mid - 1;
  }
  while (b < e && T[b + 1] <= u) ++b;
  return b;
}

// Key -> float by bit manipulation (round toward zero), no FP64 or
// conversion-pipe instruction: doubles outside the float range saturate to
// +-0 / +-inf, u64 keys keep their top 24 significant bits.  Monotone in
// the key order; only used for guesses.
__device__ __forceinline__ float key_to_float(uint64_t bits, int dt) {
  if (dt) {
    if (bits == 0) return 0.0f;
    uint32_t lz = __clzll((long long)bits);
    uint32_t e = 63 - lz;
    uint32_t mant = (uint32_t)((bits << lz) >> 40) & 0x7FFFFFu;
    return __uint_as_float(((e + 127u) << 23) | mant);
  }
  uint32_t hi = (uint32_t)(bits >> 32);
  uint32_t sign = hi & 0x80000000u;
  int32_t e = (int32_t)((hi >> 20) & 0x7FF) - 1023 + 127;
  uint32_t mant = (uint32_t)((bits >> 29) & 0x7FFFFFu);
  uint32_t f;
  if (e <= 0) f = sign;                       // zero, subnormal, underflow
  else if (e >= 255) f = sign | 0x7F800000u;  // inf or overflow
  else f = sign | ((uint32_t)e << 23) | mant;
  return __uint_as_float(f);
}

// Bucket guess from the FP32 model image (leaves in shared memory), for
// refinement scale P and offset Bg; clamped to [0, kmax].  fc (nullable):
// the leaves' clamps, without which refined guesses (P = B^2 and beyond)
// are often several buckets off where a clamp binds.
__device__ __forceinline__ uint32_t guess_bucket(const FModel& m, const FLeaf* __restrict__ fl,
                                                 const FClamp* __restrict__ fc, float Pf, float Bgf, uint32_t kmax,
                                                 uint64_t bits, int dt) {
  float x = key_to_float(bits, dt);
  x = fminf(fmaxf(x, m.xminf), m.xmaxf);
  // floor to int (saturating) and clamp as integers
  const int li = min(max(__float2int_rd(__fmaf_rn(m.raL, x - m.rx0f, m.rbL)), 0), (int)m.L - 1);
  FLeaf l = fl[li];
  float F = __fmaf_rn(l.y, x - l.x, l.z);
  if (fc) {
    const FClamp c = fc[li];
    F = fminf(fmaxf(F, c.x), c.y);
  }
  return (uint32_t)min(max(__float2int_rd(__fmaf_rn(F, Pf, -Bgf)), 0), (int)kmax);
}

// Exact bucket #{j <= kmax : T[j] <= u} from a guess: two steps either way,
// then the full branchless search.  T[0] <= every key of the item.
__device__ __forceinline__ uint32_t fix_bucket(const uint64_t* __restrict__ T, uint32_t nb_pad, uint32_t kmax,
                                               uint32_t g, uint64_t u) {
  uint32_t b = g;
  if (T[b] > u) {
    --b;
    if (T[b] > u) {
      --b;
      if (T[b] > u) {
        b = pivot_count(T, nb_pad, u);
        return b < kmax ? b : kmax;
      }
    }
    return b;
  }
  if (b < kmax && T[b + 1] <= u) {
    ++b;
    if (b < kmax && T[b + 1] <= u) {
      ++b;
      if (b < kmax && T[b + 1] <= u) {
        b = pivot_count(T, nb_pad, u);
        return b < kmax ? b : kmax;
      }
    }
  }
  return b;
}

}  // namespace lsg
