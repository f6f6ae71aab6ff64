// ls_partition.cu -- the partitioning side of learned SampleSort on GB300:
//   K1  classify + per-chunk histogram (+ homogeneity flag for the check of
//       Sec. 2.2, + NaN check), shared-memory histograms, u16 bucket ids;
//   chunk prefixes: per chunk and bucket, where the chunk's keys of that
//       bucket start (a stable counting sort's offsets, Sec. 2.4);
//   K2  per item: bucket write cursors, children (next level / base case /
//       final), level statistics;
//   K3  stable scatter: rank keys per bucket with warp votes and warp-private
//       counters, stage each tile grouped by bucket in shared memory and
//       write contiguous runs;
//   base case: warp model-placed counting sort (<= 256 keys), shared-memory
//       bitonic sort (<= 4096 keys), merge-sort fallback past max_depth;
//   key-value forms of K3 and the base cases, copies, the host-link copy.
#include <cstdio>

#include <type_traits>

#include "ls_kernels.h"

namespace lsg {

namespace {

constexpr int kTPB = 256;
constexpr int kKPT = 16;  // keys per thread per tile
constexpr uint32_t kTile = kTPB * kKPT;
static_assert(kTile == kTileKeys, "tile size shared with the host planner");
constexpr uint32_t kCopyPiece = 65536;

inline unsigned grid_for(uint64_t n, int tpb = kTPB) { return (unsigned)((n + tpb - 1) / tpb); }

// Warp-aggregated shared-memory increment; returns the key's rank among the
// keys of its bucket counted so far in this block.  b == ~0u is "no key".
__device__ __forceinline__ uint32_t agg_inc(uint32_t* h, uint32_t b) {
  unsigned peers = __match_any_sync(0xFFFFFFFFu, b);
  unsigned lane = threadIdx.x & 31;
  int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if ((int)lane == leader && b != 0xFFFFFFFFu) base = atomicAdd(&h[b], (uint32_t)__popc(peers));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  return base + __popc(peers & ((1u << lane) - 1u));
}

struct Cls {
  uint64_t dir_lo, dir_hi;
  double P, Bg;
  FModel fm;
  float Pf, Bgf;
  uint32_t nb_pad, kmax, shift, B;
  int32_t model;
  uint8_t cls;
  uint8_t agg;    // warp-aggregate histogram increments (splitters: duplicates collide)
  uint8_t clamp;  // refined item (P > B): the FP32 guess applies the leaves' clamps
};

// Load item pi's classifier into shared memory (all threads).
// aux_model: the model whose FP32 leaves are in sAux (-1: none); items that
// refine one global model share them, so they are copied once per block.
__device__ void load_cls(const PassArgs& a, const RunParams& rp, uint32_t pi, Cls& c, uint64_t* sT, void* sAux,
                         int32_t& aux_model) {
  const Plan& pl = a.plans[pi];
  c.cls = pl.cls;
  c.nb_pad = pl.nb_pad;
  c.kmax = pl.kmax;
  c.dir_lo = pl.dir_lo;
  c.dir_hi = pl.dir_hi;
  c.shift = pl.dir_shift;
  c.P = pl.P;
  c.Bg = pl.Bg;
  c.Pf = (float)pl.P;
  c.Bgf = (float)pl.Bg;
  c.B = rp.B;
  c.model = pl.model;
  c.agg = pl.decision != LS_DEC_LEARNED;
  c.clamp = pl.P > (double)rp.B;  // at P = B the unclamped guess is already within one bucket
  if (c.cls == CLS_DIRECT) {
    c.kmax = rp.B - 1;
    return;
  }
  if (c.cls == CLS_RADIX) return;  // no table: the bucket is a bit field of ord
  const uint64_t* T = a.pivots + pl.tab_off;
  for (uint32_t j = threadIdx.x; j < c.nb_pad; j += blockDim.x) sT[j] = T[j];
  if (c.cls == CLS_DIR) {
    const uint16_t* D = a.dirs + pl.dir_off;
    uint16_t* sD = static_cast<uint16_t*>(sAux);
    for (uint32_t j = threadIdx.x; j <= pl.dir_cells; j += blockDim.x) sD[j] = D[j];
  } else if (c.cls == CLS_GUESS) {
    c.fm = a.fmodels[pl.model];
    if (aux_model != pl.model) {
      const FLeaf* F = a.fleaves + c.fm.leaf_off;
      const FClamp* C = a.fclamps + c.fm.leaf_off;
      FLeaf* sF = static_cast<FLeaf*>(sAux);
      FClamp* sC = reinterpret_cast<FClamp*>(sF + c.fm.L);
      for (uint32_t j = threadIdx.x; j < c.fm.L; j += blockDim.x) {
        sF[j] = F[j];
        sC[j] = C[j];
      }
      aux_model = pl.model;
    }
  }
}

// ------------------------------------------------------------------ K1

// Exact bucket #{j <= kmax : T[j] <= u} - 1 from a guess g in [0, kmax]
// that is usually right or one off: the two table entries around g are read
// together and decide -1 / 0 / +1; a third read confirms the step, and only
// a guess two or more off takes the full search.  T[0] <= every key of the
// item, so a guess can be too high only when g >= 1.
__device__ __forceinline__ uint32_t fix_guess(const uint64_t* __restrict__ T, uint32_t nb_pad, uint32_t kmax,
                                              uint32_t g, uint64_t u) {
  const uint32_t g1 = g < kmax ? g + 1 : kmax;
  const uint64_t A = T[g], B1 = T[g1];
  const bool lo = A > u;
  const bool hi = g < kmax && B1 <= u;
  const uint32_t g2 = g1 < kmax ? g1 + 1 : kmax;
  const uint64_t C = T[lo ? (g ? g - 1 : 0) : g2];
  const bool far = lo ? (g == 0 || C > u) : (hi && g1 < kmax && C <= u);
  uint32_t b = g - (uint32_t)lo + (uint32_t)hi;
  if (far) {
    b = pivot_count(T, nb_pad, u);
    b = b < kmax ? b : kmax;
  }
  return b;
}

// fix_guess for guesses that are almost always exact (root items, P = B:
// the FP32 image's error is far below a bucket): the two table entries
// around g confirm it, and only the rare miss takes the general fix.
__device__ __forceinline__ uint32_t fix_guess_likely(const uint64_t* __restrict__ T, uint32_t nb_pad, uint32_t kmax,
                                                     uint32_t g, uint64_t u) {
  const uint32_t g1 = g < kmax ? g + 1 : kmax;
  if (T[g] <= u && (g == kmax || T[g1] > u)) return g;
  return fix_guess(T, nb_pad, kmax, g, u);
}

// Bucket of one key for a classifier kind and key type known at compile time.
template <int CLS, int DT>
__device__ __forceinline__ uint32_t classify_as(uint64_t bits, const Cls& c, const uint64_t* sT, const void* sAux,
                                                const DModel* models, const Leaf* leaves) {
  if (CLS == CLS_DIRECT) {
    const DModel& m = models[c.model];
    return refine_id(m, leaves + m.leaf_off, key_value(bits, DT), c.P, c.Bg, c.B);
  }
  const uint64_t u = ord_of(bits, DT);
  if (CLS == CLS_RADIX) return (uint32_t)(u >> c.shift) & c.kmax;  // kmax = buckets - 1, a power of two minus 1
  if (CLS == CLS_GUESS) {
    const FLeaf* sF = static_cast<const FLeaf*>(sAux);
    const FClamp* sC = c.clamp ? reinterpret_cast<const FClamp*>(sF + c.fm.L) : nullptr;
    const uint32_t g = guess_bucket(c.fm, sF, sC, c.Pf, c.Bgf, c.kmax, bits, DT);
    return c.clamp ? fix_guess(sT, c.nb_pad, c.kmax, g, u) : fix_guess_likely(sT, c.nb_pad, c.kmax, g, u);
  }
  const uint32_t b = (CLS == CLS_DIR)
                         ? pivot_count_dir(sT, static_cast<const uint16_t*>(sAux), c.dir_lo, c.dir_hi, c.shift, c.kmax, u)
                         : pivot_count(sT, c.nb_pad, u);
  return b < c.kmax ? b : c.kmax;
}

// Histogram increment that stays cheap when a warp's keys all share one
// bucket (duplicates under equality buckets): one add of the lane count.
__device__ __forceinline__ void hist_add(uint32_t* sH, uint32_t b, bool agg) {
  if (agg) {
    const unsigned act = __activemask();
    const uint32_t lo = __reduce_min_sync(act, b), hi = __reduce_max_sync(act, b);
    if (lo == hi) {
      if ((threadIdx.x & 31) == (unsigned)(__ffs(act) - 1) && b != 0xFFFFFFFFu) atomicAdd(&sH[b], (uint32_t)__popc(act));
      return;
    }
  }
  if (b != 0xFFFFFFFFu) atomicAdd(&sH[b], 1u);
}

// One chunk of K1: classify, store ids, histogram; OR every key's ord into
// `diff` XOR the item's first key's ord (zero <=> the item is homogeneous;
// its highest bit is the highest bit in which two keys differ) and, when
// NANCHK, flag NaNs (|bits| above infinity's).
// K1 keys per thread per step and resident blocks per SM (register budget):
// the guess classifier is short and gains from more warps; the search
// classifiers are chains of dependent table reads and gain from more
// independent keys per thread.
__host__ __device__ constexpr int k1_kpt(int cls) { return (cls == CLS_GUESS || cls == CLS_RADIX) ? 8 : 16; }
__host__ __device__ constexpr int k1_blocks(int cls) { return (cls == CLS_GUESS || cls == CLS_RADIX) ? 4 : 3; }

template <int CLS, int DT, bool NANCHK>
__device__ __forceinline__ void k1_chunk(const PassArgs& a, const Cls& c, const uint64_t* sT, const void* sD,
                                         uint32_t* sH, const uint64_t* src, uint16_t* idout, uint64_t clen,
                                         uint64_t first, uint64_t& diff, bool& nan) {
  constexpr uint64_t kAbs = 0x7FFFFFFFFFFFFFFFull, kInf = 0x7FF0000000000000ull;
  constexpr int kK1KPT = k1_kpt(CLS);
  constexpr uint32_t kK1Tile = kTPB * kK1KPT;
  for (uint64_t t0 = 0; t0 < clen; t0 += kK1Tile) {
    const uint32_t len = clen - t0 < kK1Tile ? (uint32_t)(clen - t0) : kK1Tile;
    const uint64_t* s = src + t0 + threadIdx.x;
    uint16_t* d = idout + t0 + threadIdx.x;
    if (CLS == CLS_GUESS && len == kK1Tile) {
      // the guess classifier in steps over groups of the thread's keys, so
      // that their shared-memory reads are in flight together: the guesses
      // (leaf reads), the table entries around them, then the rare keys
      // whose guess is two or more buckets off (the full search)
      constexpr int KG = 2;
      uint64_t v[kK1KPT];
#pragma unroll
      for (int k = 0; k < kK1KPT; ++k) v[k] = s[k * kTPB];
      const FLeaf* sF = static_cast<const FLeaf*>(sD);
      const FClamp* sC = c.clamp ? reinterpret_cast<const FClamp*>(sF + c.fm.L) : nullptr;
      const uint32_t kmax = c.kmax;
#pragma unroll
      for (int h = 0; h < kK1KPT; h += KG) {
        uint32_t g[KG];
#pragma unroll
        for (int k = 0; k < KG; ++k) {
          const uint64_t bits = v[h + k];
          if (NANCHK) nan |= (bits & kAbs) > kInf;
          diff |= ord_of(bits, DT) ^ first;
          g[k] = guess_bucket(c.fm, sF, sC, c.Pf, c.Bgf, kmax, bits, DT);
        }
        uint32_t miss = 0;
        if (c.clamp) {  // often one off: the reads on both sides decide -1 / 0 / +1
#pragma unroll
          for (int k = 0; k < KG; ++k) {
            const uint64_t u = ord_of(v[h + k], DT);
            const uint32_t gk = g[k], g1 = gk < kmax ? gk + 1 : kmax;
            const uint32_t g2 = g1 < kmax ? g1 + 1 : kmax, gm = gk ? gk - 1 : 0u;
            const uint64_t A = sT[gk], B1 = sT[g1], Cm = sT[gm], C2 = sT[g2];
            const bool lo = A > u;
            const bool hi = gk < kmax && B1 <= u;
            const bool far = lo ? (gk == 0 || Cm > u) : (hi && g1 < kmax && C2 <= u);
            g[k] = gk - (uint32_t)lo + (uint32_t)hi;
            if (far) miss |= 1u << k;
          }
          if (miss) {
#pragma unroll
            for (int k = 0; k < KG; ++k)
              if (miss & (1u << k)) {
                const uint32_t b = pivot_count(sT, c.nb_pad, ord_of(v[h + k], DT));
                g[k] = b < kmax ? b : kmax;
              }
          }
        } else {  // almost always exact: the two reads around the guess confirm it
#pragma unroll
          for (int k = 0; k < KG; ++k) {
            const uint64_t u = ord_of(v[h + k], DT);
            const uint32_t gk = g[k], g1 = gk < kmax ? gk + 1 : kmax;
            if (!(sT[gk] <= u && (gk == kmax || sT[g1] > u))) miss |= 1u << k;
          }
          if (miss) {
#pragma unroll
            for (int k = 0; k < KG; ++k)
              if (miss & (1u << k)) g[k] = fix_guess(sT, c.nb_pad, kmax, g[k], ord_of(v[h + k], DT));
          }
        }
#pragma unroll
        for (int k = 0; k < KG; ++k) {
          d[(h + k) * kTPB] = (uint16_t)g[k];
          hist_add(sH, g[k], c.agg);
        }
      }
    } else if (len == kK1Tile) {
      uint64_t v[kK1KPT];
#pragma unroll
      for (int k = 0; k < kK1KPT; ++k) v[k] = s[k * kTPB];
#pragma unroll
      for (int k = 0; k < kK1KPT; ++k) {
        const uint64_t bits = v[k];
        if (NANCHK) nan |= (bits & kAbs) > kInf;
        diff |= ord_of(bits, DT) ^ first;
        const uint32_t b = classify_as<CLS, DT>(bits, c, sT, sD, a.models, a.leaves);
        d[k * kTPB] = (uint16_t)b;
        hist_add(sH, b, c.agg);
      }
    } else {
      for (int k = 0; k < kK1KPT; ++k) {
        const uint32_t idx = k * kTPB + threadIdx.x;
        uint32_t b = 0xFFFFFFFFu;
        if (idx < len) {
          const uint64_t bits = s[k * kTPB];
          if (NANCHK) nan |= (bits & kAbs) > kInf;
          diff |= ord_of(bits, DT) ^ first;
          b = classify_as<CLS, DT>(bits, c, sT, sD, a.models, a.leaves);
          d[k * kTPB] = (uint16_t)b;
        }
        hist_add(sH, b, c.agg);
      }
    }
  }
}

// Classify every key of every chunk whose item uses classifier CLS,
// histogram per chunk in shared memory; write the chunk's bucket counts
// (dense row, read by the chunk-prefix kernels), add them to the item's
// totals, store each key's bucket id, and flag items that are not
// homogeneous.  One kernel per classifier kind, key type and NaN check keeps
// each instance's registers and instructions to what it needs.
template <int CLS, int DT, bool NANCHK>
__global__ void __launch_bounds__(kTPB, k1_blocks(CLS)) k_classify_hist(PassArgs a, RunParams rp) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* sT = reinterpret_cast<uint64_t*>(smem);
  void* sD = sT + a.nb_pad_max;  // directory or FP32 leaves (aux_bytes, 16-byte aligned)
  uint32_t* sH = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(sD) + a.aux_bytes);
  for (uint32_t j = threadIdx.x; j < a.nb_pad_max; j += blockDim.x) sH[j] = 0;
  uint32_t cur = 0xFFFFFFFFu;
  int32_t aux_model = -1;
  Cls c;
  bool nan = false;
  const uint64_t nch = batch_chunks(a), ckeys = batch_chunk_keys(a);
  for (uint64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const uint32_t pi = a.chunk_plan[ch];
    if (a.plans[pi].cls != CLS) continue;  // uniform across the block
    if (pi != cur) {
      __syncthreads();
      load_cls(a, rp, pi, c, sT, sD, aux_model);
      cur = pi;
      __syncthreads();
    }
    const Item& it = a.items[pi];
    const Plan& pl = a.plans[pi];
    const uint64_t c0 = (ch - pl.chunk_begin) * ckeys;
    const uint64_t clen = it.n - c0 < ckeys ? it.n - c0 : ckeys;
    const uint64_t* keys = it.buf ? a.keysB : a.keysA;
    uint64_t diff = 0;
    k1_chunk<CLS, DT, NANCHK>(a, c, sT, sD, sH, keys + it.lo + c0, a.ids + it.lo + c0, clen,
                              ord_of(keys[it.lo], DT), diff, nan);
    __syncthreads();
    uint32_t* row = a.agg + ch * a.nb_pad_max;
    for (uint32_t j = threadIdx.x; j < c.nb_pad; j += blockDim.x) {
      const uint32_t h = sH[j];
      row[j] = h;
      if (h) {
        atomicAdd(&a.counts[pl.cnt_off + j], (unsigned long long)h);
        sH[j] = 0;
      }
    }
    unsigned long long d = diff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d |= __shfl_xor_sync(0xFFFFFFFFu, d, o);
    if ((threadIdx.x & 31) == 0 && d) {
      if ((a.plans[pi].odiff | d) != a.plans[pi].odiff) atomicOr(&a.plans[pi].odiff, d);
      if (!a.plans[pi].mixed) atomicExch(&a.plans[pi].mixed, 1u);
    }
    __syncthreads();
  }
  if (NANCHK && __syncthreads_or(nan ? 1 : 0) && threadIdx.x == 0) atomicCAS(a.status, 0u, (unsigned)LS_ENAN);
}

// ------------------------------------------------------------------ K3

// Rank of this lane's key among the keys of the same id that the warp has
// seen so far (its earlier steps, then lower lanes of this step), and the
// advance of the warp's counter for that id.  The lanes holding the same id
// are found with one warp vote per id bit (ids below 2^NB): a lane keeps the
// voters that agree with it on every bit.  Votes need no shared memory and
// their cost grows with log2 of the bucket count only.  The warp's 16-bit
// counter for the id is read by every lane of the group and advanced by the
// group's lowest lane (the other warp sharing the word owns its other half).
// FULL: every lane holds a key; otherwise lanes with id 0xFFFF take no part.
template <bool FULL, uint32_t NB>
__device__ __forceinline__ uint32_t rank_step(uint32_t b, uint32_t* myc, unsigned lane, uint32_t wsh, unsigned lt) {
  const bool valid = FULL || b != 0xFFFFu;
  const uint32_t bb = valid ? b : 0u;
  uint16_t* c16 = reinterpret_cast<uint16_t*>(myc + bb) + (wsh >> 4);
  const uint32_t old = *c16;
  unsigned p = FULL ? 0xFFFFFFFFu : __ballot_sync(0xFFFFFFFFu, valid);
#pragma unroll
  for (uint32_t i = 0; i < NB; ++i) {
    const bool on = (bb >> i) & 1u;
    const unsigned v = __ballot_sync(0xFFFFFFFFu, on);
    p &= on ? v : ~v;
  }
  if (!valid) p = 0;
  if ((int)lane == __ffs(p) - 1) *c16 = (uint16_t)(old + __popc(p));
  __syncwarp();  // the next step's reads see this step's counters
  return old + __popc(p & lt);
}

// Stable scatter, one tile of kTile keys at a time.  Chunks are taken in
// order from a global counter; a chunk's per-bucket start comes from the
// chunk-prefix kernels (bucket cursor + keys of the bucket in the item's
// earlier chunks).  Inside a tile each warp owns kTile/(TPB/32) consecutive
// keys and ranks them in order with warp-private counters; a per-bucket
// prefix over the warps and a scan over the buckets place every key in a
// staging buffer grouped by bucket, which is written out with runs of
// consecutive destinations.  Keys keep their relative order within a bucket
// (the stable counting sort of the partitioning step).  Counters of warps 2i
// and 2i+1 share a word, 16 bits each (a warp ranks at most 512 keys).
// TPB: threads per block; QM: bucket ranges of TPB buckets (nb_pad <= QM*TPB).

// Payload type of a key-value sort: VB bytes per value (0: keys only).
template <int VB>
using ValT = typename std::conditional<VB == 8, uint64_t, uint32_t>::type;

// Resident blocks per SM the register budget is sized for (shared memory
// allows as many for 1024- and 2048-bucket tables).
constexpr int k3_min_blocks(int tpb, int qm, int vb) {
  return tpb == 512 ? (vb == 8 ? 1 : 2) : qm <= 8 ? (vb == 8 ? 1 : 2) : 1;
}

template <int TPB, int QM, int VB>
__global__ void __launch_bounds__(TPB, k3_min_blocks(TPB, QM, VB)) k_scatter(PassArgs a, RunParams rp) {
  pdl_wait();
  constexpr uint32_t kW = TPB / 32;          // warps
  constexpr uint32_t kKT = kTile / TPB;      // keys per thread per tile
  constexpr uint32_t kWK = kTile / kW;       // keys of a tile ranked by one warp
  constexpr uint32_t kNB = QM * TPB <= 1024 ? 10 : QM * TPB <= 2048 ? 11 : 12;  // id bits (ids < nb_pad)
  static_assert(kWK <= 0xFFFFu && QM * kW <= 128, "warp counters are 16 bits; 128 warp totals");
  using V = ValT<VB>;
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t nbp = a.nb_pad_max;
  uint64_t* sRun = reinterpret_cast<uint64_t*>(smem);          // next destination per bucket
  uint64_t* stage = sRun + nbp;                                // kTile keys, grouped by bucket
  uint32_t* sLs = reinterpret_cast<uint32_t*>(stage + kTile);  // tile-local start per bucket
  uint32_t* sCnt = sLs + nbp;                                  // tile count per bucket
  uint32_t* wcnt = sCnt + nbp;                                 // [kW/2][nbp] packed warp counters
  uint16_t* sid = reinterpret_cast<uint16_t*>(wcnt + (kW / 2) * nbp);  // bucket of each staged key
  V* const sv = reinterpret_cast<V*>(sid + kTile);                     // staged values (key-value sorts)
  __shared__ uint32_t wsum[128];
  __shared__ unsigned long long s_chunk[2];
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t wsh = 16 * (wid & 1);
  uint32_t* myc = wcnt + (wid >> 1) * nbp;
  const unsigned lt = (1u << lane) - 1u;
  for (uint32_t j = threadIdx.x; j < (kW / 2) * nbp; j += TPB) wcnt[j] = 0;
  bool oob = false;
  const uint64_t nch = batch_chunks(a), ckeys = batch_chunk_keys(a);
  for (int par = 0;; par ^= 1) {
    if (threadIdx.x == 0) s_chunk[par] = atomicAdd(a.chunk_ctr, 1ull);
    __syncthreads();
    const uint64_t ch = s_chunk[par];
    if (ch >= nch) break;
    const uint32_t pi = a.chunk_plan[ch];
    const Plan& pl = a.plans[pi];
    // uniform across the block; items of the buffered scatter are K3b's
    if ((pl.flags & FLAG_SKIP_SCATTER) || buffered_scatter_ok(pl, rp, a.vbytes)) continue;
    const Item& it = a.items[pi];
    const uint32_t nbk = pl.nb_pad;
    const unsigned long long* ex = a.excl + ch * nbp;
    for (uint32_t b = threadIdx.x; b < nbk; b += TPB) {
      sRun[b] = a.cursors[pl.cnt_off + b] + ex[b];
      sCnt[b] = 0;
      sLs[b] = 0;
    }
    const uint64_t c0 = (ch - pl.chunk_begin) * ckeys;
    const uint64_t clen = it.n - c0 < ckeys ? it.n - c0 : ckeys;
    const uint64_t* src = (it.buf ? a.keysB : a.keysA) + it.lo + c0;
    const uint16_t* idin = a.ids + it.lo + c0;
    uint64_t* dst = it.buf ? a.outA : a.outB;
    const V* vsrc = VB ? static_cast<const V*>(it.buf ? a.valsB : a.valsA) + it.lo + c0 : nullptr;
    V* vdst = VB ? static_cast<V*>(it.buf ? a.valsA : a.valsB) : nullptr;
    const uint64_t lo = it.lo, n = it.n;
    const uint32_t Q = (nbk + TPB - 1) / TPB;  // bucket ranges of TPB (at most QM)
    uint64_t v[kKT];
    uint32_t bk[kKT];
    V vv[VB ? kKT : 1];
    auto load_tile = [&](uint64_t t0) {
      const uint32_t len = clen - t0 < kTile ? (uint32_t)(clen - t0) : kTile;
      const uint64_t* s = src + t0 + wid * kWK + lane;
      const uint16_t* d = idin + t0 + wid * kWK + lane;
      if (len == kTile) {
#pragma unroll
        for (int k = 0; k < (int)kKT; ++k) {
          v[k] = s[k * 32];
          bk[k] = d[k * 32];
          if constexpr (VB != 0) vv[k] = vsrc[t0 + wid * kWK + lane + k * 32];
        }
      } else {
#pragma unroll
        for (int k = 0; k < (int)kKT; ++k) {
          const uint32_t pos = wid * kWK + k * 32 + lane;
          v[k] = pos < len ? s[k * 32] : 0;
          bk[k] = pos < len ? (uint32_t)d[k * 32] : 0xFFFFu;
          if constexpr (VB != 0) vv[k] = pos < len ? vsrc[t0 + pos] : V(0);
        }
      }
    };
    load_tile(0);
    auto tile = [&](uint64_t t0, uint32_t len, auto full_tag) {
      constexpr bool FULL = decltype(full_tag)::value;
      // rank: bk[k] becomes id | (rank among the warp's keys of that id) << 16
#pragma unroll
      for (int k = 0; k < (int)kKT; ++k) bk[k] |= rank_step<FULL, kNB>(bk[k], myc, lane, wsh, lt) << 16;
      __syncthreads();
      // per bucket b = q*TPB + tid: advance the run by the previous tile's
      // count, prefix over the warps (in place), tile count; then one scan
      // over all buckets (ranges q-major, then warps, then lanes)
      uint32_t cnt[QM];
#pragma unroll
      for (uint32_t q = 0; q < QM; ++q) {
        const uint32_t b = q * TPB + threadIdx.x;
        cnt[q] = 0;
        if (q < Q && b < nbk) {
          sRun[b] += sLs[b] + sCnt[b];  // undo the previous tile's offset, advance past its keys
          uint32_t t = 0;
#pragma unroll
          for (uint32_t w2 = 0; w2 < kW / 2; ++w2) {
            const uint32_t x = wcnt[w2 * nbp + b];
            const uint32_t t1 = t + (x & 0xFFFFu);
            wcnt[w2 * nbp + b] = t | (t1 << 16);
            t = t1 + (x >> 16);
          }
          sCnt[b] = t;
          cnt[q] = t;
        }
      }
      uint32_t inc[QM];
#pragma unroll
      for (uint32_t q = 0; q < QM; ++q) inc[q] = cnt[q];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
        for (uint32_t q = 0; q < QM; ++q) {
          if (q < Q) {  // uniform
            const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc[q], d);
            if (lane >= (unsigned)d) inc[q] += o;
          }
        }
      }
#pragma unroll
      for (uint32_t q = 0; q < QM; ++q) {
        const uint32_t b = q * TPB + threadIdx.x;
        if (q < Q) {
          if (lane == 31) wsum[q * kW + wid] = inc[q];
          if (b < nbk) sLs[b] = inc[q] - cnt[q];  // exclusive within the warp's 32 buckets
        }
      }
      __syncthreads();
      if (wid == 0) {  // scan the Q*kW warp totals, 4 per lane
        uint32_t e[4], s4 = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint32_t idx = lane * 4 + i;
          e[i] = idx < Q * kW ? wsum[idx] : 0u;
          s4 += e[i];
        }
        uint32_t x = s4;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, x, d);
          if (lane >= (unsigned)d) x += o;
        }
        uint32_t run = x - s4;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint32_t idx = lane * 4 + i;
          if (idx < Q * kW) wsum[idx] = run;
          run += e[i];
        }
      }
      __syncthreads();
      for (uint32_t q = 0; q < Q; ++q) {
        const uint32_t b = q * TPB + threadIdx.x;
        if (b < nbk) {
          const uint32_t ls = sLs[b] + wsum[q * kW + wid];
          sLs[b] = ls;
          sRun[b] -= ls;  // destination of staged position p is sRun[b] + p
        }
      }
      __syncthreads();
      // stage grouped by bucket; in a partial tile the empty lanes write a
      // zero key to the last slot, which no key of the tile uses
#pragma unroll
      for (int k = 0; k < (int)kKT; ++k) {
        const uint32_t b = bk[k] & 0xFFFFu;
        const bool valid = FULL || b != 0xFFFFu;
        const uint32_t bb = valid ? b : 0u;
        uint32_t p = sLs[bb] + ((myc[bb] >> wsh) & 0xFFFFu) + (bk[k] >> 16);
        if (!FULL && !valid) p = kTile - 1;
        stage[p] = v[k];
        sid[p] = (uint16_t)bb;
        if constexpr (VB != 0) sv[p] = vv[k];
      }
      // prefetch the next tile while the staged one is written out
      if (t0 + kTile < clen) load_tile(t0 + kTile);
      __syncthreads();
      auto put = [&](uint32_t p) {
        const uint64_t o = sRun[sid[p]] + p;
        const uint64_t x = stage[p];
        const bool ok = o - lo < n;  // K1 and K3 disagree: never write outside the item
        if (ok) {
          dst[o] = x;
          if constexpr (VB != 0) vdst[o] = sv[p];
        }
        oob |= !ok;
      };
      if constexpr (FULL) {
#pragma unroll 4
        for (uint32_t p = threadIdx.x; p < kTile; p += TPB) put(p);
      } else {
        for (uint32_t p = threadIdx.x; p < len; p += TPB) put(p);
      }
      for (uint32_t j = threadIdx.x; j < (kW / 2) * nbp / 4; j += TPB)
        reinterpret_cast<uint4*>(wcnt)[j] = make_uint4(0, 0, 0, 0);
      __syncthreads();
    };
    for (uint64_t t0 = 0; t0 < clen; t0 += kTile) {
      const uint32_t len = clen - t0 < kTile ? (uint32_t)(clen - t0) : kTile;
      if (len == kTile) tile(t0, len, std::true_type{});
      else tile(t0, len, std::false_type{});
    }
  }
  if (__syncthreads_or(oob ? 1 : 0) && threadIdx.x == 0) atomicCAS(a.status, 0u, (unsigned)LS_EDEVICE);
}

// ------------------------------------------------------------------ K3b

// Buffered scatter for items whose order inside a bucket does not matter
// (buffered_scatter_ok: no child is partitioned again): the partitioning of LearnedSort 2.0 (Sec. 2.2) and
// IPS4o (Sec. 2.4), where every bucket has a buffer that is written out when
// it is full.  Here a buffer is one line of kLineKeys keys in shared memory,
// lines are aligned to the destination's addresses, and each key claims the
// next position of its bucket with a shared-memory atomic, so the keys of a
// bucket do not keep their input order.  A block takes a run of one item's
// keys; the run's keys of bucket b fill one contiguous region of the
// destination that starts at the bucket's cursor plus the keys of b in the
// item before the run (the chunk prefixes, plus a count over the ids of the
// run's first chunk when the run starts inside it).  Complete lines leave as
// whole 64-byte writes; only the first and last line of a region are written
// in part.  Positions inside a region count from the line boundary before
// its start, so a key's buffer slot is its position mod kLineKeys.  Per
// tile: phase A claims the positions of a thread's keys (the atomics
// issued together), puts each key that falls in its bucket's buffered line
// into the buffer and lists the lines that complete (the thread whose key
// fills a line's last slot; one append for all of a thread's lines); after
// a barrier the listed
// lines are written (four lanes per line) and their line
// ends advanced; after a second barrier phase B places the keys past the
// buffered line (whole lines straight out, the new partial line into the
// buffer).  Phase B of one tile and phase A of the next touch different
// slots, and line ends change only in the flush, so two barriers per tile
// suffice.  Every global write is checked against the item's range.
constexpr uint32_t kBufTPB = 512;
constexpr uint32_t kBufKT = 6;
constexpr uint32_t kBufTile = kBufTPB * kBufKT;
constexpr uint32_t kLineKeys = 8;
constexpr size_t kBufSmem = (size_t)kBufMaxBuckets * (kLineKeys * 8 + 8 + 4 + 4 + 4 + 2);

__global__ void __launch_bounds__(kBufTPB, 2)
    k_scatter_buffered(PassArgs a, RunParams rp, const BufRun* __restrict__ runs, uint32_t nruns) {
  pdl_wait();
  constexpr uint64_t M = ~(uint64_t)(kLineKeys - 1);
  constexpr uint32_t kLPL = kLineKeys / 2;  // lanes per line (16-byte stores)
  constexpr uint32_t kLPI = 32 / kLPL;      // lines per warp step
  constexpr uint32_t kW = kBufTPB / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* buf = reinterpret_cast<uint64_t*>(smem);                  // [bucket][kLineKeys]
  uint64_t* rs = buf + kBufMaxBuckets * kLineKeys;                    // region start (address / 8)
  uint32_t* cur = reinterpret_cast<uint32_t*>(rs + kBufMaxBuckets);  // keys claimed in the region
  uint32_t* le = cur + kBufMaxBuckets;                                // end of the buffered line, from rs
  uint32_t* fe = le + kBufMaxBuckets;                                 // listed line: its old line end
  uint16_t* fb = reinterpret_cast<uint16_t*>(fe + kBufMaxBuckets);   // listed line: its bucket
  __shared__ uint32_t s_nfl[2];
  __shared__ unsigned long long s_run;
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  bool bad = false;
  const uint64_t ckeys = batch_chunk_keys(a);
  if (a.bd) nruns = a.bd->nruns;
  for (;;) {
    __syncthreads();  // the previous run is done with the block's buffers
    if (threadIdx.x == 0) s_run = atomicAdd(a.chunk_ctr + 1, 1ull);
    __syncthreads();
    const uint64_t ri = s_run;
    if (ri >= nruns) break;
    const BufRun rn = runs[ri];
    const Plan& pl = a.plans[rn.plan];
    // uniform across the block; the stable scatter takes the other items
    if ((pl.flags & FLAG_SKIP_SCATTER) || !buffered_scatter_ok(pl, rp, a.vbytes)) continue;
    const Item& it = a.items[rn.plan];
    const uint32_t nbk = pl.nb_pad;
    uint64_t* dst = it.buf ? a.outA : a.outB;
    const uint64_t* src = (it.buf ? a.keysB : a.keysA) + it.lo;
    const uint16_t* ids = a.ids + it.lo;
    const uint64_t ab = (uint64_t)(uintptr_t)dst >> 3;  // dst[0] as a key address
    const uint64_t alo = ab + it.lo, ahi = alo + it.n;    // the item's destination
    const uint64_t ch = rn.off / ckeys;                   // the run's first chunk (item-relative)
    const unsigned long long* ex = a.excl + (pl.chunk_begin + ch) * a.nb_pad_max;
    for (uint32_t b = threadIdx.x; b < nbk; b += kBufTPB) cur[b] = 0;
    if (threadIdx.x == 0) s_nfl[0] = s_nfl[1] = 0;
    __syncthreads();
    for (uint64_t i = ch * ckeys + threadIdx.x; i < rn.off; i += kBufTPB) {
      const uint32_t b = ids[i];
      if (b < nbk) atomicAdd(&cur[b], 1u);
      else bad = true;
    }
    __syncthreads();
    // positions within a region are counted from the line boundary before
    // its start: a key's slot in the line buffer is its position mod 8, and
    // the buffered line ends at a multiple of 8
    for (uint32_t b = threadIdx.x; b < nbk; b += kBufTPB) {
      const uint64_t x = ab + a.cursors[pl.cnt_off + b] + ex[b] + cur[b];
      rs[b] = x;
      cur[b] = (uint32_t)(x & (kLineKeys - 1));
      le[b] = kLineKeys;
    }
    __syncthreads();
    uint64_t v[kBufKT];
    uint32_t bk[kBufKT], rr[kBufKT];
    auto load_tile = [&](uint64_t t0) {
      const uint64_t len = rn.len - t0 < kBufTile ? rn.len - t0 : kBufTile;
#pragma unroll
      for (int k = 0; k < (int)kBufKT; ++k) {
        const uint32_t j = k * kBufTPB + threadIdx.x;
        const bool in = j < len;
        v[k] = in ? src[rn.off + t0 + j] : 0ull;
        bk[k] = in ? (uint32_t)ids[rn.off + t0 + j] : 0xFFFFu;
      }
    };
    load_tile(0);
    uint32_t par = 0;
    for (uint64_t t0 = 0; t0 < rn.len; t0 += kBufTile, par ^= 1) {
      // the thread's claims first (independent atomics, in flight together),
      // then the buffer stores
      uint32_t late = 0, full = 0;
#pragma unroll
      for (int k = 0; k < (int)kBufKT; ++k) rr[k] = bk[k] < nbk ? atomicAdd(&cur[bk[k]], 1u) : 0u;
#pragma unroll
      for (int k = 0; k < (int)kBufKT; ++k) {
        const uint32_t b = bk[k];
        if (b < nbk) {
          const uint32_t e = le[b];
          if (rr[k] < e) {
            buf[b * kLineKeys + (rr[k] & (kLineKeys - 1))] = v[k];
            if (rr[k] == e - 1) full |= 1u << k;
          } else {
            late |= 1u << k;
          }
        } else if (b != 0xFFFFu) {
          bad = true;  // K1 and K3 disagree
        }
      }
      if (full) {  // lines this thread completed (about one key in eight): one append for all of them
        uint32_t q = atomicAdd(&s_nfl[par], (uint32_t)__popc(full));
#pragma unroll
        for (int k = 0; k < (int)kBufKT; ++k)
          if (full & (1u << k)) {
            fb[q] = (uint16_t)bk[k];
            fe[q] = rr[k] + 1;
            ++q;
          }
      }
      __syncthreads();
      // write the completed lines and advance their line ends
      const uint32_t nf = s_nfl[par];
      for (uint32_t i = wid * kLPI + lane / kLPL; i < nf; i += kW * kLPI) {
        const uint32_t b = fb[i];
        const uint64_t r0 = rs[b];
        const uint64_t ls = (r0 & M) + fe[i] - kLineKeys;
        const uint32_t q = lane % kLPL;
        if (q == 0) le[b] = (cur[b] & ~(kLineKeys - 1)) + kLineKeys;
        if (ls >= r0) {
          if (ls >= alo && ls + kLineKeys <= ahi)
            reinterpret_cast<uint4*>(ls << 3)[q] = reinterpret_cast<const uint4*>(buf + b * kLineKeys)[q];
          else
            bad = true;
        } else {
          for (uint32_t j = 2 * q; j < 2 * q + 2; ++j) {
            const uint64_t g = ls + j;
            if (g < r0) continue;
            if (g >= alo && g < ahi) *reinterpret_cast<uint64_t*>(g << 3) = buf[b * kLineKeys + j];
            else bad = true;
          }
        }
      }
      if (threadIdx.x == 0) s_nfl[par ^ 1] = 0;
      __syncthreads();
      // keys past the buffered line: whole lines straight out, the new
      // partial line into the buffer
#pragma unroll
      for (int k = 0; k < (int)kBufKT; ++k) {
        if (!(late & (1u << k))) continue;
        const uint32_t b = bk[k];
        if (rr[k] < le[b] - kLineKeys) {
          const uint64_t g = (rs[b] & M) + rr[k];
          if (g >= alo && g < ahi) *reinterpret_cast<uint64_t*>(g << 3) = v[k];
          else bad = true;
        } else {
          buf[b * kLineKeys + (rr[k] & (kLineKeys - 1))] = v[k];
        }
      }
      if (t0 + kBufTile < rn.len) load_tile(t0 + kBufTile);
    }
    __syncthreads();
    // the regions' last (partial) lines
    for (uint32_t i = threadIdx.x; i < nbk * kLineKeys; i += kBufTPB) {
      const uint32_t b = i / kLineKeys, j = i % kLineKeys;
      const uint64_t r0 = rs[b], e = (r0 & M) + cur[b];
      const uint64_t g = (e & M) + j;
      if (g < e && g >= r0) {
        if (g >= alo && g < ahi) *reinterpret_cast<uint64_t*>(g << 3) = buf[i];
        else bad = true;
      }
    }
  }
  if (__syncthreads_or(bad ? 1 : 0) && threadIdx.x == 0) atomicCAS(a.status, 0u, (unsigned)LS_EDEVICE);
}

// ------------------------------------------------------------------ chunk prefixes

// Run pass: for each bucket column, the exclusive running sum of the K1
// counts over the run's chunks; the run's total replaces the count in the
// run's first row when the item has several runs (that row is read only by
// the thread that owns the column, before it is written).
__global__ void k_chunk_prefix(const ChunkSeg* __restrict__ segs, const Plan* __restrict__ plans, uint32_t* agg,
                               unsigned long long* __restrict__ excl, uint32_t nbp, const BatchDesc* bd) {
  pdl_wait();
  const uint32_t ns = bd ? bd->nsegs : gridDim.x;
  for (uint32_t si = blockIdx.x; si < ns; si += gridDim.x) {
    const ChunkSeg sg = segs[si];
    const uint32_t b = blockIdx.y * blockDim.x + threadIdx.x;
    if (b >= plans[sg.plan].nb_pad) continue;
    uint32_t v[kSegChunks];
#pragma unroll
    for (uint32_t j = 0; j < kSegChunks; ++j) v[j] = j < sg.nch ? agg[(sg.c0 + j) * nbp + b] : 0u;
    unsigned long long run = 0;
#pragma unroll
    for (uint32_t j = 0; j < kSegChunks; ++j) {
      if (j < sg.nch) excl[(sg.c0 + j) * nbp + b] = run;
      run += v[j];
    }
    agg[sg.c0 * nbp + b] = (uint32_t)run;  // at most kSegChunks * kChunkKeys
  }
}

// Carry scan: for each item with several runs and each bucket column, the
// exclusive prefix over its runs of the run totals, in place (the total in
// the run's first row becomes the keys of that bucket in the item's earlier
// runs).  One thread per column; the loads of eight runs are issued together.
__global__ void k_run_scan(const uint2* __restrict__ multi, const ChunkSeg* __restrict__ segs,
                           const Plan* __restrict__ plans, uint32_t* agg, uint32_t nbp, const BatchDesc* bd) {
  pdl_wait();
  const uint32_t nm = bd ? bd->nmulti : gridDim.x;
  for (uint32_t mi_ = blockIdx.x; mi_ < nm; mi_ += gridDim.x) {
    const uint2 mi = multi[mi_];  // (first run, number of runs)
    const ChunkSeg f = segs[mi.x];
    const uint32_t b = blockIdx.y * blockDim.x + threadIdx.x;
    if (b >= plans[f.plan].nb_pad) continue;
    const uint64_t c0 = f.c0;
    uint32_t run = 0;
    for (uint32_t r0 = 0; r0 < mi.y; r0 += 8) {
      uint32_t t[8];
#pragma unroll
      for (uint32_t k = 0; k < 8; ++k)
        t[k] = r0 + k < mi.y ? agg[(c0 + (uint64_t)(r0 + k) * kSegChunks) * nbp + b] : 0u;
#pragma unroll
      for (uint32_t k = 0; k < 8; ++k) {
        if (r0 + k < mi.y) agg[(c0 + (uint64_t)(r0 + k) * kSegChunks) * nbp + b] = run;
        run += t[k];
      }
    }
  }
}

// Carry pass: add each run's carry (from k_run_scan) to its chunks.
__global__ void k_chunk_carry(const ChunkSeg* __restrict__ segs, const Plan* __restrict__ plans,
                              const uint32_t* __restrict__ agg, unsigned long long* __restrict__ excl, uint32_t nbp,
                              const BatchDesc* bd) {
  pdl_wait();
  const uint32_t ns = bd ? bd->nsegs : gridDim.x;
  for (uint32_t si = blockIdx.x; si < ns; si += gridDim.x) {
    const ChunkSeg sg = segs[si];
    if (si == sg.first) continue;
    const uint32_t b = blockIdx.y * blockDim.x + threadIdx.x;
    if (b >= plans[sg.plan].nb_pad) continue;
    const unsigned long long carry = agg[sg.c0 * nbp + b];
    for (uint32_t j = 0; j < sg.nch; ++j) excl[(sg.c0 + j) * nbp + b] += carry;
  }
}

// ------------------------------------------------------------------ K2

constexpr int kK2Threads = 256;
constexpr int kK2Warps = kK2Threads / 32;

// Block-wide exchange for K2: exclusive scans of N uint32 per thread (totals
// to every thread) and sums of M uint64 per thread (to every thread), with
// one pass through shared memory.  s32 holds kK2Warps*N words, s64
// kK2Warps*M; the caller separates reuses of them with a barrier.
template <int N, int M>
__device__ __forceinline__ void k2_exchange(uint32_t (&x)[N], uint32_t (&tot)[N], unsigned long long (&y)[M],
                                            uint32_t* s32, unsigned long long* s64) {
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc[N];
#pragma unroll
  for (int k = 0; k < N; ++k) inc[k] = x[k];
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc[k], d);
      if (lane >= (unsigned)d) inc[k] += o;
    }
  }
#pragma unroll
  for (int k = 0; k < M; ++k)
    for (int d = 16; d > 0; d >>= 1) y[k] += __shfl_xor_sync(0xFFFFFFFFu, y[k], d);
  if (lane == 31)
#pragma unroll
    for (int k = 0; k < N; ++k) s32[wid * N + k] = inc[k];
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < M; ++k) s64[wid * M + k] = y[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) {
    uint32_t before = 0, all = 0;
    for (unsigned w = 0; w < (unsigned)kK2Warps; ++w) {
      const uint32_t v = s32[w * N + k];
      before += w < wid ? v : 0u;
      all += v;
    }
    x[k] = inc[k] - x[k] + before;
    tot[k] = all;
  }
#pragma unroll
  for (int k = 0; k < M; ++k) {
    unsigned long long t = 0;
    for (unsigned w = 0; w < (unsigned)kK2Warps; ++w) t += s64[w * M + k];
    y[k] = t;
  }
}

enum { L_NEXT = 0, L_SMALL, L_MID, L_LARGE, L_COPY, L_FALLBACK, L_N };

// K2, one block per item: bucket starts and write cursors from the counts,
// the item's level statistics, and the children lists (next level, base
// cases, copies, fallback).  Thread t owns a contiguous range of buckets, so
// the lists keep bucket order within an item.
__global__ void __launch_bounds__(kK2Threads) k_children(ChildArgs a, RunParams rp) {
  pdl_wait();
  uint32_t pi = blockIdx.x;
  if (a.bd && pi >= a.bd->nitems) return;  // device-planned batch: the grid covers the largest batch
  const Item& it = a.items[pi];
  Plan& pl = a.plans[pi];
  __shared__ uint32_t s32[kK2Warps * L_N];
  __shared__ unsigned long long s64[kK2Warps * 6];
  __shared__ unsigned long long smax[kK2Warps];
  __shared__ unsigned long long s_base[L_N];
  __shared__ uint32_t s_bb, s_nf[kK2Threads + 1];
  uint32_t level = it.level;
  uint32_t cl = level + 1 < LS_MAX_LEVELS ? level + 1 : LS_MAX_LEVELS - 1;
  DevLevelStats* ls = a.stats + (level < LS_MAX_LEVELS ? level : LS_MAX_LEVELS - 1);
  DevLevelStats* cs = a.stats + cl;
  uint8_t dest = it.buf ^ 1;
  // Homogeneity check (Sec. 2.2): an all-equal item is already sorted.
  if (it.n > 0 && !pl.mixed) {
    if (threadIdx.x == 0) {
      pl.flags |= FLAG_SKIP_SCATTER | FLAG_HOMOGENEOUS;
      atomicAdd(&ls->homogeneous, 1ull);
      if (it.buf == 1) {
        uint64_t np = (it.n + kCopyPiece - 1) / kCopyPiece;
        unsigned long long b = atomicAdd(&a.ctr->n_copy, (unsigned long long)np);
        if (b + np > a.copy_cap) {
          atomicExch(&a.ctr->overflow, 1ull);
        } else {
          for (uint64_t q = 0; q < np; ++q) {
            uint64_t off = q * kCopyPiece;
            uint64_t len = it.n - off < kCopyPiece ? it.n - off : kCopyPiece;
            a.copy[b + q] = Span{it.lo + off, (uint32_t)len, 1u};
          }
        }
      }
    }
    return;
  }
  uint32_t nb = pl.nb;
  const unsigned long long* cnt = a.counts + pl.cnt_off;
  bool eq = pl.decision == LS_DEC_SPLITTER_EQ;
  bool learned = pl.decision == LS_DEC_LEARNED;
  const bool radix = pl.decision == LS_DEC_RADIX;
  const uint64_t* T = a.pivots + pl.tab_off;
  bool has_T = pl.cls != CLS_DIRECT && pl.cls != CLS_RADIX;
  uint32_t per = (nb + blockDim.x - 1) / blockDim.x;
  uint32_t b0 = threadIdx.x * per < nb ? threadIdx.x * per : nb;
  uint32_t b1 = b0 + per < nb ? b0 + per : nb;
  // exclusive scan of counts -> bucket starts (uint32 is enough per item:
  // items are shorter than 2^32 keys), largest bucket, sum of squares, and
  // the no-progress test (one bucket holds the whole item)
  unsigned long long mxc = 0, sq[2] = {0, 0};
  uint32_t sc1[1] = {0}, tot1[1];
  for (uint32_t b = b0; b < b1; ++b) {
    uint64_t sz = cnt[b];
    sc1[0] += (uint32_t)sz;
    mxc = sz > mxc ? sz : mxc;
    sq[0] += sz * sz;
    if (sz == it.n && !(eq && (b & 1))) {
      sq[1] = 1;
      s_bb = b;  // the one bucket that holds the whole item
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, mxc, d);
    mxc = o > mxc ? o : mxc;
  }
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mxc;
  k2_exchange<1, 2>(sc1, tot1, sq, s32, s64);
  uint64_t run = sc1[0];
  unsigned long long tmax = 0;
  for (int w = 0; w < kK2Warps; ++w) tmax = smax[w] > tmax ? smax[w] : tmax;
  const bool noprog = sq[1] != 0;
  // level statistics of this item
  if (threadIdx.x == 0) {
    atomicAdd(&ls->items, 1ull);
    atomicAdd(&ls->keys, (unsigned long long)it.n);
    if (learned) atomicAdd(&ls->learned, 1ull);
    else if (radix) atomicAdd(&ls->radix, 1ull);
    else if (eq) atomicAdd(&ls->splitter_eq, 1ull);
    else atomicAdd(&ls->splitter, 1ull);
    atomicMax(&ls->max_child, tmax);
    atomicAdd(&ls->sumsq_child, sq[0]);
  }
  const bool refine_children = learned && rp.recurse == LS_RECURSE_REFINE_GLOBAL;
  const uint32_t mk = (it.kind == KIND_REFINE) ? it.mk : 0;
  const uint64_t mg = (it.kind == KIND_REFINE) ? it.mg : 0;
  // Under REFINE_GLOBAL no bucket below a learned item draws a new sample
  // (LearnedSort 2.0 trains once, Sec. 2.2): a child the model did not split
  // (no progress), or one that would refine past the FP64 limit, takes the
  // radix split on the bits where this item's keys differ (they all agree
  // above bit top_bits); a radix item's children split the next bits down.
  const uint32_t top_bits = pl.odiff ? 64u - (uint32_t)__clzll((long long)pl.odiff) : 0u;
  const bool radix_past_limit = refine_children && beyond_refine_limit(rp.B, mk + 2);
  if (noprog) {
    // no-progress guard: redo the same range at the next level with the
    // splitter tree (keys stay where they are).
    if (threadIdx.x == 0) {
      pl.flags |= FLAG_SKIP_SCATTER | FLAG_NOPROGRESS;
      atomicAdd(&ls->noprogress, 1ull);
      const uint32_t bb = s_bb;
      if (level + 1 > rp.max_depth) {
        atomicAdd(&cs->fallback_items, 1ull);
        atomicAdd(&cs->fallback_keys, (unsigned long long)it.n);
        unsigned long long q = atomicAdd(&a.ctr->n_fallback, 1ull);
        if (q < a.fallback_cap) a.fallback[q] = Span{it.lo, (uint32_t)it.n, it.buf};
        else atomicExch(&a.ctr->overflow, 1ull);
      } else {
        Item ch = it;
        ch.level = (uint16_t)(level + 1);
        ch.gidx = it.gidx * nb + bb;
        if (radix || refine_children) {
          ch.kind = KIND_RADIX;
          ch.mk = (uint16_t)(radix ? pl.dir_shift : top_bits);
        } else {
          ch.kind = KIND_FORCE_SPLITTER;
          ch.mk = 0;
        }
        ch.model = -1;
        ch.mg = 0;
        if (has_T) {
          if (bb >= 1) ch.ord_lo = T[bb] > it.ord_lo ? T[bb] : it.ord_lo;
          if (bb < pl.kmax) ch.ord_hi = T[bb + 1] - 1;
        }
        unsigned long long q = atomicAdd(&a.ctr->n_next, 1ull);
        if (q < a.next_cap) a.next[q] = ch;
        else atomicExch(&a.ctr->overflow, 1ull);
      }
    }
    return;
  }
  // bucket starts (item-relative) and "final" flags in shared memory:
  // a bucket is final when it is an equality bucket or holds <= 1 key.
  extern __shared__ __align__(16) unsigned char k2smem[];
  uint64_t* s_start = reinterpret_cast<uint64_t*>(k2smem);      // nb + 1
  uint8_t* s_fin = reinterpret_cast<uint8_t*>(s_start + nb + 1);  // nb
  {
    uint64_t r = run;
    for (uint32_t b = b0; b < b1; ++b) {
      s_start[b] = r;
      a.cursors[pl.cnt_off + b] = it.lo + r;  // destination of the bucket's first key
      uint64_t sz = cnt[b];
      s_fin[b] = (uint8_t)((eq && (b & 1)) || sz <= 1);
      r += sz;
    }
    if (threadIdx.x == 0) s_start[nb] = it.n;
  }
  __syncthreads();
  // s_nf[t]: the first non-final bucket at or after thread t's range (nb if
  // none), so that a run of final buckets finds its end without a serial
  // walk over the run
  if (dest == 1) {
    uint32_t f = nb;
    for (uint32_t b = b0; b < b1; ++b)
      if (!s_fin[b]) {
        f = b;
        break;
      }
    s_nf[threadIdx.x] = f;
    if (threadIdx.x == 0) s_nf[kK2Threads] = nb;
    __syncthreads();
    if (threadIdx.x < 32) {  // suffix minimum, one warp over kK2Threads / 32 entries per lane
      constexpr uint32_t kPer = kK2Threads / 32;
      uint32_t loc[kPer], m = nb;
#pragma unroll
      for (int i = kPer - 1; i >= 0; --i) {
        m = min(m, s_nf[threadIdx.x * kPer + i]);
        loc[i] = m;
      }
      uint32_t suf = m;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_down_sync(0xFFFFFFFFu, suf, d);
        if (threadIdx.x + d < 32) suf = min(suf, o);
      }
      uint32_t after = __shfl_down_sync(0xFFFFFFFFu, suf, 1);
      if (threadIdx.x == 31) after = nb;
#pragma unroll
      for (int i = 0; i < (int)kPer; ++i) s_nf[threadIdx.x * kPer + i] = min(loc[i], after);
    }
    __syncthreads();
  }
  // end of the run of final buckets that starts at b (b in this thread's range)
  auto run_end = [&](uint32_t b) {
    for (uint32_t e = b + 1; e < b1; ++e)
      if (!s_fin[e]) return e;
    return s_nf[threadIdx.x + 1];
  };
  // count list entries: base case / fallback / next level per non-final
  // bucket; one copy run per maximal run of final buckets (only when the
  // destination is the workspace buffer)
  unsigned long long eqk = 0, bk = 0, bki = 0, fbk = 0, fbi = 0;
  uint32_t nl[L_N] = {0, 0, 0, 0, 0, 0};
  for (uint32_t b = b0; b < b1; ++b) {
    uint64_t sz = cnt[b];
    if (eq && (b & 1)) eqk += sz;
    if (s_fin[b]) {
      if (dest == 1 && (b == 0 || !s_fin[b - 1])) {
        const uint32_t e = run_end(b);
        uint64_t len = s_start[e] - s_start[b];
        nl[L_COPY] += (uint32_t)((len + kCopyPiece - 1) / kCopyPiece);
      }
      continue;
    }
    if (sz <= rp.T) {
      if (sz <= kWarpSmallMax) nl[L_SMALL]++;
      else if (sz <= kWarpSortMax) nl[L_MID]++;
      else nl[L_LARGE]++;
      bki++;
      bk += sz;
    } else if (level + 1 > rp.max_depth) {
      nl[L_FALLBACK]++;
      fbi++;
      fbk += sz;
    } else {
      nl[L_NEXT]++;
    }
  }
  uint32_t tot[L_N];
  unsigned long long sums[5] = {eqk, bk, bki, fbk, fbi};
  __syncthreads();  // the first exchange's words are read by every thread before they are reused
  k2_exchange<L_N, 5>(nl, tot, sums, s32, s64);
  if (threadIdx.x == 0) {
    // No child is partitioned again: every child is final, a base case or
    // a depth-limit span, so no bucket of this item is ever sampled and the
    // order of keys inside its buckets does not matter (the buffered
    // scatter may take it).
    if (tot[L_NEXT] == 0) pl.flags |= FLAG_ORDER_FREE;
    for (int q = 0; q < L_N; ++q) {
      unsigned long long* ctr = (q == L_NEXT)    ? &a.ctr->n_next
                                : (q == L_SMALL) ? &a.ctr->n_base_small
                                : (q == L_MID)   ? &a.ctr->n_base_mid
                                : (q == L_LARGE) ? &a.ctr->n_base_large
                                : (q == L_COPY)  ? &a.ctr->n_copy
                                                 : &a.ctr->n_fallback;
      s_base[q] = tot[q] ? atomicAdd(ctr, (unsigned long long)tot[q]) : 0ull;
    }
    if (sums[0]) atomicAdd(&ls->eq_keys, sums[0]);
    if (sums[2]) {
      atomicAdd(&cs->base_items, sums[2]);
      atomicAdd(&cs->base_keys, sums[1]);
    }
    if (sums[4]) {
      atomicAdd(&cs->fallback_items, sums[4]);
      atomicAdd(&cs->fallback_keys, sums[3]);
    }
  }
  __syncthreads();
  unsigned long long wp[L_N];
  for (int q = 0; q < L_N; ++q) wp[q] = s_base[q] + nl[q];
  const uint64_t caps[L_N] = {a.next_cap, a.base_cap, a.mid_cap, a.large_cap, a.copy_cap, a.fallback_cap};
  bool ovf = false;
  for (uint32_t b = b0; b < b1; ++b) {
    uint64_t sz = cnt[b];
    uint64_t clo = it.lo + s_start[b];
    if (s_fin[b]) {
      if (dest == 1 && (b == 0 || !s_fin[b - 1])) {
        const uint32_t e = run_end(b);
        uint64_t len = s_start[e] - s_start[b];
        for (uint64_t off = 0; off < len; off += kCopyPiece) {
          uint64_t pl_len = len - off < kCopyPiece ? len - off : kCopyPiece;
          if (wp[L_COPY] < caps[L_COPY]) a.copy[wp[L_COPY]] = Span{clo + off, (uint32_t)pl_len, 1u};
          else ovf = true;
          wp[L_COPY]++;
        }
      }
      continue;
    }
    if (sz <= rp.T) {
      const int q = sz <= kWarpSmallMax ? L_SMALL : sz <= kWarpSortMax ? L_MID : L_LARGE;
      Span* lst = q == L_SMALL ? a.base_small : q == L_MID ? a.base_mid : a.base_large;
      if (wp[q] < caps[q]) lst[wp[q]] = Span{clo, (uint32_t)sz, dest};
      else ovf = true;
      wp[q]++;
    } else if (level + 1 > rp.max_depth) {
      if (wp[L_FALLBACK] < caps[L_FALLBACK]) a.fallback[wp[L_FALLBACK]] = Span{clo, (uint32_t)sz, dest};
      else ovf = true;
      wp[L_FALLBACK]++;
    } else {
      Item ch;
      ch.lo = clo;
      ch.n = sz;
      ch.gidx = it.gidx * nb + b;
      ch.segment = it.segment;
      ch.level = (uint16_t)(level + 1);
      ch.buf = dest;
      ch.pad = 0;
      ch.ord_lo = it.ord_lo;
      ch.ord_hi = it.ord_hi;
      if (has_T) {
        if (b >= 1) ch.ord_lo = T[b] > it.ord_lo ? T[b] : it.ord_lo;
        if (b < pl.kmax) ch.ord_hi = T[b + 1] - 1;
      }
      if (radix || radix_past_limit) {
        ch.kind = KIND_RADIX;
        ch.model = -1;
        ch.mk = (uint16_t)(radix ? pl.dir_shift : top_bits);
        ch.mg = 0;
      } else if (refine_children) {
        ch.kind = KIND_REFINE;
        ch.model = pl.model;
        ch.mk = (uint16_t)(mk + 1);
        ch.mg = mg * rp.B + b;
      } else {
        ch.kind = KIND_FRESH;
        ch.model = -1;
        ch.mk = 0;
        ch.mg = 0;
      }
      if (wp[L_NEXT] < caps[L_NEXT]) a.next[wp[L_NEXT]] = ch;
      else ovf = true;
      wp[L_NEXT]++;
    }
  }
  if (ovf) atomicExch(&a.ctr->overflow, 1ull);
}

// ------------------------------------------------------------- base case

// Warp bitonic sort of up to 32*E keys held E per lane (element index
// lane*E + r); padding is ~0 (largest ord).
template <int E>
__device__ __forceinline__ void warp_bitonic(uint64_t (&v)[E]) {
  const unsigned lane = threadIdx.x & 31;
  constexpr uint32_t P = 32 * E;
#pragma unroll
  for (uint32_t k = 2; k <= P; k <<= 1) {
#pragma unroll
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      if (j >= (uint32_t)E) {
        const int lm = (int)(j / E);
#pragma unroll
        for (int r = 0; r < E; ++r) {
          uint32_t i = lane * E + r;
          uint64_t o = __shfl_xor_sync(0xFFFFFFFFu, v[r], lm);
          bool up = (i & k) == 0;
          bool lower = (i & j) == 0;
          uint64_t mn = v[r] < o ? v[r] : o;
          uint64_t mx = v[r] < o ? o : v[r];
          v[r] = (lower == up) ? mn : mx;
        }
      } else {
#pragma unroll
        for (int r = 0; r < E; ++r) {
          if ((r & (int)j) == 0) {
            uint32_t i = lane * E + r;
            bool up = (i & k) == 0;
            uint64_t x = v[r], y = v[r ^ j];
            if ((x > y) == up) {
              v[r] = y;
              v[r ^ j] = x;
            }
          }
        }
      }
    }
  }
}

template <int E>
__device__ __forceinline__ void warp_sort_span(const Span& s, uint64_t* A, const uint64_t* Bbuf, int dt) {
  const unsigned lane = threadIdx.x & 31;
  const uint64_t* src = s.buf ? Bbuf : A;
  uint64_t v[E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    uint32_t i = lane * E + r;
    v[r] = i < s.n ? ord_of(src[s.lo + i], dt) : ~0ull;
  }
  warp_bitonic<E>(v);
#pragma unroll
  for (int r = 0; r < E; ++r) {
    uint32_t i = lane * E + r;
    if (i < s.n) A[s.lo + i] = unord(v[r], dt);
  }
}

// Key-value forms of the base cases: the networks and the slot sort order
// (ord key, position in the span) pairs, so equal keys keep their input
// order (a stable sort), and each output position takes the value of the
// input position it ended with.

// Warp bitonic network over 32E (key, index) pairs held E per lane.
template <int E>
__device__ __forceinline__ void warp_bitonic_kv(uint64_t (&v)[E], uint32_t (&ix)[E]) {
  const unsigned lane = threadIdx.x & 31;
  constexpr uint32_t P = 32 * E;
#pragma unroll
  for (uint32_t k = 2; k <= P; k <<= 1) {
#pragma unroll
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      if (j >= (uint32_t)E) {
        const int lm = (int)(j / E);
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const uint32_t i = lane * E + r;
          const uint64_t o = __shfl_xor_sync(0xFFFFFFFFu, v[r], lm);
          const uint32_t oi = __shfl_xor_sync(0xFFFFFFFFu, ix[r], lm);
          const bool up = (i & k) == 0, lower = (i & j) == 0;
          const bool mine_less = v[r] < o || (v[r] == o && ix[r] < oi);
          const bool keep = (lower == up) == mine_less;  // keep the smaller when lower==up
          v[r] = keep ? v[r] : o;
          ix[r] = keep ? ix[r] : oi;
        }
      } else {
#pragma unroll
        for (int r = 0; r < E; ++r) {
          if ((r & (int)j) == 0) {
            const uint32_t i = lane * E + r;
            const bool up = (i & k) == 0;
            const uint64_t x = v[r], y = v[r ^ j];
            const uint32_t xi = ix[r], yi = ix[r ^ j];
            const bool gt = x > y || (x == y && xi > yi);
            if (gt == up) {
              v[r] = y;
              v[r ^ j] = x;
              ix[r] = yi;
              ix[r ^ j] = xi;
            }
          }
        }
      }
    }
  }
}

template <int E, int VB>
__device__ __forceinline__ void warp_sort_span_kv(const Span& s, uint64_t* A, const uint64_t* Bbuf, void* VA,
                                                  const void* VBuf, int dt) {
  using V = ValT<VB>;
  const unsigned lane = threadIdx.x & 31;
  const uint64_t* src = s.buf ? Bbuf : A;
  const V* vsrc = static_cast<const V*>(s.buf ? VBuf : VA) + s.lo;
  uint64_t v[E];
  uint32_t ix[E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const uint32_t i = lane * E + r;
    v[r] = i < s.n ? ord_of(src[s.lo + i], dt) : ~0ull;
    ix[r] = i;
  }
  warp_bitonic_kv<E>(v, ix);
  V val[E];
#pragma unroll
  for (int r = 0; r < E; ++r) val[r] = lane * E + r < s.n ? vsrc[ix[r]] : V(0);
  __syncwarp();  // every value is read before any is overwritten (vsrc may be VA)
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const uint32_t i = lane * E + r;
    if (i < s.n) {
      A[s.lo + i] = unord(v[r], dt);
      static_cast<V*>(VA)[s.lo + i] = val[r];
    }
  }
}

// Model-placed base case for one span of <= 256 keys, done by one warp (the
// GPU form of LearnedSort 2.0's counting sort by predicted position plus an
// insertion-sort fix, Sec. 2.2): inside a bucket the keys are close to
// uniform in ord space, so a linear map between the span's extremes places
// them into 32 R SPK slots (R = ceil(n / 32) keys per lane, SPK slots per
// key); a counting sort by slot and a rank count inside each slot (the
// insertion-sort fix done as one comparison pass per key, without a
// dependent chain) give the exact order.  Spans
// whose largest slot holds more than kMaxSlot keys (clustered data) return
// false and take the bitonic network instead.
constexpr uint32_t kSlots = 256;  // slots of the largest size class (32 per key register)
constexpr uint32_t kMaxSlot = 24;
constexpr int kSlotsShort = 2, kSlotsMid = 1;  // slots per key of the two warp classes

// Counting sort by predicted slot of one span of n keys, 32(R-1) < n <= 32R.
// The map: with hmin / hmax the smallest / largest high word of the ords,
// base = hmin:0 and w = the top 32 bits of (u - base) << clz(hmax - hmin)
// (or, when every key has the same high word, w = (low - lmin) <<
// clz(lmax - lmin)); slot = floor(w Q 32 / 2^32) with Q = R SPK slots per
// lane.  Monotone in u, so sorting by slot and then inside slots sorts the
// span.  Slot s belongs to lane s / Q (= w >> 27) and is stored at
// (s mod Q) * 32 + s / Q, so the per-lane reads of the scan hit distinct
// banks; after the scan the word holds the slot's start and count.
template <int R, int SPK>
__device__ __forceinline__ bool warp_placed_sort(const Span& s, uint64_t* A, const uint64_t* Bbuf, int dt,
                                                 uint64_t* sk, uint32_t* sc) {
  constexpr uint32_t Q = R * SPK;  // slots per lane
  constexpr uint32_t NS = 32 * Q;
  const unsigned lane = threadIdx.x & 31;
  const uint64_t* src = (s.buf ? Bbuf : A) + s.lo;
  const uint32_t n = s.n;
  uint64_t u[R];
  uint32_t hmin = ~0u, hmax = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const bool ok = r < R - 1 || lane + 32 * r < n;
    u[r] = ok ? ord_of(src[lane + 32 * r], dt) : 0ull;
    const uint32_t h = (uint32_t)(u[r] >> 32);
    if (ok) {
      hmin = min(hmin, h);
      hmax = max(hmax, h);
    }
  }
  hmin = __reduce_min_sync(0xFFFFFFFFu, hmin);
  hmax = __reduce_max_sync(0xFFFFFFFFu, hmax);
  uint32_t w[R];
  if (hmin == hmax) {  // uniform: one high word, exact low-word extremes
    uint32_t lmin = ~0u, lmax = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r < R - 1 || lane + 32 * r < n) {
        lmin = min(lmin, (uint32_t)u[r]);
        lmax = max(lmax, (uint32_t)u[r]);
      }
    }
    lmin = __reduce_min_sync(0xFFFFFFFFu, lmin);
    lmax = __reduce_max_sync(0xFFFFFFFFu, lmax);
    if (lmin == lmax) {  // all equal: already sorted; bring home if needed
      if (s.buf)
        for (uint32_t i = lane; i < n; i += 32) A[s.lo + i] = src[i];
      return true;
    }
    const uint32_t sh = __clz(lmax - lmin);
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = ((uint32_t)u[r] - lmin) << sh;
  } else {
    const uint64_t base = (uint64_t)hmin << 32;
    const uint32_t sh = __clz(hmax - hmin);
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = (uint32_t)(((u[r] - base) << sh) >> 32);
  }
#pragma unroll
  for (int q = 0; q < (int)Q; ++q) sc[q * 32 + lane] = 0;
  __syncwarp();
  uint32_t at[R], rk[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t slot = __umulhi(w[r], NS), owner = w[r] >> 27;
    at[r] = (slot - owner * Q) * 32 + owner;
    rk[r] = (r < R - 1 || lane + 32 * r < n) ? atomicAdd(&sc[at[r]], 1u) : 0u;
  }
  __syncwarp();
  // exclusive scan of the slot counts (slots lane*R .. lane*R+R-1 per lane)
  uint32_t c[Q], loc = 0, big = 0;
#pragma unroll
  for (int q = 0; q < (int)Q; ++q) {
    c[q] = sc[q * 32 + lane];
    loc += c[q];
    big = max(big, c[q]);
  }
  uint32_t incl = loc;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane >= (unsigned)d) incl += o;
  }
  if (__reduce_max_sync(0xFFFFFFFFu, big) > kMaxSlot) return false;  // uniform across the warp
  uint32_t run = incl - loc;
#pragma unroll
  for (int q = 0; q < (int)Q; ++q) {
    sc[q * 32 + lane] = run | (c[q] << 16);  // slot start and count
    run += c[q];
  }
  __syncwarp();
  uint32_t e[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    e[r] = sc[at[r]];
    if (r < R - 1 || lane + 32 * r < n) sk[(e[r] & 0xFFFFu) + rk[r]] = u[r];
  }
  __syncwarp();
  // order inside the slots: a key's place is its slot's start plus the keys
  // of the slot before it (smaller, or equal and staged earlier); the reads
  // are independent, so a slot of c keys costs c loads, not a chain.  The
  // warp takes as many steps as its largest slot holds, each step one
  // comparison for each of a lane's keys whose slot is that long.
  uint32_t pos[R], a0[R], cn[R], mx = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    a0[r] = e[r] & 0xFFFFu;
    cn[r] = (r < R - 1 || lane + 32 * r < n) ? e[r] >> 16 : 0u;
    pos[r] = a0[r];
    mx = max(mx, cn[r]);
  }
  mx = __reduce_max_sync(0xFFFFFFFFu, mx);
  for (uint32_t i = 0; i < mx; ++i) {
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (i < cn[r]) {
        const uint64_t x = sk[a0[r] + i];
        pos[r] += (x < u[r]) | ((x == u[r]) & (i < rk[r]));
      }
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (r < R - 1 || lane + 32 * r < n) A[s.lo + pos[r]] = unord(u[r], dt);
  __syncwarp();
  return true;
}

// Warp base case in two size classes with lists of their own, so that the
// short spans (up to kWarpSmallMax keys, most of them) run in an instance
// with fewer registers and more warps per SM: RHI = 4 takes spans of up to
// 128 keys, RHI = 8 any span of up to 256.  RLO: spans of at most 32 RLO
// keys are left to the other instance (0: none).
template <int RLO, int RHI, int MINB>
__global__ void __launch_bounds__(kTPB, MINB) k_base_small(const Span* spans, uint64_t n, uint64_t* A,
                                                          const uint64_t* Bbuf, int dt, const unsigned long long* dn) {
  pdl_wait();
  if (dn) n = *dn;  // span count written on the device
  __shared__ uint64_t s_keys[kTPB / 32][32 * RHI];
  constexpr int kSPK = RHI <= 4 ? kSlotsShort : kSlotsMid;  // slots per key
  __shared__ uint32_t s_cnt[kTPB / 32][32 * RHI * kSPK];
  const unsigned wid = threadIdx.x >> 5;
  uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  uint64_t nw = (gridDim.x * (uint64_t)blockDim.x) >> 5;
  for (; w < n; w += nw) {
    const Span s = spans[w];
    const uint32_t R = (s.n + 31) >> 5;
    if (R <= RLO || R > RHI) continue;  // the other class's span (uniform across the warp)
    if (s.n < 2) {  // nothing to order; bring home if needed
      if (s.n == 1 && s.buf && (threadIdx.x & 31) == 0) A[s.lo] = Bbuf[s.lo];
      continue;
    }
    uint64_t* sk = s_keys[wid];
    uint32_t* sc = s_cnt[wid];
    bool done;
    if (RHI <= 4) {
      switch (R) {  // uniform across the warp
        case 1: done = warp_placed_sort<1, kSPK>(s, A, Bbuf, dt, sk, sc); break;
        case 2: done = warp_placed_sort<2, kSPK>(s, A, Bbuf, dt, sk, sc); break;
        case 3: done = warp_placed_sort<3, kSPK>(s, A, Bbuf, dt, sk, sc); break;
        default: done = warp_placed_sort<4, kSPK>(s, A, Bbuf, dt, sk, sc); break;
      }
    } else {
      switch (R) {
        case 1: done = warp_placed_sort<1, kSPK>(s, A, Bbuf, dt, sk, sc); break;
        case 2: done = warp_placed_sort<2, kSPK>(s, A, Bbuf, dt, sk, sc); break;
        case 3: done = warp_placed_sort<3, kSPK>(s, A, Bbuf, dt, sk, sc); break;
        case 4: done = warp_placed_sort<4, kSPK>(s, A, Bbuf, dt, sk, sc); break;
        case 5: done = warp_placed_sort<5, kSPK>(s, A, Bbuf, dt, sk, sc); break;
        case 6: done = warp_placed_sort<6, kSPK>(s, A, Bbuf, dt, sk, sc); break;
        case 7: done = warp_placed_sort<7, kSPK>(s, A, Bbuf, dt, sk, sc); break;
        default: done = warp_placed_sort<8, kSPK>(s, A, Bbuf, dt, sk, sc); break;
      }
    }
    if (done) continue;
    if (RHI <= 4) {
      if (s.n <= 32) warp_sort_span<1>(s, A, Bbuf, dt);
      else if (s.n <= 64) warp_sort_span<2>(s, A, Bbuf, dt);
      else warp_sort_span<4>(s, A, Bbuf, dt);
    } else {
      if (s.n <= 32) warp_sort_span<1>(s, A, Bbuf, dt);
      else if (s.n <= 64) warp_sort_span<2>(s, A, Bbuf, dt);
      else if (s.n <= 128) warp_sort_span<4>(s, A, Bbuf, dt);
      else warp_sort_span<8>(s, A, Bbuf, dt);
    }
  }
}
static_assert(kWarpSortMax == 256, "the warp base case classes cover spans of up to 8 keys per lane");

// warp_placed_sort for a key-value span: the slots order (ord key, index)
// pairs (si holds each staged key's index in the span), and the values are
// gathered by index at the end.  Same slot map as the keys-only form.
template <int R, int VB>
__device__ __forceinline__ bool warp_placed_sort_kv(const Span& s, uint64_t* A, const uint64_t* Bbuf, void* VA,
                                                    const void* VBuf, int dt, uint64_t* sk, uint16_t* si,
                                                    uint32_t* sc) {
  using V = ValT<VB>;
  constexpr uint32_t NS = 32 * R;
  const unsigned lane = threadIdx.x & 31;
  const uint64_t* src = (s.buf ? Bbuf : A) + s.lo;
  const V* vsrc = static_cast<const V*>(s.buf ? VBuf : VA) + s.lo;
  const uint32_t n = s.n;
  uint64_t u[R];
  uint32_t hmin = ~0u, hmax = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const bool ok = r < R - 1 || lane + 32 * r < n;
    u[r] = ok ? ord_of(src[lane + 32 * r], dt) : 0ull;
    const uint32_t h = (uint32_t)(u[r] >> 32);
    if (ok) {
      hmin = min(hmin, h);
      hmax = max(hmax, h);
    }
  }
  hmin = __reduce_min_sync(0xFFFFFFFFu, hmin);
  hmax = __reduce_max_sync(0xFFFFFFFFu, hmax);
  uint32_t w[R];
  if (hmin == hmax) {
    uint32_t lmin = ~0u, lmax = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r < R - 1 || lane + 32 * r < n) {
        lmin = min(lmin, (uint32_t)u[r]);
        lmax = max(lmax, (uint32_t)u[r]);
      }
    }
    lmin = __reduce_min_sync(0xFFFFFFFFu, lmin);
    lmax = __reduce_max_sync(0xFFFFFFFFu, lmax);
    if (lmin == lmax) {  // all equal: input order is the stable order
      if (s.buf)
        for (uint32_t i = lane; i < n; i += 32) {
          A[s.lo + i] = src[i];
          static_cast<V*>(VA)[s.lo + i] = vsrc[i];
        }
      return true;
    }
    const uint32_t sh = __clz(lmax - lmin);
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = ((uint32_t)u[r] - lmin) << sh;
  } else {
    const uint64_t base = (uint64_t)hmin << 32;
    const uint32_t sh = __clz(hmax - hmin);
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = (uint32_t)(((u[r] - base) << sh) >> 32);
  }
#pragma unroll
  for (int q = 0; q < R; ++q) sc[q * 32 + lane] = 0;
  __syncwarp();
  uint32_t at[R], rk[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t slot = __umulhi(w[r], NS), owner = w[r] >> 27;
    at[r] = (slot - owner * R) * 32 + owner;
    rk[r] = (r < R - 1 || lane + 32 * r < n) ? atomicAdd(&sc[at[r]], 1u) : 0u;
  }
  __syncwarp();
  uint32_t c[R], loc = 0, big = 0;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    c[q] = sc[q * 32 + lane];
    loc += c[q];
    big = max(big, c[q]);
  }
  uint32_t incl = loc;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane >= (unsigned)d) incl += o;
  }
  if (__reduce_max_sync(0xFFFFFFFFu, big) > kMaxSlot) return false;
  uint32_t run = incl - loc;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    sc[q * 32 + lane] = run | (c[q] << 16);  // slot start and count
    run += c[q];
  }
  __syncwarp();
  uint32_t e[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    e[r] = sc[at[r]];
    if (r < R - 1 || lane + 32 * r < n) {
      const uint32_t p = (e[r] & 0xFFFFu) + rk[r];
      sk[p] = u[r];
      si[p] = (uint16_t)(lane + 32 * r);
    }
  }
  __syncwarp();
  // order inside the slots by (key, input index): a pair's place is its
  // slot's start plus the pairs of the slot that precede it
  uint32_t pos[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t a0 = e[r] & 0xFFFFu, me = lane + 32 * r;
    const uint32_t cn = (r < R - 1 || lane + 32 * r < n) ? e[r] >> 16 : 0u;
    uint32_t p = a0;
#pragma unroll 4
    for (uint32_t i = a0; i < a0 + cn; ++i) {
      const uint64_t x = sk[i];
      p += (x < u[r]) | ((x == u[r]) & ((uint32_t)si[i] < me));
    }
    pos[r] = p;
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (r < R - 1 || lane + 32 * r < n) {
      sk[pos[r]] = u[r];
      si[pos[r]] = (uint16_t)(lane + 32 * r);
    }
  __syncwarp();
  V val[R];
#pragma unroll
  for (int r = 0; r < R; ++r)
    val[r] = (r < R - 1 || lane + 32 * r < n) ? vsrc[si[lane + 32 * r]] : V(0);
  __syncwarp();  // every value is read before any is overwritten (vsrc may be VA)
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (r < R - 1 || lane + 32 * r < n) {
      A[s.lo + lane + 32 * r] = unord(sk[lane + 32 * r], dt);
      static_cast<V*>(VA)[s.lo + lane + 32 * r] = val[r];
    }
  __syncwarp();
  return true;
}

template <int VB>
__global__ void __launch_bounds__(kTPB, 3) k_base_small_kv(const Span* spans, uint64_t n, uint64_t* A,
                                                        const uint64_t* Bbuf, void* VA, const void* VBuf, int dt) {
  pdl_wait();
  using V = ValT<VB>;
  __shared__ uint64_t s_keys[kTPB / 32][kWarpSortMax];
  __shared__ uint16_t s_idx[kTPB / 32][kWarpSortMax];
  __shared__ uint32_t s_cnt[kTPB / 32][kSlots];
  const unsigned wid = threadIdx.x >> 5;
  uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = (gridDim.x * (uint64_t)blockDim.x) >> 5;
  for (; w < n; w += nw) {
    const Span s = spans[w];
    if (s.n < 2) {
      if (s.n == 1 && s.buf && (threadIdx.x & 31) == 0) {
        A[s.lo] = Bbuf[s.lo];
        static_cast<V*>(VA)[s.lo] = static_cast<const V*>(VBuf)[s.lo];
      }
      continue;
    }
    uint64_t* sk = s_keys[wid];
    uint16_t* si = s_idx[wid];
    uint32_t* sc = s_cnt[wid];
    bool done;
    switch ((s.n + 31) >> 5) {  // uniform across the warp
      case 1: done = warp_placed_sort_kv<1, VB>(s, A, Bbuf, VA, VBuf, dt, sk, si, sc); break;
      case 2: done = warp_placed_sort_kv<2, VB>(s, A, Bbuf, VA, VBuf, dt, sk, si, sc); break;
      case 3: done = warp_placed_sort_kv<3, VB>(s, A, Bbuf, VA, VBuf, dt, sk, si, sc); break;
      case 4: done = warp_placed_sort_kv<4, VB>(s, A, Bbuf, VA, VBuf, dt, sk, si, sc); break;
      case 5: done = warp_placed_sort_kv<5, VB>(s, A, Bbuf, VA, VBuf, dt, sk, si, sc); break;
      case 6: done = warp_placed_sort_kv<6, VB>(s, A, Bbuf, VA, VBuf, dt, sk, si, sc); break;
      case 7: done = warp_placed_sort_kv<7, VB>(s, A, Bbuf, VA, VBuf, dt, sk, si, sc); break;
      default: done = warp_placed_sort_kv<8, VB>(s, A, Bbuf, VA, VBuf, dt, sk, si, sc); break;
    }
    if (done) continue;
    if (s.n <= 32) warp_sort_span_kv<1, VB>(s, A, Bbuf, VA, VBuf, dt);
    else if (s.n <= 64) warp_sort_span_kv<2, VB>(s, A, Bbuf, VA, VBuf, dt);
    else if (s.n <= 128) warp_sort_span_kv<4, VB>(s, A, Bbuf, VA, VBuf, dt);
    else warp_sort_span_kv<8, VB>(s, A, Bbuf, VA, VBuf, dt);
  }
}

// Block bitonic network over P (ord key, index) pairs in shared memory.
__device__ void block_bitonic_smem_kv(uint64_t* sm, uint32_t* si, uint32_t P) {
  for (uint32_t k = 2; k <= P; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const uint64_t x = sm[i], y = sm[ixj];
          const uint32_t xi = si[i], yi = si[ixj];
          const bool up = (i & k) == 0;
          const bool gt = x > y || (x == y && xi > yi);
          if (gt == up) {
            sm[i] = y;
            sm[ixj] = x;
            si[i] = yi;
            si[ixj] = xi;
          }
        }
      }
      __syncthreads();
    }
  }
}

// CTA base case (257 .. 8192 keys) of a key-value sort.
template <int VB>
__global__ void __launch_bounds__(1024) k_base_large_kv(const Span* spans, uint64_t n, uint64_t* A,
                                                        const uint64_t* Bbuf, void* VA, const void* VBuf, int dt) {
  pdl_wait();
  using V = ValT<VB>;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* sm = reinterpret_cast<uint64_t*>(smem);
  for (uint64_t w = blockIdx.x; w < n; w += gridDim.x) {
    const Span s = spans[w];
    const uint64_t* src = s.buf ? Bbuf : A;
    const V* vsrc = static_cast<const V*>(s.buf ? VBuf : VA) + s.lo;
    uint32_t P = 2;
    while (P < s.n) P <<= 1;
    uint32_t* si = reinterpret_cast<uint32_t*>(sm + P);
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
      sm[i] = i < s.n ? ord_of(src[s.lo + i], dt) : ~0ull;
      si[i] = i;
    }
    __syncthreads();
    block_bitonic_smem_kv(sm, si, P);
    // values gathered into registers first: the source may be the destination
    V val[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const uint32_t i = threadIdx.x + r * blockDim.x;
      val[r] = i < s.n ? vsrc[si[i]] : V(0);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const uint32_t i = threadIdx.x + r * blockDim.x;
      if (i < s.n) {
        A[s.lo + i] = unord(sm[i], dt);
        static_cast<V*>(VA)[s.lo + i] = val[r];
      }
    }
    __syncthreads();
  }
}

template <int VB>
__global__ void k_copy_spans_kv(const Span* spans, uint64_t n, uint64_t* A, const uint64_t* Bbuf, void* VA,
                                const void* VBuf) {
  pdl_wait();
  using V = ValT<VB>;
  for (uint64_t w = blockIdx.x; w < n; w += gridDim.x) {
    const Span s = spans[w];
    for (uint32_t i = threadIdx.x; i < s.n; i += blockDim.x) {
      A[s.lo + i] = Bbuf[s.lo + i];
      static_cast<V*>(VA)[s.lo + i] = static_cast<const V*>(VBuf)[s.lo + i];
    }
  }
}

// Depth-limit fallback of a key-value sort: runs of 2048 sorted by (ord,
// index) in shared memory with their values gathered, then stable merge
// passes (equal keys: the left run first) moving (key, value) pairs between
// the two buffers; the result lands in A.
template <int VB>
__global__ void __launch_bounds__(1024) k_fallback_kv(const Span* spans, uint64_t n, uint64_t* A, uint64_t* Bbuf,
                                                      void* VA, void* VBuf, int dt) {
  pdl_wait();
  using V = ValT<VB>;
  __shared__ uint64_t sm[kSortChunk];
  __shared__ uint32_t si[kSortChunk];
  for (uint64_t w = blockIdx.x; w < n; w += gridDim.x) {
    const Span s = spans[w];
    uint64_t* src = s.buf ? Bbuf : A;
    uint64_t* oth = s.buf ? A : Bbuf;
    V* vsrc = static_cast<V*>(s.buf ? VBuf : VA);
    V* voth = static_cast<V*>(s.buf ? VA : VBuf);
    for (uint64_t r0 = 0; r0 < s.n; r0 += kSortChunk) {
      const uint32_t len = (uint32_t)(s.n - r0 < kSortChunk ? s.n - r0 : kSortChunk);
      for (uint32_t i = threadIdx.x; i < kSortChunk; i += blockDim.x) {
        sm[i] = i < len ? ord_of(src[s.lo + r0 + i], dt) : ~0ull;
        si[i] = i;
      }
      __syncthreads();
      block_bitonic_smem_kv(sm, si, kSortChunk);
      for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
        oth[s.lo + r0 + i] = sm[i];
        voth[s.lo + r0 + i] = vsrc[s.lo + r0 + si[i]];
      }
      __syncthreads();
    }
    uint64_t* cur = oth;
    uint64_t* nxt = src;
    V* vcur = voth;
    V* vnxt = vsrc;
    for (uint64_t wd = kSortChunk; wd < s.n; wd *= 2) {
      for (uint64_t o = (uint64_t)threadIdx.x * 8; o < s.n; o += (uint64_t)blockDim.x * 8) {
        const uint64_t a0 = (o / (2 * wd)) * (2 * wd);
        const uint64_t a1 = a0 + wd < s.n ? a0 + wd : s.n;
        const uint64_t b1 = a0 + 2 * wd < s.n ? a0 + 2 * wd : s.n;
        const uint64_t na = a1 - a0, nbb = b1 - a1;
        const uint64_t* X = cur + s.lo + a0;
        const uint64_t* Y = cur + s.lo + a1;
        const V* XV = vcur + s.lo + a0;
        const V* YV = vcur + s.lo + a1;
        const uint64_t diag = o - a0;
        uint64_t lo = diag > nbb ? diag - nbb : 0, hi = diag < na ? diag : na;
        while (lo < hi) {  // stable merge path: X[i] goes before Y[j] when X[i] <= Y[j]
          const uint64_t mid = (lo + hi) >> 1;
          if (X[mid] <= Y[diag - 1 - mid]) lo = mid + 1;
          else hi = mid;
        }
        uint64_t i = lo, j = diag - lo;
        const uint64_t lim = b1 - o < 8 ? b1 - o : 8;
        for (uint64_t k = 0; k < lim; ++k) {
          const bool takeX = (j >= nbb) || (i < na && X[i] <= Y[j]);
          if (takeX) {
            nxt[s.lo + o + k] = X[i];
            vnxt[s.lo + o + k] = XV[i++];
          } else {
            nxt[s.lo + o + k] = Y[j];
            vnxt[s.lo + o + k] = YV[j++];
          }
        }
      }
      __syncthreads();
      uint64_t* t = cur;
      cur = nxt;
      nxt = t;
      V* tv = vcur;
      vcur = vnxt;
      vnxt = tv;
    }
    V* VAv = static_cast<V*>(VA);
    for (uint64_t i = threadIdx.x; i < s.n; i += blockDim.x) {
      const uint64_t k = cur[s.lo + i];
      const V v = vcur[s.lo + i];
      A[s.lo + i] = unord(k, dt);  // cur may be A itself: same index, read first
      VAv[s.lo + i] = v;
    }
    __syncthreads();
  }
}

__device__ void block_bitonic_smem(uint64_t* sm, uint32_t P) {
  for (uint32_t k = 2; k <= P; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        uint32_t ixj = i ^ j;
        if (ixj > i) {
          uint64_t x = sm[i], y = sm[ixj];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            sm[i] = y;
            sm[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Model-placed base case for one span of 257..4096 keys by one 256-thread
// block: the warp form's linear map between the span's extremes, counting
// sort by slot and rank count inside slots, with block-wide reductions.
// Slot s (of 256R) belongs to thread s / R (= w >> 24) and is stored at
// (s mod R) * 256 + s / R.  Returns false (uniformly) when a slot holds
// more than kMaxSlotL keys; the caller then sorts the span with the
// bitonic network.
constexpr uint32_t kLargeTPB = 256;
constexpr int kLargeR = 16;  // keys per thread: spans of up to 4096 keys
constexpr uint32_t kMaxSlotL = 32;

template <int RR>
__device__ __forceinline__ bool block_placed_sort(const Span& s, uint64_t* A, const uint64_t* Bbuf, int dt,
                                                  uint64_t* sk, uint32_t* sc, uint32_t* red) {
  const uint32_t n = s.n, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr uint32_t kW = kLargeTPB / 32;
  const uint32_t R = (n + kLargeTPB - 1) / kLargeTPB;
  const uint64_t* src = (s.buf ? Bbuf : A) + s.lo;
  uint64_t u[RR];
  uint32_t hmin = ~0u, hmax = 0;
#pragma unroll
  for (int r = 0; r < RR; ++r) {
    const uint32_t i = tid + kLargeTPB * r;
    u[r] = i < n ? ord_of(src[i], dt) : 0ull;
    if (i < n) {
      hmin = min(hmin, (uint32_t)(u[r] >> 32));
      hmax = max(hmax, (uint32_t)(u[r] >> 32));
    }
  }
  auto block_minmax = [&](uint32_t& mn, uint32_t& mx) {
    mn = __reduce_min_sync(0xFFFFFFFFu, mn);
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    if (lane == 0) {
      red[wid] = mn;
      red[kW + wid] = mx;
    }
    __syncthreads();
    mn = red[0];
    mx = red[kW];
    for (uint32_t q = 1; q < kW; ++q) {
      mn = min(mn, red[q]);
      mx = max(mx, red[kW + q]);
    }
    __syncthreads();
  };
  block_minmax(hmin, hmax);
  uint32_t w[RR];
  if (hmin == hmax) {  // uniform: one high word, exact low-word extremes
    uint32_t lmin = ~0u, lmax = 0;
#pragma unroll
    for (int r = 0; r < RR; ++r)
      if (tid + kLargeTPB * r < n) {
        lmin = min(lmin, (uint32_t)u[r]);
        lmax = max(lmax, (uint32_t)u[r]);
      }
    block_minmax(lmin, lmax);
    if (lmin == lmax) {  // all equal: already sorted; bring home if needed
      if (s.buf)
        for (uint32_t i = tid; i < n; i += kLargeTPB) A[s.lo + i] = src[i];
      return true;
    }
    const uint32_t sh = __clz(lmax - lmin);
#pragma unroll
    for (int r = 0; r < RR; ++r) w[r] = ((uint32_t)u[r] - lmin) << sh;
  } else {
    const uint64_t base = (uint64_t)hmin << 32;
    const uint32_t sh = __clz(hmax - hmin);
#pragma unroll
    for (int r = 0; r < RR; ++r) w[r] = (uint32_t)(((u[r] - base) << sh) >> 32);
  }
  const uint32_t NS = kLargeTPB * R;
  for (uint32_t i = tid; i < NS; i += kLargeTPB) sc[i] = 0;
  __syncthreads();
  uint32_t at[RR], rk[RR];
#pragma unroll
  for (int r = 0; r < RR; ++r) {
    const uint32_t slot = __umulhi(w[r], NS), owner = w[r] >> 24;
    at[r] = (slot - owner * R) * kLargeTPB + owner;
    rk[r] = tid + kLargeTPB * r < n ? atomicAdd(&sc[at[r]], 1u) : 0u;
  }
  __syncthreads();
  // exclusive scan of the slot counts in slot order (thread t: slots tR..tR+R-1)
  uint32_t loc = 0, big = 0;
#pragma unroll
  for (int q = 0; q < RR; ++q)
    if ((uint32_t)q < R) {
      const uint32_t c = sc[q * kLargeTPB + tid];
      loc += c;
      big = max(big, c);
    }
  uint32_t incl = loc;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane >= (unsigned)d) incl += o;
  }
  big = __reduce_max_sync(0xFFFFFFFFu, big);
  if (lane == 31) red[wid] = incl;
  if (lane == 0) red[kW + wid] = big;
  __syncthreads();
  uint32_t before = 0, bmax = 0;
  for (uint32_t q = 0; q < kW; ++q) {
    before += q < wid ? red[q] : 0u;
    bmax = max(bmax, red[kW + q]);
  }
  __syncthreads();
  if (bmax > kMaxSlotL) return false;  // uniform across the block
  uint32_t run = before + incl - loc;
#pragma unroll
  for (int q = 0; q < RR; ++q)
    if ((uint32_t)q < R) {
      const uint32_t c = sc[q * kLargeTPB + tid];
      sc[q * kLargeTPB + tid] = run | (c << 16);  // slot start and count
      run += c;
    }
  __syncthreads();
  uint32_t e[RR];
#pragma unroll
  for (int r = 0; r < RR; ++r) {
    e[r] = tid + kLargeTPB * r < n ? sc[at[r]] : 0u;
    if (tid + kLargeTPB * r < n) sk[(e[r] & 0xFFFFu) + rk[r]] = u[r];
  }
  __syncthreads();
  // a key's place: its slot's start plus the keys of the slot before it
#pragma unroll
  for (int r = 0; r < RR; ++r) {
    const uint32_t a0 = e[r] & 0xFFFFu, cn = e[r] >> 16, me = a0 + rk[r];
    uint32_t p = a0;
#pragma unroll 4
    for (uint32_t i = a0; i < a0 + cn; ++i) {
      const uint64_t x = sk[i];
      p += (x < u[r]) | ((x == u[r]) & (i < me));
    }
    e[r] = p;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RR; ++r)
    if (tid + kLargeTPB * r < n) sk[e[r]] = u[r];
  __syncthreads();
  for (uint32_t i = tid; i < n; i += kLargeTPB) A[s.lo + i] = unord(sk[i], dt);
  __syncthreads();
  return true;
}

// Spans of kWarpSortMax+1 .. T keys: the placed block sort, else (clustered
// spans, or spans above 4096 keys) a bitonic network over P = 2^ceil(log2 n)
// keys in shared memory.  sk holds cap keys, then the slot words.  One
// instance per size class (spans in (lo, hi]): RR keys per thread held in
// registers, so the classes of shorter spans use fewer registers and run
// more blocks per SM; each instance walks the whole list and takes its own
// spans.
template <int RR, int MINB>
__global__ void __launch_bounds__(kLargeTPB, MINB) k_base_large(const Span* spans, uint64_t n, uint64_t* A,
                                                                const uint64_t* Bbuf, int dt, uint32_t cap,
                                                                uint32_t lo, uint32_t hi,
                                                                const unsigned long long* dn) {
  pdl_wait();
  if (dn) n = *dn;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* sm = reinterpret_cast<uint64_t*>(smem);
  uint32_t* sc = reinterpret_cast<uint32_t*>(sm + cap);
  __shared__ uint32_t red[2 * (kLargeTPB / 32)];
  for (uint64_t w = blockIdx.x; w < n; w += gridDim.x) {
    Span s = spans[w];
    if (s.n <= lo || s.n > hi) continue;  // another class's span (uniform across the block)
    if (s.n <= kLargeTPB * RR && block_placed_sort<RR>(s, A, Bbuf, dt, sm, sc, red)) continue;
    const uint64_t* src = s.buf ? Bbuf : A;
    uint32_t P = 2;
    while (P < s.n) P <<= 1;
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) sm[i] = i < s.n ? ord_of(src[s.lo + i], dt) : ~0ull;
    __syncthreads();
    block_bitonic_smem(sm, P);
    for (uint32_t i = threadIdx.x; i < s.n; i += blockDim.x) A[s.lo + i] = unord(sm[i], dt);
    __syncthreads();
  }
}

__global__ void k_copy_spans(const Span* spans, uint64_t n, uint64_t* A, const uint64_t* Bbuf,
                             const unsigned long long* dn) {
  pdl_wait();
  if (dn) n = *dn;
  for (uint64_t w = blockIdx.x; w < n; w += gridDim.x) {
    Span s = spans[w];
    for (uint32_t i = threadIdx.x; i < s.n; i += blockDim.x) A[s.lo + i] = Bbuf[s.lo + i];
  }
}

// Fallback for spans past max_depth: one block merge-sorts the span through
// the other buffer (bitonic runs of 2048 in shared memory, then merge-path
// passes), leaving the result in A.
__global__ void __launch_bounds__(1024) k_fallback(const Span* spans, uint64_t n, uint64_t* A, uint64_t* Bbuf,
                                                   int dt, const unsigned long long* dn) {
  pdl_wait();
  if (dn) n = *dn;
  __shared__ uint64_t sm[kSortChunk];
  for (uint64_t w = blockIdx.x; w < n; w += gridDim.x) {
    Span s = spans[w];
    uint64_t* src = s.buf ? Bbuf : A;
    uint64_t* oth = s.buf ? A : Bbuf;
    // runs of 2048 sorted by ord, written to `oth`
    for (uint64_t r0 = 0; r0 < s.n; r0 += kSortChunk) {
      uint32_t len = (uint32_t)(s.n - r0 < kSortChunk ? s.n - r0 : kSortChunk);
      for (uint32_t i = threadIdx.x; i < kSortChunk; i += blockDim.x)
        sm[i] = i < len ? ord_of(src[s.lo + r0 + i], dt) : ~0ull;
      __syncthreads();
      block_bitonic_smem(sm, kSortChunk);
      for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) oth[s.lo + r0 + i] = sm[i];
      __syncthreads();
    }
    uint64_t* cur = oth;
    uint64_t* nxt = src;
    for (uint64_t wd = kSortChunk; wd < s.n; wd *= 2) {
      for (uint64_t o = (uint64_t)threadIdx.x * 8; o < s.n; o += (uint64_t)blockDim.x * 8) {
        uint64_t a0 = (o / (2 * wd)) * (2 * wd);
        uint64_t a1 = a0 + wd < s.n ? a0 + wd : s.n;
        uint64_t b1 = a0 + 2 * wd < s.n ? a0 + 2 * wd : s.n;
        uint64_t na = a1 - a0, nbb = b1 - a1;
        const uint64_t* X = cur + s.lo + a0;
        const uint64_t* Y = cur + s.lo + a1;
        uint64_t diag = o - a0;
        uint64_t lo = diag > nbb ? diag - nbb : 0, hi = diag < na ? diag : na;
        while (lo < hi) {
          uint64_t mid = (lo + hi) >> 1;
          if (X[mid] <= Y[diag - 1 - mid]) lo = mid + 1;
          else hi = mid;
        }
        uint64_t i = lo, j = diag - lo;
        uint64_t lim = b1 - o < 8 ? b1 - o : 8;
        for (uint64_t k = 0; k < lim; ++k) {
          bool takeX = (j >= nbb) || (i < na && X[i] <= Y[j]);
          nxt[s.lo + o + k] = takeX ? X[i++] : Y[j++];
        }
      }
      __syncthreads();
      uint64_t* t = cur;
      cur = nxt;
      nxt = t;
    }
    // cur holds ord values; write keys to A
    for (uint64_t i = threadIdx.x; i < s.n; i += blockDim.x) A[s.lo + i] = unord(cur[s.lo + i], dt);
    __syncthreads();
  }
}

// ---------------------------------------------------- host <-> device

// Copy `bytes` (a multiple of 8) between device memory and page-locked host
// memory mapped into the device's address space, with loads and stores over
// the host link instead of a copy engine (the engines stay free for a
// concurrent sort's small copies).  16-byte words when both ends allow.
__global__ void k_link_copy(const unsigned char* __restrict__ src, unsigned char* __restrict__ dst, size_t bytes) {
  pdl_wait();
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    const size_t n16 = bytes / 16;
    for (; i + 3 * stride < n16; i += 4 * stride) {
      const uint4 a = s4[i], b = s4[i + stride], c = s4[i + 2 * stride], d = s4[i + 3 * stride];
      d4[i] = a;
      d4[i + stride] = b;
      d4[i + 2 * stride] = c;
      d4[i + 3 * stride] = d;
    }
    for (; i < n16; i += stride) d4[i] = s4[i];
    if (bytes % 16 && blockIdx.x == 0 && threadIdx.x == 0)
      *reinterpret_cast<uint2*>(dst + bytes - 8) = *reinterpret_cast<const uint2*>(src + bytes - 8);
  } else {
    const uint2* s2 = reinterpret_cast<const uint2*>(src);
    uint2* d2 = reinterpret_cast<uint2*>(dst);
    for (const size_t n8 = bytes / 8; i < n8; i += stride) d2[i] = s2[i];
  }
}

// ---------------------------------------------------- ls_classify kernels

__global__ void k_direct_classify(const DModel* mp, const Leaf* leaves, const uint64_t* __restrict__ keys, uint64_t n,
                                  int dt, double P, double Bg, uint32_t B, uint32_t* ids,
                                  unsigned long long* hist) {
  pdl_wait();
  DModel m = *mp;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t b = refine_id(m, leaves + m.leaf_off, key_value(keys[i], dt), P, Bg, B);
    if (ids) ids[i] = b;
    if (hist) atomicAdd(&hist[b], 1ull);
  }
}

__global__ void k_table_classify(const Plan* plan, const uint64_t* pivots, const uint16_t* dirs,
                                 const uint64_t* __restrict__ keys, uint64_t n, int dt, uint32_t* ids,
                                 unsigned long long* hist, uint32_t nb_pad, uint32_t cells, const FModel* fmp,
                                 const FLeaf* flp, uint32_t aux_bytes) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* sT = reinterpret_cast<uint64_t*>(smem);
  void* sAux = sT + nb_pad;
  uint32_t* sH = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(sAux) + aux_bytes);
  uint16_t* sD = static_cast<uint16_t*>(sAux);
  FLeaf* sF = static_cast<FLeaf*>(sAux);
  Plan pl = *plan;
  FModel fm;
  if (pl.cls == CLS_GUESS) fm = *fmp;
  for (uint32_t j = threadIdx.x; j < nb_pad; j += blockDim.x) {
    sT[j] = pivots[pl.tab_off + j];
    sH[j] = 0;
  }
  if (pl.cls == CLS_DIR)
    for (uint32_t j = threadIdx.x; j <= cells; j += blockDim.x) sD[j] = dirs[pl.dir_off + j];
  if (pl.cls == CLS_GUESS)
    for (uint32_t j = threadIdx.x; j < fm.L; j += blockDim.x) sF[j] = flp[fm.leaf_off + j];
  const float Pf = (float)pl.P, Bgf = (float)pl.Bg;
  __syncthreads();
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t nround = (n + stride - 1) / stride;
  for (uint64_t rd = 0; rd < nround; ++rd) {
    uint64_t i = rd * stride + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint32_t b = 0xFFFFFFFFu;
    if (i < n) {
      uint64_t bits = keys[i];
      uint64_t u = ord_of(bits, dt);
      if (pl.cls == CLS_GUESS) {
        b = fix_bucket(sT, nb_pad, pl.kmax, guess_bucket(fm, sF, nullptr, Pf, Bgf, pl.kmax, bits, dt), u);
      } else {
        b = (pl.cls == CLS_DIR) ? pivot_count_dir(sT, sD, pl.dir_lo, pl.dir_hi, pl.dir_shift, pl.kmax, u)
                                : pivot_count(sT, nb_pad, u);
        b = b < pl.kmax ? b : pl.kmax;
      }
      if (ids) ids[i] = b;
    }
    agg_inc(sH, b);
  }
  __syncthreads();
  if (hist)
    for (uint32_t j = threadIdx.x; j < nb_pad; j += blockDim.x)
      if (sH[j]) atomicAdd(&hist[j], (unsigned long long)sH[j]);
}

// ------------------------------------------------------------------ scan

__global__ void k_scan_block(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, size_t n,
                             uint64_t* __restrict__ bsum) {
  pdl_wait();
  __shared__ uint64_t w[32];
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  uint64_t x = i < n ? in[i] : 0;
  unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t incl = x;
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t o = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane >= (unsigned)d) incl += o;
  }
  if (lane == 31) w[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint64_t v = lane < (blockDim.x >> 5) ? w[lane] : 0;
    for (int d = 1; d < 32; d <<= 1) {
      uint64_t o = __shfl_up_sync(0xFFFFFFFFu, v, d);
      if (lane >= (unsigned)d) v += o;
    }
    w[lane] = v;
  }
  __syncthreads();
  uint64_t excl = incl - x + (wid > 0 ? w[wid - 1] : 0);
  if (i < n) out[i] = excl;
  if (threadIdx.x == blockDim.x - 1) bsum[blockIdx.x] = w[(blockDim.x >> 5) - 1];
}

__global__ void k_scan_add(uint64_t* __restrict__ out, size_t n, const uint64_t* __restrict__ boff) {
  pdl_wait();
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] += boff[blockIdx.x];
}

__global__ void k_scan_total(uint64_t* out, size_t n, const uint64_t* in) {
  pdl_wait();
  // out[n] = out[n-1] + in[n-1]
  if (n == 0) out[0] = 0;
  else out[n] = out[n - 1] + in[n - 1];
}

__global__ void k_fill_u64(uint64_t* p, uint64_t v, size_t n) {
  pdl_wait();
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

constexpr int kScanTPB = 1024;

}  // namespace

// ===================================================== host launchers

size_t scan_tmp_elems(size_t n) {
  size_t t = 0;
  while (n > 1) {
    n = (n + kScanTPB - 1) / kScanTPB;
    t += 2 * n + 2;
  }
  return t + 4;
}

// out[0..n] = exclusive prefix sums of in[0..n) (out[n] = total).
void launch_scan_exclusive_u64(const uint64_t* in, uint64_t* out, size_t n, uint64_t* tmp, size_t tmp_elems,
                               cudaStream_t st) {
  (void)tmp_elems;
  if (n == 0) {
    pdl_launch(k_scan_total, 1, 1, 0, st, out, 0, in);
    return;
  }
  size_t nb = (n + kScanTPB - 1) / kScanTPB;
  uint64_t* bsum = tmp;
  uint64_t* boff = tmp + nb + 1;
  pdl_launch(k_scan_block, (unsigned)nb, kScanTPB, 0, st, in, out, n, bsum);
  if (nb > 1) {
    launch_scan_exclusive_u64(bsum, boff, nb, tmp + 2 * nb + 2, 0, st);
    pdl_launch(k_scan_add, (unsigned)nb, kScanTPB, 0, st, out, n, boff);
  }
  pdl_launch(k_scan_total, 1, 1, 0, st, out, n, in);
}

void launch_fill_u64(uint64_t* p, uint64_t v, size_t n, cudaStream_t st) {
  if (n) pdl_launch(k_fill_u64, grid_for(n), kTPB, 0, st, p, v, n);
}

static int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// Raise a kernel's dynamic shared memory limit once per device.
template <typename F>
static void allow_smem(F* f, size_t sm, size_t* set) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (sm > set[dev]) {
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    set[dev] = sm;
  }
}

static size_t k1_smem(const PassArgs& a) {
  return a.nb_pad_max * (8 + 4) + a.aux_bytes + 16;
}
static size_t k3_smem(const PassArgs& a, uint32_t tpb, uint32_t vb) {
  return a.nb_pad_max * (8 + 4 + 4 + 2 * (tpb / 32)) + kTile * (8 + 2 + vb) + 16;
}

template <int CLS, int DT, bool NANCHK>
static void launch_k1(const PassArgs& a, const RunParams& rp, cudaStream_t st) {
  static size_t set[64] = {};
  size_t sm = k1_smem(a);
  allow_smem(k_classify_hist<CLS, DT, NANCHK>, sm, set);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_classify_hist<CLS, DT, NANCHK>, kTPB, sm);
  if (per < 1) per = 1;
  uint64_t grid = (uint64_t)sm_count() * per;
  if (grid > a.nchunks) grid = a.nchunks;
  pdl_launch(k_classify_hist<CLS, DT, NANCHK>, (unsigned)grid, kTPB, sm, st, a, rp);
}

template <int CLS>
static void launch_k1_cls(const PassArgs& a, const RunParams& rp, cudaStream_t st) {
  if (rp.dt == LS_U64) launch_k1<CLS, LS_U64, false>(a, rp, st);
  else if (a.check_nan) launch_k1<CLS, LS_F64, true>(a, rp, st);
  else launch_k1<CLS, LS_F64, false>(a, rp, st);
}

int launch_classify_hist(const PassArgs& a, const RunParams& rp, cudaStream_t st) {
  if (!a.nchunks) return 0;
  int n = 0;
  if (a.cls_mask & (1u << CLS_GUESS)) launch_k1_cls<CLS_GUESS>(a, rp, st), ++n;
  if (a.cls_mask & (1u << CLS_TREE)) launch_k1_cls<CLS_TREE>(a, rp, st), ++n;
  if (a.cls_mask & (1u << CLS_DIR)) launch_k1_cls<CLS_DIR>(a, rp, st), ++n;
  if (a.cls_mask & (1u << CLS_DIRECT)) launch_k1_cls<CLS_DIRECT>(a, rp, st), ++n;
  if (a.cls_mask & (1u << CLS_RADIX)) launch_k1_cls<CLS_RADIX>(a, rp, st), ++n;
  return n;
}

int launch_chunk_prefix(const ChunkSeg* segs, uint32_t nsegs, const uint2* multi, uint32_t nmulti,
                        const Plan* plans, uint32_t* agg, unsigned long long* excl, uint32_t nbp, cudaStream_t st,
                        const BatchDesc* bd, int parts) {
  // with bd the counts are read on the device and nsegs / nmulti bound the
  // grids (each block strides over the runs)
  if (!nsegs) return 0;
  const unsigned cols = (nbp + kTPB - 1) / kTPB;
  int n = 0;
  if (parts & 1) pdl_launch(k_chunk_prefix, dim3(nsegs, cols), kTPB, 0, st, segs, plans, agg, excl, nbp, bd), ++n;
  if (!nmulti || !(parts & 2)) return n;
  pdl_launch(k_run_scan, dim3(nmulti, cols), kTPB, 0, st, multi, segs, plans, agg, nbp, bd);
  pdl_launch(k_chunk_carry, dim3(nsegs, cols), kTPB, 0, st, segs, plans, agg, excl, nbp, bd);
  return n + 2;
}

template <int TPB, int QM, int VB>
static void launch_k3(const PassArgs& a, const RunParams& rp, cudaStream_t st) {
  const size_t sm = k3_smem(a, TPB, VB);
  static size_t set[64] = {};
  allow_smem(k_scatter<TPB, QM, VB>, sm, set);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_scatter<TPB, QM, VB>, TPB, sm);
  if (per < 1) per = 1;
  uint64_t grid = (uint64_t)sm_count() * per;
  if (grid > a.nchunks) grid = a.nchunks;
  pdl_launch(k_scatter<TPB, QM, VB>, (unsigned)grid, TPB, sm, st, a, rp);
}

// Up to 1024 buckets: 16-warp blocks (two per SM); larger tables keep the
// warp counters of 8-warp blocks within shared memory.
template <int VB>
static void launch_k3_vb(const PassArgs& a, const RunParams& rp, cudaStream_t st) {
  if (a.nb_pad_max <= 1024) launch_k3<512, 2, VB>(a, rp, st);
  else if (a.nb_pad_max <= 2048) launch_k3<256, 8, VB>(a, rp, st);
  else launch_k3<256, 16, VB>(a, rp, st);
}

void launch_scatter(const PassArgs& a, const RunParams& rp, cudaStream_t st) {
  if (!a.nchunks) return;
  if (a.vbytes == 8) launch_k3_vb<8>(a, rp, st);
  else if (a.vbytes == 4) launch_k3_vb<4>(a, rp, st);
  else launch_k3_vb<0>(a, rp, st);
}

uint32_t buffered_scatter_slots() { return (uint32_t)sm_count() * 2; }

void launch_scatter_buffered(const PassArgs& a, const RunParams& rp, const BufRun* runs, uint32_t nruns,
                             cudaStream_t st) {
  if (!nruns) return;
  static size_t set[64] = {};
  allow_smem(k_scatter_buffered, kBufSmem, set);
  const uint32_t grid = nruns < buffered_scatter_slots() ? nruns : buffered_scatter_slots();
  pdl_launch(k_scatter_buffered, grid, kBufTPB, kBufSmem, st, a, rp, runs, nruns);
}

void launch_children(const ChildArgs& a, const RunParams& rp, cudaStream_t st) {
  if (!a.nitems) return;
  size_t sm = (size_t)(LS_MAX_FANOUT + 1) * 8 + LS_MAX_FANOUT + 16;
  static size_t set[64] = {};
  allow_smem(k_children, sm, set);
  pdl_launch(k_children, a.nitems, kK2Threads, sm, st, a, rp);
}

// Keys-only warp base case of one list: mid = false for the short class
// (spans of up to kWarpSmallMax keys), true for the long one.
static void launch_small_class(bool mid, const Span* spans, uint64_t n, uint64_t blocks, uint64_t* A,
                               const uint64_t* Bbuf, int dt, const unsigned long long* dn, cudaStream_t st) {
  if (mid) pdl_launch(k_base_small<0, 8, 4>, (unsigned)blocks, kTPB, 0, st, spans, n, A, Bbuf, dt, dn);
  else pdl_launch(k_base_small<0, 4, 5>, (unsigned)blocks, kTPB, 0, st, spans, n, A, Bbuf, dt, dn);
}

void launch_base_small(const Span* spans, uint64_t n, uint64_t* A, const uint64_t* Bbuf, void* VA, const void* VBuf,
                       uint32_t vb, int dt, cudaStream_t st, bool mid) {
  if (!n) return;
  uint64_t warps = n;
  uint64_t blocks = (warps * 32 + kTPB - 1) / kTPB;
  uint64_t cap = (uint64_t)sm_count() * 16;
  if (blocks > cap) blocks = cap;
  if (vb == 8) pdl_launch(k_base_small_kv<8>, (unsigned)blocks, kTPB, 0, st, spans, n, A, Bbuf, VA, VBuf, dt);
  else if (vb == 4) pdl_launch(k_base_small_kv<4>, (unsigned)blocks, kTPB, 0, st, spans, n, A, Bbuf, VA, VBuf, dt);
  else launch_small_class(mid, spans, n, blocks, A, Bbuf, dt, nullptr, st);
}

template <typename F>
static void launch_large(F* f, const Span* spans, uint64_t n, uint32_t P, size_t sm, cudaStream_t st, size_t* set,
                         uint64_t* A, const uint64_t* Bbuf, void* VA, const void* VBuf, int dt) {
  allow_smem(f, sm, set);
  uint32_t tpb = P >= 1024 ? 1024 : (P < 64 ? 64 : P);
  uint64_t grid = n < (uint64_t)sm_count() * 8 ? n : (uint64_t)sm_count() * 8;
  pdl_launch(f, (unsigned)grid, tpb, sm, st, spans, n, A, Bbuf, VA, VBuf, dt);
}

// Keys-only block base case in three size classes, (kWarpSortMax, 1024],
// (1024, 2048], (2048, max_len]; n bounds the grid, dn (when set) holds the
// span count on the device.
static int launch_large_classes(const Span* spans, uint64_t n, uint32_t max_len, uint64_t* A, const uint64_t* Bbuf,
                                int dt, const unsigned long long* dn, cudaStream_t st) {
  int launched = 0;
  auto run = [&](auto kern, uint32_t rr, uint32_t lo, uint32_t hi, size_t* set) {
    if (hi <= lo) return;
    uint32_t Pc = 2;
    while (Pc < hi) Pc <<= 1;
    const uint32_t cap = Pc > kLargeTPB * rr ? Pc : kLargeTPB * rr;
    const size_t sm = (size_t)cap * 8 + (size_t)kLargeTPB * rr * 4;
    allow_smem(kern, sm, set);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kLargeTPB, sm);
    if (per < 1) per = 1;
    const uint64_t grid = n < (uint64_t)sm_count() * per ? n : (uint64_t)sm_count() * per;
    pdl_launch(kern, (unsigned)grid, kLargeTPB, sm, st, spans, n, A, Bbuf, dt, cap, lo, hi, dn);
    ++launched;
  };
  static size_t set4[64] = {}, set8[64] = {}, set16[64] = {};
  const uint32_t top = max_len > kWarpSortMax ? max_len : kWarpSortMax;
  run(k_base_large<4, 4>, 4, kWarpSortMax, top < 1024 ? top : 1024, set4);
  run(k_base_large<8, 3>, 8, 1024, top < 2048 ? top : 2048, set8);
  run(k_base_large<16, 2>, 16, 2048, top, set16);
  return launched;
}

int launch_base_large(const Span* spans, uint64_t n, uint32_t max_len, uint64_t* A, const uint64_t* Bbuf, void* VA,
                      const void* VBuf, uint32_t vb, int dt, cudaStream_t st) {
  if (!n) return 0;
  uint32_t P = 2;
  while (P < max_len) P <<= 1;
  if (vb) {  // (key, index) pairs: 12 bytes per slot
    static size_t set8[64] = {}, set4[64] = {};
    if (vb == 8) launch_large(k_base_large_kv<8>, spans, n, P, (size_t)P * 12, st, set8, A, Bbuf, VA, VBuf, dt);
    else launch_large(k_base_large_kv<4>, spans, n, P, (size_t)P * 12, st, set4, A, Bbuf, VA, VBuf, dt);
    return 1;
  }
  return launch_large_classes(spans, n, max_len, A, Bbuf, dt, nullptr, st);
}

void launch_copy_spans(const Span* spans, uint64_t n, uint64_t* A, const uint64_t* Bbuf, void* VA, const void* VBuf,
                       uint32_t vb, cudaStream_t st) {
  if (!n) return;
  uint64_t grid = n < (uint64_t)sm_count() * 16 ? n : (uint64_t)sm_count() * 16;
  if (vb == 8) pdl_launch(k_copy_spans_kv<8>, (unsigned)grid, kTPB, 0, st, spans, n, A, Bbuf, VA, VBuf);
  else if (vb == 4) pdl_launch(k_copy_spans_kv<4>, (unsigned)grid, kTPB, 0, st, spans, n, A, Bbuf, VA, VBuf);
  else pdl_launch(k_copy_spans, (unsigned)grid, kTPB, 0, st, spans, n, A, Bbuf,
                  static_cast<const unsigned long long*>(nullptr));
}

void launch_fallback(const Span* spans, uint64_t n, uint64_t* A, uint64_t* Bbuf, void* VA, void* VBuf, uint32_t vb,
                     int dt, cudaStream_t st) {
  if (!n) return;
  uint64_t grid = n < (uint64_t)sm_count() * 2 ? n : (uint64_t)sm_count() * 2;
  if (vb == 8) pdl_launch(k_fallback_kv<8>, (unsigned)grid, 1024, 0, st, spans, n, A, Bbuf, VA, VBuf, dt);
  else if (vb == 4) pdl_launch(k_fallback_kv<4>, (unsigned)grid, 1024, 0, st, spans, n, A, Bbuf, VA, VBuf, dt);
  else pdl_launch(k_fallback, (unsigned)grid, 1024, 0, st, spans, n, A, Bbuf, dt,
                  static_cast<const unsigned long long*>(nullptr));
}

int launch_spans_device(int which, const LevelCounters* ctr, const Span* small, const Span* mid, const Span* large,
                        const Span* copy, const Span* fallback, uint64_t n_max, uint32_t max_len, uint64_t* A,
                        uint64_t* Bbuf, int dt, cudaStream_t st) {
  const uint64_t sms = (uint64_t)sm_count();
  const uint64_t cap = n_max ? n_max : 1;
  const uint64_t gs = cap < sms * 16 ? cap : sms * 16;
  int launched = 0;
  if (which & SPANS_SMALL) {
    launch_small_class(false, small, cap, gs, A, static_cast<const uint64_t*>(Bbuf), dt, &ctr->n_base_small, st);
    launch_small_class(true, mid, cap, gs, A, static_cast<const uint64_t*>(Bbuf), dt, &ctr->n_base_mid, st);
    launched += 2;
  }
  if (which & SPANS_LARGE) launched += launch_large_classes(large, cap, max_len, A, Bbuf, dt, &ctr->n_base_large, st);
  if (which & SPANS_COPY) {
    pdl_launch(k_copy_spans, (unsigned)gs, kTPB, 0, st, copy, cap, A, static_cast<const uint64_t*>(Bbuf),
               &ctr->n_copy);
    ++launched;
  }
  if (which & SPANS_FALLBACK) {
    const uint64_t gf = cap < sms * 2 ? cap : sms * 2;
    pdl_launch(k_fallback, (unsigned)gf, 1024, 0, st, fallback, cap, A, Bbuf, dt, &ctr->n_fallback);
    ++launched;
  }
  return launched;
}

void launch_link_copy(const void* src, void* dst, size_t bytes, cudaStream_t st) {
  if (!bytes) return;
  k_link_copy<<<16, 512, 0, st>>>(static_cast<const unsigned char*>(src), static_cast<unsigned char*>(dst), bytes);
}

void launch_direct_classify(const DModel* m, const Leaf* leaves, const uint64_t* keys, uint64_t n, int dt, double P,
                            double Bg, uint32_t B, uint32_t* ids, unsigned long long* hist, cudaStream_t st) {
  if (!n) return;
  uint64_t grid = grid_for(n);
  uint64_t cap = (uint64_t)sm_count() * 8;
  if (grid > cap) grid = cap;
  pdl_launch(k_direct_classify, (unsigned)grid, kTPB, 0, st, m, leaves, keys, n, dt, P, Bg, B, ids, hist);
}

void launch_table_classify(const Plan* plan, const uint64_t* pivots, const uint16_t* dirs, const uint64_t* keys,
                           uint64_t n, int dt, uint32_t* ids, unsigned long long* hist, uint32_t nb_pad,
                           uint32_t cells, cudaStream_t st, const FModel* fm, const FLeaf* fl) {
  if (!n) return;
  uint32_t aux = (uint32_t)((((cells + 1) * 2 > LS_MAX_FANOUT * 16 ? (cells + 1) * 2 : LS_MAX_FANOUT * 16) + 15) & ~15u);
  size_t sm = (size_t)nb_pad * 12 + aux + 16;
  static size_t set[64] = {};
  allow_smem(k_table_classify, sm, set);
  uint64_t grid = grid_for(n);
  uint64_t cap = (uint64_t)sm_count() * 4;
  if (grid > cap) grid = cap;
  pdl_launch(k_table_classify, (unsigned)grid, kTPB, sm, st, plan, pivots, dirs, keys, n, dt, ids, hist, nb_pad, cells, fm,
                                                      fl, aux);
}

}  // namespace lsg
